"""Gates shared by the GPU parity tests: marginals of the CUDA path against the FP64 oracle.

Trajectory gate (the workloads' settings: Adam, lr 0.1, beta 0.05 -> 5): the marginals
after each checkpoint of the first 50 fp32 steps must agree within TOL_P = 1e-4 max-abs.

Conditioning.  Adam and RMSprop divide by D = sqrt(v_hat) + eps (eps = 1e-8), so an
absolute gradient rounding error d moves an update by about lr * d / D.  Where a
gradient passes within ~1e-6 of zero (at step 1 Adam's update is lr * sign(g)), an
fp32 and an fp64 trajectory can take different directions, and the difference is
rounding amplified by the optimizer, not a kernel error.  Elements whose oracle
denominator fell below D_COND at some step so far are therefore

* capped: at most MAX_ILL of the compared elements;
* bounded: within TOL_ILL of the oracle on the trajectory;
* checked one step at a time: from the GPU's own fp32 state (h, m, v) at the previous
  checkpoint, written back with fem_write_state, both sides advance one step; every
  element, the excluded ones by name, must then agree within TOL_P.  From the same
  state the gradient rounding enters one update only, so this pins the kernel's step
  on exactly the elements the trajectory gate could not.
* where even that one step is ill-conditioned (Adam's first step moves by
  lr g / (|g| + eps), whose slope in g is lr / eps = 1e7 at g = 0, so a gradient of
  ~1e-8 carries its rounding into the marginal at ~1e-4), the gradient the kernel
  applied is read back from its first moment, g = (m' - beta1 m) / (1 - beta1), and
  must equal the oracle's within G_TOL = 1e-8 + 1e-5 |g| (the fp32 accuracy of a sum
  of O(10) terms of size <= 1e-2; a wrong or missing term errs by ~1e-3); the
  oracle's optimizer fed with that gradient must then give the kernel's h within
  TOL_P.  Elements over TOL_P in the one-step check must be excluded ones, and this
  applies to Adam steps (every trajectory gate runs Adam).

Every comparison prints one ``PARITY`` line: compared elements, excluded elements and
their share, disagreeing replicas (paper mode), and the errors.
"""
import os

import numpy as np

import oracle as O

TOL_P = 1e-4      # marginals, max-abs
D_COND = 1e-6     # well-conditioned: optimizer denominator >= D_COND at every step so far
MAX_ILL = 5e-3    # at most this share of compared elements may be excluded
TOL_ILL = 0.05    # loose bound on excluded elements along the trajectory
G_TOL_ABS, G_TOL_REL = 1e-8, 1e-5   # applied gradient of an ill-conditioned one-step element


def sigmoid(h):
    return O.sigmoid(np.asarray(h, np.float64))


def softmax(h):
    h = np.asarray(h, np.float64)
    e = np.exp(h - h.max(axis=-1, keepdims=True))
    return e / e.sum(axis=-1, keepdims=True)


def _where(where):
    node = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    path, _, test = node.partition("::")
    return f"{os.path.basename(path)[:-3]}::{test} {where}"


def opt_state(opt):
    """(m, v) of an oracle optimizer in the library's two state slots."""
    if isinstance(opt, O.Adam):
        return opt.m, opt.v
    if isinstance(opt, O.RMSprop):
        return opt.buf, opt.v
    return opt.buf, np.zeros_like(opt.buf)


def set_opt_state(opt, m, v):
    if isinstance(opt, O.Adam):
        opt.m, opt.v = m, v
    elif isinstance(opt, O.RMSprop):
        opt.buf, opt.v = m, v
    else:
        opt.buf = m


def gpu_windows(P, h0, checkpoints, n_steps, **run_kw):
    """Anneal P from h0 in windows ending at each checkpoint.  Returns the fields and the
    full fp32 state (h, m, v) after each checkpoint; state[0] is the start (h0, 0, 0)."""
    got = {}
    state = {0: (h0, np.zeros_like(h0), np.zeros_like(h0))}
    t = 0
    for T in checkpoints:
        P.anneal(h_init=h0 if t == 0 else None, replicas=h0.shape[1], n_steps=n_steps, t_begin=t,
                 t_end=T, **run_kw)
        got[T] = P.fields()
        state[T] = P.state()
        t = T
    return got, state


def one_step_from(gpu_step, problem, n_steps, optimizer="adam", opt_kw=None, mode="exact", sched=None):
    """A function (T, (h, m, v)) -> (GPU fields, oracle fields, extra) after one step from
    that fp32 state on both sides; gpu_step(T, h, m, v) runs the GPU step and returns the
    fields and first moment it leaves.  extra["cond"] holds the oracle's optimizer
    denominators of the step; for Adam, extra also holds the applied gradients."""
    sched = dict(sched or {})

    def step(T, state):
        h, m, v = (np.ascontiguousarray(x, dtype=np.float32) for x in state)
        got, m_got = gpu_step(T, h, m, v)
        o = O.make_optimizer(optimizer, h.shape, **(opt_kw or dict(lr=0.1)))
        set_opt_state(o, m.astype(np.float64), v.astype(np.float64))
        cd = {T + 1: None}
        ref, o = O.anneal(problem, h.astype(np.float64), n_steps, t_begin=T, t_end=T + 1,
                          optimizer=optimizer, opt=o, mode=mode, cond=cd, **sched)
        extra = dict(cond=cd[T + 1])   # the oracle's denominators of this step
        if optimizer == "adam":
            b1 = o.b1
            g_got = (m_got.astype(np.float64) - b1 * m.astype(np.float64)) / (1.0 - b1)
            g_ref = (o.m - b1 * m.astype(np.float64)) / (1.0 - b1)

            def replay(g):   # the oracle's optimizer step from the same state with gradient g
                o2 = O.make_optimizer(optimizer, h.shape, **(opt_kw or dict(lr=0.1)))
                set_opt_state(o2, m.astype(np.float64), v.astype(np.float64))
                o2.wd = 0.0   # g already holds the weight-decay term
                hh = h.astype(np.float64).copy()
                o2.step(hh, g, T + 1)
                return hh
            # the fp32 rounding of the moments the gradient is read back from
            g_rb = 2.0 ** -23 * (b1 * np.abs(m.astype(np.float64)) + np.abs(m_got.astype(np.float64))) / (1.0 - b1)
            extra.update(g_got=g_got, g_ref=g_ref, g_readback=g_rb, replay=replay)
        return got, ref, extra

    return step


def one_step(P, problem, n_steps, optimizer="adam", opt_kw=None, mode="exact", sched=None,
             **run_kw):
    """one_step_from with the GPU step of problem P: its state written with
    fem_write_state (T > 0) or a fresh start (T = 0), then one anneal step."""

    def gpu_step(T, h, m, v):
        if T == 0:    # a step count of 0 is a fresh start: fields from h_init, zero state
            P.anneal(h_init=h, n_steps=n_steps, t_end=1, optimizer=optimizer, **run_kw)
        else:
            P.set_state(h, m, v, steps_done=T)
            P.anneal(n_steps=n_steps, t_begin=T, t_end=T + 1, optimizer=optimizer, replicas=h.shape[1],
                     **run_kw)
        got, m_got, _ = P.state()
        return got, m_got

    return one_step_from(gpu_step, problem, n_steps, optimizer, opt_kw, mode, sched)


def compare(got, ref, cond, where, marg=sigmoid, agree=None, forced=None, prev=None, prev_state=None):
    """One checkpoint.  got / ref: fields [n, R] or [n, R, q]; cond: the oracle's
    denominator record of the same shape; agree: replicas compared (paper mode).
    A q-state element is excluded when any of its q denominators is.  forced: the
    one_step function, run from (prev, prev_state) when anything is excluded."""
    got = np.asarray(got)
    qstate = got.ndim == 3
    err = np.abs(marg(got) - marg(ref))
    okr = cond >= D_COND
    if qstate:
        okr = np.broadcast_to(okr.all(axis=-1, keepdims=True), got.shape)
    pool = np.ones(got.shape, bool)
    n_dis = 0
    if agree is not None:
        n_dis = int(agree.size - agree.sum())
        pool = np.broadcast_to(agree[None, :, None] if qstate else agree[None, :], got.shape)
    ok = pool & okr
    ill = pool & ~okr
    n_pool, n_ill = int(pool.sum()), int(ill.sum())
    e_ok = float(err[ok].max()) if ok.any() else 0.0
    e_ill = float(err[ill].max()) if ill.any() else 0.0
    n_over = int((err[ill] > TOL_P).sum())
    line = (f"PARITY {_where(where)}: {n_pool} compared, {n_ill} excluded ({n_ill / max(1, n_pool):.1e}, "
            f"{n_over} of them over {TOL_P:g}), {n_dis} replicas disagree | max err {e_ok:.2e}, "
            f"excluded {e_ill:.2e}")
    e1 = e1_ill = None
    over = None
    if n_ill and forced is not None:
        g1, r1, extra = forced(prev, prev_state)
        err1 = np.abs(marg(g1) - marg(r1))
        e1, e1_ill = float(err1.max()), float(err1[ill].max())
        line += f" | one step from t={prev}: max err {e1:.2e}, excluded {e1_ill:.2e}"
        over = err1 > TOL_P
        if over.any():
            if qstate:   # a q-state element's fields share one conditioning record
                over = np.broadcast_to(over.any(axis=-1, keepdims=True), got.shape)
            assert not (over & ~ill).any(), (where, "over TOL_P in one step and not excluded")
            assert "g_got" in extra, (where, "gradient read-back needs an Adam step")
            gg, gr = extra["g_got"][over], extra["g_ref"][over]
            dg = float((np.abs(gg - gr) - (G_TOL_ABS + G_TOL_REL * np.abs(gr) + extra["g_readback"][over])).max())
            e_rep = float(np.abs(marg(extra["replay"](extra["g_got"]))[over] - marg(g1)[over]).max())
            line += (f"; {int(over.sum())} ill-conditioned in that step: applied gradient within "
                     f"{float(np.abs(gg - gr).max()):.1e} of the oracle's (|g| <= {float(np.abs(gr).max()):.1e}), "
                     f"replayed update err {e_rep:.1e}")
            assert dg <= 0.0, (where, "applied gradient", dg)
            assert e_rep <= TOL_P, (where, "optimizer replay", e_rep)
    print(line)
    assert n_ill <= MAX_ILL * max(1, n_pool), (where, "excluded share", n_ill / max(1, n_pool))
    assert e_ok <= TOL_P, (where, e_ok)
    assert e_ill <= TOL_ILL, (where, "excluded", e_ill)
    if e1 is not None and over is not None:
        err1_rest = err1[~over] if over.any() else err1
        assert float(err1_rest.max() if err1_rest.size else 0.0) <= TOL_P, (where, "one step from the GPU state")
    return ill


def compare_trajectory(got, ref, cd, checkpoints, where, marg=sigmoid, agree=None, forced=None,
                       state=None):
    """compare() at every checkpoint; the one-step check starts from the GPU's state at the
    previous checkpoint (state[0] is the initial one)."""
    prev = 0
    for T in checkpoints:
        compare(got[T], ref[T], cd[T], (where, T), marg=marg, agree=agree, forced=forced, prev=prev,
                prev_state=None if state is None else state[prev])
        prev = T
