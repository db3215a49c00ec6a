// Definitions shared by the host and every kernel: the bits of a problem's sticky
// device error word and the per-step scalars a step kernel reads.
#pragma once

#include <stdint.h>

namespace fem {

// Bits of the sticky device error word.
enum : int32_t { ERR_BOUNDS = 1, ERR_TIMEOUT = 2 };

// Per-step scalars, computed on the host in double and rounded to float once.
// The optimizer fields hold the PyTorch update constants of the step's count t+1.
struct StepScalars {
  float inv_beta;      // 1 / beta(t)
  float lambda;        // lambda(t) (bMinCut)
  float gq;            // gamma_grad / 4 (single field) or gamma_grad (q states)
  float lr;            // Adam: lr / (1 - beta1^(t+1)); RMSprop, SGD: lr
  float b1, omb1;      // Adam: beta1, 1-beta1 | RMSprop: alpha, 1-alpha | SGD: momentum, 1-dampening
  float b2, omb2;      // Adam: beta2, 1-beta2
  float inv_sqrt_bc2;  // Adam: 1 / sqrt(1 - beta2^(t+1))
  float eps;
  float wd;            // L2 weight decay
  float momentum;      // RMSprop momentum
  int32_t first;       // SGD: 1 at the first step (momentum buffer starts as g)
  int32_t pad[3];
};
static_assert(sizeof(StepScalars) == 64, "StepScalars must stay 64 bytes");

}  // namespace fem
