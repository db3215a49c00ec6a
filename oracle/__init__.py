"""FP64 CPU oracle for the Free-Energy Machine (FEM) - TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, fp64 restatement of the method, written from the
paper's equations so that it can be read against them line by line.  It exists
to check the CUDA path; it is never part of it.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import or call anything here.  The CUDA library and its Python binding never
import this package, and this package never imports them: the two share no code.
The one thing both sides consume is the seeded input generator module, which
holds no arithmetic of the method.

Parity status of each function is given in its module header.  Functions whose
only check is the oracle itself are marked "parity unpinned" there.
"""
from .fem import *  # noqa: F401,F403
from .brute import *  # noqa: F401,F403
from .mpnn import *  # noqa: F401,F403
