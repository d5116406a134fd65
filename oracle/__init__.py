"""FP64 CPU oracle for the k-ISDF fragment-ERI path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library (no kernels, headers, helpers or tables); the only module both
sides read is the seeded input generator ``paper_2601_16379_gb300.workloads``,
which holds no k-ISDF arithmetic.

Every k-sum here is a direct double sum over the k-mesh (O(Nk^2)), written as
the paper's equations define it, not the FFT convolution that the method uses
for speed (Algorithm 1, Algorithm 2).  See ``isdf_oracle`` for the functions
and the passage each one follows.
"""
from .isdf_oracle import *  # noqa: F401,F403
