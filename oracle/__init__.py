"""Oracle for the aggregation-shattering Smoluchowski solver: TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 CPU restatement of what the paper computes (Matveev, Zhilin,
Smirnov, "Adaptive time-stepping for aggregation-shattering kinetics"):

* the right-hand side S(n) of the truncated aggregation-shattering system, Eq. (4),
  by the direct double sums that define it, and by the low-rank FFT route the paper
  relies on (Sec. 1 and Sec. 2: K_ij = sum_a U_ia V_aj, O(M R log M));
* the explicit RK2, RK4 and RKF45 schemes of Sec. 2, step doubling for RK2/RK4 with
  the step-size rule of Eq. (6) or the halve/double rule that follows it, and the
  Fehlberg rule for RKF45 (Sec. 2, last paragraph);
* diagnostics: total mass, number density and the truncation mass flux.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package. The CUDA library never calls it and shares no code with it.
"""
from .smol import *  # noqa: F401,F403
