"""FP64 CPU oracle of the messenger Gibbs sampler (Jasche & Lavaux 2014).

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
product path (``paper_1402_1763_gb300``) never imports it and shares no code
with it; the two meet only through the seeded inputs of ``mockgen``.

Modules:
  philox   Philox4x32-10 and Box-Muller normals (Sec. 3.4's per-core RNGs)
  bins     k-shell table, dof weights, conjugate partners (Sec. 3.2)
  sampler  tau and N~ (Sec. 2), Alg. 1, Alg. 2 on shells, the chain driver
  adjoint  torch FP64 autograd of a fixed-P chain of sweeps (differentiation workload)
  mixing   the mixing sampler of Sec. 3.3 (Alg. 3) on k-shells
  summary  correlation length and quantiles of a recorded P(k) trace

Every function is pinned by CPU tests (tests/test_oracle_*.py) against values
the paper or the mathematics fixes, not against the oracle itself.
"""
from . import philox, bins, sampler, mixing, summary  # noqa: F401
