"""CPU FP64 oracle for the filtered Paterson-Stockmeyer scheme (PSSCF).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It is plain and slow on purpose and
shares no code with the CUDA library in ``paper_2208_05683_gb300``.

What it computes, with the paper passage each part follows:
  sparse.matmul_add   matrix products of Eq. (11) and Eq. (14)
  sparse.axpy         the blocks B-hat_i of Eq. (13) and the g = 1 step
  sparse.norm1        ||.||_1 with exactly rounded column sums (Sec. 2.2)
  sparse.alg1         Algorithm 1 (Sec. 3.1.1)
  sparse.horner_dense dense Horner (Eq. 1), for small tests
  planner             Eqs. (5), (6), (24)-(28), (34)-(37), Lemma 1
  psscf.psscf         Algorithm 2 (Sec. 3.2.3), filtered and unfiltered; with
                      square=True on W = Z^2 for even or odd series
                      (planner.split_even_odd, an adjacent variant)
  normest             deterministic estimates of ||Z^k||_1, k <= 10 (Sec. 3.2.2)

Pinned by ``tests/test_oracle_*.py`` against closed forms, exact rational
arithmetic, library routines and invariants.  Parity unpinned: Algorithm 1's
exact pass counts on the configured workloads (only its invariants are
pinned), and the paper's Table 1/2 errors (their matrices are not available).
"""
from .sparse import CSR, Alg1Result, OracleNotConverged, alg1, axpy, exact_abs_sum, horner_dense, matmul_add, norm1
from . import planner
from .psscf import Result, StepStat, block, power_norms, psscf
from . import normest
from ._lib import build

__all__ = [
    "CSR", "Alg1Result", "OracleNotConverged", "alg1", "axpy", "exact_abs_sum", "horner_dense",
    "matmul_add", "norm1", "planner", "Result", "StepStat", "block", "power_norms", "psscf", "normest", "build",
]
