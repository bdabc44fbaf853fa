"""Float64 CPU oracle for the randQB_EI / randQB_FP hot path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs
of ``bench.py`` may import it.  It shares no code with the CUDA library under
``paper_1606_09402_gb300/`` and neither imports the other.

Pinned functions (see ``tests/test_oracle_*.py``): philox4x32_10 (published known-answer
vectors), omega (distribution, pairing, column addressing), randqb_ei (Theorem 1/2 identity,
Proposition 1 against randqb_b, Eckart-Young floor, exact low rank, Table 4 ranks),
randqb_fp (Proposition 2 against randqb_ei and randqb), qb_fixed_rank_adjoint (central finite
differences and torch autograd), svd_from_qb (exact SVD of exactly low-rank inputs, singular
value interlacing, the single-pass setting of Sect. 5.3).  randqb_b and randqb serve as
equivalence pins only.
"""
from .philox import philox4x32_10, omega, omega_f32
from .qb import (QB_OK, QB_NOT_CONVERGED, QB_WARN_TOL_FLOOR, QBResult, frob2, orth, qr_pos,
                 randqb, randqb_b, randqb_ei, randqb_fp, qb_fixed_rank, qb_fixed_rank_adjoint,
                 orth_loss, thm3_floor)
from .svd import svd_from_qb

__all__ = ["philox4x32_10", "omega", "omega_f32", "QB_OK", "QB_NOT_CONVERGED",
           "QB_WARN_TOL_FLOOR", "QBResult", "frob2", "orth", "qr_pos", "randqb", "randqb_b",
           "randqb_ei", "randqb_fp", "qb_fixed_rank", "qb_fixed_rank_adjoint", "orth_loss",
           "thm3_floor", "svd_from_qb"]
