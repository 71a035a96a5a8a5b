"""FP64 CPU oracle for the block-AMR finite-volume hot path.

TEST INFRASTRUCTURE ONLY: a plain, slow, obviously-correct restatement of the paper's
method (Sections 2.1.3, 2.3 and 3.1; Figs. 1-2) in numpy. Only the tests, the smoke check
(__graft_entry__.smoke) and the bench's CPU-baseline leg may import it. It shares no
code with the CUDA library; the product path never calls it.

Parity status per part is recorded beside the pins in tests/test_oracle_*.py.
"""
from .physics import HD, MHD, SRHD, make_physics  # noqa: F401
from .solver import Config, Solver, minmod, vanleer, restrict8, morton3  # noqa: F401
