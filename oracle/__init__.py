"""Oracle: a plain, slow, FP64 CPU implementation of the relaxed FMM-BEM hot path's
definition (dense collocation BEM at the same quadrature, textbook GMRES and the
relaxation schedule).

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import, call, link or execute anything here. The product
path (paper_1506_05957_gb300) never imports it, and the oracle imports nothing
from the product path: the two share only the seeded input generators in synth/.

Parity status per function is stated in each module's header.
"""
from . import quadrature, panels, dense, gmres, schedule, richardson  # noqa: F401
