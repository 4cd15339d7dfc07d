"""FP64 CPU oracle for the multivariate matrix-pencil Prony method (arXiv 2012.11430).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) imports, links or executes anything here.  Only tests/, the
smoke check in __graft_entry__ and the benchmark's CPU-baseline / reference
leg may use it.  It shares no code, tables or constants with the CUDA path;
the only code both sides see is the seeded input generator in `workloads`.
"""
from . import philox, prony_oracle, classical  # noqa: F401
