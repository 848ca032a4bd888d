"""FP64 CPU oracle of the phase-field thermocapillary LBM (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It shares no code with the CUDA library.
"""
from .oracle import OracleSim, build_oracle, lattice, node_ops  # noqa: F401
