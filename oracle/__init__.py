"""FP64 CPU oracle (test infrastructure only).

Only the test-suite, the package smoke check and the benchmark's CPU-baseline leg may
import this package.  The product path never does, and it shares no code with the CUDA
library.
"""
from . import definitions, lt_oracle  # noqa: F401
