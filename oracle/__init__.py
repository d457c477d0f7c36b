"""FP64 CPU oracle for the ECS Helmholtz solver -- test infrastructure only.

Only the test suite, the package smoke check and the benchmark's CPU-baseline leg use this
package.  It shares no code with the CUDA library.
"""
from .oracle import (Oracle, OracleError, build_oracle, get_threads, lib_path, select_precond,  # noqa: F401
                     set_threads)
