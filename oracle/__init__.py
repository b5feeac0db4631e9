"""FP64 CPU oracle of DCF-PCA (test infrastructure only).

This package is the plain, slow, obviously-correct restatement of the
method used to check the CUDA path.  Only the test-suite, the package's
``smoke()`` self-check and the CPU-baseline leg of the benchmark may import
it; the library itself never does, and this package never imports the
library.  Everything is float64 numpy; a library primitive (a matrix
product, a Cholesky factorisation) serves as a step where the paper's
formula is a plain linear-algebra definition.
"""
from .dcf_oracle import *  # noqa: F401,F403
from .dcf_oracle import __all__  # noqa: F401
