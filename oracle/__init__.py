"""CPU oracle for the regularised multifrontal LDL^T (test infrastructure).

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this package.  It shares no code with the CUDA library.
"""
from .oracle import Oracle, build_oracle, choose_form, front_factor, backward_error, FORM_AS, FORM_NE  # noqa: F401
