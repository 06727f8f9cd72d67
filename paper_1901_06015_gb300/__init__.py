"""GB300-native mixed-datatype gemm (arXiv 1901.06015): C := beta*C + alpha*op(A)*op(B)
with A, B, C each stored as s/d/c/z and a separate computation precision.

The compute path is the CUDA library ``_build/libmxgemm.so`` behind the C ABI in
``include/mxgemm.h``; ``mxgemm.py`` is a thin ctypes binding to it (argument
marshalling only). There is no CPU fallback: if the library is missing, calls raise.
"""
from .mxgemm import (  # noqa: F401
    MxgError, Handle, PlanInfo, Problem, Group, Server, lib, mxgemm, mxgemm_ex, mxgemm_noalloc, mxgemm_noalloc_check_device_error, mxgemm_grouped,
    mxg_plan, mxg_tune_save, mxg_tune_load, make_problems, mxg_strerror,
    METHODS, DT_CODES, TRANS_CODES, PREC_CODES, CASE_NAMES, dt_of,
)
