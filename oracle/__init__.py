"""Oracle for mixed-datatype gemm (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package. The library (``paper_1901_06015_gb300``) never does, and
this package imports nothing from the library.
"""
from .oracle import (  # noqa: F401
    DT_CODES, TRANS_CODES, build, oracle_mxgemm, oracle_case_of, oracle_round, OracleError,
)
