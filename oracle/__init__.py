"""CPU oracle for the three sparse primitives (permutation, extraction, assignment).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The library (``paper_2509_20776_gb300``) never imports it and shares no code with it.
"""
from .sparse_oracle import (  # noqa: F401
    CSR, OracleError, build_csr, assign, exclusive_scan, extract, extract_row,
    assign_row, inverse_map, kept_counts, permute, permute_row,
    to_dense, from_dense, canonical_check,
)
