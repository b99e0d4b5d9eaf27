"""GB300-native sparse matrix permutation, extraction and assignment (arXiv 2509.20776).

The compute path is the CUDA library ``libspgb.so`` (C ABI: ``include/sp.h``); this
package only builds it (``build.build()``) and binds it (``Context``).
"""
from ._binding import (  # noqa: F401
    CSR, Context, ExtractBatch, SpError, load_library, LIB_PATH, SP_ASSIGN_REPLACE, SP_ASSIGN_SELECT2ND,
    SP_ASSIGN_PLUS, SP_OPT_SPIN_LIMIT, SP_OPT_SCAN_HOLD_TILE, SP_OPT_VALIDATE, SP_OPT_TIMING, SIGNATURES, PHASES,
)
