"""GB300-native sparse matrix permutation, extraction and assignment (arXiv 2509.20776).

The compute path is the CUDA library ``libspgb.so`` (C ABI: ``include/sp.h``); this
package only builds it (``build.build()``), binds it (``Context``), schedules requests
over it (``serving``) and tunes its run-time kernel shapes (``autotune``).
"""
from ._binding import (  # noqa: F401
    CSR, Context, ExtractBatch, PermuteBatch, SpError, load_library, LIB_PATH, SP_ASSIGN_REPLACE, SP_ASSIGN_SELECT2ND,
    SP_ASSIGN_PLUS, SP_OPT_SPIN_LIMIT, SP_OPT_SCAN_HOLD_TILE, SP_OPT_VALIDATE, SP_OPT_TIMING, SIGNATURES, PHASES,
    SP_OPT_TILE_SHAPE, SP_OPT_HEAVY, SP_OPT_COUNT_ROWS, SP_OPT_FILL_ROWS, SP_OPT_BATCH_ROWS, SP_OPT_IDENTIFY, SP_OPT_OVERLAP,
    TorchAllocator, sp_allocator, sp_csr, tune_entries,
)
