"""GB300-native supernodal selected inversion (thin Python binding).

Everything numeric runs inside ``libpselinv.so`` (CUDA, sm_103a) behind the
C ABI declared in ``include/pselinv.h``; this module only marshals
arguments.  There is no CPU fallback: if the library has not been built,
every entry point raises ``LibraryMissing``.
"""
from .binding import (  # noqa: F401
    supernodal_coordinates,
    inverse_coordinates,
    order_nd,
    LibraryMissing,
    PselinvError,
    SelInv,
    lib_path,
    load_library,
    exported_symbols,
    F64,
    C128,
    PREC_FP64,
    PREC_OZAKI_FP16,
    SCHED_LEVEL,
    SCHED_PER_SUPERNODE,
    LAYOUT_PATTERN_A,
    LAYOUT_SUPERNODAL,
    LAYOUT_FACTORS,
    CostModel,
    InstanceGroup,
    TUNE_RESET,
    TUNE_EXHAUSTIVE,
    TUNE_MODEL,
)
