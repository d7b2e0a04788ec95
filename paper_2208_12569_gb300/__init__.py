"""fqsl: squashing factor Q and twist number Tw of magnetic field lines on one
GB300 (sm_103a), after Zhang et al. (2022), FastQSL. The computation lives in
the CUDA library libfqsl.so (C ABI in include/fqsl.h); ``fqsl`` is its Python
binding."""
from .fqsl import (  # noqa: F401
    F32, F32_ACC64, F64, LINE_BAD, LINE_CHORD, LINE_MAXSTEPS, LINE_MIXED, LINE_NULL_B, LINE_OUTSIDE, LINE_ROTATED, LINE_STALL,
    Batch, Field, FqslError, QTwPlane, STATIC_MAX_SEEDS, alloc_out, backward, debug_alloc_cap, loss_logq_tw, params,
    qmap_plane,
    qmap_plane_static, qmap_volume, tape_export, Tape, twist, version,
)
