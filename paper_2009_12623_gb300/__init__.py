"""GB300-native checkpointed FWI gradient with lossy checkpoint compression.

Kukreja et al., "Lossy Checkpoint Compression in Full Waveform Inversion":
a 3D isotropic-acoustic finite-difference forward sweep whose checkpoints go
through a fixed-accuracy (absolute tolerance) block codec into a compressed
store in HBM, followed by the adjoint sweep that decompresses them and
accumulates the imaging condition.  The compute path is the C-ABI CUDA
library ``libfwi.so`` (include/fwi.h); this package binds it.
"""
from .api import (  # noqa: F401
    FWI_CKPT_BINOMIAL,
    FWI_CKPT_EVERY_K,
    FWI_CKPT_FULL,
    FWI_CKPT_SUBSAMPLE,
    Batch,
    CheckpointStore,
    FwiError,
    Geometry,
    ckpt_schedule,
    dot_f64,
    forward,
    gradient,
    gradient_host,
    gradient_per_shot,
    kernel_launch_count,
    misfit,
    ShotSpec,
    zfp_compress,
    zfp_decompress,
    zfp_max_compressed_bytes,
)
