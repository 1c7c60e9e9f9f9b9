"""FlashSplat on GB300: optimal 3D-GS segmentation from 2D masks (arXiv 2409.08270).

The hot path -- EWA projection, tile binning with a device radix sort,
front-to-back alpha blending with per-label accumulation of alpha*T, and the
closed-form biased argmax -- runs in hand-written sm_103a CUDA kernels behind
the C-ABI library ``libflashsplat.so`` (declared in ``include/flashsplat.h``).
``flashsplat`` is the thin ctypes binding; ``synth`` makes seeded workloads.
The CUDA library is loaded on first use, not at import.
"""
