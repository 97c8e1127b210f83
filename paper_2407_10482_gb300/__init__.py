"""GB300-native NGP-RT render path (arXiv 2407.10482): occupancy-distance ray
marching, multi-level hash gathers, lightweight attention fusion, alpha
compositing and the deferred MLP, as sm_103a CUDA kernels behind the C ABI of
``include/ngprt.h``.  ``paper_2407_10482_gb300.ngprt`` is the Python binding."""

__all__ = ["ngprt", "scenes"]
