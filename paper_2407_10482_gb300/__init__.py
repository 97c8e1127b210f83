"""GB300-native NGP-RT render path (arXiv 2407.10482): occupancy-distance ray
marching, multi-level hash gathers, lightweight attention fusion (and the other
aggregation forms of Table 3), alpha compositing and the deferred MLP, with their
reverse pass and the training objective, as sm_103a CUDA kernels behind the C ABI of
``include/ngprt.h``.

Modules: ``ngprt`` (the binding: device scenes, renderer, every entry point),
``scenes`` (seeded synthetic scenes and cameras), ``fit`` (fitting a scene to images),
``proposal`` (the learned interval proposal), ``groundtruth`` (analytic images of
the synthetic fields), ``checkpoint`` (scene files), ``train_step`` (one timed
training step), ``build`` (nvcc build of libngprt.so)."""

__all__ = ["ngprt", "scenes", "fit", "proposal", "groundtruth", "checkpoint", "train_step", "build"]
