"""B300-native (sm_103a) implementation of the SwinGS hot path (arXiv
2409.07759): differentiable tile-based splatting of the frame-t active set,
the SGLD noise / relocation step and per-frame slice replacement, as hand-
written CUDA behind the C ABI of include/swgs.h.

Submodules: ``api`` (torch-facing API and autograd), ``_abi`` (ctypes
binding), ``synth`` (seeded inputs), ``window`` (batched training window),
``serving`` (continuous-batching playback loop), ``autotune``, ``build``.
The torch-facing names are imported lazily so that ``synth`` can be used
without CUDA.
"""
__all__ = ["GaussianState", "GaussianGrads", "Renderer", "render", "slice_range", "SwgsError"]


def __getattr__(name):
    if name in __all__:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
