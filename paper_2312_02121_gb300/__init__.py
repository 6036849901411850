"""GB300-native differentiable 3D Gaussian-splatting rasteriser (arXiv 2312.02121).

The compute path is the C-ABI library ``libgsplat103.so`` (hand-written CUDA
kernels for sm_103a, declared in ``include/gsplat103.h``).  ``binding`` marshals
torch tensors into it; ``autograd`` wraps the forward/backward in a
``torch.autograd.Function``; ``batch`` renders many views/scenes per launch;
``train`` runs the graph-captured optimisation loop; ``shard`` splits a batch of
views or scenes over ranks; ``debug`` holds the GS_DEBUG invariant checks.
``workloads`` only draws seeded synthetic inputs.

Submodules are imported lazily so that ``workloads`` can be used without torch
or a GPU.
"""
import importlib

__all__ = ["binding", "autograd", "batch", "build", "debug", "pipeline", "shard", "train", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
