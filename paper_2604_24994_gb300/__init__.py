"""GB300 (sm_103a) tile rasterizer for bounded power-diagram cells
(Power Foam, arxiv 2604.24994): forward render, hand-written adjoint and a
continuous-batching server behind a C ABI (include/powerfoam.h), with
pinhole and fisheye views, the optional face displacement, learned detail
sites and view-dependent site colours, per-cell contributions, the
connectivity loss (over the neighbour lists or the exact Cech adjacency),
and GPU neighbour lists.

    from paper_2604_24994_gb300 import inputs, DeviceScene, Renderer, render
    from paper_2604_24994_gb300 import build_neighbours, connect_loss, connect_loss_cech
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "DeviceScene", "Renderer", "RenderFunction", "render", "connect_loss", "connect_loss_cech",
           "build_neighbours", "build_library"]


def build_library(force: bool = False) -> str:
    from .build import build
    return build(force=force)


def __getattr__(name):
    if name in ("DeviceScene", "Renderer", "RenderFunction", "render", "Plan", "connect_loss", "connect_loss_cech",
                "build_neighbours"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
