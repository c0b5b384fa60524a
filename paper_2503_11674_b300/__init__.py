"""B300-native timing hot path of path-based timing-driven global placement.

``TimingGraph`` (sta_propagate, extract_critical_paths,
attraction_update_pairs, attraction_loss_fwd/bwd) and ``AttractionLoss`` wrap
the CUDA library built from ``csrc/`` for sm_103a; see ``include/tdp.h``.
"""
from . import _abi  # noqa: F401

__all__ = ["TimingGraph", "AttractionLoss", "attraction_loss", "build"]


def __getattr__(name):
    if name in ("TimingGraph", "AttractionLoss", "attraction_loss"):
        from . import timing
        return getattr(timing, name)
    if name == "build":
        from .build import build
        return build
    raise AttributeError(name)
