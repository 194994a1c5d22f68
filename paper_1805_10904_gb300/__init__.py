"""GB300 (sm_103a) synchronous parallel Louvain community detection.

The method is that of Forster, "Parallel Louvain Community Detection Optimized
for GPUs" (arXiv 1805.10904): synchronous local moving with the minimum-label
heuristics, followed by renumbering and graph induction, level after level.
All of it runs in the CUDA library built from ``csrc/`` (C ABI in
``include/louvain.h``); this package is its Python binding.
"""
from .louvain import (Config, Level, Louvain, LouvainError, Result, load, LIB_PATH,
                      PTR_DEVICE, PTR_HOST, stack_graphs)

__all__ = ["Config", "Level", "Louvain", "LouvainError", "Result", "load", "LIB_PATH",
           "PTR_DEVICE", "PTR_HOST", "build", "stack_graphs"]


def build(force: bool = False) -> str:
    from .build import build as _build
    return _build(force=force)
