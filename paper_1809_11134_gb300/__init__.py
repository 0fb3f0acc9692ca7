"""GB300-native batched fitness engine for the Quantum Encoded Quantum
Evolutionary Algorithm (Krylov & Lukac, arXiv:1809.11134).

The compute path is libqe.so (hand-written sm_103a CUDA behind the C ABI of
include/qe.h); `qe` is its thin Python binding and `workloads` builds seeded
synthetic inputs.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "qe", "build"]


def build(force=False, verbose=False):
    from . import _build
    return _build.build(force=force, verbose=verbose)
