"""GB300-native (sm_103a) FP64 hot path of the high-order gas-kinetic scheme with
hybrid WENO-AO reconstruction (arXiv 2304.05572).

The computation runs in the CUDA library behind the C ABI of ``include/hgks.h``;
``hgks`` is its Python binding (ctypes, argument marshalling only),
``problems`` holds the seeded initial data of the test problems and of the
benchmark workloads, and ``server`` is the continuous-batching solve server.
"""
from . import problems  # noqa: F401

__all__ = ["problems", "hgks", "build"]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)
