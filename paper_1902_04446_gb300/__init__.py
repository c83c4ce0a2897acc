"""Python binding of the GB300 blocked Floyd-Warshall APSP library.

Argument marshalling only: every step of a solve runs in the CUDA kernels of
``libapsp.so`` (built from ``csrc/`` by ``build.py``).  There is no CPU
fallback; importing this package without the built library raises.

The names follow the C ABI in ``include/apsp.h``: ``Handle.solve``,
``Handle.solve_t``, ``Handle.solve_edges``, ``Handle.last_status``,
``Handle.int16_bound``, ``Handle.minplus``, ``Handle.submit`` / ``poll`` /
``wait`` / ``fetch`` / ``release`` / ``cancel``.  Matrices are passed as torch
CUDA tensors (device memory and streams are PyTorch's; nothing else is).
"""
from __future__ import annotations

from ._lib import (  # noqa: F401
    APSP_AUTO,
    APSP_F32,
    APSP_I32,
    APSP_U16,
    INF_I32,
    INF_U16,
    ApspError,
    STATES,
    get_lib,
    lib_path,
)
from .handle import Handle, dtype_code, tri_empty, tri_layout, tri_rows, tri_to_dense  # noqa: F401


def __getattr__(name):
    # ``paper_1902_04446_gb300.lib`` loads libapsp.so on first access
    if name == "lib":
        return get_lib()
    raise AttributeError(name)

__all__ = ["Handle", "ApspError", "get_lib", "lib_path", "dtype_code", "tri_layout", "tri_empty", "tri_rows",
           "tri_to_dense", "INF_I32", "INF_U16",
           "APSP_I32", "APSP_U16", "APSP_F32", "APSP_AUTO", "STATES"]
