"""ctypes front end of the oracle's complex128 contractor (contract.c). Test infrastructure only.

`contract(net, steps)` contracts a network along a tree given as a list of (left, right) node ids;
node ids follow the engine's export convention: leaves are 0..n-1 (tensor index) and step s
produces node n + s.  The network is anything with `degrees`, `dims`, `data` (complex128
interleaved as float64) and `edges` ([E, 4] int: u, a, v, b) attributes.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.oracle_contract.restype = ctypes.c_int
        lib.oracle_contract.argtypes = [
            ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def contract(net, steps, out_cap=None):
    """Returns (result as complex128 ndarray of the final tensor, list of its leg edge ids)."""
    lib = _load()
    degrees = np.ascontiguousarray(net.degrees, dtype=np.int32)
    dims = np.ascontiguousarray(net.dims, dtype=np.int64)
    data = np.ascontiguousarray(net.data, dtype=np.float64)
    edges = np.ascontiguousarray(np.asarray(net.edges, dtype=np.int32).reshape(-1, 4))
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.int32).reshape(-1, 2))
    n = len(degrees)
    if out_cap is None:
        open_dims = [int(dims[int(np.sum(degrees[:u])) + a]) for u, a, v, b in edges if v < 0]
        out_cap = int(np.prod(open_dims, dtype=object)) if open_dims else 1
    out = np.zeros(2 * out_cap, dtype=np.float64)
    legs = np.zeros(max(len(edges), 1), dtype=np.int32)
    rank = np.zeros(1, dtype=np.int32)
    rc = lib.oracle_contract(n, _ptr(degrees), _ptr(dims), _ptr(data), len(edges), _ptr(edges),
                             len(st), _ptr(st), _ptr(out), out_cap, _ptr(legs), _ptr(rank))
    if rc != 0:
        raise RuntimeError(f"oracle_contract failed with code {rc}")
    r = int(rank[0])
    lg = [int(x) for x in legs[:r]]
    size = 1
    edim = {}
    off = np.concatenate([[0], np.cumsum(degrees)])
    for e, (u, a, v, b) in enumerate(edges):
        edim[e] = int(dims[off[u] + a])
    for e in lg:
        size *= edim[e]
    vals = out[:2 * size].view(np.complex128).copy()
    return vals.reshape([edim[e] for e in lg]) if r else vals.reshape(()), lg


def contract_scalar(net, steps) -> complex:
    v, legs = contract(net, steps, out_cap=1)
    if legs:
        raise ValueError("network is not closed")
    return complex(v)
