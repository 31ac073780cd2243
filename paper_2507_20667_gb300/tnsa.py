"""Python binding of the C ABI in include/tnsa.h (ctypes; argument marshalling only).

Every function here has the name of the C entry point it calls and does no arithmetic of the
method: planning happens in the library's C++ planner and contraction in its CUDA kernels.  If the
shared library is missing the import fails loudly; there is no fallback.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtnsa.so")

TN_OK, TN_EINVAL, TN_ENOMEM, TN_EBUDGET, TN_ECUDA, TN_ETIMEOUT, TN_EUNSUPPORTED = range(7)
PRECISIONS = {"c128": 0, "c64": 1, "tf32": 2, "bf16": 3}
EXEC_MODES = {"persistent": 0, "graph": 1}
MODES = {"naive": 0, "directed": 1}
INITIAL = {"bfs": 0, "qubit_block": 1, "given": 2}


class TnError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class tn_edge(ctypes.Structure):
    _fields_ = [("u", ctypes.c_int32), ("a", ctypes.c_int32), ("v", ctypes.c_int32), ("b", ctypes.c_int32)]


class tn_u128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]

    def value(self) -> int:
        return int(self.lo) | (int(self.hi) << 64)


class tn_plan_opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("mode", ctypes.c_int32), ("T0", ctypes.c_double),
                ("Tf", ctypes.c_double), ("steps_per_temp", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("time_limit_s", ctypes.c_double), ("iterations", ctypes.c_int32),
                ("restart_threshold", ctypes.c_int32), ("fanin_samples", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("initial", ctypes.c_int32), ("pad0", ctypes.c_int32),
                ("initial_part", ctypes.POINTER(ctypes.c_int32)), ("position", ctypes.POINTER(ctypes.c_int32)),
                ("fanin_device", ctypes.c_int32), ("pad1", ctypes.c_int32)]


class tn_plan_info(ctypes.Structure):
    _fields_ = [("con_serial", tn_u128), ("con_dist", tn_u128), ("con_par", tn_u128), ("mem", tn_u128),
                ("initial_con_dist", tn_u128), ("k", ctypes.c_int32), ("n_steps", ctypes.c_int32),
                ("sa_iterations", ctypes.c_int32), ("sa_accepted", ctypes.c_int32),
                ("sa_restarts", ctypes.c_int32), ("plan_seconds", ctypes.c_double)]


class tn_run_info(ctypes.Structure):
    _fields_ = [("device_ms", ctypes.c_double), ("launches", ctypes.c_int32), ("n_gather", ctypes.c_int32),
                ("n_tile", ctypes.c_int32), ("n_dot", ctypes.c_int32), ("n_tc", ctypes.c_int32),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double), ("arena_bytes", ctypes.c_size_t),
                ("h2d_bytes", ctypes.c_double), ("n_local", ctypes.c_int32), ("n_local_steps", ctypes.c_int32),
                ("dyn_smem", ctypes.c_int32), ("n_warp_progs", ctypes.c_int32),
                ("bytes_warp", ctypes.c_double), ("bytes_block", ctypes.c_double), ("bytes_tc", ctypes.c_double),
                ("bytes_flow", ctypes.c_double)]

    def as_dict(self):
        return {f: (getattr(self, f)) for f, _ in self._fields_}


class tn_compile_stats(ctypes.Structure):
    _fields_ = [("global_steps", ctypes.c_int32), ("n_rows", ctypes.c_int32), ("n_tile", ctypes.c_int32),
                ("n_dot", ctypes.c_int32), ("n_local", ctypes.c_int32), ("n_local_steps", ctypes.c_int32),
                ("max_local_smem", ctypes.c_int32), ("levels", ctypes.c_int32), ("total_tiles", ctypes.c_int64),
                ("arena_bytes", ctypes.c_size_t), ("flops", ctypes.c_double), ("bytes", ctypes.c_double),
                ("n_warp_progs", ctypes.c_int32), ("n_warp_steps", ctypes.c_int32),
                ("n_chained", ctypes.c_int32), ("pad", ctypes.c_int32)]


class tn_exec_config(ctypes.Structure):
    _fields_ = [("local_budget", ctypes.c_int32), ("big_programs", ctypes.c_int32),
                ("warp_programs", ctypes.c_int32), ("tc_min_m", ctypes.c_int32), ("tc_min_n", ctypes.c_int32),
                ("tc_min_k", ctypes.c_int32), ("rows_chains", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32),
                ("graph_capture", ctypes.c_int32), ("schedule", ctypes.c_int32), ("tc_tile_n", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class tn_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("launched_requests", ctypes.c_int64),
                ("max_in_flight", ctypes.c_int32), ("pad", ctypes.c_int32), ("pool_used", ctypes.c_size_t)]


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_SIGS = {
    "tn_build": (_I32, [_I32, _P, _P, _P, _I32, _P, ctypes.POINTER(_P)]),
    "tn_net_set_tensor": (_I32, [_P, _I32, _P]),
    "tn_net_info": (_I32, [_P, _P, _P, _P]),
    "tn_net_free": (None, [_P]),
    "tn_plan_opts_default": (None, [ctypes.POINTER(tn_plan_opts)]),
    "tn_plan_create": (_I32, [_P, ctypes.POINTER(tn_plan_opts), ctypes.POINTER(_P)]),
    "tn_plan_import": (_I32, [_P, _I32, _P, _I32, _P, ctypes.POINTER(_P)]),
    "tn_plan_counts": (_I32, [_P, ctypes.POINTER(tn_u128), ctypes.POINTER(tn_u128), ctypes.POINTER(tn_u128)]),
    "tn_plan_eval_states": (_I32, [_P, _I32, _I32, _I32, _I32, _P, _P, _P, _P, _P]),
    "tn_plan_slice": (_I32, [_P, _P, tn_u128, _I32, _P, _P, _P, _P, _P, _P]),
    "tn_contract_sliced": (_I32, [_P, _P, _P, _I32, _I32, _P, _I32, ctypes.c_int64, ctypes.c_int64, _P, _P, _P]),
    "tn_plan_get_info": (_I32, [_P, ctypes.POINTER(tn_plan_info)]),
    "tn_plan_export": (_I32, [_P, _P, _P, _P, _P]),
    "tn_plan_free": (None, [_P]),
    "tn_plan_compile_stats": (_I32, [_P, _P, _I32, _I32, ctypes.POINTER(tn_compile_stats)]),
    "tn_plan_compile_steps": (_I32, [_P, _P, _I32, _I32, _P, _I32, _P]),
    "tn_ctx_create": (_I32, [_I32, _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "tn_ctx_free": (None, [_P]),
    "tn_ctx_synchronize": (_I32, [_P]),
    "tn_ctx_device": (_I32, [_P, ctypes.POINTER(_I32)]),
    "tn_serve_create": (_I32, [_P, _I32, ctypes.c_size_t, _I32, ctypes.POINTER(_P)]),
    "tn_serve_register": (_I32, [_P, _P, _P, ctypes.POINTER(_I32)]),
    "tn_serve_model_info": (_I32, [_P, _I32, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_double)]),
    "tn_serve_submit": (_I32, [_P, _I32, _I32, _P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "tn_serve_poll": (_I32, [_P, ctypes.c_uint64, ctypes.c_double, _P, ctypes.POINTER(_I32),
                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I32)]),
    "tn_serve_get_stats": (_I32, [_P, ctypes.POINTER(tn_serve_stats)]),
    "tn_serve_free": (None, [_P]),
    "tn_ctx_set_exec_mode": (_I32, [_P, _I32]),
    "tn_ctx_set_local_budget": (_I32, [_P, _I32]),
    "tn_ctx_get_config": (_I32, [_P, ctypes.POINTER(tn_exec_config)]),
    "tn_ctx_set_config": (_I32, [_P, ctypes.POINTER(tn_exec_config)]),
    "tn_ctx_autotune": (_I32, [_P, _I32, _P, _P, _I32, _I32, ctypes.POINTER(tn_exec_config),
                               ctypes.POINTER(ctypes.c_double), _P, _I32, ctypes.POINTER(_I32)]),
    "tn_batch_create": (_I32, [_P, _I32, _P, _P, _I32, ctypes.POINTER(_P)]),
    "tn_batch_run": (_I32, [_P, _P]),
    "tn_batch_results": (_I32, [_P, _P, _P, _P]),
    "tn_batch_footprint": (_I32, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "tn_batch_last_info": (_I32, [_P, ctypes.POINTER(tn_run_info)]),
    "tn_batch_kernel_ms": (_I32, [_P, _I32, ctypes.POINTER(ctypes.c_double)]),
    "tn_batch_set_tensors": (_I32, [_P, _I32, _P, _P, _P]),
    "tn_batch_set_profiling": (_I32, [_P, _I32]),
    "tn_batch_debug_hold": (_I32, [_P, _I32, _I32]),
    "tn_batch_kernel_times": (_I32, [_P, _I32, _P]),
    "tn_batch_profile": (_I32, [_P, _P, _P]),
    "tn_batch_free": (None, [_P]),
    "tn_batch_contract": (_I32, [_P, _I32, _P, _P, _I32, _P, _P]),
    "tn_program_create": (_I32, [_P, _P, _P, _I32, ctypes.POINTER(_P)]),
    "tn_program_run": (_I32, [_P, _P]),
    "tn_program_footprint": (_I32, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "tn_program_last_info": (_I32, [_P, ctypes.POINTER(tn_run_info)]),
    "tn_program_free": (None, [_P]),
    "tn_contract": (_I32, [_P, _P, _P, _I32, _P, _P, ctypes.POINTER(tn_run_info)]),
    "tn_permute": (_I32, [_P, _P, _P, _I32, _I32, _P, _P]),
    "tn_dot_noalloc": (_I32, [_I32, _P, _P, _P, ctypes.c_int64, _I32, _P]),
    "tn_status_str": (ctypes.c_char_p, [_I32]),
    "tn_last_error": (ctypes.c_char_p, []),
    "tn_version": (ctypes.c_char_p, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2507_20667_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _check(status):
    if status != TN_OK:
        raise TnError(status, lib.tn_last_error().decode() or lib.tn_status_str(status).decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


_LIVE = {name: weakref.WeakSet() for name in ("tn_serve_free", "tn_batch_free", "tn_program_free", "tn_ctx_free",
                                               "tn_plan_free", "tn_net_free")}


class _Handle:
    _free = None

    def __init__(self, ptr, keep=()):
        self.ptr = ptr
        self._keep = keep
        if self._free:
            _LIVE[self._free].add(self)

    def close(self):
        if getattr(self, "ptr", None) and self._free is not None and lib is not None:
            getattr(lib, self._free)(self.ptr)
        self.ptr = None

    def __del__(self):
        self.close()

    @property
    def _as_parameter_(self):
        return self.ptr


@atexit.register
def _free_all():
    """Release every live handle, dependents first, while the CUDA runtime is still up (at process
    exit the interpreter would otherwise free them in arbitrary order, possibly after the runtime's
    own teardown)."""
    for name in ("tn_serve_free", "tn_batch_free", "tn_program_free", "tn_ctx_free", "tn_plan_free", "tn_net_free"):
        for h in list(_LIVE[name]):
            h.close()


class Net(_Handle):
    _free = "tn_net_free"


class Plan(_Handle):
    _free = "tn_plan_free"


class Ctx(_Handle):
    _free = "tn_ctx_free"


class Program(_Handle):
    _free = "tn_program_free"


class Batch(_Handle):
    _free = "tn_batch_free"


class Server(_Handle):
    _free = "tn_serve_free"


def tn_build(network) -> Net:
    """network: any object with degrees, dims, data (float64 interleaved) and edges ([E,4])."""
    degrees = np.ascontiguousarray(network.degrees, dtype=np.int32)
    dims = np.ascontiguousarray(network.dims, dtype=np.int64)
    data = np.ascontiguousarray(network.data, dtype=np.float64)
    edges = np.ascontiguousarray(np.asarray(network.edges, dtype=np.int32).reshape(-1, 4))
    out = ctypes.c_void_p()
    _check(lib.tn_build(len(degrees), _ptr(degrees), _ptr(dims), _ptr(data), len(edges), _ptr(edges),
                        ctypes.byref(out)))
    return Net(out.value)


def tn_net_set_tensor(net: Net, t: int, values) -> None:
    v = np.ascontiguousarray(np.asarray(values, dtype=np.complex128)).view(np.float64)
    _check(lib.tn_net_set_tensor(net, int(t), _ptr(v)))


def tn_net_info(net: Net):
    n, e, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib.tn_net_info(net, ctypes.byref(n), ctypes.byref(e), ctypes.byref(c)))
    return n.value, e.value, bool(c.value)


def tn_plan_opts_default() -> tn_plan_opts:
    o = tn_plan_opts()
    lib.tn_plan_opts_default(ctypes.byref(o))
    return o


def tn_plan_create(net: Net, k=1, mode="directed", T0=None, Tf=None, steps_per_temp=None, threads=None,
                   time_limit_s=None, iterations=None, restart_threshold=None, fanin_samples=None,
                   seed=None, initial_part=None, initial=None, position=None, fanin_device=None) -> Plan:
    """initial: "bfs", "qubit_block" (needs `position`, e.g. each tensor's qubit) or "given" (needs
    `initial_part`); when omitted, "given" if initial_part is passed, else "qubit_block" if position
    is passed, else "bfs"."""
    o = tn_plan_opts_default()
    o.k = int(k)
    o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    for name, val in (("T0", T0), ("Tf", Tf), ("steps_per_temp", steps_per_temp), ("threads", threads),
                      ("time_limit_s", time_limit_s), ("iterations", iterations),
                      ("restart_threshold", restart_threshold), ("fanin_samples", fanin_samples),
                      ("seed", seed), ("fanin_device", fanin_device)):
        if val is not None:
            setattr(o, name, val)
    if initial is None:
        initial = "given" if initial_part is not None else ("qubit_block" if position is not None else "bfs")
    o.initial = INITIAL[initial] if isinstance(initial, str) else int(initial)
    keep = []
    for field, arr in (("initial_part", initial_part), ("position", position)):
        if arr is not None:
            a = np.ascontiguousarray(arr, dtype=np.int32)
            keep.append(a)
            setattr(o, field, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    out = ctypes.c_void_p()
    _check(lib.tn_plan_create(net, ctypes.byref(o), ctypes.byref(out)))
    return Plan(out.value)


def tn_plan_import(net: Net, steps, part=None, k=None) -> Plan:
    st = np.ascontiguousarray(np.asarray(steps, dtype=np.int32).reshape(-1, 2))
    if part is None:
        pa, kk = None, 1
    else:
        pa = np.ascontiguousarray(part, dtype=np.int32)
        kk = int(k if k is not None else pa.max() + 1)
    out = ctypes.c_void_p()
    _check(lib.tn_plan_import(net, kk, _ptr(pa) if pa is not None else None, len(st), _ptr(st),
                              ctypes.byref(out)))
    return Plan(out.value)


def tn_plan_eval_states(net: Net, k: int, parts, fanin_samples: int = 32, device: int = -1):
    """Counts of many states (parts: [n_states, n_tensors]): (con_serial, con_dist, mem,
    saturated) as lists of Python ints / bools."""
    p = np.ascontiguousarray(np.asarray(parts, dtype=np.int32))
    n_states = p.shape[0] if p.ndim == 2 else 0
    cs = (tn_u128 * max(n_states, 1))()
    cd = (tn_u128 * max(n_states, 1))()
    mm = (tn_u128 * max(n_states, 1))()
    sat = np.zeros(max(n_states, 1), np.int32)
    _check(lib.tn_plan_eval_states(net, int(k), int(fanin_samples), int(device), n_states, _ptr(p),
                                   ctypes.cast(cs, ctypes.c_void_p), ctypes.cast(cd, ctypes.c_void_p),
                                   ctypes.cast(mm, ctypes.c_void_p), _ptr(sat)))
    return ([cs[i].value() for i in range(n_states)], [cd[i].value() for i in range(n_states)],
            [mm[i].value() for i in range(n_states)], [bool(x) for x in sat[:n_states]])


def _u128(x: int) -> tn_u128:
    return tn_u128(x & (2 ** 64 - 1), x >> 64)


def tn_plan_slice(net: Net, plan: Plan, target_mem: int, max_edges: int = 64) -> dict:
    """Edges to slice so that the plan's per-slice mem is at most target_mem, with the counts."""
    edges = np.zeros(max(max_edges, 1), np.int32)
    n = ctypes.c_int32()
    ns, sc, sm, tc = tn_u128(), tn_u128(), tn_u128(), tn_u128()
    _check(lib.tn_plan_slice(net, plan, _u128(int(target_mem)), int(max_edges), _ptr(edges), ctypes.byref(n),
                             ctypes.byref(ns), ctypes.byref(sc), ctypes.byref(sm), ctypes.byref(tc)))
    return {"edges": edges[:n.value].tolist(), "n_slices": ns.value(), "slice_con": sc.value(),
            "slice_mem": sm.value(), "total_con": tc.value()}


def tn_contract_sliced(ctx: Ctx, net: Net, plan: Plan, sliced, precision="c64", max_jobs=1024, first_slice=0,
                       slice_count=0):
    """(mantissa, exp2, number of slices) of the sliced contraction (slice_count 0: all slices)."""
    e = np.ascontiguousarray(np.asarray(sliced, dtype=np.int32))
    amp = np.zeros(2, np.float64)
    ex = ctypes.c_int32()
    ns = ctypes.c_int64()
    _check(lib.tn_contract_sliced(ctx, net, plan, PRECISIONS[precision], len(e), _ptr(e) if len(e) else None,
                                  int(max_jobs), int(first_slice), int(slice_count), _ptr(amp), ctypes.byref(ex),
                                  ctypes.byref(ns)))
    return complex(amp[0], amp[1]), ex.value, ns.value


def tn_plan_counts(plan: Plan):
    t, c, m = tn_u128(), tn_u128(), tn_u128()
    _check(lib.tn_plan_counts(plan, ctypes.byref(t), ctypes.byref(c), ctypes.byref(m)))
    return t.value(), c.value(), m.value()


def tn_plan_get_info(plan: Plan) -> dict:
    i = tn_plan_info()
    _check(lib.tn_plan_get_info(plan, ctypes.byref(i)))
    out = {}
    for f, _ in tn_plan_info._fields_:
        v = getattr(i, f)
        out[f] = v.value() if isinstance(v, tn_u128) else v
    return out


def tn_plan_export(plan: Plan, n_tensors: int):
    part = np.zeros(n_tensors, np.int32)
    steps = np.zeros((max(n_tensors - 1, 0), 3), np.int32)
    sp = np.zeros(max(n_tensors - 1, 0), np.int32)
    ns = ctypes.c_int32()
    _check(lib.tn_plan_export(plan, _ptr(part), _ptr(steps), _ptr(sp), ctypes.byref(ns)))
    return part, steps[: ns.value], sp[: ns.value]


def tn_plan_compile_stats(net: Net, plan: Plan, precision="c64", local_budget=0) -> dict:
    st = tn_compile_stats()
    _check(lib.tn_plan_compile_stats(net, plan, PRECISIONS[precision], int(local_budget), ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in tn_compile_stats._fields_ if f != "pad"}


def tn_plan_compile_steps(net: Net, plan: Plan, precision="c64", local_budget=0) -> np.ndarray:
    """[n, 8] int64: kind, M, N, K, tiles, level, program steps, program shared-memory bytes."""
    n = ctypes.c_int32()
    _check(lib.tn_plan_compile_steps(net, plan, PRECISIONS[precision], int(local_budget), None, 0, ctypes.byref(n)))
    out = np.zeros((n.value, 8), np.int64)
    _check(lib.tn_plan_compile_steps(net, plan, PRECISIONS[precision], int(local_budget), _ptr(out), n.value,
                                     ctypes.byref(n)))
    return out


def tn_ctx_create(device=0, stream=None, hbm_budget_bytes=0) -> Ctx:
    out = ctypes.c_void_p()
    _check(lib.tn_ctx_create(int(device), ctypes.c_void_p(stream) if stream else None,
                             int(hbm_budget_bytes), ctypes.byref(out)))
    return Ctx(out.value)


def tn_ctx_synchronize(ctx: Ctx) -> None:
    _check(lib.tn_ctx_synchronize(ctx))


def tn_ctx_set_exec_mode(ctx: Ctx, mode="persistent") -> None:
    _check(lib.tn_ctx_set_exec_mode(ctx, EXEC_MODES[mode] if isinstance(mode, str) else int(mode)))


def tn_ctx_set_local_budget(ctx: Ctx, nbytes: int = -1) -> None:
    _check(lib.tn_ctx_set_local_budget(ctx, int(nbytes)))


def tn_ctx_get_config(ctx: Ctx) -> dict:
    cfg = tn_exec_config()
    _check(lib.tn_ctx_get_config(ctx, ctypes.byref(cfg)))
    return cfg.as_dict()


def tn_ctx_set_config(ctx: Ctx, **fields) -> None:
    """Change fields of the context's execution configuration (local_budget, big_programs,
    warp_programs, tc_min_m, tc_min_n, tc_min_k, rows_chains, wait_limit_us, graph_capture, schedule,
    tc_tile_n); the others keep their values."""
    cfg = tn_exec_config()
    _check(lib.tn_ctx_get_config(ctx, ctypes.byref(cfg)))
    for k, v in fields.items():
        if k not in cfg.as_dict():
            raise ValueError(f"unknown configuration field {k}")
        setattr(cfg, k, int(v))
    _check(lib.tn_ctx_set_config(ctx, ctypes.byref(cfg)))


def tn_ctx_autotune(ctx: Ctx, nets, plans, precision="c64", runs=5):
    """Times the batch under each candidate configuration, keeps the fastest in ctx.
    Returns (best configuration dict, its ms per run, [ms of every candidate])."""
    if len(nets) != len(plans):
        raise ValueError("nets and plans must have the same length")
    pn, keep_n = _handle_array(nets)
    pp, keep_p = _handle_array(plans)
    best = tn_exec_config()
    ms = ctypes.c_double()
    cand = np.zeros(32, np.float64)
    nc = _I32()
    _check(lib.tn_ctx_autotune(ctx, len(nets), pn, pp, PRECISIONS[precision], int(runs), ctypes.byref(best),
                               ctypes.byref(ms), _ptr(cand), len(cand), ctypes.byref(nc)))
    return best.as_dict(), ms.value, cand[:min(nc.value, len(cand))].tolist()


def _handle_array(hs):
    arr = (ctypes.c_void_p * len(hs))(*[h.ptr for h in hs])
    return ctypes.cast(arr, ctypes.c_void_p), arr


def tn_batch_create(ctx: Ctx, nets, plans, precision="c64") -> Batch:
    if len(nets) != len(plans):
        raise ValueError("nets and plans must have the same length")
    pn, keep_n = _handle_array(nets)
    pp, keep_p = _handle_array(plans)
    out = ctypes.c_void_p()
    _check(lib.tn_batch_create(ctx, len(nets), pn, pp, PRECISIONS[precision], ctypes.byref(out)))
    b = Batch(out.value, keep=(ctx, tuple(nets), tuple(plans)))
    b.n_jobs = len(nets)
    return b


def tn_batch_run(batch: Batch, d_results: int = 0) -> None:
    _check(lib.tn_batch_run(batch, ctypes.c_void_p(d_results) if d_results else None))


def tn_batch_results(batch: Batch, n: int = None):
    """Returns (mantissas complex128 [n], exp2 int32 [n], status int32 [n]) for all n jobs of the
    batch (the call writes every job's result, so n must be the batch's job count)."""
    jobs = getattr(batch, "n_jobs", None)
    if n is None:
        n = jobs
    elif jobs is not None and n != jobs:
        raise ValueError(f"the batch has {jobs} jobs, not {n}: every job's result is written")
    amps = np.zeros(2 * n, np.float64)
    e = np.zeros(n, np.int32)
    st = np.zeros(n, np.int32)
    _check(lib.tn_batch_results(batch, _ptr(amps), _ptr(e), _ptr(st)))
    return amps.view(np.complex128).copy(), e, st


def tn_batch_set_tensors(batch: Batch, jobs, tensors, data) -> None:
    """data: complex128 entries of all (job, tensor) pairs back to back."""
    j = np.ascontiguousarray(jobs, dtype=np.int32)
    t = np.ascontiguousarray(tensors, dtype=np.int32)
    d = np.ascontiguousarray(np.asarray(data, dtype=np.complex128).ravel()).view(np.float64)
    _check(lib.tn_batch_set_tensors(batch, len(j), _ptr(j), _ptr(t), _ptr(d)))


def tn_batch_debug_hold(batch: Batch, job: int, step: int) -> None:
    _check(lib.tn_batch_debug_hold(batch, int(job), int(step)))


def tn_batch_set_profiling(batch: Batch, on: bool = True) -> None:
    _check(lib.tn_batch_set_profiling(batch, 1 if on else 0))


def tn_batch_profile(batch: Batch):
    """(cycles int64 [16], items int64 [16]) accumulated by the persistent kernel."""
    c = np.zeros(16, np.int64)
    i = np.zeros(16, np.int64)
    _check(lib.tn_batch_profile(batch, _ptr(c), _ptr(i)))
    return c, i


def tn_batch_footprint(batch: Batch) -> int:
    b = ctypes.c_size_t()
    _check(lib.tn_batch_footprint(batch, ctypes.byref(b)))
    return b.value


def tn_batch_last_info(batch: Batch) -> dict:
    i = tn_run_info()
    _check(lib.tn_batch_last_info(batch, ctypes.byref(i)))
    return i.as_dict()


def tn_batch_kernel_times(batch: Batch, n_runs: int) -> dict:
    """Mean device time (ms) per kernel class over the last n_runs runs."""
    out = np.zeros(5, np.float64)
    _check(lib.tn_batch_kernel_times(batch, int(n_runs), _ptr(out)))
    return dict(zip(("warp_programs", "block_programs", "tc_pack", "tc_gemm", "dataflow"), out.tolist()))


def tn_batch_kernel_ms(batch: Batch, n_runs: int) -> float:
    v = ctypes.c_double()
    _check(lib.tn_batch_kernel_ms(batch, int(n_runs), ctypes.byref(v)))
    return v.value


def tn_batch_contract(ctx: Ctx, nets, plans, precision="c64"):
    pn, keep_n = _handle_array(nets)
    pp, keep_p = _handle_array(plans)
    n = len(nets)
    amps = np.zeros(2 * n, np.float64)
    e = np.zeros(n, np.int32)
    _check(lib.tn_batch_contract(ctx, n, pn, pp, PRECISIONS[precision], _ptr(amps), _ptr(e)))
    return amps.view(np.complex128).copy(), e


def tn_program_create(ctx: Ctx, net: Net, plan: Plan, precision="c64") -> Program:
    out = ctypes.c_void_p()
    _check(lib.tn_program_create(ctx, net, plan, PRECISIONS[precision], ctypes.byref(out)))
    # the program refers to ctx, net and plan: keep them alive as long as it lives
    return Program(out.value, keep=(ctx, net, plan))


def tn_program_run(prog: Program, d_result: int) -> None:
    _check(lib.tn_program_run(prog, ctypes.c_void_p(d_result)))


def tn_program_footprint(prog: Program) -> int:
    b = ctypes.c_size_t()
    _check(lib.tn_program_footprint(prog, ctypes.byref(b)))
    return b.value


def tn_program_last_info(prog: Program) -> dict:
    i = tn_run_info()
    _check(lib.tn_program_last_info(prog, ctypes.byref(i)))
    return i.as_dict()


def tn_contract(ctx: Ctx, net: Net, plan: Plan, precision="c64"):
    """Returns (amplitude mantissa as complex, exp2, run info); amplitude = mantissa * 2**exp2."""
    amp = np.zeros(2, np.float64)
    e = ctypes.c_int32()
    info = tn_run_info()
    _check(lib.tn_contract(ctx, net, plan, PRECISIONS[precision], _ptr(amp), ctypes.byref(e),
                           ctypes.byref(info)))
    return complex(amp[0], amp[1]), e.value, info.as_dict()


def tn_permute(ctx: Ctx, d_in: int, d_out: int, elem_bytes: int, dims, perm) -> None:
    d = np.ascontiguousarray(dims, dtype=np.int64)
    p = np.ascontiguousarray(perm, dtype=np.int32)
    _check(lib.tn_permute(ctx, ctypes.c_void_p(d_in), ctypes.c_void_p(d_out), int(elem_bytes), len(d),
                          _ptr(d), _ptr(p)))


def tn_dot_noalloc(device: int, stream: int, d_a: int, d_b: int, n: int, precision: str, d_out: int) -> None:
    """Inner product of two device vectors into d_out (device double[2]) without allocating."""
    _check(lib.tn_dot_noalloc(int(device), ctypes.c_void_p(stream) if stream else None, ctypes.c_void_p(d_a),
                              ctypes.c_void_p(d_b), int(n), PRECISIONS[precision], ctypes.c_void_p(d_out)))


def tn_ctx_device(ctx: Ctx) -> int:
    d = ctypes.c_int32()
    _check(lib.tn_ctx_device(ctx, ctypes.byref(d)))
    return d.value


def tn_serve_create(ctx: Ctx, precision="c64", hbm_budget_bytes=1 << 30, max_batch=64) -> Server:
    out = ctypes.c_void_p()
    _check(lib.tn_serve_create(ctx, PRECISIONS[precision], int(hbm_budget_bytes), int(max_batch), ctypes.byref(out)))
    return Server(out.value, keep=(ctx,))


def tn_serve_register(server: Server, net: Net, plan: Plan) -> int:
    m = ctypes.c_int32()
    _check(lib.tn_serve_register(server, net, plan, ctypes.byref(m)))
    return m.value


def tn_serve_model_info(server: Server, model: int):
    b = ctypes.c_size_t()
    f = ctypes.c_double()
    _check(lib.tn_serve_model_info(server, int(model), ctypes.byref(b), ctypes.byref(f)))
    return b.value, f.value


def tn_serve_submit(server: Server, model: int, tensors=(), data=()) -> int:
    t = np.ascontiguousarray(tensors, dtype=np.int32)
    d = np.ascontiguousarray(np.asarray(data, dtype=np.complex128).ravel()).view(np.float64)
    tk = ctypes.c_uint64()
    _check(lib.tn_serve_submit(server, int(model), len(t), _ptr(t), _ptr(d), ctypes.byref(tk)))
    return tk.value


def tn_serve_poll(server: Server, ticket: int, timeout_s: float = 0.0):
    """None if not finished; else (mantissa complex, exp2, latency_s).  Raises TnError for a
    request that failed (TN_EBUDGET: larger than the pool)."""
    amp = np.zeros(2, np.float64)
    e = ctypes.c_int32()
    lat = ctypes.c_double()
    done = ctypes.c_int32()
    _check(lib.tn_serve_poll(server, ctypes.c_uint64(ticket), float(timeout_s), _ptr(amp), ctypes.byref(e),
                             ctypes.byref(lat), ctypes.byref(done)))
    if not done.value:
        return None
    return complex(amp[0], amp[1]), e.value, lat.value


def tn_serve_get_stats(server: Server) -> dict:
    st = tn_serve_stats()
    _check(lib.tn_serve_get_stats(server, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in tn_serve_stats._fields_ if f != "pad"}


def tn_version() -> str:
    return lib.tn_version().decode()


def amplitude(mantissa: complex, exp2: int) -> complex:
    """value = mantissa * 2**exp2 (a representation change of the returned pair, for callers)."""
    return complex(mantissa) * (2.0 ** exp2)
