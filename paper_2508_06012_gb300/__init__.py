"""GB300-native batched in-line atomistic EOS evaluation (arXiv 2508.06012, Sec. III).

Thin Python binding over the C ABI in ``include/mdeos.h``: ctypes marshalling only.
Every step of the lifting -> MD -> restriction path runs in the CUDA library
``libmdeos.so`` (built for sm_103a by :func:`build`).  There is no CPU fallback: if
the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmdeos.so")

MDEOS_OK, MDEOS_PENDING = 0, 1
MDEOS_EINVAL, MDEOS_ENOMEM, MDEOS_EUNPHYS, MDEOS_EBOX = -1, -2, -3, -4
MDEOS_ETIMEDOUT, MDEOS_ECUDA, MDEOS_ECANCELLED, MDEOS_ENBR = -5, -6, -7, -8
MDEOS_REF_ECOLD, MDEOS_REF_FIXED = 0, 1
MDEOS_REQ_TEMPERATURE, MDEOS_REQ_COLD = 1, 2
PATH_ALLPAIRS, PATH_ALLPAIRS_MI, PATH_NLIST = 0, 1, 2
CLOSURE_IDEAL_GAS, CLOSURE_MIE_GRUNEISEN, CLOSURE_MD = 0, 1, 2
BC_WALL, BC_FREE = 0, 1

EXPORTED = [
    "mdeos_config_default", "mdeos_create", "mdeos_submit", "mdeos_poll", "mdeos_destroy",
    "mdeos_last_error", "mdeos_batch_create", "mdeos_batch_launch",
    "mdeos_batch_device_results", "mdeos_batch_results", "mdeos_batch_destroy",
    "mdeos_batch_info", "mdeos_stats", "mdeos_debug_lift", "mdeos_debug_forces",
    "mdeos_debug_md", "mdeos_debug_force_bench", "mdeos_submit_noalloc", "mdeos_warm_export",
    "mdeos_warm_import", "mdeos_warm_reset", "mdeos_hydro_config_default", "mdeos_hydro_create", "mdeos_hydro_step",
    "mdeos_hydro_state", "mdeos_hydro_eos_results", "mdeos_hydro_destroy",
    "mdeos_serve_config_default", "mdeos_serve_create", "mdeos_serve_clock",
    "mdeos_serve_enqueue", "mdeos_serve_completed", "mdeos_serve_stats",
    "mdeos_serve_store_stats", "mdeos_serve_destroy",
    "mdeos_surrogate_create", "mdeos_surrogate_set_params", "mdeos_surrogate_get_params",
    "mdeos_surrogate_grads", "mdeos_surrogate_train", "mdeos_surrogate_predict",
    "mdeos_surrogate_gated_eval", "mdeos_surrogate_destroy", "mdeos_surrogate_set_infer_path",
    "mdeos_surrogate_infer_device", "mdeos_surrogate_set_output_transform",
    "mdeos_surrogate_fit_misfit", "mdeos_surrogate_misfit",
    "mdeos_surrogate_set_misfit_threshold",
    "mdeos_debug_gemm_bf16", "mdeos_debug_tanh",
    "mdeos_autotune",
]
SURROGATE_NPARAM = 33666
SURROGATE_INFER_TC, SURROGATE_INFER_MMA = 0, 1
SURROGATE_P_LINEAR, SURROGATE_P_ASINH = 0, 1


class mdeos_config(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int32), ("lift_iters", ctypes.c_int32),
        ("rescale_every_equil", ctypes.c_int32), ("rescale_every_avg", ctypes.c_int32),
        ("se_blocks", ctypes.c_int32), ("energy_ref_mode", ctypes.c_int32),
        ("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("mass", ctypes.c_double),
        ("rc", ctypes.c_double), ("dt", ctypes.c_double), ("skin", ctypes.c_double),
        ("hbm_budget_bytes", ctypes.c_size_t), ("cuda_stream", ctypes.c_void_p),
        ("warm_lift_iters", ctypes.c_int32), ("warm_slots", ctypes.c_int32),
        ("warm_atoms", ctypes.c_int32), ("nlist_capacity", ctypes.c_int32),
        ("max_cluster", ctypes.c_int32),
    ]


class mdeos_request(ctypes.Structure):
    _fields_ = [
        ("rho", ctypes.c_double), ("e", ctypes.c_double), ("e_ref", ctypes.c_double),
        ("natoms", ctypes.c_int32), ("steps_equil", ctypes.c_int32),
        ("steps_avg", ctypes.c_int32), ("flags", ctypes.c_uint32),
        ("seed", ctypes.c_uint64), ("element_id", ctypes.c_uint64),
    ]


class mdeos_result(ctypes.Structure):
    _fields_ = [
        ("P", ctypes.c_double), ("T", ctypes.c_double), ("sigma", ctypes.c_double * 6),
        ("epot", ctypes.c_double), ("ekin", ctypes.c_double), ("e_achieved", ctypes.c_double),
        ("P_se", ctypes.c_double), ("T_se", ctypes.c_double), ("T_target", ctypes.c_double),
        ("e_cold", ctypes.c_double), ("L", ctypes.c_double), ("pairs_per_step", ctypes.c_double),
        ("cand_per_step", ctypes.c_double), ("element_id", ctypes.c_uint64),
        ("natoms", ctypes.c_int32), ("status", ctypes.c_int32),
        ("nlist_builds", ctypes.c_int32), ("path", ctypes.c_int32),
        ("warm", ctypes.c_int32), ("nlist_retries", ctypes.c_int32),
    ]


class mdeos_hydro_config(ctypes.Structure):
    _fields_ = [
        ("nzones", ctypes.c_int32), ("closure", ctypes.c_int32),
        ("bc_left", ctypes.c_int32), ("bc_right", ctypes.c_int32),
        ("q_quad", ctypes.c_double), ("q_lin", ctypes.c_double),
        ("cfl", ctypes.c_double), ("dt_grow", ctypes.c_double), ("dt_fixed", ctypes.c_double),
        ("gamma", ctypes.c_double), ("mg_rho0", ctypes.c_double), ("mg_c", ctypes.c_double),
        ("mg_s", ctypes.c_double), ("mg_gamma", ctypes.c_double),
        ("natoms", ctypes.c_int32), ("steps_equil", ctypes.c_int32),
        ("steps_avg", ctypes.c_int32), ("steps_equil_first", ctypes.c_int32),
        ("steps_avg_first", ctypes.c_int32), ("first_temperature", ctypes.c_int32),
        ("e_ref", ctypes.c_double), ("sound_gamma", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("element_base", ctypes.c_uint64),
    ]


class mdeos_serve_config(ctypes.Structure):
    _fields_ = [
        ("max_inflight", ctypes.c_int32), ("max_batch", ctypes.c_int32),
        ("max_wait_s", ctypes.c_double), ("max_queue", ctypes.c_int32),
        ("idle_ms", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_size_t),
        ("warm", ctypes.c_int32), ("cluster", ctypes.c_int32), ("warm_bytes", ctypes.c_size_t),
    ]


RESULT_DTYPE = np.dtype([
    ("P", "f8"), ("T", "f8"), ("sigma", "f8", (6,)), ("epot", "f8"), ("ekin", "f8"),
    ("e_achieved", "f8"), ("P_se", "f8"), ("T_se", "f8"), ("T_target", "f8"),
    ("e_cold", "f8"), ("L", "f8"), ("pairs_per_step", "f8"), ("cand_per_step", "f8"),
    ("element_id", "u8"), ("natoms", "i4"), ("status", "i4"), ("nlist_builds", "i4"),
    ("path", "i4"), ("warm", "i4"), ("nlist_retries", "i4"),
])
REQUEST_DTYPE = np.dtype([
    ("rho", "f8"), ("e", "f8"), ("e_ref", "f8"), ("natoms", "i4"), ("steps_equil", "i4"),
    ("steps_avg", "i4"), ("flags", "u4"), ("seed", "u8"), ("element_id", "u8"),
])
SERVED_DTYPE = np.dtype([("id", "u8"), ("t_arrival", "f8"), ("t_launch", "f8"),
                         ("t_done", "f8"), ("result", RESULT_DTYPE)])
assert RESULT_DTYPE.itemsize == ctypes.sizeof(mdeos_result)
assert REQUEST_DTYPE.itemsize == ctypes.sizeof(mdeos_request)


class MdeosError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"mdeos status {status}: {msg}")
        self.status = status


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library (nvcc, sm_103a) in-tree."""
    from . import buildlib as _b
    return _b.build(force=force, verbose=verbose)


_lib = None


def lib():
    """Load libmdeos.so; raise if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MdeosError(MDEOS_ECUDA, f"{LIB_PATH} missing: run build() first")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp, i32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
        L.mdeos_config_default.argtypes = [P(mdeos_config)]
        L.mdeos_config_default.restype = None
        L.mdeos_create.argtypes = [P(mdeos_config), P(vp)]
        L.mdeos_submit.argtypes = [vp, vp, i32, P(ctypes.c_uint64)]
        L.mdeos_poll.argtypes = [vp, ctypes.c_uint64, vp, i32]
        L.mdeos_destroy.argtypes = [vp]
        L.mdeos_last_error.restype = ctypes.c_char_p
        L.mdeos_batch_create.argtypes = [vp, vp, i32, P(vp)]
        L.mdeos_batch_launch.argtypes = [vp, vp]
        L.mdeos_batch_device_results.argtypes = [vp]
        L.mdeos_batch_device_results.restype = vp
        L.mdeos_batch_results.argtypes = [vp, vp]
        L.mdeos_batch_destroy.argtypes = [vp]
        L.mdeos_batch_info.argtypes = [vp, P(i32), P(i32), P(i32), P(ctypes.c_size_t)]
        L.mdeos_stats.argtypes = [vp, P(ctypes.c_size_t), P(ctypes.c_size_t),
                                  P(ctypes.c_longlong), P(ctypes.c_size_t)]
        L.mdeos_debug_lift.argtypes = [P(mdeos_config), i32, d, d, ctypes.c_uint64, vp, vp, vp,
                                       P(d), vp]
        L.mdeos_debug_forces.argtypes = [P(mdeos_config), vp, i32, d, i32, d, vp, vp, vp, vp]
        L.mdeos_debug_md.argtypes = [P(mdeos_config), vp, vp, i32, d, i32, d, i32, i32, d, vp,
                                     vp, vp, vp]
        L.mdeos_submit_noalloc.argtypes = [P(mdeos_config), vp, i32, vp, vp]
        L.mdeos_debug_force_bench.argtypes = [P(mdeos_config), vp, i32, i32, d, d, i32, i32, vp,
                                              vp]
        u64 = ctypes.c_uint64
        L.mdeos_warm_export.argtypes = [vp, u64, i32, vp, vp, P(d)]
        L.mdeos_warm_import.argtypes = [vp, u64, i32, vp, vp, d]
        L.mdeos_warm_reset.argtypes = [vp]
        L.mdeos_hydro_config_default.argtypes = [P(mdeos_hydro_config)]
        L.mdeos_hydro_config_default.restype = None
        L.mdeos_hydro_create.argtypes = [vp, P(mdeos_hydro_config), vp, vp, vp, vp, P(vp)]
        L.mdeos_hydro_step.argtypes = [vp, i32]
        L.mdeos_hydro_state.argtypes = [vp] + [vp] * 8
        L.mdeos_hydro_eos_results.argtypes = [vp, vp]
        L.mdeos_hydro_destroy.argtypes = [vp]
        L.mdeos_serve_config_default.argtypes = [P(mdeos_serve_config)]
        L.mdeos_serve_config_default.restype = None
        L.mdeos_serve_create.argtypes = [vp, P(mdeos_serve_config), P(vp)]
        L.mdeos_serve_clock.argtypes = [vp]
        L.mdeos_serve_clock.restype = d
        L.mdeos_serve_enqueue.argtypes = [vp, vp, i32, vp]
        L.mdeos_serve_completed.argtypes = [vp, vp, i32, P(i32)]
        L.mdeos_serve_stats.argtypes = [vp, vp, vp]
        L.mdeos_serve_store_stats.argtypes = [vp, vp, vp]
        L.mdeos_serve_destroy.argtypes = [vp]
        L.mdeos_surrogate_create.argtypes = [vp, i32, i32, ctypes.c_uint64, P(vp)]
        L.mdeos_surrogate_set_params.argtypes = [vp, vp, vp]
        L.mdeos_surrogate_get_params.argtypes = [vp, vp, vp]
        L.mdeos_surrogate_grads.argtypes = [vp, vp, vp, i32, vp, P(d)]
        L.mdeos_surrogate_train.argtypes = [vp, vp, vp, i32, i32, i32, d, ctypes.c_uint64, i32, vp]
        L.mdeos_surrogate_predict.argtypes = [vp, vp, i32, vp, vp, vp]
        L.mdeos_surrogate_gated_eval.argtypes = [vp, vp, i32, d, i32, vp, vp]
        L.mdeos_surrogate_destroy.argtypes = [vp]
        L.mdeos_surrogate_set_infer_path.argtypes = [vp, i32]
        L.mdeos_surrogate_set_output_transform.argtypes = [vp, i32]
        L.mdeos_surrogate_fit_misfit.argtypes = [vp, vp, vp, i32, i32, i32]
        L.mdeos_surrogate_misfit.argtypes = [vp, vp, i32, vp]
        L.mdeos_surrogate_set_misfit_threshold.argtypes = [vp, d]
        L.mdeos_surrogate_infer_device.argtypes = [vp, vp, i32, vp, vp, vp]
        L.mdeos_autotune.argtypes = [vp, vp, i32, i32, vp, i32, P(i32)]
        i64 = ctypes.c_int64
        L.mdeos_debug_tanh.argtypes = [vp, vp, i32, vp]
        L.mdeos_debug_gemm_bf16.argtypes = [vp, vp, vp, i32, i32, i32, i64, i64, i64, i64, i64,
                                            i64, vp]
        for name in EXPORTED:
            fn = getattr(L, name)
            if name not in ("mdeos_config_default", "mdeos_last_error",
                            "mdeos_batch_device_results", "mdeos_hydro_config_default",
                            "mdeos_serve_config_default", "mdeos_serve_clock"):
                fn.restype = ctypes.c_int
        _lib = L
    return _lib


def mdeos_last_error() -> str:
    return lib().mdeos_last_error().decode()


def _check(st: int):
    if st != MDEOS_OK:
        raise MdeosError(st, mdeos_last_error())


def mdeos_config_default(**over) -> mdeos_config:
    c = mdeos_config()
    lib().mdeos_config_default(ctypes.byref(c))
    for k, v in over.items():
        setattr(c, k, v)
    return c


def mdeos_create(cfg: mdeos_config | None = None) -> ctypes.c_void_p:
    cfg = cfg or mdeos_config_default()
    h = ctypes.c_void_p()
    _check(lib().mdeos_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def mdeos_destroy(h) -> None:
    _check(lib().mdeos_destroy(h))


def as_requests(reqs) -> np.ndarray:
    """Structured request array (REQUEST_DTYPE) from a list of dicts or an array."""
    if isinstance(reqs, np.ndarray) and reqs.dtype == REQUEST_DTYPE:
        return np.ascontiguousarray(reqs)
    arr = np.zeros(len(reqs), dtype=REQUEST_DTYPE)
    for k, r in enumerate(reqs):
        for f in REQUEST_DTYPE.names:
            if f in r:
                arr[k][f] = r[f]
    return arr


def mdeos_submit(h, reqs) -> int:
    arr = as_requests(reqs)
    t = ctypes.c_uint64()
    _check(lib().mdeos_submit(h, arr.ctypes.data_as(ctypes.c_void_p), len(arr), ctypes.byref(t)))
    return t.value


def mdeos_poll(h, ticket: int, n: int, timeout_us: int = -1):
    """Results (RESULT_DTYPE array) or None while pending."""
    out = np.zeros(n, dtype=RESULT_DTYPE)
    st = lib().mdeos_poll(h, ticket, out.ctypes.data_as(ctypes.c_void_p), timeout_us)
    if st == MDEOS_PENDING:
        return None
    _check(st)
    return out


def mdeos_batch_create(h, reqs) -> ctypes.c_void_p:
    arr = as_requests(reqs)
    b = ctypes.c_void_p()
    _check(lib().mdeos_batch_create(h, arr.ctypes.data_as(ctypes.c_void_p), len(arr),
                                    ctypes.byref(b)))
    return b


def mdeos_batch_launch(b, stream: int | None = None) -> None:
    _check(lib().mdeos_batch_launch(b, ctypes.c_void_p(stream or 0)))


def mdeos_batch_device_results(b) -> int:
    return lib().mdeos_batch_device_results(b)


def mdeos_batch_results(b, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=RESULT_DTYPE)
    _check(lib().mdeos_batch_results(b, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def mdeos_batch_info(b) -> dict:
    ni, nc, sm = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    sc = ctypes.c_size_t()
    _check(lib().mdeos_batch_info(b, ctypes.byref(ni), ctypes.byref(nc), ctypes.byref(sm),
                                  ctypes.byref(sc)))
    return {"items": ni.value, "ctas": nc.value, "smem": sm.value, "scratch_bytes": sc.value}


def mdeos_batch_destroy(b) -> None:
    _check(lib().mdeos_batch_destroy(b))


def mdeos_stats(h) -> dict:
    a, b, d = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    c = ctypes.c_longlong()
    _check(lib().mdeos_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                             ctypes.byref(d)))
    return {"h2d": a.value, "d2h": b.value, "launches": c.value, "device_bytes": d.value}


def mdeos_submit_noalloc(reqs, d_results_ptr: int, cfg: mdeos_config | None = None,
                         stream: int | None = None) -> None:
    """Queue a batch without any device allocation by the library; results land in
    the caller's device array at d_results_ptr (n records) when the stream reaches it."""
    arr = as_requests(reqs)
    cfg = cfg or mdeos_config_default()
    _check(lib().mdeos_submit_noalloc(ctypes.byref(cfg), arr.ctypes.data_as(ctypes.c_void_p),
                                      len(arr), ctypes.c_void_p(d_results_ptr),
                                      ctypes.c_void_p(stream or 0)))


def _dptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _stream_ptr(stream) -> ctypes.c_void_p:
    return ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)


def mdeos_debug_lift(n: int, rho: float, T: float, seed: int, cfg: mdeos_config | None = None,
                     stream=None):
    """Device lifting of one box: (x4, v4 torch cuda float32 [n,4], E_cold, L)."""
    import torch
    cfg = cfg or mdeos_config_default()
    x4 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    v4 = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = ctypes.c_double()
    _check(lib().mdeos_debug_lift(ctypes.byref(cfg), n, rho, T, seed, _dptr(x4), _dptr(v4),
                                  _dptr(e), ctypes.byref(L), _stream_ptr(stream)))
    return x4, v4, float(e.item()), L.value


def mdeos_debug_forces(x4, L: float, path: int, skin: float = 0.3,
                       cfg: mdeos_config | None = None, stream=None):
    """Device forces on positions x4 (torch cuda float32 [n,4]): (f4, ew[7], pairs)."""
    import torch
    cfg = cfg or mdeos_config_default()
    n = x4.shape[0]
    f4 = torch.zeros_like(x4)
    ew = torch.zeros(7, dtype=torch.float64, device=x4.device)
    pc = torch.zeros(1, dtype=torch.int64, device=x4.device)
    _check(lib().mdeos_debug_forces(ctypes.byref(cfg), _dptr(x4), n, L, path, skin, _dptr(f4),
                                    _dptr(ew), _dptr(pc), _stream_ptr(stream)))
    return f4, ew, int(pc.item())


def mdeos_debug_md(x4, v4, L: float, steps: int, path: int, skin: float = 0.3,
                   T_target: float = 0.0, rescale_every: int = 0,
                   cfg: mdeos_config | None = None, stream=None, cycles=None):
    """Device velocity-Verlet on one box, in place; returns (epot[steps], ekin[steps]).
    `cycles`, if given, is a cuda int64 tensor of 11 receiving per-phase SM cycles."""
    import torch
    cfg = cfg or mdeos_config_default()
    n = x4.shape[0]
    ep = torch.zeros(max(steps, 1), dtype=torch.float64, device=x4.device)
    ek = torch.zeros(max(steps, 1), dtype=torch.float64, device=x4.device)
    _check(lib().mdeos_debug_md(ctypes.byref(cfg), _dptr(x4), _dptr(v4), n, L, steps, T_target,
                                rescale_every, path, skin, _dptr(ep), _dptr(ek),
                                _dptr(cycles) if cycles is not None else ctypes.c_void_p(0),
                                _stream_ptr(stream)))
    return ep[:steps], ek[:steps]


def mdeos_debug_force_bench(x4, L: float, skin: float, passes: int, mode: int = 0,
                            cfg: mdeos_config | None = None, stream=None):
    """Repeated force passes on resident boxes (x4: cuda float32 [nbox, n, 4]);
    returns a cuda int64 tensor [nbox, 2]: SM cycles of the passes, list entries."""
    import torch
    cfg = cfg or mdeos_config_default()
    nbox, n = x4.shape[0], x4.shape[1]
    cyc = torch.zeros((nbox, 2), dtype=torch.int64, device=x4.device)
    _check(lib().mdeos_debug_force_bench(ctypes.byref(cfg), _dptr(x4), nbox, n, L, skin, passes,
                                         mode, _dptr(cyc), _stream_ptr(stream)))
    return cyc


def mdeos_warm_export(h, element_id: int, natoms: int):
    """Stored final state of an element: (x4, v4 float32 [n,4] host arrays, L)."""
    x4 = np.zeros((natoms, 4), dtype=np.float32)
    v4 = np.zeros((natoms, 4), dtype=np.float32)
    L = ctypes.c_double()
    _check(lib().mdeos_warm_export(h, element_id, natoms, x4.ctypes.data_as(ctypes.c_void_p),
                                   v4.ctypes.data_as(ctypes.c_void_p), ctypes.byref(L)))
    return x4, v4, L.value


def mdeos_warm_import(h, element_id: int, x, v, L: float) -> None:
    """Store a state (positions x and velocities v, [n,3] or [n,4]) for an element."""
    n = len(x)
    x4 = np.zeros((n, 4), dtype=np.float32)
    v4 = np.zeros((n, 4), dtype=np.float32)
    x4[:, :3] = np.asarray(x)[:, :3]
    v4[:, :3] = np.asarray(v)[:, :3]
    _check(lib().mdeos_warm_import(h, element_id, n, x4.ctypes.data_as(ctypes.c_void_p),
                                   v4.ctypes.data_as(ctypes.c_void_p), float(L)))


def mdeos_warm_reset(h) -> None:
    _check(lib().mdeos_warm_reset(h))


def mdeos_hydro_config_default(**over) -> mdeos_hydro_config:
    c = mdeos_hydro_config()
    lib().mdeos_hydro_config_default(ctypes.byref(c))
    for k, v in over.items():
        setattr(c, k, v)
    return c


def _f8(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (n,):
        raise ValueError(f"expected {n} values, got shape {a.shape}")
    return a


class Hydro:
    """1D Lagrangian hydro on the GPU (mdeos_hydro_*); the handle must outlive it."""

    def __init__(self, h, cfg: mdeos_hydro_config, x, u, rho, e0):
        nz = cfg.nzones
        self.nz = nz
        self.cfg = cfg
        self._keep = [_f8(x, nz + 1), _f8(u, nz + 1), _f8(rho, nz), _f8(e0, nz)]
        self.hy = ctypes.c_void_p()
        vp = [a.ctypes.data_as(ctypes.c_void_p) for a in self._keep]
        _check(lib().mdeos_hydro_create(h, ctypes.byref(cfg), *vp, ctypes.byref(self.hy)))

    def step(self, nsteps: int = 1) -> None:
        _check(lib().mdeos_hydro_step(self.hy, nsteps))

    def state(self) -> dict:
        nz = self.nz
        out = {k: np.zeros(nz + 1) for k in ("x", "u")}
        out.update({k: np.zeros(nz) for k in ("rho", "e", "P", "q", "c2")})
        clock = np.zeros(3)
        ptrs = [out[k].ctypes.data_as(ctypes.c_void_p) for k in ("x", "u", "rho", "e", "P", "q", "c2")]
        _check(lib().mdeos_hydro_state(self.hy, *ptrs, clock.ctypes.data_as(ctypes.c_void_p)))
        out["t"], out["dt"], out["steps"] = clock[0], clock[1], int(clock[2])
        return out

    def eos_results(self) -> np.ndarray:
        out = np.zeros(self.nz, dtype=RESULT_DTYPE)
        _check(lib().mdeos_hydro_eos_results(self.hy, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def close(self):
        if self.hy:
            lib().mdeos_hydro_destroy(self.hy)
            self.hy = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def mdeos_serve_config_default(**over) -> mdeos_serve_config:
    c = mdeos_serve_config()
    lib().mdeos_serve_config_default(ctypes.byref(c))
    for k, v in over.items():
        setattr(c, k, v)
    return c


class Server:
    """Continuous-batching server on a handle (mdeos_serve_*); the handle must outlive it."""

    def __init__(self, h, cfg: mdeos_serve_config | None = None, **over):
        self.cfg = cfg or mdeos_serve_config_default(**over)
        self.s = ctypes.c_void_p()
        _check(lib().mdeos_serve_create(h, ctypes.byref(self.cfg), ctypes.byref(self.s)))

    def clock(self) -> float:
        return lib().mdeos_serve_clock(self.s)

    def enqueue(self, reqs) -> np.ndarray:
        arr = as_requests(reqs)
        ids = np.zeros(len(arr), dtype=np.uint64)
        _check(lib().mdeos_serve_enqueue(self.s, arr.ctypes.data_as(ctypes.c_void_p), len(arr),
                                         ids.ctypes.data_as(ctypes.c_void_p)))
        return ids

    def completed(self, max_n: int = 4096) -> np.ndarray:
        out = np.empty(max_n, dtype=SERVED_DTYPE)
        k = ctypes.c_int32()
        _check(lib().mdeos_serve_completed(self.s, out.ctypes.data_as(ctypes.c_void_p), max_n,
                                           ctypes.byref(k)))
        return out[:k.value]

    def stats(self) -> dict:
        c = np.zeros(7, dtype=np.int64)
        b = np.zeros(2, dtype=np.uint64)
        _check(lib().mdeos_serve_stats(self.s, c.ctypes.data_as(ctypes.c_void_p),
                                       b.ctypes.data_as(ctypes.c_void_p)))
        keys = ("enqueued", "admitted", "finished", "shed", "launches", "waiting", "cuda_errors")
        d = {k: int(v) for k, v in zip(keys, c)}
        d["device_bytes"], d["peak_inflight"] = int(b[0]), int(b[1])
        return d

    def store_stats(self) -> dict:
        c = np.zeros(4, dtype=np.int64)
        b = np.zeros(2, dtype=np.uint64)
        _check(lib().mdeos_serve_store_stats(self.s, c.ctypes.data_as(ctypes.c_void_p),
                                             b.ctypes.data_as(ctypes.c_void_p)))
        keys = ("warm_starts", "memory_waits", "evictions", "stored")
        d = {k: int(v) for k, v in zip(keys, c)}
        d["store_used_bytes"], d["store_bytes"] = int(b[0]), int(b[1])
        return d

    def wait_all(self, n_expected: int, timeout_s: float = 600.0) -> np.ndarray:
        """Collect completions until n_expected have arrived (or the timeout)."""
        import time
        got = []
        t0 = time.time()
        total = 0
        while total < n_expected and time.time() - t0 < timeout_s:
            c = self.completed()
            if len(c):
                got.append(c)
                total += len(c)
            else:
                time.sleep(0.0005)
        return np.concatenate(got) if got else np.zeros(0, dtype=SERVED_DTYPE)

    def close(self):
        if self.s:
            lib().mdeos_serve_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def mdeos_autotune(h, reqs, steps: int = 200) -> np.ndarray:
    """Measure the best launch shape (Verlet skin, warps per box) per atom count on
    this GPU and keep it in the handle; returns rows (natoms, skin, warps, ms of GPU
    time per box)."""
    arr = as_requests(reqs)
    tab = np.zeros((64, 4))
    k = ctypes.c_int32()
    _check(lib().mdeos_autotune(h, arr.ctypes.data_as(ctypes.c_void_p), len(arr), steps,
                                tab.ctypes.data_as(ctypes.c_void_p), 64, ctypes.byref(k)))
    return tab[:k.value]


def _vp(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Surrogate:
    """MLP-ensemble surrogate EOS on a handle (mdeos_surrogate_*)."""

    def __init__(self, h, n_models: int = 4, max_batch: int = 4096, seed: int = 1):
        self.E = n_models
        self.s = ctypes.c_void_p()
        _check(lib().mdeos_surrogate_create(h, n_models, max_batch, seed, ctypes.byref(self.s)))

    def set_params(self, params=None, norm=None):
        p = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        nm = None if norm is None else np.ascontiguousarray(norm, dtype=np.float64)
        _check(lib().mdeos_surrogate_set_params(self.s, _vp(p), _vp(nm)))

    def get_params(self):
        p = np.zeros((self.E, SURROGATE_NPARAM), dtype=np.float32)
        nm = np.zeros(8)
        _check(lib().mdeos_surrogate_get_params(self.s, _vp(p), _vp(nm)))
        return p, nm

    def grads(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        g = np.zeros((self.E, SURROGATE_NPARAM), dtype=np.float32)
        loss = ctypes.c_double()
        _check(lib().mdeos_surrogate_grads(self.s, _vp(x), _vp(y), len(x), _vp(g),
                                           ctypes.byref(loss)))
        return g, loss.value

    def train(self, x, y, epochs, batch=1024, lr=1e-3, seed=0, set_norm=True):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        out = np.zeros(max(epochs, 1))
        _check(lib().mdeos_surrogate_train(self.s, _vp(x), _vp(y), len(x), epochs, batch, lr,
                                           seed, int(set_norm), _vp(out)))
        return out[:epochs]

    def predict(self, x, per_model=False):
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = len(x)
        mean = np.zeros((n, 2))
        sd = np.zeros((n, 2))
        pm = np.zeros((self.E, n, 2), dtype=np.float32) if per_model else None
        _check(lib().mdeos_surrogate_predict(self.s, _vp(x), n, _vp(mean), _vp(sd), _vp(pm)))
        return (mean, sd, pm) if per_model else (mean, sd)

    def set_output_transform(self, mode: int):
        """SURROGATE_P_LINEAR (default) or SURROGATE_P_ASINH (learn asinh(P))."""
        _check(lib().mdeos_surrogate_set_output_transform(self.s, mode))

    def fit_misfit(self, x, y, bins: int = 32, min_count: int = 8):
        """Misfit map of the gate from MD answers y (n, 2) = (P, T) at inputs x (n, 2)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        _check(lib().mdeos_surrogate_fit_misfit(self.s, _vp(x), _vp(y), len(x), bins, min_count))

    def misfit(self, x):
        """The misfit map at inputs x (n, 2): RMS relative P residual of the cell."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros(len(x))
        _check(lib().mdeos_surrogate_misfit(self.s, _vp(x), len(x), _vp(out)))
        return out

    def set_misfit_threshold(self, threshold: float):
        """Gate also on the misfit map (math.inf: not used)."""
        _check(lib().mdeos_surrogate_set_misfit_threshold(self.s, float(threshold)))

    def set_infer_path(self, path: int):
        """SURROGATE_INFER_TC (fused tcgen05 kernel, default) or SURROGATE_INFER_MMA (the
        layered path of the training step)."""
        _check(lib().mdeos_surrogate_set_infer_path(self.s, path))

    def infer_device(self, x, mean, sd, stream=None):
        """Asynchronous prediction on device tensors: x (n, 2) float64 (rho, e) in;
        mean and sd (n, 2) float64 out; on `stream` (torch.cuda.Stream) or the handle's."""
        import torch
        for t in (x, mean, sd):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                    and tuple(t.shape) == (x.shape[0], 2)):
                raise ValueError("infer_device wants contiguous (n, 2) float64 CUDA tensors")
        _check(lib().mdeos_surrogate_infer_device(self.s, _dptr(x), x.shape[0], _dptr(mean),
                                                  _dptr(sd), _stream_ptr(stream)))

    def gated_eval(self, reqs, threshold, md_natoms=0):
        arr = as_requests(reqs)
        out = np.zeros(len(arr), dtype=RESULT_DTYPE)
        used = np.zeros(len(arr), dtype=np.int32)
        _check(lib().mdeos_surrogate_gated_eval(self.s, _vp(arr), len(arr), threshold, md_natoms,
                                                _vp(out), _vp(used)))
        return out, used

    def close(self):
        if self.s:
            lib().mdeos_surrogate_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def mdeos_debug_gemm_bf16(A_bits, B_bits, M, N, K, sa, sb, sc, stream=None):
    """C = A B on the tensor-core GEMM; A_bits/B_bits: torch cuda int16 tensors of
    bfloat16 bit patterns, strides (sa_m, sa_k), (sb_k, sb_n), (sc_m, sc_n).  Returns
    the flat output buffer (element (m, n) at m * sc_m + n * sc_n)."""
    import torch
    C = torch.zeros((M - 1) * sc[0] + (N - 1) * sc[1] + 1, dtype=torch.float32, device="cuda")
    _check(lib().mdeos_debug_gemm_bf16(_dptr(A_bits), _dptr(B_bits), _dptr(C), M, N, K, sa[0],
                                       sa[1], sb[0], sb[1], sc[0], sc[1], _stream_ptr(stream)))
    return C


def mdeos_debug_tanh(x, stream=None):
    """The surrogate's hidden-layer tanh on a torch cuda float32 tensor."""
    import torch
    x = x.contiguous()
    y = torch.empty_like(x)
    _check(lib().mdeos_debug_tanh(_dptr(x), _dptr(y), x.numel(), _stream_ptr(stream)))
    return y


def e_from_temperature(T, natoms):
    """Specific energy whose first lifting temperature (Eq. 9) is T: e = N_DOF T / (2N)."""
    return (3.0 * natoms - 3.0) * T / (2.0 * natoms)


class Engine:
    """Convenience wrapper: one handle, synchronous evaluate()."""

    def __init__(self, **cfg):
        self.cfg = mdeos_config_default(**cfg)
        self.h = mdeos_create(self.cfg)

    def evaluate(self, reqs, timeout_us: int = -1) -> np.ndarray:
        arr = as_requests(reqs)
        t = mdeos_submit(self.h, arr)
        return mdeos_poll(self.h, t, len(arr), timeout_us)

    def close(self):
        if self.h:
            mdeos_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
