"""FP64 CPU oracle of the in-line atomistic EOS evaluation (arXiv 2508.06012, Sec. III).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this package.  It shares no code
with the CUDA path (``paper_2508_06012_gb300``) and never imports it.

The numerical core is plain C (``mdeos_oracle.c``) compiled by :func:`build`; this file
is argument marshalling over ctypes.  ``oracle.hydro`` holds the 1D Lagrangian hydro
reference and the analytic EOS forms (Eq. 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdeos_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

OK, EINVAL, EUNPHYS, EBOX = 0, -1, -3, -4
REF_ECOLD, REF_FIXED = 0, 1
FORCE_ALLPAIRS, FORCE_CELL = 0, 1
REQ_TEMPERATURE = 1


class Params(ctypes.Structure):
    _fields_ = [
        ("eps", ctypes.c_double), ("sigma", ctypes.c_double), ("mass", ctypes.c_double),
        ("rc", ctypes.c_double), ("dt", ctypes.c_double),
        ("lift_iters", ctypes.c_int), ("rescale_every_equil", ctypes.c_int),
        ("rescale_every_avg", ctypes.c_int), ("se_blocks", ctypes.c_int),
        ("energy_ref_mode", ctypes.c_int), ("force_mode", ctypes.c_int),
        ("warm_lift_iters", ctypes.c_int),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("rho", ctypes.c_double), ("e", ctypes.c_double), ("e_ref", ctypes.c_double),
        ("natoms", ctypes.c_int), ("steps_equil", ctypes.c_int), ("steps_avg", ctypes.c_int),
        ("flags", ctypes.c_uint32), ("seed", ctypes.c_uint64),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("P", ctypes.c_double), ("T", ctypes.c_double), ("sigma", ctypes.c_double * 6),
        ("epot", ctypes.c_double), ("ekin", ctypes.c_double), ("e_achieved", ctypes.c_double),
        ("P_se", ctypes.c_double), ("T_se", ctypes.c_double), ("T_target", ctypes.c_double),
        ("e_cold", ctypes.c_double), ("L", ctypes.c_double), ("status", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                               os.path.getmtime(_SRC[:-2] + ".h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        _lib.orc_philox4x32_10.argtypes = [p, p, p]
        _lib.orc_lattice_fcc.argtypes = [i, d, p, p]
        _lib.orc_lattice_fcc.restype = i
        _lib.orc_init_velocities.argtypes = [i, ctypes.c_uint64, d, d, p]
        _lib.orc_lj_forces.argtypes = [i, p, d, ctypes.POINTER(Params), i, p, p]
        _lib.orc_lj_forces.restype = d
        _lib.orc_count_pairs.argtypes = [i, p, d, d]
        _lib.orc_count_pairs.restype = ctypes.c_longlong
        _lib.orc_md_steps.argtypes = [i, p, p, p, d, ctypes.POINTER(Params), i, d, i, p, p]
        _lib.orc_md_steps.restype = i
        _lib.orc_kinetic.argtypes = [i, p, d]
        _lib.orc_kinetic.restype = d
        _lib.orc_eos_eval.argtypes = [ctypes.POINTER(Request), ctypes.POINTER(Params),
                                      ctypes.POINTER(Result)]
        _lib.orc_eos_eval.restype = i
        _lib.orc_eos_batch.argtypes = [p, i, ctypes.POINTER(Params), p, i]
        _lib.orc_eos_batch.restype = i
        _lib.orc_max_threads.restype = i
        _lib.orc_eos_eval_state.argtypes = [ctypes.POINTER(Request), ctypes.POINTER(Params),
                                            p, p, d, p, p, ctypes.POINTER(Result)]
        _lib.orc_eos_eval_state.restype = i
        _lib.orc_eos_batch_state.argtypes = [p, i, ctypes.POINTER(Params), p, p, p, p, p, p, i]
        _lib.orc_eos_batch_state.restype = i
        _lib.orc_block_se.argtypes = [p, i, i, p, p]
        _lib.orc_block_se.restype = i
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_params(eps=1.0, sigma=1.0, mass=1.0, rc=2.5, dt=0.005, lift_iters=2,
                rescale_every_equil=0, rescale_every_avg=10, se_blocks=10,
                energy_ref_mode=REF_ECOLD, force_mode=FORCE_ALLPAIRS,
                warm_lift_iters=1) -> Params:
    return Params(eps, sigma, mass, rc, dt, lift_iters, rescale_every_equil,
                  rescale_every_avg, se_blocks, energy_ref_mode, force_mode, warm_lift_iters)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def lattice_fcc(n: int, rho: float):
    x = np.zeros((n, 3), dtype=np.float64)
    L = ctypes.c_double(0.0)
    st = lib().orc_lattice_fcc(n, rho, _ptr(x), ctypes.byref(L))
    if st != OK:
        raise ValueError(f"lattice_fcc status {st}")
    return x, L.value


def init_velocities(n: int, seed: int, T: float, mass: float = 1.0) -> np.ndarray:
    v = np.zeros((n, 3), dtype=np.float64)
    lib().orc_init_velocities(n, seed, T, mass, _ptr(v))
    return v


def lj_forces(x: np.ndarray, L: float, params: Params | None = None, mode: int = FORCE_ALLPAIRS):
    """Return (E_pot, forces (n,3), W[6] = sum_{i<j} r_ij (x) f_ij)."""
    params = params or make_params()
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    f = np.zeros((n, 3), dtype=np.float64)
    W = np.zeros(6, dtype=np.float64)
    E = lib().orc_lj_forces(n, _ptr(x), L, ctypes.byref(params), mode, _ptr(f), _ptr(W))
    return E, f, W


def block_se(x, nblocks: int):
    """Block-average (mean, standard error) of a series, the restriction's error bar."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    mean, se = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib().orc_block_se(_ptr(x), x.shape[0], nblocks, ctypes.byref(mean), ctypes.byref(se))
    if st != 0:
        raise ValueError("orc_block_se: invalid series or block count")
    return mean.value, se.value


def count_pairs(x: np.ndarray, L: float, rc: float = 2.5) -> int:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return int(lib().orc_count_pairs(x.shape[0], _ptr(x), L, rc))


def kinetic(v: np.ndarray, mass: float = 1.0) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return lib().orc_kinetic(v.shape[0], _ptr(v), mass)


def md_steps(x, v, L, steps, params: Params | None = None, T_target=0.0, rescale_every=0):
    """Velocity-Verlet from (x, v); returns (x, v, f, epot[steps], ekin[steps])."""
    params = params or make_params()
    x = np.ascontiguousarray(x, dtype=np.float64).copy()
    v = np.ascontiguousarray(v, dtype=np.float64).copy()
    n = x.shape[0]
    f = np.zeros((n, 3))
    W = np.zeros(6)
    lib().orc_lj_forces(n, _ptr(x), L, ctypes.byref(params), params.force_mode, _ptr(f), _ptr(W))
    ep = np.zeros(max(steps, 1))
    ek = np.zeros(max(steps, 1))
    lib().orc_md_steps(n, _ptr(x), _ptr(v), _ptr(f), L, ctypes.byref(params), steps, T_target,
                       rescale_every, _ptr(ep), _ptr(ek))
    return x, v, f, ep[:steps], ek[:steps]


RESULT_FIELDS = ("P", "T", "epot", "ekin", "e_achieved", "P_se", "T_se", "T_target",
                 "e_cold", "L", "status")


def _result_dict(r: Result) -> dict:
    d = {k: getattr(r, k) for k in RESULT_FIELDS}
    d["sigma"] = list(r.sigma)
    return d


def eos_eval(rho, e, natoms, steps_equil, steps_avg, seed, params: Params | None = None,
             e_ref=0.0, flags=0) -> dict:
    params = params or make_params()
    rq = Request(rho, e, e_ref, natoms, steps_equil, steps_avg, flags, seed)
    out = Result()
    lib().orc_eos_eval(ctypes.byref(rq), ctypes.byref(params), ctypes.byref(out))
    return _result_dict(out)


def eos_batch(reqs: list[dict], params: Params | None = None, nthreads: int = 0) -> list[dict]:
    """reqs: dicts with rho, e, natoms, steps_equil, steps_avg, seed[, e_ref, flags]."""
    params = params or make_params()
    n = len(reqs)
    arr = (Request * n)()
    for k, r in enumerate(reqs):
        arr[k] = Request(r["rho"], r["e"], r.get("e_ref", 0.0), r["natoms"], r["steps_equil"],
                         r["steps_avg"], r.get("flags", 0), r["seed"])
    out = (Result * n)()
    lib().orc_eos_batch(ctypes.cast(arr, ctypes.c_void_p), n, ctypes.byref(params),
                        ctypes.cast(out, ctypes.c_void_p), nthreads)
    return [_result_dict(out[k]) for k in range(n)]


def _req_array(reqs):
    arr = (Request * len(reqs))()
    for k, r in enumerate(reqs):
        arr[k] = Request(r["rho"], r["e"], r.get("e_ref", 0.0), r["natoms"], r["steps_equil"],
                         r["steps_avg"], r.get("flags", 0), r.get("seed", 0))
    return arr


def eos_eval_state(req: dict, params: Params | None = None, x_in=None, v_in=None, L_in=0.0):
    """One evaluation with an optional warm start from (x_in, v_in, L_in).

    Returns (result dict, x_out (n,3), v_out (n,3)); x_out/v_out is the final
    state (None if the evaluation failed)."""
    params = params or make_params()
    n = req["natoms"]
    rq = _req_array([req])
    out = Result()
    xo = np.zeros((n, 3))
    vo = np.zeros((n, 3))
    if x_in is not None:
        xi = np.ascontiguousarray(x_in, dtype=np.float64).reshape(n, 3)
        vi = np.ascontiguousarray(v_in, dtype=np.float64).reshape(n, 3)
        px, pv = _ptr(xi), _ptr(vi)
    else:
        px = pv = None
        L_in = 0.0
    lib().orc_eos_eval_state(rq, ctypes.byref(params), px, pv, float(L_in), _ptr(xo), _ptr(vo),
                             ctypes.byref(out))
    d = _result_dict(out)
    if d["status"] != OK:
        return d, None, None
    return d, xo, vo


def eos_batch_state(reqs: list[dict], params: Params | None = None, x_in=None, v_in=None,
                    L_in=None, nthreads: int = 0):
    """Batch of equal-size requests with per-request warm starts.

    x_in, v_in: (nreq, natoms, 3) or None; L_in: (nreq,) with <= 0 meaning cold.
    Returns (list of result dicts, x_out, v_out) with the final states."""
    params = params or make_params()
    nr = len(reqs)
    n = reqs[0]["natoms"]
    assert all(r["natoms"] == n for r in reqs)
    rq = _req_array(reqs)
    out = (Result * nr)()
    xo = np.zeros((nr, n, 3))
    vo = np.zeros((nr, n, 3))
    if x_in is not None:
        xi = np.ascontiguousarray(x_in, dtype=np.float64).reshape(nr, n, 3)
        vi = np.ascontiguousarray(v_in, dtype=np.float64).reshape(nr, n, 3)
        li = np.ascontiguousarray(L_in, dtype=np.float64).reshape(nr)
        px, pv, pl = _ptr(xi), _ptr(vi), _ptr(li)
    else:
        px = pv = pl = None
    lib().orc_eos_batch_state(ctypes.cast(rq, ctypes.c_void_p), nr, ctypes.byref(params), px, pv,
                              pl, _ptr(xo), _ptr(vo), ctypes.cast(out, ctypes.c_void_p), nthreads)
    return [_result_dict(out[k]) for k in range(nr)], xo, vo


def max_threads() -> int:
    return int(lib().orc_max_threads())


def e_from_temperature(T: float, natoms: int) -> float:
    """Specific energy that makes the first lifting temperature (Eq. 9) equal T."""
    return (3.0 * natoms - 3.0) * T / (2.0 * natoms)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
