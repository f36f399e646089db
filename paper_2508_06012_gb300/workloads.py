"""Seeded synthetic inputs shaped like the paper's EOS workloads.

Only input generation lives here (densities, temperatures, atom counts, per-box
seeds); none of the method's arithmetic.  Both the CUDA path and the CPU oracle are
fed from these generators.

The paper's own workloads (Mishin-EAM copper, an ML hydrogen potential, LEOS tables)
are not available, so Lennard-Jones boxes in reduced units stand in for them, with
the paper's shape: O(10^3) atoms per box (Sec. VI), one independent box per element
and call (Sec. III), an equilibrate-then-average schedule (App. B).
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser: decorrelated 64-bit per-box seeds from (base, index)."""
    x = (x + 0x9E3779B97F4A7C15) & MASK64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & MASK64
    return x ^ (x >> 31)


def box_seed(base: int, index: int) -> int:
    return splitmix64((base * 0x100000001B3 + index) & MASK64)


def small_queries(base_seed: int = 20250806, nbox: int = 16):
    """16 independent queries: N = 256 (FCC 4x4x4), rho* ~ U[0.5, 1.0],
    T* ~ U[1.0, 2.0], 1000 equilibration + 1000 averaging steps."""
    rng = np.random.default_rng(base_seed)
    rho = rng.uniform(0.5, 1.0, nbox)
    T = rng.uniform(1.0, 2.0, nbox)
    return [dict(rho=float(rho[k]), T=float(T[k]), natoms=256, steps_equil=1000,
                 steps_avg=1000, seed=box_seed(base_seed, k), element_id=k)
            for k in range(nbox)]


def uneven_batch(base_seed: int = 20250807, nbox: int = 4096, steps_equil: int = 1000,
            steps_avg: int = 1000):
    """Batched uneven EOS: N = 4 n^3 with n ~ U{3..10} (108..4000 atoms),
    rho* ~ U[0.3, 1.2], T* log-uniform on [0.7, 3.0], 2000 steps."""
    rng = np.random.default_rng(base_seed)
    ncell = rng.integers(3, 11, nbox)
    rho = rng.uniform(0.3, 1.2, nbox)
    T = np.exp(rng.uniform(np.log(0.7), np.log(3.0), nbox))
    return [dict(rho=float(rho[k]), T=float(T[k]), natoms=int(4 * ncell[k] ** 3),
                 steps_equil=steps_equil, steps_avg=steps_avg, seed=box_seed(base_seed, k),
                 element_id=k)
            for k in range(nbox)]


def stratified(reqs, per_class: int, steps_equil: int, steps_avg: int):
    """A bounded sample of a workload: the first `per_class` boxes of every atom
    count, with a shortened step schedule (the per-step cost is unchanged)."""
    seen: dict[int, int] = {}
    out = []
    for r in reqs:
        c = seen.get(r["natoms"], 0)
        if c < per_class:
            seen[r["natoms"]] = c + 1
            q = dict(r)
            q["steps_equil"] = steps_equil
            q["steps_avg"] = steps_avg
            out.append(q)
    return out


def random_boxes(seed: int, nbox: int, nmin: int, nmax: int, rho=(0.3, 1.2), T=(0.7, 3.0),
                 steps_equil: int = 200, steps_avg: int = 200):
    """Ragged atom counts (any N, partial FCC lattices) for edge-case tests."""
    rng = np.random.default_rng(seed)
    n = rng.integers(nmin, nmax + 1, nbox)
    r = rng.uniform(rho[0], rho[1], nbox)
    t = np.exp(rng.uniform(np.log(T[0]), np.log(T[1]), nbox))
    return [dict(rho=float(r[k]), T=float(t[k]), natoms=int(n[k]), steps_equil=steps_equil,
                 steps_avg=steps_avg, seed=box_seed(seed, k), element_id=k)
            for k in range(nbox)]


def serving_stream(base_seed: int = 20250809, nreq: int = 1000, steps_equil: int = 1000,
            steps_avg: int = 1000):
    """EOS serving stream: atom counts log-uniform on [256, 32000], rho* ~ U[0.3, 1.2],
    T* log-uniform on [0.7, 3.0] (the 1000 + 1000-step schedule of the uneven batch)."""
    rng = np.random.default_rng(base_seed)
    n = np.exp(rng.uniform(np.log(256.0), np.log(32000.0), nreq)).astype(np.int64)
    rho = rng.uniform(0.3, 1.2, nreq)
    T = np.exp(rng.uniform(np.log(0.7), np.log(3.0), nreq))
    return [dict(rho=float(rho[k]), T=float(T[k]), natoms=int(n[k]), steps_equil=steps_equil,
                 steps_avg=steps_avg, seed=box_seed(base_seed, k), element_id=0)
            for k in range(nreq)]


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream of the given mean rate."""
    rng = np.random.default_rng(seed)
    n = rng.poisson(rate * duration)
    return np.sort(rng.uniform(0.0, duration, n))
