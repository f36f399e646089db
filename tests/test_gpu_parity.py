"""GPU parity of the single-box kernels against the FP64 oracle, element by element
on identical inputs, through the C ABI.

Tolerances (FP32 pair arithmetic against FP64; the largest forces and the
per-thread FP32 partial sums set the scale):
  forces     ||F_gpu - F_ref||_2 / ||F_ref||_2 <= 1e-5; per atom
             |dF_i| <= 1e-5 max(|F_ref,i|, F_rms) + 16 u sum_j |f_ij|
                       + 2 u L sum_j |df_ij/dr|   (u = 2^-24)
  energy     |E_gpu - E_ref| <= 1e-6 |E_ref| + 1e-5 N
  virial     |W_gpu - W_ref| <= 2e-5 max|W_ref| + 1e-4 N
  trajectory max |r_gpu - r_ref| <= 1e-4 sigma after 100 steps from one state
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

RC = 2.5


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06012_gb300 as m
    m.build()
    return m


def _f32_box(orc, n, rho, seed, T=1.5, steps=150):
    """A liquid-like configuration from a short oracle run, rounded to float32,
    and a float32-representable box side (both sides see identical inputs)."""
    x, L = orc.lattice_fcc(n, rho)
    v = orc.init_velocities(n, seed, T)
    x, v, _, _, _ = orc.md_steps(x, v, L, steps, orc.make_params(force_mode=1 if L > 7.5 else 0),
                                 T_target=T, rescale_every=10)
    L32 = float(np.float32(L))
    x32 = np.mod(x.astype(np.float32), np.float32(L32)).astype(np.float32)
    return x32, L32, v


def _to_dev(x32):
    import torch
    x4 = np.zeros((len(x32), 4), dtype=np.float32)
    x4[:, :3] = x32
    return torch.from_numpy(x4).cuda()


def _force_err(f_gpu, f_ref):
    """Relative force error ||F_gpu - F_ref||_2 / ||F_ref||_2 over all atoms."""
    return np.linalg.norm(f_gpu - f_ref) / np.linalg.norm(f_ref)


def _force_err_atom(f_gpu, f_ref):
    """Worst atom: |dF_i| / max(|F_i|, F_rms)."""
    fnorm = np.linalg.norm(f_ref, axis=1)
    frms = np.sqrt((fnorm ** 2).mean())
    return (np.linalg.norm(f_gpu - f_ref, axis=1) / np.maximum(fnorm, frms)).max()


def _pair_force_sums(x, L):
    """Per atom, sum_j |f_ij| and sum_j |df_ij/dr| (minimum image, r < rc): the
    scales of the FP32 rounding in an atom's force."""
    x = np.asarray(x, dtype=np.float64)
    sf, sd = np.zeros(len(x)), np.zeros(len(x))
    for i0 in range(0, len(x), 512):
        d = x[i0:i0 + 512, None, :] - x[None, :, :]
        d -= L * np.round(d / L)
        r2 = (d ** 2).sum(-1)
        with np.errstate(divide="ignore", invalid="ignore"):
            ir = 1.0 / np.sqrt(r2)
            f = np.abs(24.0 * (2.0 * ir ** 13 - ir ** 7))
            df = np.abs(24.0 * (-26.0 * ir ** 14 + 7.0 * ir ** 8))
        out = (r2 >= RC * RC) | (r2 == 0.0)
        f[out] = 0.0
        df[out] = 0.0
        sf[i0:i0 + 512] = f.sum(1)
        sd[i0:i0 + 512] = df.sum(1)
    return sf, sd


def _fp32_atom_bound(x, L, f_ref):
    """Per-atom bound on the FP32 force error: 1e-5 max(|F_i|, F_rms), plus 16 unit
    roundoffs u = 2^-24 of sum_j |f_ij| (each pair term carries ~10 roundings -- r^2,
    the reciprocal, r^-6, the force factor -- and the list sum one more per term),
    plus the rounding of the position difference itself, u L per axis for a pair
    across the periodic boundary, times sum_j |df_ij/dr|.  Where the pair forces
    cancel to a small net force the last two terms dominate."""
    fnorm = np.linalg.norm(f_ref, axis=1)
    frms = np.sqrt((fnorm ** 2).mean())
    sf, sd = _pair_force_sums(x, L)
    u = 2.0 ** -24
    return 1e-5 * np.maximum(fnorm, frms) + 16.0 * u * sf + 2.0 * u * L * sd


def _ambiguous_pairs(x, L, rel=2e-6):
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    r2 = (d.astype(np.float64) ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    return int((np.abs(r2 - RC * RC) < rel * RC * RC).sum())


CASES = [
    # n, rho, path, seed
    (108, 0.35, 0, 1),     # all-pairs, minimum image (L = 6.7)
    (256, 0.8, 0, 2),
    (108, 1.15, 1, 3),     # all-pairs over two images per axis (L = 4.5 < 2 rc)
    (64, 0.9, 1, 4),
    (500, 0.9, 2, 5),      # Verlet list, brute-force build (L = 8.2 < 3 (rc + skin)), 1 thread per atom
    (256, 0.85, 2, 8),     # brute-force build, 4 threads per atom
    (384, 0.7, 2, 9),      # largest box with 4 threads per atom
    (385, 0.7, 2, 10),     # smallest with 1
    (2048, 1.1, 2, 6),     # Verlet list from the shared-memory cell list
    (4000, 0.3, 2, 7),     # largest box of the uneven batch, dilute
    (4000, 1.2, 2, 8),     # largest box of the uneven batch, dense
    (1111, 0.7, 2, 9),     # ragged: partial lattice, several ragged warps
    (4096, 0.85, 2, 10),   # maximum atoms per box
]


@pytest.mark.parametrize("n,rho,path,seed", CASES)
def test_forces_energy_virial_match_oracle(m, orc, n, rho, path, seed):
    x32, L, _ = _f32_box(orc, n, rho, seed)
    E, f, W = orc.lj_forces(x32.astype(np.float64), L)
    f4, ew, pairs = m.mdeos_debug_forces(_to_dev(x32), L, path, skin=0.3)
    fg = f4.cpu().numpy()[:, :3].astype(np.float64)
    ew = ew.cpu().numpy()
    assert np.isfinite(ew).all()
    assert _force_err(fg, f) <= 1e-5
    ea = _force_err_atom(fg, f)
    err = np.linalg.norm(fg - f, axis=1)
    bound = _fp32_atom_bound(x32, L, f)
    print(f"per-atom force error n={n} rho={rho} path={path}: {ea:.3e} of max(|F_i|, F_rms), "
          f"{(err / bound).max():.3f} of the FP32 bound")
    assert (err <= bound).all(), (err / bound).max()
    assert abs(ew[0] - E) <= 1e-6 * abs(E) + 1e-5 * n
    assert np.abs(ew[1:] - W).max() <= 2e-5 * np.abs(W).max() + 1e-4 * n
    # in-cutoff ordered pair count: exact except pairs within FP32 rounding of rc
    ref = orc.count_pairs(x32.astype(np.float64), L, RC)
    assert abs(pairs - ref) <= _ambiguous_pairs(x32.astype(np.float64), L)


def test_force_paths_agree_on_one_box(m, orc):
    """The three force paths of one kernel family give the same forces where
    their domains overlap (L >= 2 (rc + skin))."""
    x32, L, _ = _f32_box(orc, 864, 0.6, 11)
    fa = m.mdeos_debug_forces(_to_dev(x32), L, 0)[0].cpu().numpy()[:, :3]
    fm = m.mdeos_debug_forces(_to_dev(x32), L, 1)[0].cpu().numpy()[:, :3]
    fn = m.mdeos_debug_forces(_to_dev(x32), L, 2, skin=0.4)[0].cpu().numpy()[:, :3]
    assert _force_err(fm.astype(np.float64), fa.astype(np.float64)) <= 1e-6
    # the list path shifts the home atom to the image its build found (x +- L) where
    # the all-pairs path takes the minimum image of each difference: the two round a
    # difference across a face differently (u L per axis), so they agree within the
    # FP32 bound each has against the FP64 forces
    fn64, fa64 = fn.astype(np.float64), fa.astype(np.float64)
    assert _force_err(fn64, fa64) <= 1e-5
    err = np.linalg.norm(fn64 - fa64, axis=1)
    assert (err <= 2.0 * _fp32_atom_bound(x32, L, fa64)).all()


@pytest.mark.parametrize("n,rho,skin", [(1372, 0.9, 0.3), (2048, 0.5, 0.3), (864, 1.1, 0.2)])
def test_verlet_list_trajectory_follows_all_pairs(m, orc, n, rho, skin):
    """Same FP32 arithmetic on both paths; only the candidate set differs, so any
    missed pair (late rebuild, wrong cell) shows up as a jump, not slow chaos."""
    import torch
    x32, L, v = _f32_box(orc, n, rho, 40 + n)
    v32 = v.astype(np.float32)
    xa, va = _to_dev(x32), torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    va[:, :3] = torch.from_numpy(v32).cuda()
    xb, vb = xa.clone(), va.clone()
    dev = []
    for chunk in range(10):
        epa, _ = m.mdeos_debug_md(xa, va, L, 10, 0)
        epb, _ = m.mdeos_debug_md(xb, vb, L, 10, 2, skin=skin)
        d = (xa - xb).cpu().numpy()[:, :3]
        d -= L * np.round(d / L)
        dev.append(float(np.abs(d).max()))
    assert max(dev) <= 1e-4, dev


@pytest.mark.parametrize("n,rho,T,seed", [(256, 0.8, 1.5, 77), (108, 1.2, 0.7, 78),
                                          (500, 0.3, 3.0, 79), (4000, 1.0, 2.0, 80)])
def test_lifting_matches_oracle(m, orc, n, rho, T, seed):
    """Eq. 6-7 lattice, Eq. 9 Maxwell velocities (same Philox stream), E_cold."""
    x4, v4, e_cold, L = m.mdeos_debug_lift(n, rho, T, seed)
    xr, Lr = orc.lattice_fcc(n, rho)
    vr = orc.init_velocities(n, seed, T)
    assert abs(L - Lr) <= 1e-6 * Lr
    xg = x4.cpu().numpy()[:, :3].astype(np.float64)
    assert np.abs(xg - xr * (L / Lr)).max() <= 2e-6 * L
    vg = v4.cpu().numpy()[:, :3].astype(np.float64)
    assert np.abs(vg - vr).max() <= 1e-5 * np.sqrt(T)
    assert np.abs(vg.sum(axis=0)).max() <= 1e-4 * np.sqrt(T * n)
    assert abs((vg ** 2).sum() / (3 * n - 3) - T) <= 1e-5 * T
    Ec, _, _ = orc.lj_forces(xg, L)
    assert abs(e_cold - Ec) <= 1e-6 * abs(Ec)


@pytest.mark.parametrize("n,rho,path", [(256, 0.8, 0), (108, 1.1, 1), (1372, 0.9, 2)])
def test_trajectory_matches_oracle_100_steps(m, orc, n, rho, path):
    """Same initial state handed to both sides; NVE velocity-Verlet."""
    x32, L, v = _f32_box(orc, n, rho, 21 + n)
    v32 = v.astype(np.float32)
    import torch
    x4 = _to_dev(x32)
    v4 = torch.zeros_like(x4)
    v4[:, :3] = torch.from_numpy(v32).cuda()
    ep, ek = m.mdeos_debug_md(x4, v4, L, 100, path, skin=0.3)
    xr, vr, _, epr, ekr = orc.md_steps(x32.astype(np.float64), v32.astype(np.float64), L, 100)
    d = x4.cpu().numpy()[:, :3].astype(np.float64) - xr
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= 1e-4, (np.abs(d).max(), np.abs(ep.cpu().numpy() - epr)[::10])
    assert np.abs(ep.cpu().numpy() - epr).max() <= 1e-4 * n
    assert np.abs(ek.cpu().numpy() - ekr).max() <= 1e-4 * n


def test_thermostat_trajectory_matches_oracle(m, orc):
    x32, L, v = _f32_box(orc, 500, 0.7, 31)
    v32 = v.astype(np.float32)
    import torch
    x4 = _to_dev(x32)
    v4 = torch.zeros_like(x4)
    v4[:, :3] = torch.from_numpy(v32).cuda()
    ep, ek = m.mdeos_debug_md(x4, v4, L, 60, 2, skin=0.3, T_target=1.1, rescale_every=5)
    xr, vr, _, epr, ekr = orc.md_steps(x32.astype(np.float64), v32.astype(np.float64), L, 60,
                                       T_target=1.1, rescale_every=5)
    d = x4.cpu().numpy()[:, :3] - xr
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= 1e-4
    # after a rescale step the kinetic temperature is the target
    ndof = 3 * 500 - 3
    vg = v4.cpu().numpy()[:, :3].astype(np.float64)
    assert abs((vg ** 2).sum() / ndof - 1.1) <= 1e-5


@pytest.mark.parametrize("path", [0, 2])
def test_nve_energy_drift(m, orc, path):
    """Relative drift |E(1000) - E(0)| / (N T) <= 1e-4 on the GPU path (FP32)."""
    n, rho, T = 864, 0.8, 1.0
    x4, v4, _, L = m.mdeos_debug_lift(n, rho, T, 5)
    ep, ek = m.mdeos_debug_md(x4, v4, L, 200, path, skin=0.3)  # melt first
    ep, ek = m.mdeos_debug_md(x4, v4, L, 1000, path, skin=0.3)
    et = (ep + ek).cpu().numpy()
    assert abs(et[-1] - et[0]) / (n * T) <= 1e-4
    # full lists do not cancel pair forces exactly in FP32: the total momentum
    # random-walks; bound the centre-of-mass velocity at 1e-4 of the thermal one
    vcm = np.abs(v4.cpu().numpy()[:, :3].sum(axis=0)).max() / n
    assert vcm <= 1e-4 * np.sqrt(T)
