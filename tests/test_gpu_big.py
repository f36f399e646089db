"""GPU parity of boxes above the shared-memory limit (4097..32768 atoms: state in
global memory, one CTA per box) against the FP64 oracle, through the C ABI.

Same tolerances as the shared-memory path (tests/test_gpu_parity.py): per-atom and
global force norms, energy and virial, 100-step trajectories, NVE drift; whole EOS
evaluations against the oracle's block standard errors; bitwise alone-vs-mixed.
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


def _perturbed_lattice(orc, n, rho, seed, amp=0.08):
    """FCC lattice (first n sites, Eq. 6-7) with Gaussian displacements, in float32,
    wrapped into a float32-representable box."""
    x, L = orc.lattice_fcc(n, rho)
    rng = np.random.default_rng(seed)
    x = x + amp * rng.standard_normal(x.shape)
    L32 = float(np.float32(L))
    x32 = np.mod(x.astype(np.float32), np.float32(L32)).astype(np.float32)
    x32[x32 >= np.float32(L32)] = 0.0
    return x32, L32


def _to_dev(a32):
    import torch
    a4 = np.zeros((len(a32), 4), dtype=np.float32)
    a4[:, :3] = a32
    return torch.from_numpy(a4).cuda()


def _pairs_in_band(x, L, lo, hi):
    from scipy.spatial import cKDTree
    t = cKDTree(np.mod(x, L), boxsize=L)
    c = t.count_neighbors(t, np.array([lo, hi]))
    return int(c[1] - c[0])


def _fp32_force_bound(x, L, F):
    """Per-atom bound on the FP32 force error.  In a box of side L a position
    difference across the periodic boundary is rounded at the scale of L
    (2^-24 L per component); each pair force moves by |df/dr| times that.  Bound:
    1e-4 max(|F_i|, F_rms) + 4 * 2^-24 L * sum_j |df_ij/dr| + |f(rc)| per pair of
    atom i within rounding of the cutoff."""
    from scipy.spatial import cKDTree
    t = cKDTree(np.mod(x, L), boxsize=L)
    pr = t.query_pairs(RC * (1 + 4e-6), output_type="ndarray")
    d = x[pr[:, 0]] - x[pr[:, 1]]
    d -= L * np.round(d / L)
    r = np.sqrt((d ** 2).sum(axis=1))
    g = np.abs(24.0 * (-26.0 * r ** -14 + 7.0 * r ** -8))
    stiff = np.bincount(pr[:, 0], g, minlength=len(x)) + np.bincount(pr[:, 1], g, minlength=len(x))
    # a pair within FP32 rounding of the cutoff may be in or out on either side:
    # the truncated force jumps by |f(rc)| there
    band = np.abs(r - RC) < 4e-6 * RC
    amb = np.bincount(pr[band, 0], minlength=len(x)) + np.bincount(pr[band, 1], minlength=len(x))
    f_rc = abs(24.0 * (2.0 * RC ** -13 - RC ** -7))
    fn = np.linalg.norm(F, axis=1)
    frms = np.sqrt((fn ** 2).mean())
    return 1e-4 * np.maximum(fn, frms) + 4.0 * 2.0 ** -24 * L * stiff + 1.01 * f_rc * amb


def _ordered_pairs(x, L, r):
    from scipy.spatial import cKDTree
    t = cKDTree(np.mod(x, L), boxsize=L)
    return int(t.count_neighbors(t, r)) - len(x)


@pytest.mark.parametrize("n,rho,seed", [
    (4097, 0.8, 1),      # one atom above the shared-memory limit, ragged lattice
    (6912, 0.9, 2),      # 4 x 12^3
    (13500, 0.35, 3),    # dilute, 4 x 15^3
    (32000, 1.2, 4),     # largest box of the serving stream, dense
    (32768, 0.8, 5),     # maximum atoms per box
])
def test_big_forces_energy_virial_match_oracle(m, orc, n, rho, seed):
    x32, L = _perturbed_lattice(orc, n, rho, seed)
    x64 = x32.astype(np.float64)
    E, f, W = orc.lj_forces(x64, L, orc.make_params(force_mode=orc.FORCE_CELL),
                            mode=orc.FORCE_CELL)
    f4, ew, pairs = m.mdeos_debug_forces(_to_dev(x32), L, m.PATH_NLIST, skin=0.3)
    fg = f4.cpu().numpy()[:, :3].astype(np.float64)
    ew = ew.cpu().numpy()
    assert np.isfinite(ew).all()
    assert np.linalg.norm(fg - f) / np.linalg.norm(f) <= 1e-5
    err = np.linalg.norm(fg - f, axis=1)
    bound = _fp32_force_bound(x64, L, f)
    assert (err <= bound).all(), (err / bound).max()
    assert abs(ew[0] - E) <= 1e-6 * abs(E) + 1e-5 * n
    assert np.abs(ew[1:] - W).max() <= 2e-5 * np.abs(W).max() + 1e-4 * n
    ref = _ordered_pairs(x64, L, RC)
    amb = 2 * _pairs_in_band(x64, L, RC * (1 - 1e-6), RC * (1 + 1e-6))
    assert abs(pairs - ref) <= amb


def test_big_trajectory_matches_oracle_100_steps(m, orc):
    import torch
    n, rho, T = 5324, 0.8, 1.2
    x32, L = _perturbed_lattice(orc, n, rho, 11, amp=0.05)
    v32 = orc.init_velocities(n, 12, T).astype(np.float32)
    x4 = _to_dev(x32)
    v4 = torch.zeros_like(x4)
    v4[:, :3] = torch.from_numpy(v32).cuda()
    ep, ek = m.mdeos_debug_md(x4, v4, L, 100, m.PATH_NLIST, skin=0.3)
    p = orc.make_params(force_mode=orc.FORCE_CELL)
    xr, vr, _, epr, ekr = orc.md_steps(x32.astype(np.float64), v32.astype(np.float64), L, 100,
                                       params=p)
    d = x4.cpu().numpy()[:, :3].astype(np.float64) - xr
    d -= L * np.round(d / L)
    assert np.abs(d).max() <= 1e-4, np.abs(d).max()
    assert np.abs(ep.cpu().numpy() - epr).max() <= 1e-4 * n
    assert np.abs(ek.cpu().numpy() - ekr).max() <= 1e-4 * n


def test_big_nve_energy_drift_and_momentum(m, orc):
    import torch
    n, rho, T = 6912, 0.8, 1.0
    x32, L = _perturbed_lattice(orc, n, rho, 21, amp=0.0)
    v32 = orc.init_velocities(n, 22, T).astype(np.float32)
    x4 = _to_dev(x32)
    v4 = torch.zeros_like(x4)
    v4[:, :3] = torch.from_numpy(v32).cuda()
    m.mdeos_debug_md(x4, v4, L, 200, m.PATH_NLIST, skin=0.3)      # melt
    ep, ek = m.mdeos_debug_md(x4, v4, L, 1000, m.PATH_NLIST, skin=0.3)
    et = (ep + ek).cpu().numpy()
    assert abs(et[-1] - et[0]) / (n * T) <= 1e-4
    vcm = np.abs(v4.cpu().numpy()[:, :3].sum(axis=0)).max() / n
    assert vcm <= 1e-4 * np.sqrt(T)


def test_big_eos_lifting_matches_oracle(m, orc):
    """Whole lifting -> MD -> restriction of 6912-atom boxes: the deterministic part
    of the lifting (E_cold of the lattice, Eq. 6-7) against the oracle; the
    statistical parity of the restricted values is in tests/test_gpu_ensembles.py."""
    reqs = [dict(rho=rho, e=m.e_from_temperature(T, 6912), natoms=6912, steps_equil=200,
                 steps_avg=300, seed=900 + k) for k, (rho, T) in
            enumerate([(0.7, 1.5), (0.95, 2.0), (0.4, 1.2), (1.1, 2.5)])]
    with m.Engine() as eng:
        g = eng.evaluate(reqs)
    assert (g["status"] == 0).all() and (g["path"] == m.PATH_NLIST).all()
    for k, r in enumerate(reqs):
        x, L = orc.lattice_fcc(6912, r["rho"])
        L32 = float(np.float32(L))
        E, _, _ = orc.lj_forces(x * (L32 / L), L32, orc.make_params(force_mode=orc.FORCE_CELL),
                                mode=orc.FORCE_CELL)
        # FP32 per-thread energy sums over ~550 pair terms per thread
        assert g["e_cold"][k] == pytest.approx(E / 6912, rel=5e-6)
        assert g["T_target"][k] > 0
    assert np.allclose(g["sigma"][:, :3].mean(axis=1), g["P"], rtol=1e-6, atol=1e-6)


def test_big_alone_equals_mix_and_limits(m):
    from paper_2508_06012_gb300 import workloads as w
    small = w.random_boxes(5, 12, 108, 3000, steps_equil=60, steps_avg=60)
    reqs = [dict(rho=b["rho"], e=m.e_from_temperature(b["T"], b["natoms"]), natoms=b["natoms"],
                 steps_equil=60, steps_avg=60, seed=b["seed"]) for b in small]
    big = [dict(rho=0.8, e=1.5, natoms=n, steps_equil=60, steps_avg=60, seed=70 + k)
           for k, n in enumerate((4500, 9000, 20000))]
    mix = reqs[:6] + big + reqs[6:]
    with m.Engine() as eng:
        r = eng.evaluate(mix)
        assert (r["status"][6:9] == 0).all()   # small random boxes may fail (T_k < 0)
        for k in (6, 7, 8, 0, 12):
            alone = eng.evaluate([mix[k]])[0]
            assert alone.tobytes() == r[k].tobytes()
        lim = eng.evaluate([dict(big[0], natoms=32768, rho=0.9, steps_equil=20, steps_avg=20),
                            dict(big[0], natoms=32769)])
        assert list(lim["status"]) == [0, m.MDEOS_EINVAL]


def test_noalloc_rejects_big_boxes(m):
    import torch
    reqs = [dict(rho=0.8, e=1.5, natoms=5000, steps_equil=20, steps_avg=20, seed=1),
            dict(rho=0.8, e=1.5, natoms=256, steps_equil=20, steps_avg=20, seed=2)]
    rec = m.RESULT_DTYPE.itemsize
    buf = torch.zeros(2 * rec, dtype=torch.uint8, device="cuda")
    m.mdeos_submit_noalloc(reqs, buf.data_ptr())
    torch.cuda.synchronize()
    out = np.frombuffer(buf.cpu().numpy().tobytes(), dtype=m.RESULT_DTYPE)
    assert list(out["status"]) == [m.MDEOS_EINVAL, 0]
