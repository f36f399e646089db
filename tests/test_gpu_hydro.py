"""GPU tests of the hydro caller (mdeos_hydro_*) and of the warm-start store, through
the C ABI, against the hydro oracle (oracle/hydro.py) and the warm-started EOS oracle.

Analytic closures: the device update is FP64 in the same operation order as the oracle
with no contracted multiply-adds, so states must agree bit for bit.  MD closure: the
hydro update is replayed in the oracle with the EOS answers the GPU produced (again bit
for bit), and the EOS answers themselves are checked statistically (warm vs cold, GPU
warm vs oracle warm from the same imported state).
"""
import numpy as np
import pytest

from oracle import hydro as H

pytestmark = pytest.mark.gpu
G53 = 5.0 / 3.0
CU = dict(mg_rho0=8.94, mg_c=0.3933, mg_s=1.5, mg_gamma=2.12)


@pytest.fixture(scope="module")
def m():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2508_06012_gb300 as m
    m.build()
    return m


@pytest.fixture(scope="module")
def h(m):
    hd = m.mdeos_create()
    yield hd
    m.mdeos_destroy(hd)


def _same(a, b):
    a, b = np.asarray(a), np.asarray(b)
    d = np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)) if a.size else 0.0
    return np.array_equal(a, b), d


def _compare(gs, o, what=("x", "u", "rho", "e")):
    for k in what:
        eq, d = _same(gs[k], getattr(o, k))
        assert eq, f"{k}: max rel diff {d:.3e}"


# --------------------------------------------------------------------------- analytic
@pytest.mark.parametrize("nz,steps", [(7, 40), (200, 300), (2500, 150)])
def test_ideal_gas_shock_tube_bitwise(m, h, nz, steps):
    g = G53
    o = H.shock_tube(nz, (1.0, 0.0, 2.0 / (g - 1)), (0.5, 0.0, 0.5 / (0.5 * (g - 1))),
                     H.IdealGas(g))
    cfg = m.mdeos_hydro_config_default(nzones=nz, closure=m.CLOSURE_IDEAL_GAS, gamma=g)
    with m.Hydro(h, cfg, o.x, o.u, o.rho, o.e) as hy:
        hy.step(steps)
        for _ in range(steps):
            o.step()
        s = hy.state()
    _compare(s, o)
    assert s["steps"] == steps and s["t"] == o.t
    assert np.array_equal(s["P"], o.P) and np.array_equal(s["q"], o.q)


def test_free_ends_momentum_and_energy(m, h):
    o = H.shock_tube(300, (1.0, 0.3, 1.0), (0.5, -0.2, 2.0), H.IdealGas(G53),
                     bc=(H.BC_FREE, H.BC_FREE))
    m0, p0, E0 = o.totals()
    cfg = m.mdeos_hydro_config_default(nzones=300, closure=m.CLOSURE_IDEAL_GAS, gamma=G53,
                                       bc_left=m.BC_FREE, bc_right=m.BC_FREE)
    with m.Hydro(h, cfg, o.x, o.u, o.rho, o.e) as hy:
        hy.step(250)
        s = hy.state()
    for _ in range(250):
        o.step()
    _compare(s, o)
    _, p1, E1 = o.totals()
    assert abs(p1 - p0) <= 1e-13 * m0 and abs(E1 - E0) <= 1e-13 * E0


@pytest.mark.parametrize("uI", [3.010, 6.913])
def test_cu_impact_mie_gruneisen_bitwise_and_hugoniot(m, h, uI):
    """Sec. IV plate impact (2 mm flyer, 3.6 mm target, 560 zones): device state equals
    the oracle's bit for bit, and the plateau at x = 3 mm is the Rankine-Hugoniot state."""
    nz = 560
    x = np.linspace(0.0, 0.56, nz + 1)
    u = np.where(x < 0.2 - 1e-12, 0.1 * uI, 0.0)
    rho = np.full(nz, 8.94)
    e = np.zeros(nz)
    mg = H.MieGruneisen(8.94, 0.3933, 1.5, 2.12)
    o = H.Hydro(x, u, rho, e, mg, bc_left=H.BC_FREE, bc_right=H.BC_FREE)
    cfg = m.mdeos_hydro_config_default(nzones=nz, closure=m.CLOSURE_MIE_GRUNEISEN,
                                       bc_left=m.BC_FREE, bc_right=m.BC_FREE, **CU)
    z = int(np.argmin(np.abs(o.centers() - 0.3)))
    t_end = 0.30 if uI < 5 else 0.20   # microseconds; the shock passes x = 3 mm before
    hist = []
    with m.Hydro(h, cfg, x, u, rho, e) as hy:
        k = 0
        while o.t < t_end:
            hy.step(1)
            o.step()
            k += 1
            if k % 50 == 0:
                s = hy.state()
                _compare(s, o)
            hist.append((o.t, o.P[z], o.rho[z]))
        s = hy.state()
    _compare(s, o)
    hist = np.array(hist)
    _, P, rhoH, _ = H.plate_impact(8.94, 8.94, 0.3933, 1.5, 0.1 * uI)
    t_arr = 0.1 / (0.3933 + 1.5 * 0.05 * uI)
    sel = hist[:, 0] > t_arr + 0.3 * (hist[-1, 0] - t_arr)
    assert sel.sum() > 20
    assert np.mean(hist[sel, 1]) == pytest.approx(P, rel=0.01)
    assert np.mean(hist[sel, 2]) == pytest.approx(rhoH, rel=0.005)


def test_tangled_mesh_is_reported(m, h):
    # colliding flows with a time step forced far above the CFL bound cross the nodes
    nz = 20
    x = np.linspace(0.0, 1.0, nz + 1)
    u = np.where(x < 0.5, 5.0, -5.0)
    cfg = m.mdeos_hydro_config_default(nzones=nz, closure=m.CLOSURE_IDEAL_GAS, dt_fixed=0.5,
                                       bc_left=m.BC_FREE, bc_right=m.BC_FREE)
    with m.Hydro(h, cfg, x, u, np.ones(nz), np.ones(nz)) as hy:
        with pytest.raises(m.MdeosError) as ei:
            hy.step(5)
        assert ei.value.status == m.MDEOS_EUNPHYS
        s = hy.state()
        assert 1 <= s["steps"] < 5      # stopped at the last good step


def test_hydro_rejects_bad_input(m, h):
    cfg = m.mdeos_hydro_config_default(nzones=3, closure=m.CLOSURE_IDEAL_GAS)
    with pytest.raises(m.MdeosError):
        m.Hydro(h, cfg, [0.0, 1.0, 0.5, 2.0], np.zeros(4), np.ones(3), np.ones(3))
    with pytest.raises(m.MdeosError):
        m.Hydro(h, cfg, [0.0, 1.0, 2.0, 3.0], np.zeros(4), [1.0, -1.0, 1.0], np.ones(3))


# --------------------------------------------------------------------------- MD closure
class _Replay:
    """Closure returning the EOS answers the GPU used, with its sound-speed estimate."""

    def __init__(self, sg):
        self.sg = sg
        self.P = self.T = None

    def __call__(self, rho, e):
        return self.P, self.sg * np.maximum(self.P / rho, self.T)


def _md_handle(m, nz, natoms, **over):
    cfg = m.mdeos_config_default(energy_ref_mode=m.MDEOS_REF_FIXED, warm_slots=nz,
                                 warm_atoms=natoms, **over)
    return m.mdeos_create(cfg)


def test_md_closure_replay_bitwise_conservation_and_warm(m):
    nz, natoms = 24, 256
    hd = _md_handle(m, nz, natoms)
    try:
        x = np.linspace(0.0, 24.0, nz + 1)
        rho = np.where(np.arange(nz) < nz // 2, 0.9, 0.6)
        e = np.where(np.arange(nz) < nz // 2, -3.0, -2.0)
        cfg = m.mdeos_hydro_config_default(
            nzones=nz, closure=m.CLOSURE_MD, natoms=natoms, steps_equil=60, steps_avg=100,
            steps_equil_first=200, steps_avg_first=100, seed=77, e_ref=0.0)
        rep = _Replay(cfg.sound_gamma)
        o = H.Hydro(x, np.zeros(nz + 1), rho, e, rep)
        _, _, E0 = o.totals()
        with m.Hydro(hd, cfg, x, np.zeros(nz + 1), rho, e) as hy:
            for k in range(4):
                hy.step(1)
                r = hy.eos_results()
                assert (r["status"] == 0).all()
                assert (r["warm"] == (1 if k > 0 else 0)).all()
                rep.P, rep.T = r["P"].copy(), r["T"].copy()
                o.step()
                s = hy.state()
                _compare(s, o)
        _, _, E1 = o.totals()
        assert abs(E1 - E0) <= 1e-13 * abs(E0)
        assert s["u"][nz // 2] > 0.0  # dense, hot side pushes into the light side
    finally:
        m.mdeos_destroy(hd)


def test_md_closure_first_call_at_temperature(m):
    nz, natoms = 8, 108
    hd = _md_handle(m, nz, natoms)
    try:
        T0 = np.where(np.arange(nz) < 4, 2.0, 1.0)
        cfg = m.mdeos_hydro_config_default(
            nzones=nz, closure=m.CLOSURE_MD, natoms=natoms, steps_equil=40, steps_avg=60,
            steps_equil_first=100, steps_avg_first=100, seed=3, first_temperature=1)
        x = np.linspace(0, 8, nz + 1)
        rho = np.where(np.arange(nz) < 4, 1.0, 0.5)
        with m.Hydro(hd, cfg, x, np.zeros(nz + 1), rho, T0) as hy:
            hy.step(1)
            r = hy.eos_results()
            s = hy.state()
            assert (r["status"] == 0).all() and (r["T_target"] == T0).all()
            # e after the step = achieved energy minus the step's compression work
            uh = 0.5 * s["u"]                     # nodes started at rest
            work = s["dt"] * (s["P"] + s["q"]) * (uh[1:] - uh[:-1]) / (rho * np.diff(x))
            assert np.allclose(s["e"] + work, r["e_achieved"], rtol=1e-12, atol=1e-12)
            hy.step(2)
            assert (hy.eos_results()["warm"] == 1).all()
    finally:
        m.mdeos_destroy(hd)


# --------------------------------------------------------------------------- warm store
def _reqs(rho, e, n, k, steps_equil, steps_avg, seed0, elem0, flags=0):
    return [dict(rho=rho, e=e, natoms=n, steps_equil=steps_equil, steps_avg=steps_avg,
                 seed=seed0 + i, element_id=elem0 + i, flags=flags) for i in range(k)]


def test_warm_start_matches_cold_start_statistically(m):
    k, n = 32, 500
    hd = _md_handle(m, k, n)
    try:
        r0 = m.mdeos_poll(hd, m.mdeos_submit(hd, _reqs(0.75, -3.5, n, k, 300, 100, 10, 1)), k)
        assert (r0["status"] == 0).all() and (r0["warm"] == 0).all()
        warm = m.mdeos_poll(hd, m.mdeos_submit(hd, _reqs(0.80, -3.5, n, k, 200, 300, 50, 1)), k)
        cold = m.mdeos_poll(hd, m.mdeos_submit(
            hd, _reqs(0.80, -3.5, n, k, 200, 300, 90, 1, flags=m.MDEOS_REQ_COLD)), k)
        assert (warm["warm"] == 1).all() and (cold["warm"] == 0).all()
        assert (warm["status"] == 0).all() and (cold["status"] == 0).all()
        for key in ("P", "T", "e_achieved"):
            a, b = warm[key], cold[key]
            se = np.sqrt(a.var(ddof=1) / k + b.var(ddof=1) / k)
            assert abs(a.mean() - b.mean()) <= 3 * se, (key, a.mean(), b.mean(), se)
    finally:
        m.mdeos_destroy(hd)


def test_gpu_warm_start_matches_oracle_from_same_state(m, orc):
    """Identical starting states (the oracle's final states at rho = 0.7, imported into
    the store): warm GPU and warm oracle evaluations at rho = 0.76 agree within 3 SE."""
    k, n = 12, 256
    p = orc.make_params(energy_ref_mode=orc.REF_FIXED)
    old = [dict(rho=0.70, e=-3.2, natoms=n, steps_equil=300, steps_avg=50, seed=400 + i)
           for i in range(k)]
    r0, x0, v0 = orc.eos_batch_state(old, p)
    assert all(r["status"] == 0 for r in r0)
    L0 = np.array([r["L"] for r in r0])
    new = [dict(rho=0.76, e=-3.2, natoms=n, steps_equil=200, steps_avg=400, seed=0)
           for _ in range(k)]
    ro, _, _ = orc.eos_batch_state(new, p, x0, v0, L0)
    hd = _md_handle(m, k, n)
    try:
        for i in range(k):
            m.mdeos_warm_import(hd, 100 + i, x0[i], v0[i], L0[i])
        reqs = [dict(r, element_id=100 + i) for i, r in enumerate(new)]
        g = m.mdeos_poll(hd, m.mdeos_submit(hd, reqs), k)
    finally:
        m.mdeos_destroy(hd)
    assert (g["status"] == 0).all() and (g["warm"] == 1).all()
    for key in ("P", "T", "e_achieved", "epot"):
        a = g[key]
        b = np.array([r[key] for r in ro])
        se = np.sqrt(a.var(ddof=1) / k + b.var(ddof=1) / k)
        assert abs(a.mean() - b.mean()) <= 3 * se + 1e-12, (key, a.mean(), b.mean(), se)


def test_warm_store_slot_rules(m):
    n = 108
    hd = _md_handle(m, 2, n)
    try:
        base = dict(rho=0.8, e=-3.0, natoms=n, steps_equil=40, steps_avg=40)
        # first sight: cold; a repeated element in one submit runs cold and is not stored
        r = m.mdeos_poll(hd, m.mdeos_submit(hd, [dict(base, seed=1, element_id=5),
                                                 dict(base, seed=2, element_id=5),
                                                 dict(base, seed=3, element_id=6),
                                                 dict(base, seed=4, element_id=7)]), 4)
        assert (r["status"] == 0).all() and (r["warm"] == 0).all()
        x4, v4, L = m.mdeos_warm_export(hd, 5, n)
        assert L == pytest.approx(r["L"][0]) and (x4[:, :3] >= 0).all() and (x4[:, :3] < L).all()
        ids = np.sort(x4[:, 3].view(np.int32))
        assert np.array_equal(ids, np.arange(n))          # every atom exactly once
        with pytest.raises(m.MdeosError):
            m.mdeos_warm_export(hd, 7, n)                  # store was full: not kept
        # second call: stored elements warm-start, the third (no slot) stays cold
        r = m.mdeos_poll(hd, m.mdeos_submit(hd, [dict(base, seed=1, element_id=5),
                                                 dict(base, seed=3, element_id=6),
                                                 dict(base, seed=4, element_id=7)]), 3)
        assert list(r["warm"]) == [1, 1, 0]
        # a failed evaluation invalidates the slot: the next one lifts cold
        r = m.mdeos_poll(hd, m.mdeos_submit(hd, [dict(base, e=-40.0, seed=1, element_id=5)]), 1)
        assert r["status"][0] == m.MDEOS_EUNPHYS
        with pytest.raises(m.MdeosError):
            m.mdeos_warm_export(hd, 5, n)
        r = m.mdeos_poll(hd, m.mdeos_submit(hd, [dict(base, seed=1, element_id=5)]), 1)
        assert r["status"][0] == 0 and r["warm"][0] == 0
        m.mdeos_warm_reset(hd)
        r = m.mdeos_poll(hd, m.mdeos_submit(hd, [dict(base, seed=1, element_id=6)]), 1)
        assert r["warm"][0] == 0
    finally:
        m.mdeos_destroy(hd)
