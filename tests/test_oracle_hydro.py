"""Pins of the hydro oracle (oracle/hydro.py) and of the warm-started EOS oracle.

Each pin comes from outside the code it checks: closed forms, conservation laws,
the Rankine-Hugoniot jump conditions, textbook special cases of the Riemann problem,
and the Cu impact numbers printed in the paper (Sec. IV, Tables I-III).
"""
import os

import numpy as np
import pytest

from oracle import hydro as H

GOLD = os.path.join(os.path.dirname(__file__), "golden", "cu_plate_impact_tables.txt")
G53 = 5.0 / 3.0
CU = dict(C=0.3933, s=1.5, Gamma=2.12)  # cm/us, -, - (Sec. IV.A)


def cu_rows():
    return np.loadtxt(GOLD, comments="#")


# --------------------------------------------------------------------------- closures
def test_ideal_gas_closed_form():
    P, c2 = H.IdealGas(1.4)(np.array([2.0]), np.array([3.0]))
    assert P[0] == pytest.approx(0.4 * 2.0 * 3.0, rel=1e-15)
    assert c2[0] == pytest.approx(1.4 * P[0] / 2.0, rel=1e-15)


def test_mie_gruneisen_reference_curve_and_energy_slope():
    mg = H.MieGruneisen(8.94, **CU)
    rho = np.linspace(8.0, 14.0, 13)
    eta, PH, EH = mg.reference(rho)
    P, _ = mg(rho, EH)
    assert np.allclose(P, PH, rtol=1e-14, atol=1e-16)         # P(E_ref) = P_ref (Eq. 1)
    h = 1e-6
    dPde = (mg(rho, EH + h)[0] - mg(rho, EH - h)[0]) / (2 * h)
    assert np.allclose(dPde, CU["Gamma"] * rho, rtol=1e-8)      # dP/dE = Gamma / V


def test_mie_gruneisen_hugoniot_is_the_rankine_hugoniot_locus():
    """The reference curve written in eta equals the jump conditions written in u_p."""
    mg = H.MieGruneisen(8.94, **CU)
    for up in (0.05, 0.15, 0.3):
        Us, P, rho = H.hugoniot_state(8.94, CU["C"], CU["s"], up)
        _, PH, EH = mg.reference(np.array([rho]))
        assert PH[0] == pytest.approx(P, rel=1e-13)
        assert EH[0] == pytest.approx(0.5 * up * up, rel=1e-12)   # energy jump = u_p^2 / 2


@pytest.mark.parametrize("closure,rho,e", [
    (H.IdealGas(G53), [0.3, 1.0, 2.0, 5.0], [0.5, 1.0, 3.0, 2.0]),
    (H.MieGruneisen(8.94, **CU), [9.0, 10.0, 9.5, 11.0], [0.05, 0.2, 0.1, 0.3])])
def test_sound_speed_is_isentropic_derivative(closure, rho, e):
    rho, e = np.array(rho), np.array(e)
    P, c2 = closure(rho, e)
    h = 1e-5 * rho
    de = P / rho ** 2 * h                      # de = P / rho^2 drho along an isentrope
    num = (closure(rho + h, e + de)[0] - closure(rho - h, e - de)[0]) / (2 * h)
    assert np.allclose(c2, num, rtol=1e-6)


def test_mie_gruneisen_sound_speed_at_rest_is_bulk_sound_speed():
    mg = H.MieGruneisen(8.94, **CU)
    _, c2 = mg(np.array([8.94]), np.array([0.0]))
    assert np.sqrt(c2[0]) == pytest.approx(CU["C"], rel=1e-14)


# --------------------------------------------------------------------------- Riemann
def _jumps(pre, post, S, g):
    """Residuals of mass, momentum and energy (enthalpy) jumps across a shock of speed S."""
    r0, u0, p0 = pre
    r1, u1, p1 = post
    w0, w1 = u0 - S, u1 - S
    mass = r0 * w0 - r1 * w1
    mom = r0 * w0 * w0 + p0 - (r1 * w1 * w1 + p1)
    en = g / (g - 1) * p0 / r0 + 0.5 * w0 * w0 - (g / (g - 1) * p1 / r1 + 0.5 * w1 * w1)
    return mass, mom, en


CASES = [((1.0, 0.0, 2.0), (0.5, 0.0, 0.5)),      # shock-tube states of the coupled test
         ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1)),    # strong left rarefaction, right shock
         ((1.0, 2.0, 1.0), (1.0, -2.0, 1.0)),     # colliding flows: two shocks
         ((1.0, -1.0, 1.0), (1.0, 1.0, 1.0)),     # receding flows: two rarefactions
         ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01))]  # blast wave


@pytest.mark.parametrize("L,R", CASES)
def test_riemann_solution_satisfies_jump_and_wave_invariants(L, R):
    g = G53
    ps, us = H.riemann_star(L, R, g)
    eps = 1e-9
    for side, W, sgn in (("L", L, -1.0), ("R", R, 1.0)):
        rK, uK, pK = W
        cK = np.sqrt(g * pK / rK)
        # state just on the star side of the contact
        rs, u1, p1 = (a[0] for a in H.riemann_sample(L, R, np.array([us + sgn * eps]), g))
        assert u1 == pytest.approx(us, rel=1e-12, abs=1e-12) and p1 == pytest.approx(ps, rel=1e-12)
        if ps > pK:   # shock: Rankine-Hugoniot with the speed from the mass jump
            S = (rs * us - rK * uK) / (rs - rK)
            m, mo, en = _jumps(W, (rs, us, ps), S, g)
            scale = max(rK * abs(uK - S), 1.0)
            assert abs(m) < 1e-10 * scale and abs(mo) < 1e-10 * max(pK, ps) \
                and abs(en) < 1e-10 * max(pK / rK, 1.0)
        else:         # rarefaction: isentropic, Riemann invariant carried across
            assert ps / rs ** g == pytest.approx(pK / rK ** g, rel=1e-12)
            cs = np.sqrt(g * ps / rs)
            J = uK - sgn * 2 * cK / (g - 1)
            assert us - sgn * 2 * cs / (g - 1) == pytest.approx(J, rel=1e-12, abs=1e-12)


def test_riemann_symmetric_closed_forms():
    g = G53
    # receding flows: u* = 0, c* = c - (g - 1) |u| / 2 (Riemann invariant), p* isentropic
    ps, us = H.riemann_star((1.0, -1.0, 1.0), (1.0, 1.0, 1.0), g)
    c = np.sqrt(g)
    cs = c - 0.5 * (g - 1) * 1.0
    assert us == pytest.approx(0.0, abs=1e-14)
    assert ps == pytest.approx((cs / c) ** (2 * g / (g - 1)), rel=1e-12)
    # colliding flows: u* = 0 and (p* - p)^2 A / (p* + B) = u^2 (shock relation)
    ps, us = H.riemann_star((1.0, 2.0, 1.0), (1.0, -2.0, 1.0), g)
    A, B = 2 / (g + 1), (g - 1) / (g + 1)
    a, b, cc = 1.0, -(2.0 + 4.0 / A), 1.0 - 4.0 * B / A   # (p-1)^2 = 4 (p + B) / A
    root = (-b + np.sqrt(b * b - 4 * a * cc)) / (2 * a)
    assert us == pytest.approx(0.0, abs=1e-14)
    assert ps == pytest.approx(root, rel=1e-12)


# --------------------------------------------------------------------------- hydro
def _tube(nz, bc=(H.BC_WALL, H.BC_WALL)):
    g = G53
    return H.shock_tube(nz, (1.0, 0.0, 2.0 / (g - 1)), (0.5, 0.0, 0.5 / (0.5 * (g - 1))),
                        H.IdealGas(g), bc=bc)


def test_hydro_conserves_mass_and_energy_to_roundoff():
    h = _tube(200)
    m0, _, E0 = h.totals()
    for _ in range(300):
        h.step()
    m1, _, E1 = h.totals()
    assert m1 == m0
    assert np.allclose(h.rho * (h.x[1:] - h.x[:-1]), h.m, rtol=1e-13)
    assert abs(E1 - E0) <= 1e-13 * E0


def test_hydro_free_ends_conserve_momentum():
    h = H.shock_tube(200, (1.0, 0.3, 1.0), (0.5, -0.2, 2.0), H.IdealGas(G53),
                     bc=(H.BC_FREE, H.BC_FREE))
    _, p0, E0 = h.totals()
    for _ in range(200):
        h.step()
    _, p1, E1 = h.totals()
    assert abs(p1 - p0) <= 1e-13 * h.totals()[0]
    assert abs(E1 - E0) <= 1e-13 * E0


def test_hydro_converges_to_exact_riemann_solution():
    g = G53
    errs = []
    for nz in (100, 200, 400):
        h = _tube(nz)
        h.run_until(0.2)
        r, _, _ = H.riemann_sample((1.0, 0.0, 2.0), (0.5, 0.0, 0.5), (h.centers() - 0.5) / h.t, g)
        errs.append(np.mean(np.abs(h.rho - r)))
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1]
    assert errs[2] < 3e-3


def test_hydro_uniform_state_stays_uniform():
    h = H.shock_tube(50, (1.0, 0.0, 1.5), (1.0, 0.0, 1.5), H.IdealGas(G53))
    for _ in range(50):
        h.step()
    assert np.all(h.rho == 1.0) and np.all(h.e == 1.5) and np.all(h.u == 0.0)


# --------------------------------------------------------------------------- Cu impact
def test_plate_impact_rankine_hugoniot_matches_paper_tables():
    for uI, rf, rt, Pexp, dPexp, rexp, drexp, Pan, ran in cu_rows():
        up, P, rho, _ = H.plate_impact(rf, rt, CU["C"], CU["s"], 0.1 * uI)
        P_gpa = 100.0 * P
        if uI < 5:   # low velocity: R-H, the paper's analytic EOS and experiment agree
            assert P_gpa == pytest.approx(83.29, abs=0.01)
            assert rho == pytest.approx(11.81, abs=0.005)
            assert abs(P_gpa - Pan) / Pan < 0.005 and abs(rho - ran) / ran < 0.005
            assert abs(P_gpa - Pexp) < 2 * dPexp and abs(rho - rexp) < 2 * drexp
        else:        # high velocity: the paper's 28-element run sits ~4% below R-H (its
            # Sec. IV.D attributes it to discretisation); R-H is within experiment's 2 sigma
            assert abs(P_gpa - Pexp) < 2 * dPexp and abs(rho - rexp) < 2 * drexp
            assert 0.0 < (P_gpa - Pan) / P_gpa < 0.06


def test_symmetric_equal_density_impact_halves_velocity():
    up, P, rt, rf = H.plate_impact(8.94, 8.94, CU["C"], CU["s"], 0.301)
    assert up == pytest.approx(0.1505, rel=1e-12) and rt == pytest.approx(rf, rel=1e-12)


@pytest.mark.parametrize("row", [0, 1])
def test_hydro_cu_impact_reaches_hugoniot_state(row):
    """Sec. IV set-up in 1D: 2 mm flyer onto a 3.6 mm target, state sampled 1 mm into
    the target (x = 3 mm); plateau vs the Rankine-Hugoniot state."""
    uI, rf, rt = cu_rows()[row][:3]
    rho0 = 0.5 * (rf + rt)
    mg = H.MieGruneisen(rho0, **CU)
    nz = 560
    x = np.linspace(0.0, 0.56, nz + 1)
    u = np.where(x < 0.2 - 1e-12, 0.1 * uI, 0.0)
    h = H.Hydro(x, u, np.full(nz, rho0), np.zeros(nz), mg, bc_left=H.BC_FREE,
                bc_right=H.BC_FREE)
    z = int(np.argmin(np.abs(h.centers() - 0.3)))
    hist = []
    t_end = 0.30 if uI < 5 else 0.20
    h.run_until(t_end, record=lambda hh: hist.append((hh.t, hh.P[z], hh.rho[z])))
    hist = np.array(hist)
    _, P, rho, _ = H.plate_impact(rho0, rho0, CU["C"], CU["s"], 0.1 * uI)
    t_arr = 0.1 / (CU["C"] + CU["s"] * 0.05 * uI)     # shock arrival at x = 3 mm
    sel = hist[:, 0] > t_arr + 0.3 * (t_end - t_arr)
    assert sel.sum() > 20
    assert np.mean(hist[sel, 1]) == pytest.approx(P, rel=0.01)
    assert np.mean(hist[sel, 2]) == pytest.approx(rho, rel=0.005)


# --------------------------------------------------------------------------- warm start
def _ens(orc, reqs, params, states=None):
    if states is None:
        return orc.eos_batch_state(reqs, params)
    x, v, L = states
    return orc.eos_batch_state(reqs, params, x, v, L)


def test_warm_start_agrees_with_cold_start_statistically(orc):
    """The EOS answer must not depend on where the lift started: warm starts from states
    equilibrated at a neighbouring density give the same ensemble means as cold lifts."""
    p = orc.make_params(energy_ref_mode=orc.REF_FIXED)
    n, k = 108, 8
    e = -4.0                                   # FIXED reference 0: liquid near T ~ 1.3
    old = [dict(rho=0.75, e=e, natoms=n, steps_equil=300, steps_avg=100, seed=100 + s)
           for s in range(k)]
    r0, x0, v0 = _ens(orc, old, p)
    assert all(r["status"] == 0 for r in r0)
    new = [dict(rho=0.80, e=e, natoms=n, steps_equil=300, steps_avg=600, seed=200 + s)
           for s in range(k)]
    rw, xw, vw = _ens(orc, new, p, (x0, v0, np.array([r["L"] for r in r0])))
    rc, _, _ = _ens(orc, new, p)
    assert all(r["status"] == 0 for r in rw + rc)
    for key in ("P", "T", "e_achieved"):
        a = np.array([r[key] for r in rw])
        b = np.array([r[key] for r in rc])
        se = np.sqrt(a.var(ddof=1) / k + b.var(ddof=1) / k)
        assert abs(a.mean() - b.mean()) <= 3 * se + 1e-12, (key, a.mean(), b.mean(), se)
    # final states lie in the new box
    L = rw[0]["L"]
    assert (xw >= 0).all() and (xw < L).all() and L < r0[0]["L"]


def test_warm_start_temperature_mode_and_invalid(orc):
    p = orc.make_params(energy_ref_mode=orc.REF_FIXED, warm_lift_iters=1)
    rq = dict(rho=0.8, e=1.2, natoms=108, steps_equil=50, steps_avg=50, seed=5,
              flags=orc.REQ_TEMPERATURE)
    r, x, v = orc.eos_eval_state(rq, p)
    rw, _, _ = orc.eos_eval_state(dict(rq, rho=0.82), p, x, v, r["L"])
    assert rw["status"] == 0 and rw["T_target"] == 1.2
    bad = orc.make_params(energy_ref_mode=orc.REF_FIXED, warm_lift_iters=0)
    rb, _, _ = orc.eos_eval_state(dict(rq, rho=0.82), bad, x, v, r["L"])
    assert rb["status"] == orc.EINVAL    # equilibration steps with no Eq. 10 segment


def test_coupled_md_hydro_conserves_energy(orc):
    """Compatible energy update: total energy is conserved whatever the closure returns,
    here the warm-started MD closure (6 zones of 108 atoms)."""
    clo = H.MDClosure(natoms=108, steps_equil=40, steps_avg=40, seed=9, steps_equil_first=100,
                      steps_avg_first=60)
    nz = 6
    x = np.linspace(0.0, 6.0, nz + 1)
    rho = np.array([0.9, 0.9, 0.9, 0.6, 0.6, 0.6])
    e = np.array([-3.0, -3.0, -3.0, -2.5, -2.5, -2.5])
    h = H.Hydro(x, np.zeros(nz + 1), rho, e, clo)
    _, _, E0 = h.totals()
    for _ in range(3):
        h.step()
    _, _, E1 = h.totals()
    assert clo.calls == 3 and abs(E1 - E0) <= 1e-13 * abs(E0)
    assert h.u[3] > 0.0           # the dense side pushes into the light side
