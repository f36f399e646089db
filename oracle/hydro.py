"""Plain FP64 reference of the hydro caller of the in-line EOS (arXiv 2508.06012, Sec. II).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` (and the CPU arm of ``bench.py``),
never by the product package.  Shares no code with the CUDA path.

What it computes
----------------
* One-dimensional planar Lagrangian hydrodynamics of the Euler equations (Eq. 2-4) on
  a staggered grid: node positions x_i and velocities u_i, zone masses m_z, densities
  rho_z and specific internal energies e_z.  One step (time n -> n+1):

    1. closure: P_z, c_z^2 = EOS(rho_z, e_z)                 (Eq. 5, one call per zone)
    2. artificial viscosity (von Neumann-Richtmyer quadratic plus linear term, the
       Wilkins form the paper cites; constants are not given there, the reading is
       q2 = 2, q1 = 0.5):  du_z = u_{z+1} - u_z,
       q_z = rho_z * (q2 du_z^2 - q1 c_z du_z) if du_z < 0 else 0
    3. time step: dt = cfl * min_z dx_z / (c_z + 2 q2 |min(du_z, 0)|), cfl = 0.5, at most
       dt_grow * dt of the previous step
    4. momentum (Eq. 3): F_i = (P+q)_{i-1} - (P+q)_i (outside pressure 0 at a free end),
       u_i <- u_i + dt F_i / M_i with M_i half the mass of the two adjacent zones; u = 0
       at a wall
    5. positions: x_i <- x_i + dt (u_i^n + u_i^{n+1}) / 2
    6. energy (Eq. 4): e_z <- e_z - dt (P+q)_z (u^{n+1/2}_{z+1} - u^{n+1/2}_z) / m_z, the
       compatible form: the internal energy gains exactly the work the nodal forces
       take out of the kinetic energy, so total energy is conserved to round-off
    7. mass (Eq. 2): rho_z <- m_z / (x_{z+1} - x_z)

  Every expression is written in one fixed evaluation order (the CUDA hydro kernels
  follow the same reading independently and are compiled without FMA contraction).

* Closures: ideal gas; Mie-Grueneisen with a linear U_s-u_p Hugoniot as reference curve
  (Eq. 1 with constant Gamma, P_ref = P_H, E_ref = E_H); the MD closure through the
  C oracle's warm-started EOS evaluation (warm-start reading: affine rescale of the
  previous final state, then one Eq. 10 temperature update before averaging).
* Exact Riemann solution of the ideal-gas shock tube (two-wave pressure function
  solved by Newton iteration, then the self-similar sampling; the textbook construction
  of Toro, ch. 4, restated).
* Rankine-Hugoniot states of a linear U_s-u_p material and of a plate impact.
"""
from __future__ import annotations

import numpy as np

BC_WALL, BC_FREE = 0, 1


# ---------------------------------------------------------------------------
# closures
class IdealGas:
    """P = (gamma - 1) rho e, c^2 = gamma P / rho."""

    def __init__(self, gamma: float = 5.0 / 3.0):
        self.gamma = float(gamma)

    def __call__(self, rho, e):
        P = (self.gamma - 1.0) * rho * e
        c2 = self.gamma * P / rho
        return P, c2


class MieGruneisen:
    """Eq. 1 with the Hugoniot of a linear U_s = C + s u_p material as reference curve.

    eta = 1 - rho0 / rho, P_H = rho0 C^2 eta / (1 - s eta)^2, E_H = P_H eta / (2 rho0)
    (Rankine-Hugoniot energy jump from rest at e = 0), P = P_H + Gamma rho (e - E_H)
    (Eq. 1 with V the specific volume 1 / rho and constant Gamma).
    c^2 = (dP/drho)_e + (P / rho^2) (dP/de)_rho, the isentropic sound speed squared.
    """

    def __init__(self, rho0: float, C: float, s: float, Gamma: float):
        self.rho0, self.C, self.s, self.Gamma = float(rho0), float(C), float(s), float(Gamma)

    def reference(self, rho):
        rho0, C, s = self.rho0, self.C, self.s
        eta = 1.0 - rho0 / rho
        den = 1.0 - s * eta
        PH = rho0 * C * C * eta / (den * den)
        EH = PH * eta / (2.0 * rho0)
        return eta, PH, EH

    def __call__(self, rho, e):
        rho0, C, s, G = self.rho0, self.C, self.s, self.Gamma
        eta, PH, EH = self.reference(rho)
        P = PH + G * rho * (e - EH)
        den = 1.0 - s * eta
        dPH = rho0 * C * C * (1.0 + s * eta) / (den * den * den)   # dP_H / d eta
        dEH = (PH + eta * dPH) / (2.0 * rho0)                       # dE_H / d eta
        deta = rho0 / (rho * rho)                                   # d eta / d rho
        dP_drho_e = (dPH - G * rho * dEH) * deta + G * (e - EH)
        c2 = dP_drho_e + P / (rho * rho) * (G * rho)
        return P, c2


class MDClosure:
    """The atomistic EOS (lifting -> MD -> restriction) of the C oracle, one request per
    zone per call, warm-started from each zone's previous final state after the first
    call.  Sound speed estimate (the paper gives none): c^2 = gamma_a * max(P / rho, T).
    """

    def __init__(self, natoms: int, steps_equil: int, steps_avg: int, seed: int,
                 params=None, steps_equil_first: int | None = None,
                 steps_avg_first: int | None = None, gamma_a: float = 3.0, e_ref: float = 0.0,
                 warm: bool = True):
        from . import make_params, REF_FIXED
        self.params = params or make_params(energy_ref_mode=REF_FIXED)
        self.natoms, self.steps_equil, self.steps_avg = natoms, steps_equil, steps_avg
        self.steps_equil_first = steps_equil if steps_equil_first is None else steps_equil_first
        self.steps_avg_first = steps_avg if steps_avg_first is None else steps_avg_first
        self.seed, self.gamma_a, self.e_ref, self.warm = seed, gamma_a, e_ref, warm
        self.state = None   # (x, v, L) per zone after the first call
        self.calls = 0
        self.last = None

    def __call__(self, rho, e):
        from . import eos_batch_state
        nz = len(rho)
        first = self.state is None or not self.warm
        reqs = [dict(rho=float(rho[z]), e=float(e[z]), e_ref=self.e_ref, natoms=self.natoms,
                     steps_equil=self.steps_equil_first if first else self.steps_equil,
                     steps_avg=self.steps_avg_first if first else self.steps_avg,
                     seed=int(self.seed + 7919 * z + 104729 * self.calls))
                for z in range(nz)]
        if first:
            res, xo, vo = eos_batch_state(reqs, self.params)
        else:
            x, v, L = self.state
            res, xo, vo = eos_batch_state(reqs, self.params, x, v, L)
        st = np.array([r["status"] for r in res])
        if (st != 0).any():
            raise RuntimeError(f"MD closure failed in zones {np.flatnonzero(st)[:8]}")
        self.state = (xo, vo, np.array([r["L"] for r in res]))
        self.calls += 1
        self.last = res
        P = np.array([r["P"] for r in res])
        T = np.array([r["T"] for r in res])
        c2 = self.gamma_a * np.maximum(P / rho, T)
        return P, c2


# ---------------------------------------------------------------------------
# staggered Lagrangian hydro
class Hydro:
    def __init__(self, x, u, rho, e, closure, bc_left=BC_WALL, bc_right=BC_WALL, q2=2.0,
                 q1=0.5, cfl=0.5, dt_grow=1.1, dt_fixed=None):
        self.x = np.array(x, dtype=np.float64)
        self.u = np.array(u, dtype=np.float64)
        self.rho = np.array(rho, dtype=np.float64)
        self.e = np.array(e, dtype=np.float64)
        nz = len(self.rho)
        assert self.x.shape == (nz + 1,) and self.u.shape == (nz + 1,) and self.e.shape == (nz,)
        self.m = self.rho * (self.x[1:] - self.x[:-1])
        M = np.zeros(nz + 1)
        M[:-1] += 0.5 * self.m
        M[1:] += 0.5 * self.m
        self.M = M
        self.closure = closure
        self.bc = (bc_left, bc_right)
        self.q2, self.q1, self.cfl, self.dt_grow = float(q2), float(q1), float(cfl), float(dt_grow)
        self.dt_fixed = dt_fixed
        self.dt_prev = None
        self.t = 0.0
        self.nstep = 0
        if bc_left == BC_WALL:
            self.u[0] = 0.0
        if bc_right == BC_WALL:
            self.u[-1] = 0.0
        self.P = np.zeros(nz)
        self.q = np.zeros(nz)
        self.c2 = np.zeros(nz)

    def step(self):
        x, u, rho, e, m, M = self.x, self.u, self.rho, self.e, self.m, self.M
        # 1. closure
        P, c2 = self.closure(rho, e)
        P = np.asarray(P, dtype=np.float64)
        c2 = np.asarray(c2, dtype=np.float64)
        c = np.sqrt(c2)
        # 2. artificial viscosity
        du = u[1:] - u[:-1]
        q = np.where(du < 0.0, rho * (self.q2 * du * du - self.q1 * c * du), 0.0)
        Pq = P + q
        # 3. time step
        dx = x[1:] - x[:-1]
        sig = c + 2.0 * self.q2 * np.maximum(-du, 0.0)
        if self.dt_fixed is not None:
            dt = float(self.dt_fixed)
        else:
            dt = self.cfl * np.min(dx / sig)
            if self.dt_prev is not None:
                dt = min(dt, self.dt_grow * self.dt_prev)
        # 4. momentum
        F = np.zeros_like(u)
        F[1:-1] = Pq[:-1] - Pq[1:]
        F[0] = 0.0 - Pq[0]
        F[-1] = Pq[-1] - 0.0
        un = u + dt * F / M
        if self.bc[0] == BC_WALL:
            un[0] = 0.0
        if self.bc[1] == BC_WALL:
            un[-1] = 0.0
        uh = 0.5 * (u + un)
        # 5. positions
        xn = x + dt * uh
        # 6. energy, compatible form
        en = e - dt * Pq * (uh[1:] - uh[:-1]) / m
        # 7. density
        rhon = m / (xn[1:] - xn[:-1])
        self.x, self.u, self.e, self.rho = xn, un, en, rhon
        self.P, self.q, self.c2 = P, q, c2
        self.dt_prev = dt
        self.t += dt
        self.nstep += 1
        return dt

    def run_until(self, t_end, max_steps=10 ** 7, record=None):
        """Steps until t >= t_end (the last step is shortened to land on t_end).
        record(h) is called after every step."""
        while self.t < t_end and self.nstep < max_steps:
            keep = self.dt_fixed
            dt_est = self._dt_estimate()
            if self.t + dt_est > t_end:
                self.dt_fixed = t_end - self.t
            self.step()
            self.dt_fixed = keep
            if record is not None:
                record(self)
        return self

    def _dt_estimate(self):
        if self.dt_fixed is not None:
            return float(self.dt_fixed)
        P, c2 = self.closure(self.rho, self.e) if not isinstance(self.closure, MDClosure) \
            else (self.P, self.c2)
        c = np.sqrt(np.asarray(c2))
        du = self.u[1:] - self.u[:-1]
        dx = self.x[1:] - self.x[:-1]
        sig = c + 2.0 * self.q2 * np.maximum(-du, 0.0)
        dt = self.cfl * np.min(dx / sig)
        if self.dt_prev is not None:
            dt = min(dt, self.dt_grow * self.dt_prev)
        return dt

    def totals(self):
        """(mass, momentum, total energy) = (sum m, sum M u, sum m e + sum M u^2 / 2)."""
        return (float(np.sum(self.m)), float(np.sum(self.M * self.u)),
                float(np.sum(self.m * self.e) + 0.5 * np.sum(self.M * self.u * self.u)))

    def centers(self):
        return 0.5 * (self.x[1:] + self.x[:-1])


def shock_tube(nz, left, right, closure, length=1.0, x0=0.5, bc=(BC_WALL, BC_WALL), **kw):
    """Uniform grid on [0, length]; zones with centre < x0 get left = (rho, u, e), the
    others right.  Node velocities: the left u up to the node at x0, the right u after."""
    x = np.linspace(0.0, length, nz + 1)
    xc = 0.5 * (x[1:] + x[:-1])
    L = xc < x0
    rho = np.where(L, left[0], right[0])
    e = np.where(L, left[2], right[2])
    u = np.where(x < x0, left[1], right[1]).astype(np.float64)
    u[np.isclose(x, x0)] = 0.5 * (left[1] + right[1])
    return Hydro(x, u, rho, e, closure, bc_left=bc[0], bc_right=bc[1], **kw)


# ---------------------------------------------------------------------------
# exact ideal-gas Riemann problem
def _f_side(p, rho, pK, cK, g):
    """Velocity change across the left or right wave as a function of the star pressure,
    and its derivative."""
    if p > pK:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        sq = np.sqrt(A / (p + B))
        return (p - pK) * sq, sq * (1.0 - 0.5 * (p - pK) / (B + p))
    # rarefaction
    r = (p / pK) ** ((g - 1.0) / (2.0 * g))
    return 2.0 * cK / (g - 1.0) * (r - 1.0), 1.0 / (rho * cK) * (p / pK) ** (-(g + 1.0) / (2.0 * g))


def riemann_star(left, right, gamma=5.0 / 3.0, tol=1e-14, maxit=200):
    """Star-region pressure and velocity of the ideal-gas Riemann problem; left / right
    are (rho, u, p)."""
    rL, uL, pL = left
    rR, uR, pR = right
    g = gamma
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    if 2.0 * (cL + cR) / (g - 1.0) <= uR - uL:
        raise ValueError("vacuum is generated")
    # two-rarefaction guess (exact when both waves are rarefactions)
    z = (g - 1.0) / (2.0 * g)
    p = ((cL + cR - 0.5 * (g - 1.0) * (uR - uL)) / (cL / pL ** z + cR / pR ** z)) ** (1.0 / z)
    p = max(p, 1e-12 * min(pL, pR))
    for _ in range(maxit):
        fL, dL = _f_side(p, rL, pL, cL, g)
        fR, dR = _f_side(p, rR, pR, cR, g)
        pn = p - (fL + fR + uR - uL) / (dL + dR)
        pn = max(pn, 0.5 * p) if pn <= 0 else pn
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _f_side(p, rL, pL, cL, g)
    fR, _ = _f_side(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def riemann_sample(left, right, s, gamma=5.0 / 3.0):
    """(rho, u, p) at the similarity coordinates s = (x - x0) / t (array)."""
    g = gamma
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    ps, us = riemann_star(left, right, g)
    s = np.asarray(s, dtype=np.float64)
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    gm = (g - 1.0) / (g + 1.0)
    for k, S in enumerate(s.ravel()):
        if S <= us:   # left of the contact
            if ps > pL:
                SL = uL - cL * np.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                if S <= SL:
                    w = (rL, uL, pL)
                else:
                    w = (rL * (ps / pL + gm) / (gm * ps / pL + 1.0), us, ps)
            else:
                SH = uL - cL
                cs = cL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                ST = us - cs
                if S <= SH:
                    w = (rL, uL, pL)
                elif S >= ST:
                    w = (rL * (ps / pL) ** (1.0 / g), us, ps)
                else:
                    uf = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + S)
                    cf = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - S))
                    w = (rL * (cf / cL) ** (2.0 / (g - 1.0)), uf,
                         pL * (cf / cL) ** (2.0 * g / (g - 1.0)))
        else:         # right of the contact
            if ps > pR:
                SR = uR + cR * np.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                if S >= SR:
                    w = (rR, uR, pR)
                else:
                    w = (rR * (ps / pR + gm) / (gm * ps / pR + 1.0), us, ps)
            else:
                SH = uR + cR
                cs = cR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                ST = us + cs
                if S >= SH:
                    w = (rR, uR, pR)
                elif S <= ST:
                    w = (rR * (ps / pR) ** (1.0 / g), us, ps)
                else:
                    uf = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + S)
                    cf = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - S))
                    w = (rR * (cf / cR) ** (2.0 / (g - 1.0)), uf,
                         pR * (cf / cR) ** (2.0 * g / (g - 1.0)))
        rho.flat[k], u.flat[k], p.flat[k] = w
    return rho, u, p


# ---------------------------------------------------------------------------
# Rankine-Hugoniot states of a linear U_s - u_p material
def hugoniot_state(rho0, C, s, up, P0=0.0):
    """Shocked state reached from rest at (rho0, P0) with particle velocity jump up:
    U_s = C + s up, P = P0 + rho0 U_s up (momentum jump), rho = rho0 U_s / (U_s - up)
    (mass jump).  Returns (U_s, P, rho)."""
    Us = C + s * up
    return Us, P0 + rho0 * Us * up, rho0 * Us / (Us - up)


def plate_impact(rho0_flyer, rho0_target, C, s, u_impact, tol=1e-15):
    """Flyer at u_impact onto a target at rest, both the same linear U_s - u_p material
    (up to density): pressure and velocity match at the interface.  Solves
    rho0_t (C + s up) up = rho0_f (C + s (u_I - up)) (u_I - up) for up by bisection.
    Returns (up, P, rho_target_shocked, rho_flyer_shocked)."""
    def g(up):
        return (rho0_target * (C + s * up) * up
                - rho0_flyer * (C + s * (u_impact - up)) * (u_impact - up))
    a, b = 0.0, u_impact
    for _ in range(200):
        mid = 0.5 * (a + b)
        if g(mid) > 0.0:
            b = mid
        else:
            a = mid
        if b - a <= tol * u_impact:
            break
    up = 0.5 * (a + b)
    _, P, rho_t = hugoniot_state(rho0_target, C, s, up)
    _, _, rho_f = hugoniot_state(rho0_flyer, C, s, u_impact - up)
    return up, P, rho_t, rho_f
