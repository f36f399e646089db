/*
 * mdeos_oracle.c -- plain, slow, obviously correct FP64 CPU reference of the
 * in-line atomistic EOS evaluation of arXiv 2508.06012 (Sec. III):
 *   lifting   : density -> FCC lattice (Eq. 6-7), energy -> temperature via
 *               E_cold and the two-update iteration (Eq. 8-10),
 *   evolution : velocity-Verlet with a velocity-rescale thermostat, LJ 12-6
 *               truncated-shifted pair potential,
 *   restriction: stress tensor (Eq. 11) and pressure = mean normal stress,
 *               time-averaged with block standard errors.
 *
 * TEST INFRASTRUCTURE ONLY: called from tests/, the smoke check and the CPU
 * baseline of bench.py; never from the product library.
 *
 * Readings of points the paper leaves open:
 *  - Eq. 6/7 conflict for alpha != 1; lattice constant a = (alpha/n)^(1/3)
 *    with alpha = 4 (FCC) and N = alpha * V / a^3.
 *  - N_DOF = 3N - 3 (total momentum removed).
 *  - "sample the new potential energy": mean of E_pot over the last 10% of
 *    the segment (at least one step).
 *  - the equilibration steps are split into lift_iters equal NVE segments
 *    (remainder to the last).  Segment k starts at T_k; after it, E_pot is
 *    sampled, T_{k+1} follows from Eq. 10 and velocities are rescaled to it.
 *    With lift_iters = 2 this is the paper's "two temperature update
 *    iterations"; production then runs NVT at T_2.
 *  - NVT production: velocity rescale to the last lifting temperature every
 *    rescale_every_avg steps; each averaging step is sampled before its
 *    rescale.
 *  - Eq. 11 with absolute positions is replaced by its periodic pair form
 *    W = sum_{i<j} r_ij (x) f_ij.
 */
#include "mdeos_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11.  Four 32-bit counter words, two key words, ten
 * rounds; each round multiplies words 0 and 2 by the Philox multipliers,
 * mixes hi halves with the other words and the round key, and the key is
 * bumped by the Weyl constants between rounds. */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;
static const uint32_t PHILOX_W1 = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------ */
/* Lifting of the density, Eq. 6-7 (reading: a = (4/n)^(1/3), N = 4 V/a^3).
 * The box holds N atoms at number density rho, so L = (N/rho)^(1/3).  The
 * first N sites of an nc^3-cell FCC lattice (nc the smallest integer with
 * 4 nc^3 >= N) are filled in (cell z, cell y, cell x, basis) order. */
int orc_lattice_fcc(int n, double rho, double* x, double* L_out) {
  if (n < 2 || !(rho > 0.0)) return ORC_EINVAL;
  int nc = 1;
  while (4LL * nc * nc * nc < n) ++nc;
  double L = cbrt((double)n / rho);
  double a = L / nc;
  static const double basis[4][3] = {{0, 0, 0}, {0.5, 0.5, 0}, {0.5, 0, 0.5}, {0, 0.5, 0.5}};
  int k = 0;
  for (int cz = 0; cz < nc && k < n; ++cz)
    for (int cy = 0; cy < nc && k < n; ++cy)
      for (int cx = 0; cx < nc && k < n; ++cx)
        for (int b = 0; b < 4 && k < n; ++b) {
          x[3 * k + 0] = a * (cx + basis[b][0]);
          x[3 * k + 1] = a * (cy + basis[b][1]);
          x[3 * k + 2] = a * (cz + basis[b][2]);
          ++k;
        }
  *L_out = L;
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
double orc_kinetic(int n, const double* v, double mass) {
  double s = 0.0;
  for (int i = 0; i < 3 * n; ++i) s += v[i] * v[i];
  return 0.5 * mass * s;
}

static double uniform_open(uint32_t r) { return ((double)r + 0.5) * (1.0 / 4294967296.0); }

/* Energy lifting, first guess (Eq. 9): Gaussian velocities drawn at T.
 * Atom i of a box with 64-bit seed s uses Philox key (lo(s), hi(s)) and
 * counter (i, 0, 0, 0); Box-Muller on (u0,u1) gives vx, vy and on (u2,u3)
 * gives vz.  Total momentum is removed, then velocities are scaled so that
 * 2 KE / N_DOF = T exactly. */
void orc_init_velocities(int n, uint64_t seed, double T, double mass, double* v) {
  const double two_pi = 6.283185307179586476925286766559;
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  double sd = sqrt(T / mass);
  for (int i = 0; i < n; ++i) {
    uint32_t ctr[4] = {(uint32_t)i, 0u, 0u, 0u}, r[4];
    orc_philox4x32_10(ctr, key, r);
    double u0 = uniform_open(r[0]), u1 = uniform_open(r[1]);
    double u2 = uniform_open(r[2]), u3 = uniform_open(r[3]);
    double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
    v[3 * i + 0] = sd * r01 * cos(two_pi * u1);
    v[3 * i + 1] = sd * r01 * sin(two_pi * u1);
    v[3 * i + 2] = sd * r23 * cos(two_pi * u3);
  }
  double p[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) p[d] += v[3 * i + d];
  for (int d = 0; d < 3; ++d) p[d] /= n;
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) v[3 * i + d] -= p[d];
  double ndof = 3.0 * n - 3.0;
  double Tinst = 2.0 * orc_kinetic(n, v, mass) / ndof;
  double lam = sqrt(T / Tinst);
  for (int i = 0; i < 3 * n; ++i) v[i] *= lam;
}

/* ------------------------------------------------------------------ */
/* Lennard-Jones 12-6, truncated and shifted at rc:
 *   u(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6] - u(rc)    (r < rc)
 *   f_ij = 24 eps [2 (sigma/r)^12 - (sigma/r)^6] / r^2 * r_ij
 * with r_ij = x_i - x_j taken over periodic images. */
typedef struct {
  double eps4, eps24, sig6, rc2, ucut;
} lj_consts;

static lj_consts lj_make(const orc_params* p) {
  lj_consts c;
  c.eps4 = 4.0 * p->eps;
  c.eps24 = 24.0 * p->eps;
  c.sig6 = pow(p->sigma, 6.0);
  c.rc2 = p->rc * p->rc;
  double s6 = c.sig6 / (c.rc2 * c.rc2 * c.rc2);
  c.ucut = c.eps4 * (s6 * s6 - s6);
  return c;
}

/* one pair term: adds forces on i (+) and j (-), returns the energy */
static double pair_term(const lj_consts* c, const double d[3], double r2, double* fi, double* fj,
                        double W[6]) {
  double ir2 = 1.0 / r2;
  double s6 = c->sig6 * ir2 * ir2 * ir2;
  double fr = c->eps24 * s6 * (2.0 * s6 - 1.0) * ir2;
  double fx = fr * d[0], fy = fr * d[1], fz = fr * d[2];
  fi[0] += fx; fi[1] += fy; fi[2] += fz;
  fj[0] -= fx; fj[1] -= fy; fj[2] -= fz;
  W[0] += d[0] * fx; W[1] += d[1] * fy; W[2] += d[2] * fz;
  W[3] += d[0] * fy; W[4] += d[0] * fz; W[5] += d[1] * fz;
  return c->eps4 * (s6 * s6 - s6) - c->ucut;
}

/* minimum-image displacement component in [-L/2, L/2] */
static double min_image(double d, double L) { return d - L * nearbyint(d / L); }

/* O(N^2) double loop over unordered pairs and every image within rc. */
static double forces_allpairs(int n, const double* x, double L, const lj_consts* c, double* f,
                              double W[6]) {
  double E = 0.0;
  for (int i = 0; i < n; ++i) {
    for (int j = i + 1; j < n; ++j) {
      double d0[3];
      for (int a = 0; a < 3; ++a) d0[a] = min_image(x[3 * i + a] - x[3 * j + a], L);
      /* with L >= rc only the images k in {-1,0,1}^3 can lie within rc;
       * with L >= 2 rc only the minimum image can (|d0| <= L/2 per axis) */
      int km = (L < 2.0 * sqrt(c->rc2)) ? 1 : 0;
      for (int kz = -km; kz <= km; ++kz)
        for (int ky = -km; ky <= km; ++ky)
          for (int kx = -km; kx <= km; ++kx) {
            double d[3] = {d0[0] + kx * L, d0[1] + ky * L, d0[2] + kz * L};
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < c->rc2) E += pair_term(c, d, r2, &f[3 * i], &f[3 * j], W);
          }
    }
  }
  return E;
}

/* Linked-cell variant for L >= 3 rc: cells of side >= rc, each unordered pair
 * visited once from its lower index through the 27 neighbouring cells. */
static double forces_cell(int n, const double* x, double L, const lj_consts* c, double rc,
                          double* f, double W[6]) {
  int nc = (int)floor(L / rc);
  if (nc < 3) return forces_allpairs(n, x, L, c, f, W);
  double cs = L / nc;
  int ncell = nc * nc * nc;
  int* head = (int*)malloc(sizeof(int) * ncell);
  int* next = (int*)malloc(sizeof(int) * n);
  int* cell_of = (int*)malloc(sizeof(int) * n);
  for (int k = 0; k < ncell; ++k) head[k] = -1;
  for (int i = n - 1; i >= 0; --i) {
    int ci[3];
    for (int a = 0; a < 3; ++a) {
      double w = x[3 * i + a] - L * floor(x[3 * i + a] / L);
      int q = (int)floor(w / cs);
      if (q < 0) q = 0;
      if (q >= nc) q = nc - 1;
      ci[a] = q;
    }
    int k = (ci[2] * nc + ci[1]) * nc + ci[0];
    cell_of[i] = k;
    next[i] = head[k];
    head[k] = i;
  }
  double E = 0.0;
  for (int i = 0; i < n; ++i) {
    int k = cell_of[i];
    int cx = k % nc, cy = (k / nc) % nc, cz = k / (nc * nc);
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int qx = (cx + dx + nc) % nc, qy = (cy + dy + nc) % nc, qz = (cz + dz + nc) % nc;
          for (int j = head[(qz * nc + qy) * nc + qx]; j >= 0; j = next[j]) {
            if (j <= i) continue;
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = min_image(x[3 * i + a] - x[3 * j + a], L);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 < c->rc2) E += pair_term(c, d, r2, &f[3 * i], &f[3 * j], W);
          }
        }
  }
  free(head);
  free(next);
  free(cell_of);
  return E;
}

double orc_lj_forces(int n, const double* x, double L, const orc_params* p, int mode, double* f,
                     double W[6]) {
  lj_consts c = lj_make(p);
  memset(f, 0, sizeof(double) * 3 * n);
  for (int a = 0; a < 6; ++a) W[a] = 0.0;
  if (mode == ORC_FORCE_CELL) return forces_cell(n, x, L, &c, p->rc, f, W);
  return forces_allpairs(n, x, L, &c, f, W);
}

long long orc_count_pairs(int n, const double* x, double L, double rc) {
  long long cnt = 0;
  double rc2 = rc * rc;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double d0[3];
      for (int a = 0; a < 3; ++a) d0[a] = min_image(x[3 * i + a] - x[3 * j + a], L);
      for (int kz = -1; kz <= 1; ++kz)
        for (int ky = -1; ky <= 1; ++ky)
          for (int kx = -1; kx <= 1; ++kx) {
            double d[3] = {d0[0] + kx * L, d0[1] + ky * L, d0[2] + kz * L};
            if (d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rc2) cnt += 2;
          }
    }
  return cnt;
}

/* ------------------------------------------------------------------ */
static void rescale_to(int n, double* v, double mass, double T_target) {
  double ndof = 3.0 * n - 3.0;
  double Tinst = 2.0 * orc_kinetic(n, v, mass) / ndof;
  double lam = sqrt(T_target / Tinst);
  for (int i = 0; i < 3 * n; ++i) v[i] *= lam;
}

/* One velocity-Verlet step: half kick, drift (wrapped into [0, L)), new
 * forces, half kick.  Returns the potential energy at the new positions. */
static double vv_step(int n, double* x, double* v, double* f, double L, const orc_params* p,
                      double W[6]) {
  double h = 0.5 * p->dt / p->mass;
  for (int i = 0; i < 3 * n; ++i) {
    v[i] += h * f[i];
    x[i] += p->dt * v[i];
    x[i] -= L * floor(x[i] / L);
    if (x[i] >= L) x[i] -= L;
  }
  double E = orc_lj_forces(n, x, L, p, p->force_mode, f, W);
  for (int i = 0; i < 3 * n; ++i) v[i] += h * f[i];
  return E;
}

int orc_md_steps(int n, double* x, double* v, double* f, double L, const orc_params* p, int steps,
                 double T_target, int rescale_every, double* epot_out, double* ekin_out) {
  double W[6];
  for (int s = 0; s < steps; ++s) {
    double E = vv_step(n, x, v, f, L, p, W);
    if (epot_out) epot_out[s] = E;
    if (ekin_out) ekin_out[s] = orc_kinetic(n, v, p->mass);
    if (rescale_every > 0 && (s + 1) % rescale_every == 0) rescale_to(n, v, p->mass, T_target);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
static int is_fin(double a) { return isfinite(a) ? 1 : 0; }

/* Lifting -> MD -> restriction.  Cold start (x_in == NULL): the FCC lattice of
 * Eq. 6-7 with Maxwell velocities at the Eq. 9 temperature and lift_iters
 * Eq. 10 segments.  Warm start (x_in != NULL, the previous final state of the
 * same element, box side L_in): positions scaled affinely by L / L_in, the
 * velocities kept, their mean removed and rescaled to the Eq. 10 temperature
 * of the scaled configuration, then warm_lift_iters Eq. 10 segments.  The
 * final state (positions in [0, L)) is written to x_out / v_out if given. */
static int eos_core(const orc_request* rq, const orc_params* p, const double* x_in,
                    const double* v_in, double L_in, double* x_out, double* v_out,
                    orc_result* out) {
  memset(out, 0, sizeof(*out));
  int n = rq->natoms;
  const int warm = x_in != NULL && v_in != NULL && L_in > 0.0;
  int nseg = warm ? p->warm_lift_iters : p->lift_iters;
  if (n < 2 || !(rq->rho > 0.0) || rq->steps_avg < 1 || p->se_blocks < 2 ||
      p->se_blocks > rq->steps_avg || nseg < 0 || rq->steps_equil < 0 ||
      (rq->steps_equil > 0 && rq->steps_equil < nseg) ||
      (rq->steps_equil > 0 && nseg == 0)) {
    out->status = ORC_EINVAL;
    return ORC_EINVAL;
  }
  double* x = (double*)malloc(sizeof(double) * 3 * n);
  double* v = (double*)malloc(sizeof(double) * 3 * n);
  double* f = (double*)malloc(sizeof(double) * 3 * n);
  double L;
  orc_lattice_fcc(n, rq->rho, x, &L);
  out->L = L;
  if (L < p->rc) {
    out->status = ORC_EBOX;
    free(x); free(v); free(f);
    return ORC_EBOX;
  }
  const double ndof = 3.0 * n - 3.0;
  const double V = L * L * L;
  const int temp_mode = (rq->flags & ORC_REQ_TEMPERATURE) != 0;
  double W[6];

  /* E_cold: potential energy of the lattice at rest (Sec. III). */
  double E_cold = orc_lj_forces(n, x, L, p, p->force_mode, f, W);
  out->e_cold = E_cold / n;
  double E_ref = (p->energy_ref_mode == ORC_REF_FIXED) ? n * rq->e_ref : E_cold;
  double E_tgt = n * rq->e + E_ref;

  /* Eq. 9 (or the given T) */
  double Tk = temp_mode ? rq->e : 2.0 * (E_tgt - E_cold) / ndof;
  int status = ORC_OK;
  if (!warm && (!(Tk > 0.0) || !is_fin(Tk))) status = ORC_EUNPHYS;
  if (warm) {
    /* warm start: affine scaling of the previous state, Eq. 10 temperature
     * of the scaled configuration */
    const double s = L / L_in;
    double vm[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) {
        double xi = x_in[3 * i + a] * s;
        xi -= L * floor(xi / L);
        if (xi >= L) xi -= L;
        x[3 * i + a] = xi;
        v[3 * i + a] = v_in[3 * i + a];
        vm[a] += v_in[3 * i + a];
      }
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) v[3 * i + a] -= vm[a] / n;
    double E0 = orc_lj_forces(n, x, L, p, p->force_mode, f, W);
    Tk = temp_mode ? rq->e : 2.0 * (E_tgt - E0) / ndof; /* Eq. 10 */
    if (!(Tk > 0.0) || !is_fin(Tk) || !is_fin(E0))
      status = ORC_EUNPHYS;
    else
      rescale_to(n, v, p->mass, Tk);
  } else if (status == ORC_OK) {
    orc_init_velocities(n, rq->seed, Tk, p->mass, v);
  }

  /* Equilibration: lift_iters NVE segments; after each, E_pot is sampled and
   * the temperature updated with Eq. 10, then velocities are rescaled to it.
   * After the last update the state is initialised (Sec. III). */
  if (status == ORC_OK && rq->steps_equil > 0) {
    int base = rq->steps_equil / nseg;
    for (int k = 0; k < nseg && status == ORC_OK; ++k) {
      int len = base + (k == nseg - 1 ? rq->steps_equil % nseg : 0);
      int nsamp = (len + 9) / 10;
      if (nsamp < 1) nsamp = 1;
      double acc = 0.0;
      for (int s = 0; s < len; ++s) {
        double E = vv_step(n, x, v, f, L, p, W);
        if (!is_fin(E)) { status = ORC_EUNPHYS; break; }
        if (s >= len - nsamp) acc += E;
        if (p->rescale_every_equil > 0 && (s + 1) % p->rescale_every_equil == 0)
          rescale_to(n, v, p->mass, Tk);
      }
      if (status != ORC_OK) break;
      double Ebar = acc / nsamp;
      Tk = temp_mode ? rq->e : 2.0 * (E_tgt - Ebar) / ndof; /* Eq. 10 */
      if (!(Tk > 0.0) || !is_fin(Tk)) { status = ORC_EUNPHYS; break; }
      rescale_to(n, v, p->mass, Tk);
    }
  }
  out->T_target = Tk;

  /* Production (NVT) with restriction (Eq. 11) and block averages. */
  if (status == ORC_OK) {
    int nb = p->se_blocks;
    double* serP = (double*)calloc(rq->steps_avg, sizeof(double)); /* per-step samples */
    double* serT = (double*)calloc(rq->steps_avg, sizeof(double));
    double sP = 0, sT = 0, sE = 0, sK = 0, sS[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < rq->steps_avg; ++s) {
      double E = vv_step(n, x, v, f, L, p, W);
      double K[6] = {0, 0, 0, 0, 0, 0};
      for (int i = 0; i < n; ++i) {
        const double* vi = &v[3 * i];
        K[0] += vi[0] * vi[0]; K[1] += vi[1] * vi[1]; K[2] += vi[2] * vi[2];
        K[3] += vi[0] * vi[1]; K[4] += vi[0] * vi[2]; K[5] += vi[1] * vi[2];
      }
      for (int a = 0; a < 6; ++a) K[a] *= p->mass;
      double KE = 0.5 * (K[0] + K[1] + K[2]);
      double Ps = (K[0] + K[1] + K[2] + W[0] + W[1] + W[2]) / (3.0 * V);
      double Ts = 2.0 * KE / ndof;
      if (!is_fin(E) || !is_fin(Ps) || !is_fin(Ts)) { status = ORC_EUNPHYS; break; }
      sP += Ps; sT += Ts; sE += E; sK += KE;
      for (int a = 0; a < 6; ++a) sS[a] += (K[a] + W[a]) / V;
      serP[s] = Ps;
      serT[s] = Ts;
      if (p->rescale_every_avg > 0 && (s + 1) % p->rescale_every_avg == 0)
        rescale_to(n, v, p->mass, Tk);
    }
    if (status == ORC_OK) {
      double m = rq->steps_avg;
      out->P = sP / m;
      out->T = sT / m;
      for (int a = 0; a < 6; ++a) out->sigma[a] = sS[a] / m;
      out->epot = sE / m / n;
      out->ekin = sK / m / n;
      out->e_achieved = (sK / m + sE / m - E_ref) / n;
      orc_block_se(serP, rq->steps_avg, nb, NULL, &out->P_se);
      orc_block_se(serT, rq->steps_avg, nb, NULL, &out->T_se);
    }
    free(serP); free(serT);
  }
  out->status = status;
  if (status == ORC_OK && x_out && v_out) {
    memcpy(x_out, x, sizeof(double) * 3 * n);
    memcpy(v_out, v, sizeof(double) * 3 * n);
  }
  free(x); free(v); free(f);
  return status;
}

/* Block-average standard error of the mean of a series x[0..m) (App. B averages
 * over the production steps; the error bar is the standard error of the mean
 * of nb equal-count blocks): block b holds steps s with floor(s nb / m) = b,
 * mean = (1/nb) sum_b xbar_b, se = sqrt(sum_b (xbar_b - mean)^2 / ((nb - 1) nb)).
 * For independent samples of variance s^2, E[se^2] = s^2 / m. */
int orc_block_se(const double* x, int m, int nb, double* mean_out, double* se_out) {
  if (x == NULL || m < 1 || nb < 2 || nb > m) return ORC_EINVAL;
  double* bs = (double*)calloc(nb, sizeof(double));
  int* bn = (int*)calloc(nb, sizeof(int));
  for (int s = 0; s < m; ++s) {
    int b = (int)((long long)s * nb / m);
    bs[b] += x[s];
    bn[b] += 1;
  }
  double mu = 0.0;
  for (int b = 0; b < nb; ++b) { bs[b] /= bn[b]; mu += bs[b]; }
  mu /= nb;
  double v = 0.0;
  for (int b = 0; b < nb; ++b) v += (bs[b] - mu) * (bs[b] - mu);
  if (mean_out) *mean_out = mu;
  if (se_out) *se_out = sqrt(v / (nb - 1) / nb);
  free(bs); free(bn);
  return ORC_OK;
}

int orc_eos_eval(const orc_request* rq, const orc_params* p, orc_result* out) {
  return eos_core(rq, p, NULL, NULL, 0.0, NULL, NULL, out);
}

int orc_eos_eval_state(const orc_request* rq, const orc_params* p, const double* x_in,
                       const double* v_in, double L_in, double* x_out, double* v_out,
                       orc_result* out) {
  return eos_core(rq, p, x_in, v_in, L_in, x_out, v_out, out);
}

int orc_eos_batch_state(const orc_request* rq, int n, const orc_params* p, const double* x_in,
                        const double* v_in, const double* L_in, double* x_out, double* v_out,
                        orc_result* out, int nthreads) {
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int i = 0; i < n; ++i) {
    const long long o = 3LL * rq[0].natoms * i;
    const int w = L_in != NULL && L_in[i] > 0.0;
    eos_core(&rq[i], p, w ? x_in + o : NULL, w ? v_in + o : NULL, w ? L_in[i] : 0.0,
             x_out ? x_out + o : NULL, v_out ? v_out + o : NULL, &out[i]);
  }
  (void)nthreads;
  return ORC_OK;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int orc_eos_batch(const orc_request* rq, int n, const orc_params* p, orc_result* out, int nthreads) {
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int i = 0; i < n; ++i) orc_eos_eval(&rq[i], p, &out[i]);
  (void)nthreads;
  return ORC_OK;
}
