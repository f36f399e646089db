// 1D planar Lagrangian hydrodynamics (Euler equations, Eq. 2-4) on a staggered
// grid, closed by an ideal gas, the Mie-Grueneisen form of Eq. 1, or the batched
// atomistic EOS of this library (one request per zone and step, Sec. III).
//
// The hydro state is a few thousand zones: one CTA of 1024 threads runs a whole
// step (phases separated by __syncthreads), and the analytic closures run many
// steps per launch.  With the MD closure a step is one persistent EOS batch
// launch (milliseconds of MD per zone) followed by one hydro launch (~10 us).
//
// Arithmetic is FP64 in one fixed evaluation order per expression; this file is
// compiled with -fmad=false so no multiply-add is contracted, making every
// update the correctly rounded sequence of operations written here.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mdeos_host.h"

namespace mdeos {

enum { HY_ERR_STATE = 1, HY_ERR_EOS = 2, HY_ERR_DT = 3 };

struct HydroArgs {
  double *x, *u, *M, *m, *rho, *e, *P, *q, *c2, *Pq, *uh;
  double* clock;  // [0] time, [1] last dt, [2] steps, [3] previous dt (0 = none)
  int* err;
  const mdeos_result* md;
  int nz, bcl, bcr, set_e_from_md;
  double q2, q1, cfl, grow, dt_fixed;
  double gamma, rho0, C, s, G, sg;
};

constexpr int kHydroThreads = 1024;

// zone masses m = rho dx and node masses M_i = m_i / 2 + m_{i-1} / 2
__global__ void __launch_bounds__(kHydroThreads, 1) hydro_init_kernel(HydroArgs a) {
  const int nz = a.nz;
  for (int z = threadIdx.x; z < nz; z += blockDim.x) a.m[z] = a.rho[z] * (a.x[z + 1] - a.x[z]);
  __syncthreads();
  for (int i = threadIdx.x; i <= nz; i += blockDim.x) {
    double Mi = 0.0;
    if (i < nz) Mi = Mi + 0.5 * a.m[i];
    if (i > 0) Mi = Mi + 0.5 * a.m[i - 1];
    a.M[i] = Mi;
  }
  if (threadIdx.x == 0) {
    if (a.bcl == MDEOS_BC_WALL) a.u[0] = 0.0;
    if (a.bcr == MDEOS_BC_WALL) a.u[nz] = 0.0;
    a.clock[0] = a.clock[1] = a.clock[2] = a.clock[3] = 0.0;
    *a.err = 0;
  }
}

// closure P(rho, e) and the squared sound speed
template <int CL>
__device__ __forceinline__ void closure(const HydroArgs& a, int z, double rho, double e, double& P,
                                        double& c2) {
  if (CL == MDEOS_CLOSURE_IDEAL_GAS) {
    P = (a.gamma - 1.0) * rho * e;
    c2 = a.gamma * P / rho;
  } else if (CL == MDEOS_CLOSURE_MIE_GRUNEISEN) {
    // Eq. 1, reference curve = Hugoniot of U_s = C + s u_p from rest at e = 0
    const double rho0 = a.rho0, C = a.C, s = a.s, G = a.G;
    const double eta = 1.0 - rho0 / rho;
    const double den = 1.0 - s * eta;
    const double PH = rho0 * C * C * eta / (den * den);
    const double EH = PH * eta / (2.0 * rho0);
    P = PH + G * rho * (e - EH);
    const double dPH = rho0 * C * C * (1.0 + s * eta) / (den * den * den);
    const double dEH = (PH + eta * dPH) / (2.0 * rho0);
    const double deta = rho0 / (rho * rho);
    const double dPde = (dPH - G * rho * dEH) * deta + G * (e - EH);
    c2 = dPde + P / (rho * rho) * (G * rho);
  } else {
    // atomistic EOS result of this step's batch; sound speed estimate
    const mdeos_result& r = a.md[z];
    P = r.P;
    c2 = a.sg * fmax(P / rho, r.T);
  }
}

template <int CL>
__global__ void __launch_bounds__(kHydroThreads, 1) hydro_kernel(HydroArgs a, int nsteps) {
  __shared__ double s_min[kHydroThreads / 32];
  __shared__ int s_err;
  const int nz = a.nz;
  const int tid = threadIdx.x;
  for (int step = 0; step < nsteps; ++step) {
    if (tid == 0) s_err = *a.err;
    // phase A: closure, artificial viscosity, time-step bound per zone
    double lmin = INFINITY;
    int bad = 0;
    for (int z = tid; z < nz; z += kHydroThreads) {
      const double rho = a.rho[z];
      double e = a.e[z];
      if (CL == MDEOS_CLOSURE_MD) {
        if (a.md[z].status != MDEOS_OK) bad = HY_ERR_EOS;
        if (a.set_e_from_md) e = a.md[z].e_achieved;
      }
      double P, c2;
      closure<CL>(a, z, rho, e, P, c2);
      const double c = sqrt(c2);
      const double du = a.u[z + 1] - a.u[z];
      const double q = du < 0.0 ? rho * (a.q2 * du * du - a.q1 * c * du) : 0.0;
      const double dx = a.x[z + 1] - a.x[z];
      const double sig = c + 2.0 * a.q2 * fmax(-du, 0.0);
      lmin = fmin(lmin, dx / sig);
      if (!(rho > 0.0) || !(dx > 0.0) || !isfinite(P) || !(c2 >= 0.0) || !isfinite(e))
        bad = bad ? bad : HY_ERR_STATE;
      a.P[z] = P;
      a.q[z] = q;
      a.c2[z] = c2;
      a.Pq[z] = P + q;
      if (CL == MDEOS_CLOSURE_MD && a.set_e_from_md) a.e[z] = e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmin = fmin(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    bad = __reduce_max_sync(0xffffffffu, bad);
    __syncthreads();  // s_err read of the previous step done
    if ((tid & 31) == 0) {
      s_min[tid >> 5] = lmin;
      if (bad) atomicMax(&s_err, bad);
    }
    __syncthreads();
    double dt;
    {
      double mn = s_min[0];
      for (int w = 1; w < kHydroThreads / 32; ++w) mn = fmin(mn, s_min[w]);
      dt = a.cfl * mn;
      const double prev = a.clock[3];
      if (prev > 0.0) dt = fmin(dt, a.grow * prev);
      if (a.dt_fixed > 0.0) dt = a.dt_fixed;
    }
    if (!(dt > 0.0) || !isfinite(dt)) {
      if (tid == 0) atomicMax(&s_err, HY_ERR_DT);
    }
    __syncthreads();
    if (s_err != 0) {
      if (tid == 0) *a.err = s_err;
      return;  // state left at the last good step
    }
    // phase B: nodes -- momentum (Eq. 3), positions
    for (int i = tid; i <= nz; i += kHydroThreads) {
      const double left = (i > 0) ? a.Pq[i - 1] : 0.0;
      const double right = (i < nz) ? a.Pq[i] : 0.0;
      const double F = left - right;
      const double u0 = a.u[i];
      double un = u0 + dt * F / a.M[i];
      if ((i == 0 && a.bcl == MDEOS_BC_WALL) || (i == nz && a.bcr == MDEOS_BC_WALL)) un = 0.0;
      const double uh = 0.5 * (u0 + un);
      a.u[i] = un;
      a.uh[i] = uh;
      a.x[i] = a.x[i] + dt * uh;
    }
    __syncthreads();
    // phase C: zones -- energy (Eq. 4, compatible form) and density (Eq. 2)
    for (int z = tid; z < nz; z += kHydroThreads) {
      a.e[z] = a.e[z] - dt * a.Pq[z] * (a.uh[z + 1] - a.uh[z]) / a.m[z];
      a.rho[z] = a.m[z] / (a.x[z + 1] - a.x[z]);
    }
    if (tid == 0) {
      a.clock[0] = a.clock[0] + dt;
      a.clock[1] = dt;
      a.clock[2] = a.clock[2] + 1.0;
      a.clock[3] = dt;
    }
    __syncthreads();
    if (CL == MDEOS_CLOSURE_MD) break;  // one EOS batch per step
  }
}

}  // namespace mdeos

using namespace mdeos;

struct mdeos_hydro {
  mdeos_handle* h = nullptr;
  mdeos_hydro_config cfg;
  int nz = 0;
  double* d_mem = nullptr;
  int* d_err = nullptr;
  mdeos_result* d_res = nullptr;
  HydroArgs args;
  std::vector<double> e0;   // first-call energies (temperatures with first_temperature)
  std::vector<double> h_rho, h_e;
  std::vector<mdeos_request> reqs;
  int calls = 0;
};

extern "C" void mdeos_hydro_config_default(mdeos_hydro_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->bc_left = c->bc_right = MDEOS_BC_WALL;
  c->q_quad = 2.0;
  c->q_lin = 0.5;
  c->cfl = 0.5;
  c->dt_grow = 1.1;
  c->gamma = 5.0 / 3.0;
  c->sound_gamma = 3.0;
}

#define HCK(call)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return set_error(MDEOS_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

extern "C" mdeos_status mdeos_hydro_create(mdeos_handle* h, const mdeos_hydro_config* cfg,
                                           const double* x, const double* u, const double* rho,
                                           const double* e0, mdeos_hydro** out) {
  if (!h || !cfg || !x || !u || !rho || !e0 || !out)
    return set_error(MDEOS_EINVAL, "bad hydro_create arguments");
  *out = nullptr;
  const int nz = cfg->nzones;
  if (nz < 1 || nz > (1 << 24)) return set_error(MDEOS_EINVAL, "nzones out of range");
  if (cfg->closure < 0 || cfg->closure > 2) return set_error(MDEOS_EINVAL, "unknown closure");
  if ((cfg->bc_left != MDEOS_BC_WALL && cfg->bc_left != MDEOS_BC_FREE) ||
      (cfg->bc_right != MDEOS_BC_WALL && cfg->bc_right != MDEOS_BC_FREE))
    return set_error(MDEOS_EINVAL, "unknown boundary condition");
  if (!(cfg->q_quad >= 0) || !(cfg->q_lin >= 0) || !(cfg->cfl > 0) || !(cfg->dt_grow >= 1.0) ||
      !(cfg->dt_fixed >= 0))
    return set_error(MDEOS_EINVAL, "q, cfl, dt_grow or dt_fixed out of range");
  if (cfg->closure == MDEOS_CLOSURE_IDEAL_GAS && !(cfg->gamma > 1.0))
    return set_error(MDEOS_EINVAL, "gamma must be > 1");
  if (cfg->closure == MDEOS_CLOSURE_MIE_GRUNEISEN &&
      (!(cfg->mg_rho0 > 0) || !(cfg->mg_c > 0) || !(cfg->mg_s >= 0)))
    return set_error(MDEOS_EINVAL, "Mie-Grueneisen parameters out of range");
  if (cfg->closure == MDEOS_CLOSURE_MD &&
      (cfg->natoms < 2 || cfg->steps_avg < 1 || cfg->steps_avg_first < 1 || !(cfg->sound_gamma > 0)))
    return set_error(MDEOS_EINVAL, "MD closure: natoms, steps or sound_gamma out of range");
  for (int i = 0; i < nz; ++i)
    if (!(x[i + 1] > x[i]) || !(rho[i] > 0) || !std::isfinite(e0[i]))
      return set_error(MDEOS_EINVAL, "nodes must increase, densities be > 0, energies finite");
  mdeos_hydro* hy = new mdeos_hydro();
  hy->h = h;
  hy->cfg = *cfg;
  hy->nz = nz;
  cudaStream_t st = handle_stream(h);
  cudaError_t e = cudaSetDevice(handle_device(h));
  // device layout: x u M uh (nz+1 each) | m rho e P q c2 Pq (nz each) | clock[4]
  const size_t nn = (size_t)nz + 1, nzz = (size_t)nz;
  const size_t ndbl = 4 * nn + 7 * nzz + 4;
  if (e == cudaSuccess) e = cudaMalloc(&hy->d_mem, ndbl * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&hy->d_err, sizeof(int));
  if (e == cudaSuccess && cfg->closure == MDEOS_CLOSURE_MD)
    e = cudaMalloc(&hy->d_res, nzz * sizeof(mdeos_result));
  if (e != cudaSuccess) {
    mdeos_hydro_destroy(hy);
    return set_error(MDEOS_ECUDA, std::string("hydro allocation: ") + cudaGetErrorString(e));
  }
  double* p = hy->d_mem;
  HydroArgs& a = hy->args;
  std::memset(&a, 0, sizeof(a));
  a.x = p; p += nn;
  a.u = p; p += nn;
  a.M = p; p += nn;
  a.uh = p; p += nn;
  a.m = p; p += nzz;
  a.rho = p; p += nzz;
  a.e = p; p += nzz;
  a.P = p; p += nzz;
  a.q = p; p += nzz;
  a.c2 = p; p += nzz;
  a.Pq = p; p += nzz;
  a.clock = p;
  a.err = hy->d_err;
  a.md = hy->d_res;
  a.nz = nz;
  a.bcl = cfg->bc_left;
  a.bcr = cfg->bc_right;
  a.q2 = cfg->q_quad;
  a.q1 = cfg->q_lin;
  a.cfl = cfg->cfl;
  a.grow = cfg->dt_grow;
  a.dt_fixed = cfg->dt_fixed;
  a.gamma = cfg->gamma;
  a.rho0 = cfg->mg_rho0;
  a.C = cfg->mg_c;
  a.s = cfg->mg_s;
  a.G = cfg->mg_gamma;
  a.sg = cfg->sound_gamma;
  hy->e0.assign(e0, e0 + nz);
  const bool t_first = cfg->closure == MDEOS_CLOSURE_MD && cfg->first_temperature;
  e = cudaMemcpyAsync(a.x, x, nn * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(a.u, u, nn * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(a.rho, rho, nzz * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)  // temperatures are not energies: e is set by the first EOS call
    e = t_first ? cudaMemsetAsync(a.e, 0, nzz * sizeof(double), st)
                : cudaMemcpyAsync(a.e, e0, nzz * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    hydro_init_kernel<<<1, kHydroThreads, 0, st>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    mdeos_hydro_destroy(hy);
    return set_error(MDEOS_ECUDA, std::string("hydro init: ") + cudaGetErrorString(e));
  }
  count_launch(h, 1);
  hy->h_rho.resize(nz);
  hy->h_e.resize(nz);
  hy->reqs.resize(nz);
  *out = hy;
  return MDEOS_OK;
}

static mdeos_status hydro_status(mdeos_hydro* hy, cudaStream_t st) {
  int err = 0;
  HCK(cudaMemcpyAsync(&err, hy->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HCK(cudaStreamSynchronize(st));
  if (err == HY_ERR_EOS) return set_error(MDEOS_EUNPHYS, "an EOS box of the MD closure failed");
  if (err == HY_ERR_DT) return set_error(MDEOS_EUNPHYS, "hydro time step not positive/finite");
  if (err != 0) return set_error(MDEOS_EUNPHYS, "tangled mesh or non-finite hydro state");
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_hydro_step(mdeos_hydro* hy, int32_t nsteps) {
  if (!hy || nsteps < 0) return set_error(MDEOS_EINVAL, "bad hydro_step arguments");
  if (nsteps == 0) return MDEOS_OK;
  cudaStream_t st = handle_stream(hy->h);
  HCK(cudaSetDevice(handle_device(hy->h)));
  HydroArgs a = hy->args;
  const int cl = hy->cfg.closure;
  if (cl == MDEOS_CLOSURE_IDEAL_GAS) {
    hydro_kernel<MDEOS_CLOSURE_IDEAL_GAS><<<1, kHydroThreads, 0, st>>>(a, nsteps);
    HCK(cudaGetLastError());
    count_launch(hy->h, 1);
    return hydro_status(hy, st);
  }
  if (cl == MDEOS_CLOSURE_MIE_GRUNEISEN) {
    hydro_kernel<MDEOS_CLOSURE_MIE_GRUNEISEN><<<1, kHydroThreads, 0, st>>>(a, nsteps);
    HCK(cudaGetLastError());
    count_launch(hy->h, 1);
    return hydro_status(hy, st);
  }
  const mdeos_hydro_config& c = hy->cfg;
  const int nz = hy->nz;
  for (int k = 0; k < nsteps; ++k) {
    HCK(cudaMemcpyAsync(hy->h_rho.data(), a.rho, nz * sizeof(double), cudaMemcpyDeviceToHost, st));
    HCK(cudaMemcpyAsync(hy->h_e.data(), a.e, nz * sizeof(double), cudaMemcpyDeviceToHost, st));
    HCK(cudaStreamSynchronize(st));
    const bool first = hy->calls == 0;
    for (int z = 0; z < nz; ++z) {
      mdeos_request& r = hy->reqs[z];
      std::memset(&r, 0, sizeof(r));
      r.rho = hy->h_rho[z];
      r.e = (first && c.first_temperature) ? hy->e0[z] : hy->h_e[z];
      r.e_ref = c.e_ref;
      r.natoms = c.natoms;
      r.steps_equil = first ? c.steps_equil_first : c.steps_equil;
      r.steps_avg = first ? c.steps_avg_first : c.steps_avg;
      r.flags = (first && c.first_temperature) ? MDEOS_REQ_TEMPERATURE : 0u;
      r.seed = c.seed + ((uint64_t)hy->calls << 32) + (uint64_t)z;
      r.element_id = c.element_base + (uint64_t)z + 1;
    }
    mdeos_status s = eval_into_device(hy->h, hy->reqs.data(), nz, hy->d_res);
    if (s != MDEOS_OK) return s;
    a.set_e_from_md = (first && c.first_temperature) ? 1 : 0;
    hydro_kernel<MDEOS_CLOSURE_MD><<<1, kHydroThreads, 0, st>>>(a, 1);
    HCK(cudaGetLastError());
    count_launch(hy->h, 1);
    hy->calls += 1;
    s = hydro_status(hy, st);
    if (s != MDEOS_OK) return s;
  }
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_hydro_state(mdeos_hydro* hy, double* x, double* u, double* rho,
                                          double* e, double* P, double* q, double* c2,
                                          double* clock) {
  if (!hy) return set_error(MDEOS_EINVAL, "hydro is NULL");
  cudaStream_t st = handle_stream(hy->h);
  HCK(cudaSetDevice(handle_device(hy->h)));
  const size_t nn = (size_t)hy->nz + 1, nz = (size_t)hy->nz;
  const HydroArgs& a = hy->args;
  struct {
    double* dst;
    const double* src;
    size_t n;
  } cp[] = {{x, a.x, nn}, {u, a.u, nn}, {rho, a.rho, nz}, {e, a.e, nz},
            {P, a.P, nz}, {q, a.q, nz}, {c2, a.c2, nz}, {clock, a.clock, 3}};
  for (auto& c : cp)
    if (c.dst) HCK(cudaMemcpyAsync(c.dst, c.src, c.n * sizeof(double), cudaMemcpyDeviceToHost, st));
  HCK(cudaStreamSynchronize(st));
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_hydro_eos_results(mdeos_hydro* hy, mdeos_result* out) {
  if (!hy || !out) return set_error(MDEOS_EINVAL, "bad hydro_eos_results arguments");
  if (hy->cfg.closure != MDEOS_CLOSURE_MD || hy->calls == 0)
    return set_error(MDEOS_EINVAL, "no MD-closure batch has run");
  cudaStream_t st = handle_stream(hy->h);
  HCK(cudaSetDevice(handle_device(hy->h)));
  HCK(cudaMemcpyAsync(out, hy->d_res, (size_t)hy->nz * sizeof(mdeos_result),
                      cudaMemcpyDeviceToHost, st));
  HCK(cudaStreamSynchronize(st));
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_hydro_destroy(mdeos_hydro* hy) {
  if (!hy) return MDEOS_OK;
  if (hy->h) {
    cudaSetDevice(handle_device(hy->h));
    cudaStreamSynchronize(handle_stream(hy->h));
  }
  if (hy->d_mem) cudaFree(hy->d_mem);
  if (hy->d_err) cudaFree(hy->d_err);
  if (hy->d_res) cudaFree(hy->d_res);
  delete hy;
  return MDEOS_OK;
}
