// Single-box kernels for parity tests.  Each runs one box in one CTA (one
// group of 32 warps) through the same device functions as the batch kernel.
#include "mdeos_big.cuh"

namespace mdeos {

template <int APT>
__device__ void debug_lift_body(const Group& g, const BoxDesc& bd, const RunParams& rp, double T,
                                float4* x4, float4* v4, double* e_out) {
  const BoxCtx b = make_ctx(bd, rp);
  if (g.tid < 16) g.ctrl()[g.tid] = 0;
  lattice_own<APT>(g, bd);
  gbar(g.bar, g.nt);
  ForceAcc f0;
  if (bd.path == PATH_NLIST) {
    build_nlist<APT>(g, b);
    compute_forces<APT, PATH_NLIST, true, false, false>(g, b, rp, f0);
  } else if (bd.path == PATH_ALLPAIRS_MI) {
    compute_forces<APT, PATH_ALLPAIRS_MI, true, false, false>(g, b, rp, f0);
  } else {
    compute_forces<APT, PATH_ALLPAIRS, true, false, false>(g, b, rp, f0);
  }
  double et[1];
  const long long q[1] = {(long long)f0.e};
  group_sum<1>(g, q, et);
  init_velocities<APT>(g, b, bd.seed, T, rp);
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) {
      const float4 xi = g.x()[i];
      const int id = __float_as_int(xi.w);
      x4[id] = make_float4(xi.x, xi.y, xi.z, 0.f);
      v4[id] = g.v()[i];
    }
  }
  if (g.tid == 0) e_out[0] = et[0];
}

template <int APT, int PATH>
__device__ void debug_forces_body(const Group& g, const BoxDesc& bd, const RunParams& rp,
                                  const float4* x4, float4* f4, double* ew, long long* pairs) {
  const BoxCtx b = make_ctx(bd, rp);
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) {
      const float4 xi = x4[i];
      g.x()[i] = make_float4(xi.x, xi.y, xi.z, __int_as_float(i));
      g.v()[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (g.tid < 16) g.ctrl()[g.tid] = 0;
  gbar(g.bar, g.nt);
  if (PATH == PATH_NLIST) {
    // the list is built from wrapped positions (and may re-order the atoms);
    // forces use the positions as given
    wrap_own<APT>(g, b);
    build_nlist<APT>(g, b);
    for (int a = 0; a < APT; ++a) {
      const int i = g.tid + a * g.nt;
      if (i < b.n) {
        const float4 xo = g.x()[i];
        const float4 xi = x4[__float_as_int(xo.w)];
        g.x()[i] = make_float4(xi.x, xi.y, xi.z, xo.w);
      }
    }
    gbar(g.bar, g.nt);
  }
  ForceAcc fa;
  compute_forces<APT, PATH, true, true, true>(g, b, rp, fa);
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) f4[__float_as_int(g.x()[i].w)] = g.f()[i];
  }
  const long long q[8] = {(long long)fa.e,    (long long)fa.w[0], (long long)fa.w[1],
                          (long long)fa.w[2], (long long)fa.w[3], (long long)fa.w[4],
                          (long long)fa.w[5], (long long)fa.np * 4294967296LL};
  double out[8];
  group_sum<8>(g, q, out);
  if (g.tid == 0) {
    for (int k = 0; k < 7; ++k) ew[k] = out[k];
    if (pairs) pairs[0] = (long long)llrint(out[7]);
    if (g.ctrl()[CTRL_OVERFLOW]) ew[0] = __longlong_as_double(0x7ff8000000000001ll);
  }
}

template <int APT, int PATH>
__device__ void debug_md_body(const Group& g, const BoxDesc& bd, const RunParams& rp, float4* x4,
                              float4* v4, int steps, double T_target, int rescale_every,
                              double* epot, double* ekin, long long* cyc) {
  // cyc (optional): SM cycles seen by thread 0 in [drift, list build, forces,
  // kick + reductions] summed over the steps, the number of list builds, and
  // the build's phases [count, scan, scatter, cell sort, permute, search]
  long long c_drift = 0, c_build = 0, c_force = 0, c_red = 0, nbuild = 0;
  long long bph[6] = {0, 0, 0, 0, 0, 0};
  const BoxCtx b = make_ctx(bd, rp);
  const int n = b.n;
  const double ndof = 3.0 * n - 3.0;
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < n) {
      const float4 xi = x4[i], vi = v4[i];
      g.x()[i] = make_float4(xi.x, xi.y, xi.z, __int_as_float(i));
      g.v()[i] = make_float4(vi.x, vi.y, vi.z, 0.f);
    }
  }
  if (g.tid < 16) g.ctrl()[g.tid] = 0;
  gbar(g.bar, g.nt);
  if (PATH == PATH_NLIST) {
    wrap_own<APT>(g, b);
    build_nlist<APT>(g, b);
  }
  {
    ForceAcc f0;
    compute_forces<APT, PATH, false, false, false>(g, b, rp, f0);
  }
  gbar(g.bar, g.nt);  // every force loop has read the positions before any atom moves
  for (int s = 0; s < steps; ++s) {
    const long long t0 = clock64();
    const bool need = kick_drift<APT>(g, b, rp, 1.0f);
    bool rebuilt = false;
    if (PATH == PATH_NLIST) {
      rebuilt = gbar_or(g.bar, g.nt, need);
    } else {
      gbar(g.bar, g.nt);
    }
    const long long t1 = clock64();
    if (rebuilt) {
      wrap_own<APT>(g, b);
      build_nlist<APT>(g, b, cyc ? bph : nullptr);
    }
    const long long t2 = clock64();
    ForceAcc fa;
    compute_forces<APT, PATH, true, false, false>(g, b, rp, fa);
    const long long t3 = clock64();
    long long ke = 0;
    for (int a = 0; a < APT; ++a) {
      const int i = g.tid + a * g.nt;
      if (i < n) {
        const float4 fi = g.f()[i];
        float4 vi = g.v()[i];
        vi.x = fmaf(rp.hdtm, fi.x, vi.x);
        vi.y = fmaf(rp.hdtm, fi.y, vi.y);
        vi.z = fmaf(rp.hdtm, fi.z, vi.z);
        g.v()[i] = vi;
        ke += fxp(0.5f * rp.mass_f * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z));
      }
    }
    const long long q[2] = {(long long)fa.e, ke};
    double tot[2];
    group_sum<2>(g, q, tot);
    if (g.tid == 0) {
      if (epot) epot[s] = tot[0];
      if (ekin) ekin[s] = tot[1];
      const long long t4 = clock64();
      c_drift += t1 - t0;
      c_build += t2 - t1;
      c_force += t3 - t2;
      c_red += t4 - t3;
      nbuild += rebuilt ? 1 : 0;
    }
    if (rescale_every > 0 && (s + 1) % rescale_every == 0) {
      const float lam = (float)sqrt(T_target / (2.0 * tot[1] / ndof));
      for (int a = 0; a < APT; ++a) {
        const int i = g.tid + a * g.nt;
        if (i < n) {
          float4 vi = g.v()[i];
          vi.x *= lam;
          vi.y *= lam;
          vi.z *= lam;
          g.v()[i] = vi;
        }
      }
    }
  }
  wrap_own<APT>(g, b);
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < n) {
      const float4 xi = g.x()[i], vi = g.v()[i];
      const int id = __float_as_int(xi.w);
      x4[id] = make_float4(xi.x, xi.y, xi.z, 0.f);
      v4[id] = make_float4(vi.x, vi.y, vi.z, 0.f);
    }
  }
  if (cyc && g.tid == 0) {
    cyc[0] = c_drift;
    cyc[1] = c_build;
    cyc[2] = c_force;
    cyc[3] = c_red;
    cyc[4] = nbuild;
    for (int k = 0; k < 6; ++k) cyc[5 + k] = bph[k];
  }
}

__global__ void __launch_bounds__(kCtaThreads, 1)
    debug_lift_kernel(BoxDesc bd, RunParams rp, double T, int apt, int ncell_cap, float4* x4,
                      float4* v4, double* e_out, uint16_t* nl) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Group g = make_group(smem, threadIdx.x, 32, apt, ncell_cap, 1, nl);
  switch (apt) {
    case 1: debug_lift_body<1>(g, bd, rp, T, x4, v4, e_out); break;
    case 2: debug_lift_body<2>(g, bd, rp, T, x4, v4, e_out); break;
    default: debug_lift_body<4>(g, bd, rp, T, x4, v4, e_out); break;
  }
}

template <int APT>
__device__ void debug_forces_path(const Group& g, const BoxDesc& bd, const RunParams& rp,
                                  const float4* x4, float4* f4, double* ew, long long* pairs) {
  switch (bd.path) {
    case PATH_NLIST: debug_forces_body<APT, PATH_NLIST>(g, bd, rp, x4, f4, ew, pairs); break;
    case PATH_ALLPAIRS_MI:
      debug_forces_body<APT, PATH_ALLPAIRS_MI>(g, bd, rp, x4, f4, ew, pairs);
      break;
    default: debug_forces_body<APT, PATH_ALLPAIRS>(g, bd, rp, x4, f4, ew, pairs); break;
  }
}

__global__ void __launch_bounds__(kCtaThreads, 1)
    debug_forces_kernel(BoxDesc bd, RunParams rp, int apt, int ncell_cap, const float4* x4,
                        float4* f4, double* ew, long long* pairs, uint16_t* nl) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Group g = make_group(smem, threadIdx.x, 32, apt, ncell_cap, 1, nl);
  switch (apt) {
    case 1: debug_forces_path<1>(g, bd, rp, x4, f4, ew, pairs); break;
    case 2: debug_forces_path<2>(g, bd, rp, x4, f4, ew, pairs); break;
    default: debug_forces_path<4>(g, bd, rp, x4, f4, ew, pairs); break;
  }
}

template <int APT>
__device__ void debug_md_path(const Group& g, const BoxDesc& bd, const RunParams& rp, float4* x4,
                              float4* v4, int steps, double T, int every, double* ep, double* ek,
                              long long* cyc) {
  switch (bd.path) {
    case PATH_NLIST:
      debug_md_body<APT, PATH_NLIST>(g, bd, rp, x4, v4, steps, T, every, ep, ek, cyc);
      break;
    case PATH_ALLPAIRS_MI:
      debug_md_body<APT, PATH_ALLPAIRS_MI>(g, bd, rp, x4, v4, steps, T, every, ep, ek, cyc);
      break;
    default:
      debug_md_body<APT, PATH_ALLPAIRS>(g, bd, rp, x4, v4, steps, T, every, ep, ek, cyc);
      break;
  }
}

__global__ void __launch_bounds__(kCtaThreads, 1)
    debug_md_kernel(BoxDesc bd, RunParams rp, int apt, int ncell_cap, float4* x4, float4* v4,
                    int steps, double T, int every, double* ep, double* ek, long long* cyc,
                    uint16_t* nl) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Group g = make_group(smem, threadIdx.x, 32, apt, ncell_cap, 1, nl);
  switch (apt) {
    case 1: debug_md_path<1>(g, bd, rp, x4, v4, steps, T, every, ep, ek, cyc); break;
    case 2: debug_md_path<2>(g, bd, rp, x4, v4, steps, T, every, ep, ek, cyc); break;
    default: debug_md_path<4>(g, bd, rp, x4, v4, steps, T, every, ep, ek, cyc); break;
  }
}

// ---------------------------------------------------------------------------
// The pair-force pass on its own: one resident box per CTA (positions from x4 +
// blockIdx.x * n), the Verlet list built once, then `passes` force passes exactly
// as the step loop runs them (mode 0: forces only, in list-length order; 1: forces,
// energy, virial and pair count; 2: list builds instead of force passes).  cyc[2 b] = SM cycles of the passes, cyc[2 b + 1]
// = list entries (pair candidates) per pass of box b.

template <int APT>
__device__ void debug_force_bench_body(const Group& g, const BoxDesc& bd, const RunParams& rp,
                                       const float4* x4, int passes, int mode, long long* cyc) {
  const BoxCtx b = make_ctx(bd, rp);
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) {
      const float4 xi = x4[i];
      g.x()[i] = make_float4(xi.x, xi.y, xi.z, __int_as_float(i));
      g.v()[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (g.tid < 16) g.ctrl()[g.tid] = 0;
  gbar(g.bar, g.nt);
  wrap_own<APT>(g, b);
  build_nlist<APT>(g, b);
  long long cand[1] = {0};
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) cand[0] += (long long)list_entries(__float_as_int(g.f()[i].w), b.tpa) * 4294967296LL;
  }
  double ctot[1];
  group_sum<1>(g, cand, ctot);
  ForceAcc fa;
  const long long t0 = clock64();
  for (int p = 0; p < passes; ++p) {
    if (mode == 0) {
      compute_forces<APT, PATH_NLIST, false, false, false>(g, b, rp, fa);
    } else if (mode == 1) {
      compute_forces<APT, PATH_NLIST, true, true, true>(g, b, rp, fa);
      gbar(g.bar, g.nt);
    } else {  // the Verlet-list build on its own (positions unchanged)
      build_nlist<APT>(g, b);
    }
  }
  const long long t1 = clock64();
  if (g.tid == 0) {
    cyc[0] = t1 - t0;
    cyc[1] = (long long)ctot[0];
  }
  if (fa.e == 12345ull && fa.np == -1) cyc[0] = -1;  // keeps the sums live
}

__global__ void __launch_bounds__(kCtaThreads, 1)
    debug_force_bench_kernel(BoxDesc bd, RunParams rp, int apt, int ncell_cap, const float4* x4,
                             int passes, int mode, long long* cyc, uint16_t* nl,
                             long long nl_elems) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Group g = make_group(smem, threadIdx.x, 32, apt, ncell_cap, 1,
                             nl + (long long)blockIdx.x * nl_elems);
  const float4* xb = x4 + (size_t)blockIdx.x * bd.natoms;
  long long* cb = cyc + 2 * blockIdx.x;
  switch (apt) {
    case 1: debug_force_bench_body<1>(g, bd, rp, xb, passes, mode, cb); break;
    case 2: debug_force_bench_body<2>(g, bd, rp, xb, passes, mode, cb); break;
    default: debug_force_bench_body<4>(g, bd, rp, xb, passes, mode, cb); break;
  }
}

cudaError_t launch_debug_force_bench(const BoxDesc& bd, const RunParams& rp, int apt, int ncell_cap,
                                     int smem, const float4* x4, int nbox, int passes, int mode,
                                     long long* cyc, uint16_t* nl, long long nl_elems,
                                     cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(debug_force_bench_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  debug_force_bench_kernel<<<nbox, kCtaThreads, smem, st>>>(bd, rp, apt, ncell_cap, x4, passes,
                                                             mode, cyc, nl, nl_elems);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// boxes above the shared-memory limit (global-memory state, one CTA)

__global__ void __launch_bounds__(kCtaThreads, 1)
    debug_big_forces_kernel(BoxDesc bd, RunParams rp, unsigned char* scratch, const float4* x4,
                            float4* f4, double* ew, long long* pairs) {
  __shared__ BigShared sh;
  const BigCtx b = make_big_ctx(bd, rp);
  BigClu cl = big_clu(b.n, 0, 1);
  BigMem m = big_mem(scratch, b.n, b.nc * b.nc * b.nc, cl);
  extern __shared__ __align__(128) unsigned char dyn[];
  big_pos_cache(m, dyn, 0);  // position windows, as in the batch kernel
  if (threadIdx.x < 16) sh.ctrl[threadIdx.x] = 0;
  for (int s = threadIdx.x; s < b.n; s += blockDim.x) {
    const float4 xi = x4[s];
    m.x[s] = make_float4(xi.x, xi.y, xi.z, __int_as_float(s));
    m.v[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  big_wrap(m, b.L, b.invL);
  __syncthreads();
  big_build(m, &sh, cl, b.n, b.nc, b.L, b.cinv, b.rs2, b.maxnb);
  // forces use the positions as given (the list came from the wrapped ones)
  for (int s = threadIdx.x; s < b.n; s += blockDim.x) {
    const float4 xo = m.x[s];
    const float4 xi = x4[__float_as_int(xo.w)];
    m.x[s] = make_float4(xi.x, xi.y, xi.z, xo.w);
  }
  __syncthreads();
  const FSums r = big_forces(m, b, make_lj(rp), true, true);
  for (int s = threadIdx.x; s < b.n; s += blockDim.x) f4[__float_as_int(m.x[s].w)] = m.f[s];
  const long long q[8] = {(long long)r.e,  (long long)r.w0, (long long)r.w1, (long long)r.w2,
                          (long long)r.w3, (long long)r.w4, (long long)r.w5,
                          (long long)r.np * 4294967296LL};
  double out[8];
  block_sum<8>(&sh, cl, q, out);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 7; ++k) ew[k] = out[k];
    if (pairs) pairs[0] = (long long)llrint(out[7]);
    if (sh.ctrl[CTRL_OVERFLOW]) ew[0] = __longlong_as_double(0x7ff8000000000001ll);
  }
}

__global__ void __launch_bounds__(kCtaThreads, 1)
    debug_big_md_kernel(BoxDesc bd, RunParams rp, unsigned char* scratch, float4* x4, float4* v4,
                        int steps, double T_target, int rescale_every, double* epot,
                        double* ekin, long long* cyc) {
  __shared__ BigShared sh;
  extern __shared__ __align__(128) unsigned char dyn[];
  const BigCtx b = make_big_ctx(bd, rp);
  const LJ lj = make_lj(rp);
  BigClu cl = big_clu(b.n, 0, 1);
  BigMem m = big_mem(scratch, b.n, b.nc * b.nc * b.nc, cl);
  big_pos_cache(m, dyn, 0);  // position windows, as in the batch kernel
  const int n = b.n;
  const double ndof = 3.0 * n - 3.0;
  long long nbuild = 0;
  if (threadIdx.x < 16) sh.ctrl[threadIdx.x] = 0;
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    const float4 xi = x4[s], vi = v4[s];
    m.x[s] = make_float4(xi.x, xi.y, xi.z, __int_as_float(s));
    m.v[s] = make_float4(vi.x, vi.y, vi.z, 0.f);
  }
  __syncthreads();
  big_wrap(m, b.L, b.invL);
  __syncthreads();
  big_build(m, &sh, cl, n, b.nc, b.L, b.cinv, b.rs2, b.maxnb);
  big_forces(m, b, lj, false, false);
  __syncthreads();
  for (int st = 0; st < steps; ++st) {
    const bool need = big_kick_drift(m, b, rp, 1.0f);
    if (__syncthreads_or(need)) {
      big_wrap(m, b.L, b.invL);
      __syncthreads();
      big_build(m, &sh, cl, n, b.nc, b.L, b.cinv, b.rs2, b.maxnb);
      ++nbuild;
    }
    const FSums r = big_forces(m, b, lj, true, false);
    long long ke = 0;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
      const float4 fi = m.f[s];
      float4 vi = m.v[s];
      vi.x = fmaf(rp.hdtm, fi.x, vi.x);
      vi.y = fmaf(rp.hdtm, fi.y, vi.y);
      vi.z = fmaf(rp.hdtm, fi.z, vi.z);
      m.v[s] = vi;
      ke += fxp(0.5f * rp.mass_f * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z));
    }
    const long long q[2] = {(long long)r.e, ke};
    double tot[2];
    block_sum<2>(&sh, cl, q, tot);
    if (threadIdx.x == 0) {
      if (epot) epot[st] = tot[0];
      if (ekin) ekin[st] = tot[1];
    }
    if (rescale_every > 0 && (st + 1) % rescale_every == 0) {
      const float lam = (float)sqrt(T_target / (2.0 * tot[1] / ndof));
      for (int s = threadIdx.x; s < n; s += blockDim.x) {
        float4 vi = m.v[s];
        vi.x *= lam;
        vi.y *= lam;
        vi.z *= lam;
        m.v[s] = vi;
      }
    }
    __syncthreads();
  }
  big_wrap(m, b.L, b.invL);
  __syncthreads();
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    const float4 xi = m.x[s], vi = m.v[s];
    const int id = __float_as_int(xi.w);
    x4[id] = make_float4(xi.x, xi.y, xi.z, 0.f);
    v4[id] = make_float4(vi.x, vi.y, vi.z, 0.f);
  }
  if (cyc && threadIdx.x == 0) {
    for (int k = 0; k < 11; ++k) cyc[k] = 0;
    cyc[4] = nbuild;
  }
}

// dynamic shared memory for the big-box debug kernels: position windows of the
// whole box when it fits, else all that the device allows
static int g_debug_big_smem_max = 0;
static int debug_big_smem(int n) { return std::min(16 * big_cap(n), g_debug_big_smem_max); }

cudaError_t launch_debug_big_forces(const BoxDesc& bd, const RunParams& rp, unsigned char* scratch,
                                    const float4* x4, float4* f4, double* ew, long long* pairs,
                                    cudaStream_t st) {
  debug_big_forces_kernel<<<1, kCtaThreads, debug_big_smem(bd.natoms), st>>>(bd, rp, scratch, x4,
                                                                             f4, ew, pairs);
  return cudaGetLastError();
}

cudaError_t launch_debug_big_md(const BoxDesc& bd, const RunParams& rp, unsigned char* scratch,
                                float4* x4, float4* v4, int steps, double T, int every, double* ep,
                                double* ek, long long* cyc, cudaStream_t st) {
  debug_big_md_kernel<<<1, kCtaThreads, debug_big_smem(bd.natoms), st>>>(
      bd, rp, scratch, x4, v4, steps, T, every, ep, ek, cyc);
  return cudaGetLastError();
}

cudaError_t set_debug_attributes(int max_smem) {
  cudaError_t e;
  e = cudaFuncSetAttribute(debug_lift_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(debug_forces_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(debug_md_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (e != cudaSuccess) return e;
  // the big-box kernels also hold a static BigShared
  const int big_max = max_smem - (int)sizeof(BigShared);
  e = cudaFuncSetAttribute(debug_big_forces_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big_max);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(debug_big_md_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big_max);
  if (e == cudaSuccess) g_debug_big_smem_max = big_max;
  return e;
}

cudaError_t launch_debug_lift(const BoxDesc& bd, const RunParams& rp, double T, int apt,
                              int ncell_cap, int smem, float4* x4, float4* v4, double* e_out,
                              uint16_t* nl, cudaStream_t st) {
  debug_lift_kernel<<<1, kCtaThreads, smem, st>>>(bd, rp, T, apt, ncell_cap, x4, v4, e_out, nl);
  return cudaGetLastError();
}

cudaError_t launch_debug_forces(const BoxDesc& bd, const RunParams& rp, int apt, int ncell_cap,
                                int smem, const float4* x4, float4* f4, double* ew,
                                long long* pairs, uint16_t* nl, cudaStream_t st) {
  debug_forces_kernel<<<1, kCtaThreads, smem, st>>>(bd, rp, apt, ncell_cap, x4, f4, ew, pairs, nl);
  return cudaGetLastError();
}

cudaError_t launch_debug_md(const BoxDesc& bd, const RunParams& rp, int apt, int ncell_cap,
                            int smem, float4* x4, float4* v4, int steps, double T, int every,
                            double* ep, double* ek, long long* cyc, uint16_t* nl,
                            cudaStream_t st) {
  debug_md_kernel<<<1, kCtaThreads, smem, st>>>(bd, rp, apt, ncell_cap, x4, v4, steps, T, every,
                                                ep, ek, cyc, nl);
  return cudaGetLastError();
}

}  // namespace mdeos
