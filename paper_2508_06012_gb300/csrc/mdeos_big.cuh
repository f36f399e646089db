// Boxes above the shared-memory limit (4097..32768 atoms): the same lifting ->
// MD -> restriction as run_box (Sec. III, Eq. 6-11), run by one whole CTA with
// the box state in global memory.
//
// Layout of a box's per-CTA scratch (16-byte aligned, `cap` = n rounded up to 32):
//   x, v, x2, v2, f   float4[cap] each (x.w = atom id, v.w = displacement bound,
//                     f.w = list length; x2/v2 receive the cell-ordered copy at a
//                     rebuild, then the two buffers swap roles)
//   cell counts, cell starts   int[ncell + 1] each
//   Verlet list       uint16 indices, 8 per 16-byte word, word kb of slot s at
//                     (kb * cap + s) * 16 bytes
// A rebuild sorts the atoms into cell order, so the 1024 atoms a CTA works on at
// once are spatial neighbours and their gathers stay in L1 (~100 KB of positions
// around a slab of cells).  FP64 appears only in the per-step leader-warp
// accumulation and the once-per-box lifting arithmetic, as in run_box.
#pragma once

#include "mdeos_device.cuh"

namespace mdeos {

// shared memory of a big-box CTA
constexpr int kMaxRounds = 16;  // force-pass rounds of a big box (position windows)

struct BigShared {
  long long red[32 * kRedSlots];
  double bc[8];
  double acc[kAccDoubles];
  int bcnt[kMaxSeBlocks];
  int ctrl[16];
  int scan[32];
  int wlo[kMaxRounds];  // first slot of each round's position window
  int wsz[kMaxRounds];  // its length in slots (cyclic over the box)
  int nround;           // rounds (0: no shared-memory positions)
  int rsz;              // slots per round (a multiple of the CTA's threads)
  int flag;             // a cluster-wide predicate, broadcast to the CTA
};

// A big box on a thread-block cluster of csize CTAs (csize 1: the whole box on one
// CTA).  The box state stays in one global scratch; CTA crank owns the slots
// [lo, hi), a contiguous part of the cell order (a slab of cells), and computes their
// lists, forces and updates; cells are dealt to the cluster's threads.  A CTA reads
// the slots of other CTAs from L2 only (its L1 never holds a line it did not write
// through its own slots), and phases meet at cluster barriers (release/acquire).  Box
// sums add the exact per-CTA partials in rank order, so every CTA holds the same
// integers and takes the same decisions, and every result equals the one-CTA run.
struct BigClu {
  int crank, csize;
  int lo, hi;     // the CTA's slots
  int seq;        // cluster exchanges so far (picks the partials' set)
  long long* clu;  // cluster partials, two alternating sets of kMaxCluster x kRedSlots
                   // (shared memory behind BigShared; only with csize > 1)
};

// shared memory of the cluster partials, behind BigShared (position windows follow)
constexpr int kBigCluBytes = 2 * kMaxCluster * kRedSlots * 8;

__device__ __forceinline__ BigClu big_clu(int n, int crank, int csize, long long* clu = nullptr) {
  BigClu c;
  c.crank = crank;
  c.csize = csize;
  c.lo = (int)((long long)n * crank / csize);
  c.hi = (int)((long long)n * (crank + 1) / csize);
  c.seq = 0;
  c.clu = clu;
  return c;
}

// barrier of the phases that read what other CTAs wrote
__device__ __forceinline__ void big_bar(const BigClu& cl) {
  if (cl.csize > 1)
    cluster_sync();
  else
    __syncthreads();
}

// loads of slots that other CTAs may have written: L2 only in a cluster
__device__ __forceinline__ float4 big_ld4(const float4* p, bool l2) { return l2 ? __ldcg(p) : *p; }
__device__ __forceinline__ int big_ldi(const int* p, bool l2) { return l2 ? __ldcg(p) : *p; }
__device__ __forceinline__ float big_ldw(const float4* p, bool l2) {
  return l2 ? __ldcg(reinterpret_cast<const float*>(p) + 3) : p->w;
}

// Cluster totals of per-CTA totals held by lanes k < NQ of warp 0 (called by every
// thread; the other lanes' values are ignored): every rank's partial goes into the
// same slot of every CTA, then each CTA adds them in rank order.  The two sets
// alternate, so a set is not written again before every CTA has passed the barrier
// of the exchange in between.
template <int NQ>
__device__ __forceinline__ unsigned long long big_cluster_total(BigShared* sh, BigClu& cl,
                                                                unsigned long long t) {
  if (cl.csize == 1) return t;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long* set = cl.clu + (cl.seq & 1) * (kMaxCluster * kRedSlots);
  if (warp == 0 && lane < NQ) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(set + cl.crank * kRedSlots + lane);
    for (int rk = 0; rk < cl.csize; ++rk) st_cluster_s64(cluster_map(a, rk), (long long)t);
  }
  cluster_sync();
  ++cl.seq;
  unsigned long long s = 0;
  if (warp == 0 && lane < NQ)
    for (int rk = 0; rk < cl.csize; ++rk) s += (unsigned long long)set[rk * kRedSlots + lane];
  return s;
}

// a predicate ORed over every thread of the cluster
__device__ __forceinline__ bool big_or(BigShared* sh, BigClu& cl, bool p) {
  const bool any = __syncthreads_or(p) != 0;
  if (cl.csize == 1) return any;
  const unsigned long long t = big_cluster_total<1>(sh, cl, any ? 1ull : 0ull);
  if (threadIdx.x == 0) sh->flag = t != 0;
  __syncthreads();
  return sh->flag != 0;
}

static_assert(sizeof(BigShared) <= kBigSharedBytes, "big-box shared memory");

struct BigMem {
  float4 *x, *v, *x2, *v2, *f;
  int *cnt, *start;
  uint4* nl;
  int cap;
  uint32_t sx_a;  // shared-memory position windows for the force pass (0: none)
  int sx_cap;     // their capacity in atoms
  int nround, rsz;           // force-pass rounds from the last build (0: none)
  const int *wlo, *wsz;      // their windows (shared memory)
  int lo, hi;                // this CTA's slots
  bool l2;                   // other CTAs write the box too: read their slots from L2
};

// Position windows in the dynamic shared memory from offset `off` on: address and
// capacity (in float4) of what the launch provides, at least 1024 atoms, else none.
__device__ __forceinline__ void big_pos_cache(BigMem& m, const unsigned char* dyn_base, int off) {
  uint32_t dyn;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
  const int cap = (int)(((long long)dyn - off) / 16);
  m.sx_a = cap >= 1024 ? (uint32_t)__cvta_generic_to_shared(dyn_base) + (uint32_t)off : 0u;
  m.sx_cap = cap >= 1024 ? cap : 0;
}

__device__ inline BigMem big_mem(unsigned char* p, int n, int ncell, const BigClu& cl) {
  BigMem m;
  m.lo = cl.lo;
  m.hi = cl.hi;
  m.l2 = cl.csize > 1;
  m.cap = big_cap(n);
  float4* q = reinterpret_cast<float4*>(p);
  m.x = q;
  m.v = q + m.cap;
  m.x2 = q + 2 * m.cap;
  m.v2 = q + 3 * m.cap;
  m.f = q + 4 * m.cap;
  unsigned char* c = p + (size_t)80 * m.cap;
  m.cnt = reinterpret_cast<int*>(c);
  m.start = m.cnt + ncell + 1;
  m.nl = reinterpret_cast<uint4*>(c + big_cells_bytes(ncell));
  m.sx_a = 0u;
  m.sx_cap = 0;
  m.nround = 0;
  m.rsz = n;
  m.wlo = m.wsz = nullptr;
  return m;
}

// Sum NQ per-thread fixed-point values (fxp units) over the CTA (and the cluster)
// exactly; every thread gets the totals as FP64 in real units.
template <int NQ>
__device__ void block_sum(BigShared* sh, BigClu& cl, const long long (&q)[NQ], double (&out)[NQ]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const long long s = warp_sum_ll(q[k]);
    if (lane == 0) sh->red[warp * kRedSlots + k] = s;
  }
  __syncthreads();
  unsigned long long s = 0;
  if (warp == 0 && lane < NQ)
    for (int w = 0; w < nw; ++w) s += (unsigned long long)sh->red[w * kRedSlots + lane];
  s = big_cluster_total<NQ>(sh, cl, s);
  if (warp == 0 && lane < NQ) sh->bc[lane] = (double)(long long)s * kFixInv;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NQ; ++k) out[k] = sh->bc[k];
}

// Lifted FCC lattice (Eq. 6-7), same site order as lattice_own; velocities zero.
__device__ inline void big_lattice(const BigMem& m, const BoxDesc& bd) {
  const int nc = bd.nc_lat;
  const double a = bd.L / nc;
  for (int i = m.lo + threadIdx.x; i < m.hi; i += blockDim.x) {
    const int c = i >> 2, bb = i & 3;
    const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
    const double bx = (bb == 1 || bb == 2) ? 0.5 : 0.0;
    const double by = (bb == 1 || bb == 3) ? 0.5 : 0.0;
    const double bz = (bb == 2 || bb == 3) ? 0.5 : 0.0;
    m.x[i] = make_float4((float)(a * (cx + bx)), (float)(a * (cy + by)), (float)(a * (cz + bz)),
                         __int_as_float(i));
    m.v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__device__ inline void big_wrap(const BigMem& m, float L, float invL) {
  for (int i = m.lo + threadIdx.x; i < m.hi; i += blockDim.x) {
    float4 xi = m.x[i];
    xi.x -= L * floorf(xi.x * invL);
    xi.y -= L * floorf(xi.y * invL);
    xi.z -= L * floorf(xi.z * invL);
    xi.x = fmaxf((xi.x >= L) ? xi.x - L : xi.x, 0.f);
    xi.y = fmaxf((xi.y >= L) ? xi.y - L : xi.y, 0.f);
    xi.z = fmaxf((xi.z >= L) ? xi.z - L : xi.z, 0.f);
    m.x[i] = xi;
    m.v[i].w = 0.f;
  }
}

// Verlet list from wrapped positions: counting sort into cell order (inside a
// cell by previous slot: deterministic), permutation of x and v into the second
// buffers (then swapped), 27-cell search with one image shift per cell.  In a
// cluster: cells are dealt to the cluster's threads, slots to their owners, the
// prefix sum over the cells is rank 0's, and each phase ends at a cluster barrier.
// Returns whether a list overflowed anywhere in the cluster.
static __device__ bool big_build(BigMem& m, BigShared* sh, BigClu& cl, int n, int nc, float L,
                                 float cinv, float rs2, int maxnb) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int gt = cl.crank * nt + tid, gn = cl.csize * nt;  // the thread among the cluster's
  const bool l2 = m.l2;
  const int ncell = nc * nc * nc;
  for (int c = gt; c < ncell; c += gn) m.cnt[c] = 0;
  big_bar(cl);
  for (int i = m.lo + tid; i < m.hi; i += nt) {
    const int c = cell_of(m.x[i], cinv, nc);
    m.f[i].x = __int_as_float(c);
    atomicAdd(&m.cnt[c], 1);
  }
  big_bar(cl);
  if (cl.crank == 0) {  // exclusive scan of the counts into starts; counts become cursors
    const int per = (ncell + nt - 1) / nt;
    const int lo = min(tid * per, ncell), hi = min(lo + per, ncell);
    int s = 0;
    for (int c = lo; c < hi; ++c) s += big_ldi(m.cnt + c, l2);
    const int lane = tid & 31, warp = tid >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) sh->scan[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      int v = lane < (nt >> 5) ? sh->scan[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      sh->scan[lane] = v;
    }
    __syncthreads();
    int off = (warp > 0 ? sh->scan[warp - 1] : 0) + incl - s;
    for (int c = lo; c < hi; ++c) {
      const int k = big_ldi(m.cnt + c, l2);
      m.start[c] = off;
      off += k;
      m.cnt[c] = 0;
    }
    if (tid == 0) m.start[ncell] = n;
  }
  big_bar(cl);
  for (int i = m.lo + tid; i < m.hi; i += nt) {
    const int c = __float_as_int(m.f[i].x);
    const int s = big_ldi(m.start + c, l2) + atomicAdd(&m.cnt[c], 1);
    reinterpret_cast<float*>(m.x2 + s)[3] = __int_as_float(i);
  }
  big_bar(cl);
  for (int c = gt; c < ncell; c += gn) {  // insertion sort of the previous slots
    const int lo = big_ldi(m.start + c, l2), hi = big_ldi(m.start + c + 1, l2);
    for (int a = lo + 1; a < hi; ++a) {
      const float key = big_ldw(m.x2 + a, l2);
      const int kk = __float_as_int(key);
      int b = a - 1;
      float wb;
      while (b >= lo && __float_as_int(wb = big_ldw(m.x2 + b, l2)) > kk) {
        reinterpret_cast<float*>(m.x2 + b + 1)[3] = wb;
        --b;
      }
      reinterpret_cast<float*>(m.x2 + b + 1)[3] = key;
    }
  }
  big_bar(cl);
  for (int s = m.lo + tid; s < m.hi; s += nt) {
    const int i = __float_as_int(big_ldw(m.x2 + s, l2));
    m.x2[s] = big_ld4(m.x + i, l2);
    const float4 vi = big_ld4(m.v + i, l2);
    m.v2[s] = make_float4(vi.x, vi.y, vi.z, 0.f);
  }
  big_bar(cl);
  {
    float4* t = m.x;
    m.x = m.x2;
    m.x2 = t;
    t = m.v;
    m.v = m.v2;
    m.v2 = t;
  }
  // Force-pass rounds over the CTA's slots: slots [lo + q rsz, lo + (q + 1) rsz) lie
  // in cell layers z0..z1 (cells are z-major), so their neighbours lie in layers
  // z0 - 1 .. z1 + 1 (cyclic; a neighbour across the y or x boundary can be anywhere in
  // its layer).  The slots of those whole layers (contiguous, cyclic over the box) are
  // the round's position window.  The fewest rounds whose windows all fit the shared
  // memory; none if even kMaxRounds do not.  List entries are stored relative to the
  // window start, so the pass indexes the window directly.
  const int own = m.hi - m.lo;
  if (tid == 0) {
    sh->nround = 0;
    sh->rsz = own;
    if (m.sx_cap > 0 && own > 0) {
      const int nc2 = nc * nc;
      for (int R = 1; R <= kMaxRounds; ++R) {
        const int rsz = ((own + R - 1) / R + nt - 1) / nt * nt;
        const int nr = (own + rsz - 1) / rsz;
        bool fits = true;
        for (int q = 0; q < nr && fits; ++q) {
          const int s0 = m.lo + q * rsz, s1 = min(m.hi, s0 + rsz) - 1;
          const int z0 = cell_of(m.x[s0], cinv, nc) / nc2, z1 = cell_of(m.x[s1], cinv, nc) / nc2;
          int lo = 0, sz = n;
          if (z1 - z0 + 3 < nc) {
            const int lz = (z0 - 1 + nc) % nc, hz = (z1 + 1) % nc;
            lo = big_ldi(m.start + lz * nc2, l2);
            const int hi = big_ldi(m.start + (hz + 1) * nc2, l2);
            sz = lz <= hz ? hi - lo : (n - lo) + hi;
          }
          fits = sz <= m.sx_cap;
          sh->wlo[q] = lo;
          sh->wsz[q] = sz;
        }
        if (fits) {
          sh->nround = nr;
          sh->rsz = rsz;
          break;
        }
      }
    }
  }
  __syncthreads();
  m.nround = sh->nround;
  m.rsz = sh->rsz;
  m.wlo = sh->wlo;
  m.wsz = sh->wsz;
  uint16_t* row = reinterpret_cast<uint16_t*>(m.nl);
  const size_t wstride = (size_t)m.cap * 8;  // uint16 entries between words of one slot
  // The search runs in the same rounds, candidates read from the round's window: a
  // cell's slots are contiguous in the window (the window's cyclic seam falls on a
  // cell boundary), so one offset per cell maps them.  A cell or slot outside its
  // window (impossible by construction) fails the box without any read.
  const bool win = m.nround > 0;
  for (int q = 0; q < (win ? m.nround : 1); ++q) {
    const int wl = win ? m.wlo[q] : 0, ws = win ? m.wsz[q] : n;
    const int sb = win ? m.lo + q * m.rsz : m.lo, se = win ? min(m.hi, sb + m.rsz) : m.hi;
    if (win) {
      float4* sx = reinterpret_cast<float4*>(__cvta_shared_to_generic(m.sx_a));
      for (int k = tid; k < ws; k += nt) {
        int g = wl + k;
        if (g >= n) g -= n;
        sx[k] = big_ld4(m.x + g, l2);
      }
      __syncthreads();
    }
    for (int s = sb + tid; s < se; s += nt) {
      int si = s - wl;
      if (si < 0) si += n;
      if (si >= ws) {
        atomicOr(&sh->ctrl[CTRL_OVERFLOW], 1);
        m.f[s].w = __int_as_float(0);
        continue;
      }
      const float4 xi = win ? ld_shared4(m.sx_a + 16u * (uint32_t)si) : m.x[s];
      const int cx = min((int)(xi.x * cinv), nc - 1);
      const int cy = min((int)(xi.y * cinv), nc - 1);
      const int cz = min((int)(xi.z * cinv), nc - 1);
      int k = 0;
      for (int dz = -1; dz <= 1; ++dz) {
        int zz = cz + dz;
        float sz = 0.f;
        if (zz < 0) { zz += nc; sz = -L; } else if (zz >= nc) { zz -= nc; sz = L; }
        for (int dy = -1; dy <= 1; ++dy) {
          int yy = cy + dy;
          float sy = 0.f;
          if (yy < 0) { yy += nc; sy = -L; } else if (yy >= nc) { yy -= nc; sy = L; }
          for (int dx = -1; dx <= 1; ++dx) {
            int xx = cx + dx;
            float sx_ = 0.f;
            if (xx < 0) { xx += nc; sx_ = -L; } else if (xx >= nc) { xx -= nc; sx_ = L; }
            const int c = (zz * nc + yy) * nc + xx;
            const int j0 = big_ldi(m.start + c, l2), j1 = big_ldi(m.start + c + 1, l2);
            int jb = j0 - wl;  // window index of the cell's first slot
            if (jb < 0) jb += n;
            if (jb + (j1 - j0) > ws) {
              atomicOr(&sh->ctrl[CTRL_OVERFLOW], 1);
              continue;
            }
            for (int j = j0; j < j1; ++j) {
              const int e = jb + (j - j0);  // window-relative slot (= j without windows)
              const float4 xj = win ? ld_shared4(m.sx_a + 16u * (uint32_t)e) : big_ld4(m.x + j, l2);
              const float ddx = xi.x - (xj.x + sx_), ddy = xi.y - (xj.y + sy), ddz = xi.z - (xj.z + sz);
              const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
              if (j != s && r2 < rs2) {
                if (k < maxnb) row[(size_t)(k >> 3) * wstride + (size_t)s * 8 + (k & 7)] = (uint16_t)e;
                ++k;
              }
            }
          }
        }
      }
      if (k > maxnb) atomicOr(&sh->ctrl[CTRL_OVERFLOW], 1);
      m.f[s].w = __int_as_float(min(k, maxnb));
    }
    if (win) __syncthreads();  // before the next window overwrites this one
  }
  __syncthreads();
  // a list overflow anywhere ends the box in every CTA alike
  const bool ovf = big_or(sh, cl, sh->ctrl[CTRL_OVERFLOW] != 0);
  if (tid == 0) sh->ctrl[CTRL_OVERFLOW] = ovf ? 1 : 0;
  __syncthreads();
  return ovf;
}

// Forces on every atom (strided over the CTA) from the Verlet list, minimum image
// on every entry; partial sums over the thread's atoms.  Out of line and fed
// scalars, like force_pass.  Positions come from the shared-memory copy at sx_a
// (SM) or from global memory with ordinary (L1-cached) loads: they were written by
// this CTA before the last barrier.
//
// SM: slots [s0, s1) of one round, positions from the round's window in shared
// memory (slot wl at index 0, cyclic over the n slots; list entries are window
// indices).  Otherwise all slots, positions and list entries as global slots.
template <bool EN, bool VIR, bool CNT, bool SM>
__device__ __noinline__ FSums big_force_pass(const float4* x, uint32_t sx_a, int s0, int s1,
                                             int wl, float4* f, const uint4* nl, int cap, int n,
                                             float L, float invL, bool l2, LJ c) {
  unsigned long long es = 0, ws[6] = {0, 0, 0, 0, 0, 0};
  int np = 0, bad = 0;
#pragma unroll 1
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    float e = 0.f;  // this atom's energy and virial over its list
    float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int si = s;  // the atom's own index in the position source
    if (SM) {
      si = s - wl;
      if (si < 0) si += n;
    }
    const float4 xi = SM ? ld_shared4(sx_a + 16u * (uint32_t)si) : x[s];
    const float cw = f[s].w;
    const int cn = __float_as_int(cw);
    const int nw = (cn + 7) >> 3;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    const uint4* p = nl + s;
    uint4 q = nw > 0 ? __ldcg(p) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll 1
    for (int kb = 0; kb < nw; ++kb) {
      const uint4 cur = q;
      if (kb + 1 < nw) q = __ldcg(p + (size_t)(kb + 1) * cap);
      const int left = cn - (kb << 3);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const unsigned wd = u < 2 ? cur.x : (u < 4 ? cur.y : (u < 6 ? cur.z : cur.w));
        const int jj = (int)((wd >> (16 * (u & 1))) & 0xffffu);
        const bool ok = u < left;
        const int jr = ok ? jj : si;
        const float4 xj = SM ? ld_shared4(sx_a + 16u * (uint32_t)jr) : big_ld4(x + jr, l2);
        const float dx = min_img(xi.x - xj.x, L, invL);
        const float dy = min_img(xi.y - xj.y, L, invL);
        const float dz = min_img(xi.z - xj.z, L, invL);
        lj_pair<EN, VIR>(dx, dy, dz, ok, c, fx, fy, fz, e, w, np);
      }
    }
    f[s] = make_float4(fx, fy, fz, cw);
    if (EN) {
      es += (unsigned long long)fxp(0.5f * e);
      bad |= !(fabsf(e) < 1e9f);
    }
    if (VIR) {
#pragma unroll
      for (int k = 0; k < 6; ++k) ws[k] += (unsigned long long)fxp(0.5f * w[k]);
      bad |= !(fabsf(w[0]) + fabsf(w[1]) + fabsf(w[2]) < 1e9f);
    }
  }
  FSums out = {es, ws[0], ws[1], ws[2], ws[3], ws[4], ws[5], CNT ? np : 0, bad};
  return out;
}

struct BigCtx {
  int n, nc, maxnb;
  float L, invL, half_skin, rs2, cinv;
};

__device__ inline BigCtx make_big_ctx(const BoxDesc& bd, const RunParams& rp) {
  BigCtx b;
  b.n = bd.natoms;
  b.nc = bd.nc_cell;
  b.maxnb = bd.maxnb;
  b.L = (float)bd.L;
  b.invL = (float)(1.0 / bd.L);
  b.half_skin = 0.5f * bd.skin;
  const float rs = rp.rc + bd.skin;
  b.rs2 = rs * rs;
  b.cinv = (float)(bd.nc_cell / bd.L);
  return b;
}

// Force pass.  With position windows from the last build: per round, the window's
// positions are copied into shared memory, a barrier, the round's slots, a barrier
// (before the next window overwrites it); per-thread sums add up over the rounds.
// Every caller has a barrier since the positions were last written.
template <bool EN, bool VIR, bool CNT>
__device__ __forceinline__ FSums big_forces_t(const BigMem& m, const BigCtx& b, const LJ& c) {
  if (m.nround == 0)
    return big_force_pass<EN, VIR, CNT, false>(m.x, 0u, m.lo, m.hi, 0, m.f, m.nl, m.cap, b.n, b.L,
                                               b.invL, m.l2, c);
  FSums t = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  float4* sx = reinterpret_cast<float4*>(__cvta_shared_to_generic(m.sx_a));
  for (int q = 0; q < m.nround; ++q) {
    const int wl = m.wlo[q], ws = m.wsz[q];
    for (int k = threadIdx.x; k < ws; k += blockDim.x) {
      int g = wl + k;
      if (g >= b.n) g -= b.n;
      sx[k] = big_ld4(m.x + g, m.l2);
    }
    __syncthreads();
    const int s0 = m.lo + q * m.rsz, s1 = min(m.hi, s0 + m.rsz);
    const FSums r = big_force_pass<EN, VIR, CNT, true>(m.x, m.sx_a, s0, s1, wl, m.f, m.nl, m.cap,
                                                       b.n, b.L, b.invL, m.l2, c);
    __syncthreads();
    t.e += r.e;
    t.w0 += r.w0;
    t.w1 += r.w1;
    t.w2 += r.w2;
    t.w3 += r.w3;
    t.w4 += r.w4;
    t.w5 += r.w5;
    t.np += r.np;
    t.bad |= r.bad;
  }
  return t;
}

__device__ __forceinline__ FSums big_forces(const BigMem& m, const BigCtx& b, const LJ& c, bool en,
                                            bool vir) {
  if (vir) return big_forces_t<true, true, true>(m, b, c);
  if (en) return big_forces_t<true, false, false>(m, b, c);
  return big_forces_t<false, false, false>(m, b, c);
}

// Maxwell velocities at T (Eq. 9): Philox keyed by the seed, counter = atom id,
// FP64 Box-Muller, mean removed, exact rescale to T; same arithmetic as
// init_velocities with the intermediate values kept in v instead of registers.
static __device__ void big_init_velocities(const BigMem& m, BigShared* sh, BigClu& cl, int n,
                                           unsigned long long seed, double T, const RunParams& rp) {
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffull), k1 = (uint32_t)(seed >> 32);
  const double sd = sqrt(T / rp.mass);
  const double two_m32 = 2.3283064365386962890625e-10;  // 2^-32
  long long p[3] = {0, 0, 0};
  for (int s = m.lo + threadIdx.x; s < m.hi; s += blockDim.x) {
    const uint32_t id = (uint32_t)__float_as_int(m.x[s].w);
    uint32_t c[4] = {id, 0u, 0u, 0u};
    philox4x32_10(c, k0, k1);
    const double u0 = ((double)c[0] + 0.5) * two_m32, u1 = ((double)c[1] + 0.5) * two_m32;
    const double u2 = ((double)c[2] + 0.5) * two_m32, u3 = ((double)c[3] + 0.5) * two_m32;
    const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
    double s1, c1, s3, c3;
    sincospi(2.0 * u1, &s1, &c1);
    sincospi(2.0 * u3, &s3, &c3);
    const float vx = (float)(sd * r01 * c1), vy = (float)(sd * r01 * s1), vz = (float)(sd * r23 * c3);
    m.v[s] = make_float4(vx, vy, vz, 0.f);
    p[0] += fxp(vx);
    p[1] += fxp(vy);
    p[2] += fxp(vz);
  }
  double ptot[3];
  block_sum<3>(sh, cl, p, ptot);
  const float mx = (float)(ptot[0] / n), my = (float)(ptot[1] / n), mz = (float)(ptot[2] / n);
  long long ke[1] = {0};
  for (int s = m.lo + threadIdx.x; s < m.hi; s += blockDim.x) {
    float4 vi = m.v[s];
    vi.x -= mx;
    vi.y -= my;
    vi.z -= mz;
    m.v[s] = vi;
    ke[0] += fxp(vi.x * vi.x + vi.y * vi.y + vi.z * vi.z);
  }
  double ketot[1];
  block_sum<1>(sh, cl, ke, ketot);
  const double Tinst = rp.mass * ketot[0] / (3.0 * n - 3.0);
  const float lam = (float)sqrt(T / Tinst);
  for (int s = m.lo + threadIdx.x; s < m.hi; s += blockDim.x) {
    const float4 vi = m.v[s];
    m.v[s] = make_float4(lam * vi.x, lam * vi.y, lam * vi.z, 0.f);
  }
  __syncthreads();
}

// first half kick with the pending thermostat factor, drift, displacement bound
__device__ __forceinline__ bool big_kick_drift(const BigMem& m, const BigCtx& b,
                                               const RunParams& rp, float lam) {
  bool need = false;
  for (int s = m.lo + threadIdx.x; s < m.hi; s += blockDim.x) {
    const float4 fi = m.f[s];
    float4 vi = m.v[s];
    vi.x = fmaf(lam, vi.x, rp.hdtm * fi.x);
    vi.y = fmaf(lam, vi.y, rp.hdtm * fi.y);
    vi.z = fmaf(lam, vi.z, rp.hdtm * fi.z);
    vi.w = fmaf(rp.dt, sqrtf(vi.x * vi.x + vi.y * vi.y + vi.z * vi.z), vi.w);
    m.v[s] = vi;
    float4 xi = m.x[s];
    xi.x = fmaf(rp.dt, vi.x, xi.x);
    xi.y = fmaf(rp.dt, vi.y, xi.y);
    xi.z = fmaf(rp.dt, vi.z, xi.z);
    m.x[s] = xi;
    need = need || (vi.w > b.half_skin);
  }
  return need;
}

// One big box, start to finish (same schedule and accumulation as run_box), on this
// CTA or on the csize CTAs of its thread-block cluster (rank crank; every CTA passes
// the scratch of the cluster's box, and all take the same path through it, so they
// meet at the same cluster barriers).  Rank 0 writes the result.
static __device__ __noinline__ void run_big(unsigned char* scratch, BigShared* sh, const BoxDesc& bd,
                                            const RunParams& rp, mdeos_result* out, int crank = 0,
                                            int csize = 1) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nt >> 5;
  const BigCtx b = make_big_ctx(bd, rp);
  const LJ lj = make_lj(rp);
  // in a cluster, the partials' sets follow BigShared; then the position windows in
  // the CTA's otherwise idle shared memory
  unsigned char* shb = reinterpret_cast<unsigned char*>(sh);
  BigClu cl = big_clu(b.n, crank, csize,
                      csize > 1 ? reinterpret_cast<long long*>(shb + kBigSharedBytes) : nullptr);
  BigMem m = big_mem(scratch, b.n, b.nc * b.nc * b.nc, cl);
  big_pos_cache(m, shb, kBigSharedBytes + (csize > 1 ? kBigCluBytes : 0));
  const int n = b.n;
  const double ndof = 3.0 * n - 3.0;
  const double V = bd.L * bd.L * bd.L;
  const bool temp_mode = (bd.flags & MDEOS_REQ_TEMPERATURE) != 0;
  double* acc = sh->acc;
  if (tid < 16) sh->ctrl[tid] = 0;
  for (int k = tid; k < kAccDoubles; k += nt) acc[k] = 0.0;
  for (int k = tid; k < kMaxSeBlocks; k += nt) sh->bcnt[k] = 0;
  big_lattice(m, bd);
  big_bar(cl);
  big_build(m, sh, cl, n, b.nc, b.L, b.cinv, b.rs2, b.maxnb);
  int builds = 1;
  double E_cold;
  {
    const FSums r = big_forces(m, b, lj, true, false);
    const long long q[1] = {(long long)r.e};
    double et[1];
    block_sum<1>(sh, cl, q, et);
    E_cold = et[0];
  }
  double* boxc = acc + ACC_BOX;
  const double E_ref = (rp.ref_mode == MDEOS_REF_FIXED) ? n * bd.e_ref : E_cold;
  const double E_tgt = n * bd.e + E_ref;
  double Tk = temp_mode ? bd.e : 2.0 * (E_tgt - E_cold) / ndof;  // Eq. 9
  int status = MDEOS_OK;
  if (!(Tk > 0.0) || !isfinite(Tk)) status = MDEOS_EUNPHYS;
  if (sh->ctrl[CTRL_OVERFLOW]) status = MDEOS_ENBR;
  if (tid == 0) {
    boxc[0] = E_cold;
    boxc[1] = E_ref;
    boxc[2] = E_tgt;
    boxc[3] = Tk;
  }
  const int nseg = (bd.steps_equil > 0) ? rp.lift_iters : 0;
  const int base = nseg > 0 ? bd.steps_equil / nseg : 0;
  int seg = 0, seg_pos = 0;
  int seg_len = (nseg == 1) ? bd.steps_equil : base;
  int nsamp = max(1, (seg_len + 9) / 10);
  const int total = bd.steps_equil + bd.steps_avg;
  const int nb = rp.se_blocks;
  if (status == MDEOS_OK) big_init_velocities(m, sh, cl, n, bd.seed, Tk, rp);
  const double invV = 1.0 / V, inv3V = 1.0 / (3.0 * V), inv_ndof = 1.0 / ndof;
  float lam = 1.0f;
  for (int step = 0; step < total && status == MDEOS_OK; ++step) {
    const bool avg = step >= bd.steps_equil;
    const int s_avg = step - bd.steps_equil;
    const bool seg_end = !avg && (seg_pos == seg_len - 1);
    const bool esamp = !avg && !temp_mode && (seg_pos >= seg_len - nsamp);
    const bool need = big_kick_drift(m, b, rp, lam);
    const bool rebuild = big_or(sh, cl, need);  // also publishes the new positions
    {
      // written by warp 0 last step (non-finite state): stop before a rebuild
      // bins such positions into cells
      const int st = sh->ctrl[CTRL_STATUS];
      if (st != 0 || sh->ctrl[CTRL_OVERFLOW] != 0) {
        status = st != 0 ? st : MDEOS_ENBR;
        break;
      }
    }
    if (rebuild) {
      big_wrap(m, b.L, b.invL);
      big_bar(cl);
      const bool ovf = big_build(m, sh, cl, n, b.nc, b.L, b.cinv, b.rs2, b.maxnb);
      ++builds;
      if (ovf) {
        status = MDEOS_ENBR;
        break;
      }
    }
    const FSums r = big_forces(m, b, lj, avg || esamp, avg);
    // second half kick; per-atom kinetic energy and kinetic stress into exact sums
    unsigned long long ke = 0, kt[6] = {0, 0, 0, 0, 0, 0};
    int cand = 0;
    bool bad = r.bad != 0;
    for (int s = m.lo + tid; s < m.hi; s += nt) {
      const float4 fi = m.f[s];
      float4 vi = m.v[s];
      vi.x = fmaf(rp.hdtm, fi.x, vi.x);
      vi.y = fmaf(rp.hdtm, fi.y, vi.y);
      vi.z = fmaf(rp.hdtm, fi.z, vi.z);
      m.v[s] = vi;
      const float ka = 0.5f * rp.mass_f * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z);
      bad |= !(ka < 1e9f);
      ke += (unsigned long long)fxp(ka);
      if (avg) {
        kt[0] += (unsigned long long)fxp(rp.mass_f * vi.x * vi.x);
        kt[1] += (unsigned long long)fxp(rp.mass_f * vi.y * vi.y);
        kt[2] += (unsigned long long)fxp(rp.mass_f * vi.z * vi.z);
        kt[3] += (unsigned long long)fxp(rp.mass_f * vi.x * vi.y);
        kt[4] += (unsigned long long)fxp(rp.mass_f * vi.x * vi.z);
        kt[5] += (unsigned long long)fxp(rp.mass_f * vi.y * vi.z);
        cand += __float_as_int(fi.w);
      }
    }
    {
      long long* red = sh->red + warp * kRedSlots;
      const long long s = warp_sum_ll((long long)ke);
      const bool any_bad = __any_sync(0xffffffffu, bad);
      if (lane == 0) {
        red[7] = s;
        red[10] = any_bad ? 1 : 0;
      }
      if (avg || esamp) {
        const long long se = warp_sum_ll((long long)r.e);
        if (lane == 0) red[6] = se;
      }
      if (avg) {
        const unsigned long long wv[6] = {r.w0, r.w1, r.w2, r.w3, r.w4, r.w5};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const long long sk = warp_sum_ll((long long)(kt[k] + wv[k]));
          if (lane == 0) red[k] = sk;
        }
        const long long sp = warp_sum_ll(r.np), sc = warp_sum_ll(cand);
        if (lane == 0) {
          red[8] = sp;
          red[9] = sc;
        }
      }
    }
    // thermostat steps and segment ends rescale the velocities
    const bool resc = seg_end ||
                      (!avg && rp.rescale_every_equil > 0 &&
                       (seg_pos + 1) % rp.rescale_every_equil == 0) ||
                      (avg && rp.rescale_every_avg > 0 && (s_avg + 1) % rp.rescale_every_avg == 0);
    __syncthreads();
    // box sums of the step: exact sums of the warp partials (lane k of warp 0 holds
    // quantity k), over the cluster's CTAs in rank order; the thermostat's kinetic
    // temperature comes from the same sum
    unsigned long long qsum = 0;
    if (warp == 0) qsum = (unsigned long long)warp_partials_ll(sh->red, nwarps, lane);
    qsum = big_cluster_total<kRedSlots>(sh, cl, qsum);
    if (warp == 0) {
      const long long qi = (long long)qsum;
      const double q = lane < 8 ? (double)qi * kFixInv : (double)qi;
      const double s0 = __shfl_sync(0xffffffffu, q, 0), s1 = __shfl_sync(0xffffffffu, q, 1);
      const double s2 = __shfl_sync(0xffffffffu, q, 2), k7 = __shfl_sync(0xffffffffu, q, 7);
      const double Ps = (s0 + s1 + s2) * inv3V;  // Eq. 11, mean normal stress
      const double Ts = 2.0 * k7 * inv_ndof;
      if ((lane == 7 && !(Ts > 0.0)) || (lane == 10 && qi != 0))
        sh->ctrl[CTRL_STATUS] = MDEOS_EUNPHYS;
      int slot = -1;
      double val = 0.0;
      if (avg) {
        const int blk = (int)(((long long)s_avg * nb) / bd.steps_avg);
        if (lane < 6) { slot = ACC_RUN + lane; val = q * invV; }
        else if (lane < 10) { slot = ACC_RUN + lane; val = q; }
        else if (lane == 10) { slot = ACC_RUN + 10; val = Ps; }
        else if (lane == 11) { slot = ACC_RUN + 11; val = Ts; }
        else if (lane == 12) { slot = ACC_BP + blk; val = Ps; sh->bcnt[blk] += 1; }
        else if (lane == 13) { slot = ACC_BT + blk; val = Ts; }
      } else if (esamp && lane == 6) {
        slot = ACC_RUN + 12;
        val = q;
      }
      if (slot >= 0) acc[slot] += val;
      double Tn = Tk;
      if (seg_end && lane == 6) {
        const double Ebar = acc[ACC_RUN + 12] / nsamp;
        Tn = temp_mode ? bd.e : 2.0 * (boxc[2] - Ebar) / ndof;  // Eq. 10
        sh->bc[0] = Tn;
        acc[ACC_RUN + 12] = 0.0;
      }
      // velocity-rescale factor towards the (new) target temperature
      if (resc) {
        Tn = __shfl_sync(0xffffffffu, Tn, 6);
        if (lane == 7)
          sh->bc[5] = (Tn > 0.0 && Ts > 0.0 && isfinite(Tn) && isfinite(Ts)) ? sqrt(Tn / Ts) : -1.0;
      }
    }
    // the rescale is applied with the next first half-kick
    lam = 1.0f;
    if (resc) {
      __syncthreads();
      const double lam_d = sh->bc[5];
      if (!(lam_d > 0.0)) {
        status = MDEOS_EUNPHYS;
        break;
      }
      if (seg_end) {
        Tk = sh->bc[0];
        if (tid == 0) boxc[3] = Tk;
      }
      lam = (float)lam_d;
    }
    if (seg_end) {
      ++seg;
      seg_pos = 0;
      seg_len = (seg == nseg - 1) ? base + bd.steps_equil % nseg : base;
      nsamp = max(1, (seg_len + 9) / 10);
    } else if (!avg) {
      ++seg_pos;
    }
  }
  __syncthreads();
  if (status == MDEOS_OK && sh->ctrl[CTRL_STATUS] != 0) status = sh->ctrl[CTRL_STATUS];
  if (tid == 0 && cl.crank == 0) {
    const double m_ = bd.steps_avg;
    mdeos_result res;
    for (int k = 0; k < 6; ++k) res.sigma[k] = acc[ACC_RUN + k] / m_;
    res.P = acc[ACC_RUN + 10] / m_;
    res.T = acc[ACC_RUN + 11] / m_;
    res.epot = acc[ACC_RUN + 6] / m_ / n;
    res.ekin = acc[ACC_RUN + 7] / m_ / n;
    res.e_achieved = (acc[ACC_RUN + 7] / m_ + acc[ACC_RUN + 6] / m_ - boxc[1]) / n;
    double mP = 0.0, mT = 0.0;
    for (int k = 0; k < nb; ++k) {
      const double c = sh->bcnt[k] > 0 ? (double)sh->bcnt[k] : 1.0;
      acc[ACC_BP + k] /= c;
      acc[ACC_BT + k] /= c;
      mP += acc[ACC_BP + k];
      mT += acc[ACC_BT + k];
    }
    mP /= nb;
    mT /= nb;
    double vP = 0.0, vT = 0.0;
    for (int k = 0; k < nb; ++k) {
      vP += (acc[ACC_BP + k] - mP) * (acc[ACC_BP + k] - mP);
      vT += (acc[ACC_BT + k] - mT) * (acc[ACC_BT + k] - mT);
    }
    res.P_se = sqrt(vP / (nb - 1) / nb);
    res.T_se = sqrt(vT / (nb - 1) / nb);
    res.T_target = boxc[3];
    res.e_cold = boxc[0] / n;
    res.L = bd.L;
    res.pairs_per_step = acc[ACC_RUN + 8] / m_;
    res.cand_per_step = acc[ACC_RUN + 9] / m_;
    res.element_id = bd.element_id;
    res.natoms = n;
    res.status = status;
    res.nlist_builds = builds;
    res.path = PATH_NLIST;
    res.warm = 0;
    res.nlist_retries = 0;
    if (status != MDEOS_OK) {
      res.P = res.T = res.epot = res.ekin = res.e_achieved = res.P_se = res.T_se = 0.0;
      for (int k = 0; k < 6; ++k) res.sigma[k] = 0.0;
    }
    *out = res;
  }
  big_bar(cl);  // no CTA leaves while another may still store into its shared memory
}

}  // namespace mdeos
