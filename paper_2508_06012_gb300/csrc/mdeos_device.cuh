// Device code of the batched in-line atomistic EOS evaluation
// (arXiv 2508.06012, Sec. III: lifting Eq. 6-10, MD, restriction Eq. 11).
//
// Execution model (GB300, sm_103a):
//  * A group of warps runs one box start to finish: lattice, E_cold,
//    velocities, every MD step and the restriction.  Groups are synchronised
//    by a named barrier; several groups share a 1024-thread CTA.
//  * The box lives in shared memory for its whole run: positions, forces and
//    velocities as float4 (the force array doubles as the cell-sorted copy
//    while the Verlet list is rebuilt).  Thread t owns atoms t, t + nt, ...
//    for the whole run, so per-atom state needs no cross-thread exchange
//    except positions.
//  * Pair forces are FP32 (rcp.approx + FMA), each atom's sum over its list in
//    list order.  Box sums (energy, virial, kinetic energy and stress, momentum)
//    add per-atom FP32 values converted to 64-bit fixed point (2^-32 units):
//    integer sums are exact and independent of their order, so no result
//    depends on how many threads run a box or which thread holds which atom.
//    Time accumulation and the restriction are FP64.
//  * The Verlet list (uint16 atom indices, eight per 16-byte word, words laid
//    out so one warp load is contiguous) lives in global scratch.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mdeos_internal.h"

namespace mdeos {

// ---------------------------------------------------------------------------
// primitives

__device__ __forceinline__ void gbar(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Thread-block clusters: rank and size, the cluster-wide barrier (every thread of
// every CTA; release/acquire, so shared-memory stores into other CTAs before it are
// visible after it), and stores into another CTA's shared memory (mapa maps a local
// shared address to the same offset in CTA `rank`).
__device__ __forceinline__ int cluster_rank() {
  int r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ int cluster_size() {
  int r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
               ::: "memory");
}

__device__ __forceinline__ uint32_t cluster_map(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_cluster_v4(uint32_t a, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}

__device__ __forceinline__ void st_cluster_s64(uint32_t a, long long v) {
  asm volatile("st.shared::cluster.s64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_s32(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// barrier that also ORs a predicate over the participating threads
__device__ __forceinline__ bool gbar_or(int id, int n, bool p) {
  int r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\t"
      "setp.ne.s32 pi, %3, 0;\n\t"
      "bar.red.or.pred po, %1, %2, pi;\n\t"
      "selp.s32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"(id), "r"(n), "r"((int)p)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 64-bit fixed point of the box sums: v * 2^32 rounded to the nearest integer
// (exact for |v| >= 2^-9, where the scaled float is already an integer).  Values
// are kept below 2^30 in magnitude by the callers' finiteness checks.
constexpr float kFixScale = 4294967296.0f;         // 2^32
constexpr double kFixInv = 2.3283064365386963e-10;  // 2^-32
__device__ __forceinline__ long long fxp(float v) { return __float2ll_rn(v * kFixScale); }

// exact warp sum of 64-bit integers (two's complement wraps instead of overflow UB)
__device__ __forceinline__ long long warp_sum_ll(long long v) {
  unsigned long long u = (unsigned long long)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) u += (unsigned long long)__shfl_xor_sync(0xffffffffu, (long long)u, o);
  return (long long)u;
}

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the two-multiplier
// bijection, the key advanced by the Weyl increments between rounds.
__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t lo0 = m0 * c[0], hi0 = __umulhi(m0, c[0]);
    uint32_t lo1 = m1 * c[2], hi1 = __umulhi(m1, c[2]);
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// ---------------------------------------------------------------------------
// group of warps running one box; shared-memory layout as group_smem_bytes()

// FP64 accumulator slots (group shared memory)
enum { ACC_BP = 0, ACC_BT = kMaxSeBlocks, ACC_RUN = 2 * kMaxSeBlocks, ACC_BOX = 2 * kMaxSeBlocks + 16 };
// running sums at ACC_RUN + k: 0..5 stress / V, 6 E_pot, 7 E_kin, 8 in-cutoff pairs,
// 9 candidates, 10 P, 11 T, 12 lifting E_pot sample; box constants at ACC_BOX + 0..3
enum { CTRL_STATUS = 0, CTRL_OVERFLOW = 1, CTRL_WARM = 2 };

struct Group {
  unsigned char* base;
  uint16_t* nl;  // neighbour scratch: word (kb, i) at ((kb * npad + i) * 8) uint16 units
  int tid, nt, bar, npad, nwarps, off_red, off_clu;
  // thread-block cluster sharing the box (csize 1: none): every CTA holds the whole
  // box and advances it alike; CTA crank computes the forces and lists of its share
  // of the atoms and sends them to the others
  int crank, csize;
  __device__ __forceinline__ int warp() const { return tid >> 5; }
  __device__ __forceinline__ int lane() const { return tid & 31; }
  __device__ __forceinline__ float4* x() const { return reinterpret_cast<float4*>(base); }
  __device__ __forceinline__ float4* f() const { return reinterpret_cast<float4*>(base) + npad; }
  __device__ __forceinline__ float4* v() const { return reinterpret_cast<float4*>(base) + 2 * npad; }
  __device__ __forceinline__ int* cell() const {
    return reinterpret_cast<int*>(base + (size_t)48 * npad);
  }
  __device__ __forceinline__ long long* red() const {
    return reinterpret_cast<long long*>(base + off_red);
  }
  __device__ __forceinline__ double* bc() const {
    return reinterpret_cast<double*>(base + off_red + nwarps * kRedSlots * 8);
  }
  __device__ __forceinline__ double* acc() const { return bc() + 8; }
  __device__ __forceinline__ int* bcnt() const { return reinterpret_cast<int*>(acc() + kAccDoubles); }
  __device__ __forceinline__ int* ctrl() const { return bcnt() + kMaxSeBlocks; }
  __device__ __forceinline__ long long* clu() const {
    return reinterpret_cast<long long*>(base + off_clu);
  }
};

__device__ inline Group make_group(unsigned char* base, int tid, int warps, int apt, int ncell_cap,
                                   int bar, uint16_t* nl) {
  Group g;
  g.base = base;
  g.nl = nl;
  g.tid = tid;
  g.nt = warps * 32;
  g.bar = bar;
  g.npad = warps * 32 * apt;
  g.nwarps = warps;
  g.off_red = group_red_offset(warps, apt, ncell_cap);
  g.off_clu = group_cluster_offset(warps, apt, ncell_cap);
  g.crank = 0;
  g.csize = 1;
  return g;
}

// Sum NQ per-thread fixed-point values (fxp units) over the group exactly; every
// thread gets the totals as FP64 in real units.
template <int NQ>
__device__ void group_sum(const Group& g, const long long (&q)[NQ], double (&out)[NQ]) {
#pragma unroll
  for (int k = 0; k < NQ; ++k) {
    const long long s = warp_sum_ll(q[k]);
    if (g.lane() == 0) g.red()[g.warp() * kRedSlots + k] = s;
  }
  gbar(g.bar, g.nt);
  if (g.warp() == 0 && g.lane() < NQ) {
    unsigned long long s = 0;
    for (int w = 0; w < g.nwarps; ++w) s += (unsigned long long)g.red()[w * kRedSlots + g.lane()];
    g.bc()[g.lane()] = (double)(long long)s * kFixInv;
  }
  gbar(g.bar, g.nt);
#pragma unroll
  for (int k = 0; k < NQ; ++k) out[k] = g.bc()[k];
}

// Leader-warp combination of one step's per-warp partials (red[w * kRedSlots + k],
// k < kRedSlots): lane k returns the exact sum over warps of quantity k.
__device__ __forceinline__ long long warp_partials_ll(const long long* red, int nwarps, int lane) {
  unsigned long long s = 0;
  if (lane < kRedSlots)
    for (int w = 0; w < nwarps; ++w) s += (unsigned long long)red[w * kRedSlots + lane];
  return (long long)s;
}

// Per-box constants in registers.
struct BoxCtx {
  int n, maxnb, nc;
  int tpa;  // threads per atom of the list passes (brute_tpa for lists without cells)
  float L, invL, half_skin, rcs2, cinv;
};

__device__ inline BoxCtx make_ctx(const BoxDesc& bd, const RunParams& rp) {
  BoxCtx b;
  b.n = bd.natoms;
  b.maxnb = bd.maxnb;
  b.nc = bd.nc_cell;
  b.tpa = (bd.path == PATH_NLIST && bd.nc_cell == 0) ? brute_tpa(bd.natoms) : 1;
  b.L = (float)bd.L;
  b.invL = (float)(1.0 / bd.L);
  b.half_skin = 0.5f * bd.skin;
  float rs = rp.rc + bd.skin;
  b.rcs2 = rs * rs;
  b.cinv = bd.nc_cell > 0 ? (float)(bd.nc_cell / bd.L) : 0.f;
  return b;
}

// ---------------------------------------------------------------------------
// Lennard-Jones 12-6 pair term, truncated and shifted:
//   u(r) = 4 eps [(s/r)^12 - (s/r)^6] - u(rc),
//   f_ij = 24 eps [2 (s/r)^12 - (s/r)^6] / r^2 * r_ij
// `ok` masks the term (the atom itself, padding).

// pair constants, passed by value into the force pass
struct LJ {
  float rc2, eps4, eps24, eps48, sig6, ucut;
};

__device__ __forceinline__ LJ make_lj(const RunParams& rp) {
  LJ c;
  c.rc2 = rp.rc2;
  c.eps4 = rp.eps4;
  c.eps24 = rp.eps24;
  c.eps48 = 2.0f * rp.eps24;
  c.sig6 = rp.sig6;
  c.ucut = rp.ucut;
  return c;
}

template <bool EN, bool VIR>
__device__ __forceinline__ void lj_pair(float dx, float dy, float dz, bool ok, const LJ& c,
                                        float& fx, float& fy, float& fz, float& e, float (&w)[6],
                                        int& npair) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float ir2 = rcp_approx(r2);
  const float s6 = c.sig6 * ir2 * ir2 * ir2;
  const float fr = s6 * fmaf(c.eps48, s6, -c.eps24) * ir2;  // 24 eps s6 (2 s6 - 1) / r^2
  // outside the cutoff (or a masked entry, whose r^2 may be 0 and fr not finite)
  // nothing is accumulated: the sums are predicated, not multiplied by a zero
  if (ok && r2 < c.rc2) {
    fx = fmaf(fr, dx, fx);
    fy = fmaf(fr, dy, fy);
    fz = fmaf(fr, dz, fz);
    if (EN) e += fmaf(c.eps4 * s6, s6 - 1.0f, -c.ucut);
    if (VIR) {
      const float tx = fr * dx, ty = fr * dy, tz = fr * dz;
      w[0] = fmaf(tx, dx, w[0]);
      w[1] = fmaf(ty, dy, w[1]);
      w[2] = fmaf(tz, dz, w[2]);
      w[3] = fmaf(tx, dy, w[3]);
      w[4] = fmaf(tx, dz, w[4]);
      w[5] = fmaf(ty, dz, w[5]);
    }
    ++npair;
  }
}

// 16-byte shared-memory load from a 32-bit shared address (the force pass is not
// inlined, so its pointers would otherwise be generic)
__device__ __forceinline__ float4 ld_shared4(uint32_t a) {
  float4 v;
  asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "r"(a));
  return v;
}

// Minimum image of a coordinate difference, d - L k with k the integer nearest to
// d / L, on the FP32 pipe (no conversion instructions): one fused multiply-add adds
// 1.5 * 2^23 to the exact product d * invL, which leaves no fraction bits for
// |d * invL| < 2^22, and subtracting the constant again gives k (ties to even).  Only
// where d is within rounding of +-L/2 can k differ from rintf(d * invL); such a pair
// is beyond the cutoff on every path that uses one image (L >= 2 rc).
__device__ __forceinline__ float min_img(float d, float L, float invL) {
  const float magic = 12582912.0f;
  const float k = __fsub_rn(__fmaf_rn(d, invL, magic), magic);
  return fmaf(-L, k, d);
}

// Verlet-list pair from a home position already shifted to the entry's image
template <bool EN, bool VIR>
__device__ __forceinline__ void nl_pair_sh(uint32_t xs_a, int j, bool ok, float hx, float hy,
                                           float hz, const LJ& c, float& fx, float& fy, float& fz,
                                           float& e, float (&w)[6], int& np) {
  const float4 xj = ld_shared4(xs_a + 16u * (uint32_t)j);
  lj_pair<EN, VIR>(hx - xj.x, hy - xj.y, hz - xj.z, ok, c, fx, fy, fz, e, w, np);
}

// Verlet-list pair: minimum image across the periodic box; `ok` masks padding
template <bool EN, bool VIR>
__device__ __forceinline__ void nl_pair_bd(uint32_t xs_a, int j, bool ok, const float4& xi,
                                           float L, float invL, const LJ& c, float& fx, float& fy,
                                           float& fz, float& e, float (&w)[6], int& np) {
  const float4 xj = ld_shared4(xs_a + 16u * (uint32_t)j);
  const float dx = min_img(xi.x - xj.x, L, invL);
  const float dy = min_img(xi.y - xj.y, L, invL);
  const float dz = min_img(xi.z - xj.z, L, invL);
  lj_pair<EN, VIR>(dx, dy, dz, ok, c, fx, fy, fz, e, w, np);
}

__device__ __forceinline__ void st_shared_u16(uint32_t a, int v) {
  asm volatile("st.shared.u16 [%0], %1;" ::"r"(a), "h"((unsigned short)v) : "memory");
}

__device__ __forceinline__ uint4 ld_shared_u4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a)
               : "memory");
  return v;
}

__device__ __forceinline__ int ld_shared_u16(uint32_t a) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return (int)v;
}

// List words of boxes searched without cells: `tpa` sub-lists per atom (sub-list p
// holds the neighbours among slots p, p + tpa, p + 2 tpa, ...: slots of these boxes
// keep their lattice order, so interleaved slots give every sub-list about the same
// share of an atom's neighbours), sub-list p of slot i being unit u = i tpa + p with
// word kb at kb * npad * tpa + u.
// The slot's list word packs the entry counts of its sub-lists (8 bits each for 4,
// 16 bits each for 2).
__device__ __forceinline__ int sub_entries(int meta, int tpa, int p) {
  return tpa == 4 ? (meta >> (8 * p)) & 0xff : (tpa == 2 ? (meta >> (16 * p)) & 0xffff
                                                         : (int)((unsigned)meta >> 16));
}

// list entries of a slot (without padding), from its list word
__device__ __forceinline__ int list_entries(int meta, int tpa) {
  if (tpa == 1) return (int)((unsigned)meta >> 16);
  int k = 0;
  for (int p = 0; p < tpa; ++p) k += sub_entries(meta, tpa, p);
  return k;
}

// lanes of the tpa-group of the calling lane (tpa consecutive lanes, one atom)
__device__ __forceinline__ unsigned tpa_mask(int tpa) {
  const int lane = threadIdx.x & 31;
  return (tpa >= 32 ? 0xffffffffu : ((1u << tpa) - 1u)) << (lane & ~(tpa - 1));
}

// per-thread partial sums of one force pass: energy and virial in fxp units
// (already halved: each pair appears in two atoms' lists), wrapping integer adds
struct FSums {
  unsigned long long e, w0, w1, w2, w3, w4, w5;
  int np;
  int bad;  // an atom's energy or virial is not finite or above 1e9
};

// Forces on the thread's own slots tid, tid + nt, ... (written to fs), with
// optional energy, virial and pair-count sums: per atom in FP32 over its list,
// then added to the thread's exact fixed-point sums.  Not inlined and fed only
// scalars: it runs with the whole register budget for the pair loop while the
// caller's step state is saved once per call, and positions are read with
// explicit shared-memory loads.
//
// CODED (Verlet path): lists with image codes (cell search) or with the minimum image
// per entry (search without cells); separate instances keep each loop's registers.
template <int APT, int PATH, bool EN, bool VIR, bool CNT, bool CODED>
__device__ __noinline__ FSums force_pass(uint32_t xs_a, float4* fs, const uint16_t* nl, int tid,
                                         int nt, int npad, int n, int tpa, int u0, int u1,
                                         float L, float invL, LJ c) {
  unsigned long long es = 0, ws[6] = {0, 0, 0, 0, 0, 0};
  int np = 0, bad = 0;
  // units u0 .. u1 - 1 (u0 a multiple of tpa); unit u = i tpa + p: sub-list p of atom
  // i (tpa = 1 but for lists without cells)
  const int sh = tpa == 4 ? 2 : (tpa == 2 ? 1 : 0);
#pragma unroll 1
  for (int u = u0 + tid; u < u1; u += nt) {
    const int i = u >> sh, p = u & (tpa - 1);
    {
      const float4 xi = ld_shared4(xs_a + 16u * (uint32_t)i);
      const float cw = fs[i].w;  // packed list lengths (Verlet path), kept across steps
      float fx = 0.f, fy = 0.f, fz = 0.f;
      float e = 0.f;  // this atom's energy and virial over its list
      float w[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (PATH == PATH_NLIST) {
        // Row of slot i: eight uint16 entries per 16-byte word, word (k/8) of slot
        // i at (k/8) * npad + i, so a warp's word loads are contiguous.  The list
        // is rewritten inside this kernel at every rebuild, so it is read with
        // L2-only loads (never the read-only cache); the next word is fetched while
        // the current one is processed.  Positions are not wrapped between list
        // builds, so the image of every entry stays the one the build found: the
        // word's code selects, per axis, the home position or its image (+-L by the
        // slot's direction bits), and the pair takes the plain difference.  Lists
        // without codes (boxes searched without cells) take the minimum image per
        // entry.  The build pads partial words with the atom's own slot, so every
        // word is processed whole and the self entries are masked by index.
        const uint4* lp = reinterpret_cast<const uint4*>(nl) + u;
        const size_t wst = (size_t)npad * tpa;  // words between word kb and kb + 1
        const int meta = __float_as_int(cw);
        const int nw = CODED ? meta & 0xfff : (sub_entries(meta, tpa, p) + 7) >> 3;
        uint4 q = nw > 0 ? __ldcg(lp) : make_uint4(0u, 0u, 0u, 0u);
        if (CODED) {
          // home shift along an axis: +L for atoms in the lower half of the grid
#define MDEOS_SHIFT(bit) ((meta & (bit)) ? -L : L)
          const float xa = xi.x + MDEOS_SHIFT(0x1000), ya = xi.y + MDEOS_SHIFT(0x2000);
          const float za = xi.z + MDEOS_SHIFT(0x4000);
#pragma unroll 1
          for (int kb = 0; kb < nw; ++kb) {
            const uint4 cur = q;
            if (kb + 1 < nw) q = __ldcg(lp + (size_t)(kb + 1) * wst);
            const float hx = (cur.x & 0x1000u) ? xa : xi.x;
            const float hy = (cur.x & 0x2000u) ? ya : xi.y;
            const float hz = (cur.x & 0x4000u) ? za : xi.z;
            const int j0 = (int)(cur.x & 0xfffu), j1 = (int)(cur.x >> 16);
            const int j2 = (int)(cur.y & 0xffffu), j3 = (int)(cur.y >> 16);
            const int j4 = (int)(cur.z & 0xffffu), j5 = (int)(cur.z >> 16);
            const int j6 = (int)(cur.w & 0xffffu), j7 = (int)(cur.w >> 16);
            const float px = fx, py = fy, pz = fz;  // the force before this word
            // the virial is taken per atom below, not per pair
            nl_pair_sh<EN, false>(xs_a, j0, j0 != i, hx, hy, hz, c, fx, fy, fz, e, w, np);
            nl_pair_sh<EN, false>(xs_a, j1, j1 != i, hx, hy, hz, c, fx, fy, fz, e, w, np);
            nl_pair_sh<EN, false>(xs_a, j2, j2 != i, hx, hy, hz, c, fx, fy, fz, e, w, np);
            nl_pair_sh<EN, false>(xs_a, j3, j3 != i, hx, hy, hz, c, fx, fy, fz, e, w, np);
            nl_pair_sh<EN, false>(xs_a, j4, j4 != i, hx, hy, hz, c, fx, fy, fz, e, w, np);
            nl_pair_sh<EN, false>(xs_a, j5, j5 != i, hx, hy, hz, c, fx, fy, fz, e, w, np);
            nl_pair_sh<EN, false>(xs_a, j6, j6 != i, hx, hy, hz, c, fx, fy, fz, e, w, np);
            nl_pair_sh<EN, false>(xs_a, j7, j7 != i, hx, hy, hz, c, fx, fy, fz, e, w, np);
            if (VIR) {
              // image term of the word: its shift S (per axis: sx, sy, sz or 0) times
              // its force G, symmetrised, into w (xx, yy, zz, xy, xz, yz)
              const float gx = fx - px, gy = fy - py, gz = fz - pz;
              if (cur.x & 0x1000u) {
                const float sh = MDEOS_SHIFT(0x1000);
                w[0] = fmaf(sh, gx, w[0]);
                w[3] = fmaf(0.5f * sh, gy, w[3]);
                w[4] = fmaf(0.5f * sh, gz, w[4]);
              }
              if (cur.x & 0x2000u) {
                const float sh = MDEOS_SHIFT(0x2000);
                w[1] = fmaf(sh, gy, w[1]);
                w[3] = fmaf(0.5f * sh, gx, w[3]);
                w[5] = fmaf(0.5f * sh, gz, w[5]);
              }
              if (cur.x & 0x4000u) {
                const float sh = MDEOS_SHIFT(0x4000);
                w[2] = fmaf(sh, gz, w[2]);
                w[4] = fmaf(0.5f * sh, gx, w[4]);
                w[5] = fmaf(0.5f * sh, gy, w[5]);
              }
            }
          }
#undef MDEOS_SHIFT
          if (VIR) {
            // Virial of the box from the atom's total force: with full lists and
            // f_ji = -f_ij, sum_{i<j} d_ij (x) f_ij = sum_i [x_i (x) F_i +
            // 1/2 sum_w S_w (x) F_i,w] (x_i the positions the forces were taken at,
            // F_i,w the force from word w, S_w its image shift), symmetrised; w held
            // the image terms, and the halving of the per-pair form below is undone
            w[0] = 2.0f * fmaf(xi.x, fx, 0.5f * w[0]);
            w[1] = 2.0f * fmaf(xi.y, fy, 0.5f * w[1]);
            w[2] = 2.0f * fmaf(xi.z, fz, 0.5f * w[2]);
            w[3] = 2.0f * fmaf(0.5f * xi.x, fy, fmaf(0.5f * xi.y, fx, 0.5f * w[3]));
            w[4] = 2.0f * fmaf(0.5f * xi.x, fz, fmaf(0.5f * xi.z, fx, 0.5f * w[4]));
            w[5] = 2.0f * fmaf(0.5f * xi.y, fz, fmaf(0.5f * xi.z, fy, 0.5f * w[5]));
          }
        } else {
#pragma unroll 1
          for (int kb = 0; kb < nw; ++kb) {
            const uint4 cur = q;
            if (kb + 1 < nw) q = __ldcg(lp + (size_t)(kb + 1) * wst);
            const int j0 = (int)(cur.x & 0xffffu), j1 = (int)(cur.x >> 16);
            const int j2 = (int)(cur.y & 0xffffu), j3 = (int)(cur.y >> 16);
            const int j4 = (int)(cur.z & 0xffffu), j5 = (int)(cur.z >> 16);
            const int j6 = (int)(cur.w & 0xffffu), j7 = (int)(cur.w >> 16);
            nl_pair_bd<EN, VIR>(xs_a, j0, j0 != i, xi, L, invL, c, fx, fy, fz, e, w, np);
            nl_pair_bd<EN, VIR>(xs_a, j1, j1 != i, xi, L, invL, c, fx, fy, fz, e, w, np);
            nl_pair_bd<EN, VIR>(xs_a, j2, j2 != i, xi, L, invL, c, fx, fy, fz, e, w, np);
            nl_pair_bd<EN, VIR>(xs_a, j3, j3 != i, xi, L, invL, c, fx, fy, fz, e, w, np);
            nl_pair_bd<EN, VIR>(xs_a, j4, j4 != i, xi, L, invL, c, fx, fy, fz, e, w, np);
            nl_pair_bd<EN, VIR>(xs_a, j5, j5 != i, xi, L, invL, c, fx, fy, fz, e, w, np);
            nl_pair_bd<EN, VIR>(xs_a, j6, j6 != i, xi, L, invL, c, fx, fy, fz, e, w, np);
            nl_pair_bd<EN, VIR>(xs_a, j7, j7 != i, xi, L, invL, c, fx, fy, fz, e, w, np);
          }
        }
      } else if (PATH == PATH_ALLPAIRS) {
        for (int j = 0; j < n; ++j) {
          const float4 xj = ld_shared4(xs_a + 16u * (uint32_t)j);
          const float dx = min_img(xi.x - xj.x, L, invL);
          const float dy = min_img(xi.y - xj.y, L, invL);
          const float dz = min_img(xi.z - xj.z, L, invL);
          lj_pair<EN, VIR>(dx, dy, dz, j != i, c, fx, fy, fz, e, w, np);
        }
      } else {  // PATH_ALLPAIRS_MI: rc <= L < 2 rc, the two nearest images per axis
        for (int j = 0; j < n; ++j) {
          const float4 xj = ld_shared4(xs_a + 16u * (uint32_t)j);
          const float d0x = min_img(xi.x - xj.x, L, invL);
          const float d0y = min_img(xi.y - xj.y, L, invL);
          const float d0z = min_img(xi.z - xj.z, L, invL);
          const float d1x = d0x - copysignf(L, d0x);
          const float d1y = d0y - copysignf(L, d0y);
          const float d1z = d0z - copysignf(L, d0z);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float dx = (k & 1) ? d1x : d0x;
            const float dy = (k & 2) ? d1y : d0y;
            const float dz = (k & 4) ? d1z : d0z;
            lj_pair<EN, VIR>(dx, dy, dz, (j != i) || (k != 0), c, fx, fy, fz, e, w, np);
          }
        }
      }
      if (tpa > 1) {  // the partial forces of the atom's units, in a fixed order
        const unsigned m = tpa_mask(tpa);
        fx += __shfl_xor_sync(m, fx, 1);
        fy += __shfl_xor_sync(m, fy, 1);
        fz += __shfl_xor_sync(m, fz, 1);
        if (tpa > 2) {
          fx += __shfl_xor_sync(m, fx, 2);
          fy += __shfl_xor_sync(m, fy, 2);
          fz += __shfl_xor_sync(m, fz, 2);
        }
      }
      if (p == 0) fs[i] = make_float4(fx, fy, fz, cw);
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
  }
  FSums out = {es, ws[0], ws[1], ws[2], ws[3], ws[4], ws[5], CNT ? np : 0, bad};
  return out;
}

// Per-thread sums of a force pass: energy and virial (fxp units, halved), pair
// count, and the non-finite flag.
struct ForceAcc {
  unsigned long long e = 0, w[6] = {0, 0, 0, 0, 0, 0};
  int np = 0, bad = 0;
};

// Cluster form of a force pass's end: the sums of this CTA's threads (exact), sent
// with the forces of its own atoms (a0 .. a1 - 1) to every CTA of the cluster; after
// the cluster barrier thread 0 of every CTA holds the cluster's sums (added over the
// ranks in order: the same integers everywhere) and the other threads none.
static __device__ void cluster_exchange(const Group& g, FSums& r, int a0, int a1) {
  long long q[9] = {(long long)r.e,  (long long)r.w0, (long long)r.w1,
                    (long long)r.w2, (long long)r.w3, (long long)r.w4,
                    (long long)r.w5, (long long)r.np, (long long)r.bad};
#pragma unroll
  for (int k = 0; k < 9; ++k) q[k] = warp_sum_ll(q[k]);
  long long* red = g.red();
  if (g.lane() == 0)
#pragma unroll
    for (int k = 0; k < 9; ++k) red[g.warp() * kRedSlots + k] = q[k];
  gbar(g.bar, g.nt);
  const uint32_t f_a = (uint32_t)__cvta_generic_to_shared(g.f());
  for (int i = a0 + g.tid; i < a1; i += g.nt) {
    const float4 fi = g.f()[i];
    for (int rk = 0; rk < g.csize; ++rk)
      if (rk != g.crank) st_cluster_v4(cluster_map(f_a + 16u * (uint32_t)i, rk), fi);
  }
  // lane k < 9 of warp 0: the CTA's sum of quantity k, into slot (crank, k) of every CTA
  const int lane = g.lane();
  if (g.warp() == 0 && lane < 9) {
    long long t = 0;
    for (int w = 0; w < g.nwarps; ++w) t += red[w * kRedSlots + lane];
    const uint32_t c_a =
        (uint32_t)__cvta_generic_to_shared(g.clu() + g.crank * kRedSlots + lane);
    for (int rk = 0; rk < g.csize; ++rk) st_cluster_s64(cluster_map(c_a, rk), t);
  }
  cluster_sync();
  FSums z = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0, 0};
  if (g.warp() == 0) {
    long long t = 0;
    if (lane < 9)
      for (int rk = 0; rk < g.csize; ++rk) t += g.clu()[rk * kRedSlots + lane];
    long long v[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) v[k] = __shfl_sync(0xffffffffu, t, k);
    if (lane == 0) {
      z.e = (unsigned long long)v[0];
      z.w0 = (unsigned long long)v[1];
      z.w1 = (unsigned long long)v[2];
      z.w2 = (unsigned long long)v[3];
      z.w3 = (unsigned long long)v[4];
      z.w4 = (unsigned long long)v[5];
      z.w5 = (unsigned long long)v[6];
      z.np = (int)v[7];
      z.bad = v[8] != 0;
    }
  }
  r = z;
}

// the atoms a CTA of the cluster computes (all of them without a cluster)
__device__ __forceinline__ void own_atoms(const Group& g, int n, int& a0, int& a1) {
  const int A = (n + g.csize - 1) / g.csize;
  a0 = min(n, g.crank * A);
  a1 = min(n, a0 + A);
}

template <int APT, int PATH, bool EN, bool VIR, bool CNT>
__device__ __forceinline__ void compute_forces(const Group& g, const BoxCtx& b, const RunParams& rp,
                                               ForceAcc& acc) {
  const uint32_t xs_a = (uint32_t)__cvta_generic_to_shared(g.x());
  int a0, a1;
  own_atoms(g, b.n, a0, a1);
  // before another CTA's forces land here, every CTA has read its forces of the
  // last pass (the half kicks)
  if (g.csize > 1) cluster_sync();
  FSums r =
      (PATH != PATH_NLIST || b.nc > 0)
          ? force_pass<APT, PATH, EN, VIR, CNT, true>(xs_a, g.f(), g.nl, g.tid, g.nt, g.npad, b.n,
                                                      b.tpa, a0 * b.tpa, a1 * b.tpa, b.L, b.invL,
                                                      make_lj(rp))
          : force_pass<APT, PATH, EN, VIR, CNT, false>(xs_a, g.f(), g.nl, g.tid, g.nt, g.npad,
                                                       b.n, b.tpa, a0 * b.tpa, a1 * b.tpa, b.L,
                                                       b.invL, make_lj(rp));
  // with several threads per atom an atom's force is written by the first thread of
  // its group, not by the thread that owns the atom in the step
  if (b.tpa > 1 || g.csize > 1) gbar(g.bar, g.nt);
  if (g.csize > 1) cluster_exchange(g, r, a0, a1);
  if (EN) acc.e += r.e;
  if (VIR) {
    acc.w[0] += r.w0;
    acc.w[1] += r.w1;
    acc.w[2] += r.w2;
    acc.w[3] += r.w3;
    acc.w[4] += r.w4;
    acc.w[5] += r.w5;
  }
  if (CNT) acc.np += r.np;
  acc.bad |= r.bad;
}

// ---------------------------------------------------------------------------
// Verlet list build from positions wrapped into [0, L).
//
// Cell path (a grid of cells of side >= (rc + skin) / 2, at most 12 per axis; any
// box with L >= 2 (rc + skin)): a shared-memory counting sort re-orders the box
// into cell order -- positions (original atom id carried in x.w) and velocities
// are permuted in place, and ownership follows the slot -- so the 32 lanes of a
// warp hold neighbouring atoms and scan overlapping cells, and later force-loop
// gathers touch nearby shared-memory words.  Inside a cell atoms keep their
// previous relative order (sorted by previous slot), so the order, the list and
// every result are deterministic.
// Without a grid (nc_cell = 0: boxes of at most kBruteMaxAtoms atoms, where a scan
// of all atoms with broadcast loads is cheaper than the cell search) every atom is
// scanned with the minimum image, without re-ordering.
// The list length of slot s is kept in f[s].w (as int bits).

__device__ __forceinline__ int cell_of(const float4& x, float cinv, int nc) {
  const int cx = min((int)(x.x * cinv), nc - 1);
  const int cy = min((int)(x.y * cinv), nc - 1);
  const int cz = min((int)(x.z * cinv), nc - 1);
  return (cz * nc + cy) * nc + cx;
}

__device__ __forceinline__ int ld_shared_s32(uint32_t a) {
  int v;
  asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
  return v;
}

__device__ __forceinline__ void st_shared_v4(uint32_t a, float4 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w)
               : "memory");
}

// List layout shared by the searches and the force pass.  Entries are uint16 slots,
// eight to a 16-byte word.  The word's bits 12..14 of its first entry (slots stay
// below 4096) say on which axes (x, y, z) its entries lie across a face of the box
// from the home atom, so the force pass shifts the home atom once per word instead
// of taking the minimum image per entry.  Along each axis only one face can be
// crossed within R < L / 2: the upper one for an atom in the lower half of the cell
// grid (the home atom is then shifted by +L), the lower one otherwise (-L); that
// direction per axis is a bit of the slot's list word.  The list word of a slot (the
// w component of its force entry) packs the word count (bits 0..11), the directions
// (bits 12..14, x, y, z: 1 = shift by -L) and the entry count without padding (bits
// 16..31).  Lists without codes (the minimum image per entry) carry no directions.
__device__ __forceinline__ int list_meta(int nw, int dirs, int k) {
  return nw | (dirs << 12) | (k << 16);
}

// One output stream of the cell search: eight entries assembled in four registers,
// each new entry entering at the top (after eight the first sits in the low half of
// w0), with the image code of the entries it holds.
struct LStream {
  uint32_t w0, w1, w2, w3;
  int cnt, code;
};

__device__ __forceinline__ void ls_push(LStream& s, uint32_t e) {
  s.w0 = __funnelshift_r(s.w0, s.w1, 16);
  s.w1 = __funnelshift_r(s.w1, s.w2, 16);
  s.w2 = __funnelshift_r(s.w2, s.w3, 16);
  s.w3 = __funnelshift_r(s.w3, e, 16);
}

// store the assembled word as word kw of the slot's row (counted beyond the capacity)
__device__ __forceinline__ void ls_store(LStream& s, uint4* lrow, int npad, int& kw, int maxw) {
  if (kw < maxw)
    lrow[(size_t)kw * npad] = make_uint4(s.w0 | ((uint32_t)s.code << 12), s.w1, s.w2, s.w3);
  ++kw;
  s.cnt = 0;
}

// a partial word is completed with the slot itself (masked by index in the force pass)
__device__ __forceinline__ void ls_flush(LStream& s, uint32_t pad, uint4* lrow, int npad, int& kw,
                                         int maxw) {
  if (s.cnt > 0) {
#pragma unroll 1
    for (int u = s.cnt; u < 8; ++u) ls_push(s, pad);
    ls_store(s, lrow, npad, kw, maxw);
  }
}

// entries of slots t0..t1-1 within R of the (shifted) home position a, into stream s
// under image code `code`; a code change first closes the stream's partial word
__device__ __forceinline__ void ls_scan(LStream& s, int code, int t0, int t1, float ax, float ay,
                                        float az, uint32_t xs_a, int sl, float rcs2, uint4* lrow,
                                        int npad, int& kw, int maxw, int& k) {
  if (t0 >= t1) return;
  if (s.code != code) {
    ls_flush(s, (uint32_t)sl, lrow, npad, kw, maxw);
    s.code = code;
  }
#pragma unroll 1
  for (int t = t0; t < t1; t += 2) {
    const float4 xa = ld_shared4(xs_a + 16u * (uint32_t)t);
    const float4 xb = ld_shared4(xs_a + 16u * (uint32_t)min(t + 1, t1 - 1));
    const float dax = ax - xa.x, day = ay - xa.y, daz = az - xa.z;
    const float dbx = ax - xb.x, dby = ay - xb.y, dbz = az - xb.z;
    const float ra = fmaf(dax, dax, fmaf(day, day, daz * daz));
    const float rb = fmaf(dbx, dbx, fmaf(dby, dby, dbz * dbz));
    if (ra < rcs2 && t != sl) {
      ls_push(s, (uint32_t)t);
      ++k;
      if (++s.cnt == 8) ls_store(s, lrow, npad, kw, maxw);
    }
    if (rb < rcs2 && t + 1 != sl && t + 1 < t1) {
      ls_push(s, (uint32_t)(t + 1));
      ++k;
      if (++s.cnt == 8) ls_store(s, lrow, npad, kw, maxw);
    }
  }
}

// Verlet-list search over the cell-ordered box (cells of side h >= R / 2, R = rc +
// skin, at least 4 per axis).  Every lane walks 5 x 5 rows of cells around its home
// cell (z and y offsets -2..2), and in each row only the x range of cells that can
// hold an atom within R of its own: R^2 less the squared distance to the row's y-z
// rectangle bounds the x extent.  A row's cells are contiguous slots in cell order;
// the part of the range inside the box goes to one output stream, the part across
// an x face (at most one side) to a second one with its image shift applied to the
// home atom.  The rows are taken in an order that keeps rows crossing the same y and
// z faces together (offsets that cross no face first along each axis, then blocks
// (z inside, y inside), (z inside, y across), (z across, y inside), (z across, y
// across)), so each stream changes its image code at most three times and few words
// are closed early.  Ranges use R enlarged by 1e-5 so rounding drops no cell, and the
// home position is clamped into [0, L] so the indices stay in range even for a state
// that has blown up (the box then fails on its temperature); entries are accepted on
// r^2 < R^2.  A cell reached through two images (grids of 4 cells) holds at most one
// image of each atom within R, since L >= 2 R.  At the end the slot's force entry
// receives (0, 0, 0, list word).  Out of line and fed only scalars and shared-memory
// addresses, so the search has the whole register budget.
template <int APT>
__device__ __noinline__ void nl_search(uint32_t xs_a, uint32_t meta_a, uint32_t cs_a,
                                       uint32_t ovf_a, uint16_t* nl, int tid, int nt, int npad,
                                       int n, int nc, float L, float cinv, float rcs2, int maxnb) {
  const float Rs = 1.00001f * sqrtf(rcs2);
  const float Rs2 = Rs * Rs;
  const float h = L / (float)nc;
  const int maxw = maxnb >> 3;
#pragma unroll 1
  for (int a = 0; a < APT; ++a) {
    const int sl = tid + a * nt;
    if (sl >= n) break;
    float4 xi = ld_shared4(xs_a + 16u * (uint32_t)sl);
    xi.x = fminf(fmaxf(xi.x, 0.f), L);
    xi.y = fminf(fmaxf(xi.y, 0.f), L);
    xi.z = fminf(fmaxf(xi.z, 0.f), L);
    const int cx = min((int)(xi.x * cinv), nc - 1), cy = min((int)(xi.y * cinv), nc - 1);
    const int cz = min((int)(xi.z * cinv), nc - 1);
    // the face an axis can cross: upper half of the grid -> the upper face
    const int hx = 2 * cx >= nc, hy = 2 * cy >= nc, hz = 2 * cz >= nc;
    // offsets (of -2..2) that cross it, and the rotation putting the others first
    const int wy = hy ? max(cy + 3 - nc, 0) : max(2 - cy, 0);
    const int wz = hz ? max(cz + 3 - nc, 0) : max(2 - cz, 0);
    const int ny0 = 5 - wy, nz0 = 5 - wz;
    const int ry = hy ? 0 : wy, rz = hz ? 0 : wz;
    uint4* lrow = reinterpret_cast<uint4*>(nl) + sl;  // word w at lrow + w * npad
    LStream s0 = {0u, 0u, 0u, 0u, 0, 0}, s1 = {0u, 0u, 0u, 0u, 0, 1};
    int kw = 0, k = 0;
    int yb = 0, zb = 0, iy = 0, iz = 0;  // block (z across, y across) and offsets in it
#pragma unroll 1
    for (int r = 0; r < 25; ++r) {
      const int dz = (iz + rz < 5 ? iz + rz : iz + rz - 5) - 2;
      const int dy = (iy + ry < 5 ? iy + ry : iy + ry - 5) - 2;
      const int qz = cz + dz, qy = cy + dy;
      const float zl = (float)qz * h;
      const float ez = fmaxf(fmaxf(zl - xi.z, xi.z - (zl + h)), 0.f);
      const int wzc = qz < 0 ? qz + nc : (qz >= nc ? qz - nc : qz);
      const float az = xi.z - (qz < 0 ? -L : (qz >= nc ? L : 0.f));
      const float yl = (float)qy * h;
      const float ey = fmaxf(fmaxf(yl - xi.y, xi.y - (yl + h)), 0.f);
      const int wyc = qy < 0 ? qy + nc : (qy >= nc ? qy - nc : qy);
      const float ay = xi.y - (qy < 0 ? -L : (qy >= nc ? L : 0.f));
      const float rx2 = Rs2 - ez * ez - ey * ey;
      // x cells within the radius left over (none when the row is out of range)
      const float rx = sqrtf(fmaxf(rx2, 0.f));
      const int x0 = max((int)floorf((xi.x - rx) * cinv), cx - 2);
      int x1 = min((int)floorf((xi.x + rx) * cinv), cx + 2);
      if (rx2 < 0.f) x1 = x0 - 1;
      const uint32_t rowa = cs_a + 4u * (uint32_t)((wzc * nc + wyc) * nc);
      const int code = (yb << 1) | (zb << 2);
      {  // cells inside the box
        const int lo = max(x0, 0), hi = min(x1, nc - 1);
        if (lo <= hi)
          ls_scan(s0, code, ld_shared_s32(rowa + 4u * (uint32_t)lo),
                  ld_shared_s32(rowa + 4u * (uint32_t)(hi + 1)), xi.x, ay, az, xs_a, sl, rcs2,
                  lrow, npad, kw, maxw, k);
      }
      {  // cells across the lower (x0 < 0) or upper (x1 >= nc) x face
        const int lo = x0 < 0 ? x0 + nc : max(x0, nc) - nc;
        const int hi = x0 < 0 ? min(x1, -1) + nc : x1 - nc;
        if (lo <= hi)
          ls_scan(s1, code | 1, ld_shared_s32(rowa + 4u * (uint32_t)lo),
                  ld_shared_s32(rowa + 4u * (uint32_t)(hi + 1)), xi.x + (x0 < 0 ? L : -L), ay,
                  az, xs_a, sl, rcs2, lrow, npad, kw, maxw, k);
      }
      // next row: the block's y offsets, then its z offsets, then the next block
      if (++iy == (yb ? 5 : ny0)) {
        iy = yb ? ny0 : 0;
        if (++iz == (zb ? 5 : nz0)) {
          if (yb == 0 && wy > 0) {
            yb = 1;
          } else {
            yb = 0;
            zb = 1;
          }
          iz = zb ? nz0 : 0;
          iy = yb ? ny0 : 0;
        }
      }
    }
    ls_flush(s0, (uint32_t)sl, lrow, npad, kw, maxw);
    ls_flush(s1, (uint32_t)sl, lrow, npad, kw, maxw);
    if (kw > maxw) {
      atomicOr(reinterpret_cast<int*>(__cvta_shared_to_generic(ovf_a)), 1);
      kw = maxw;
    }
    st_shared_v4(meta_a + 16u * (uint32_t)sl,
                 make_float4(0.f, 0.f, 0.f,
                             __int_as_float(list_meta(kw, hx | (hy << 1) | (hz << 2), k))));
  }
}

// Verlet-list search without cells (small boxes): unit u = i tpa + p scans the
// slots p, p + tpa, ... with the minimum image; the lanes of a warp with the same p
// load the same position (a broadcast), four candidates at a time.  The
// minimum image is taken again per entry in the force pass (no image codes).
// Entries are assembled eight at a time in registers and stored as one 16-byte
// word; the last word is padded with the atom's own slot.  Out of line, scalars and
// shared-memory addresses only.
static __device__ __noinline__ void nl_search_all(uint32_t xs_a, uint32_t meta_a, uint32_t ovf_a,
                                                  uint16_t* nl, int tid, int nt, int npad, int n,
                                                  int tpa, int u0, int u1, float L, float invL,
                                                  float rcs2, int maxnb) {
  const int maxw = (maxnb / tpa) >> 3;
  const size_t wstride = (size_t)npad * tpa;  // words between word kb and kb + 1
#pragma unroll 1
  for (int u = u0 + tid; u < u1; u += nt) {
    const int i = u / tpa, p = u - i * tpa;
    const int jlast = n - 1 - (n - 1 - p) % tpa;  // the last slot of this sub-list's share
    const float4 xi = ld_shared4(xs_a + 16u * (uint32_t)i);
    uint4* lrow = reinterpret_cast<uint4*>(nl) + u;
    LStream st = {0u, 0u, 0u, 0u, 0, 0};
    int k = 0, kw = 0;
#pragma unroll 1
    for (int jb = p; jb < n; jb += 4 * tpa) {
      float r2[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 xo = ld_shared4(xs_a + 16u * (uint32_t)min(jb + q * tpa, jlast));
        const float dx = min_img(xi.x - xo.x, L, invL);
        const float dy = min_img(xi.y - xo.y, L, invL);
        const float dz = min_img(xi.z - xo.z, L, invL);
        r2[q] = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = jb + q * tpa;
        if (r2[q] < rcs2 && j != i && j < n) {
          ls_push(st, (uint32_t)j);
          ++k;
          if (++st.cnt == 8) {
            if (kw < maxw) lrow[(size_t)kw * wstride] = make_uint4(st.w0, st.w1, st.w2, st.w3);
            ++kw;
            st.cnt = 0;
          }
        }
      }
    }
    if (st.cnt > 0) {
#pragma unroll 1
      for (int q = st.cnt; q < 8; ++q) ls_push(st, (uint32_t)i);
      if (kw < maxw) lrow[(size_t)kw * wstride] = make_uint4(st.w0, st.w1, st.w2, st.w3);
      ++kw;
    }
    if (kw > maxw) {
      atomicOr(reinterpret_cast<int*>(__cvta_shared_to_generic(ovf_a)), 1);
      k = maxw * 8;
    }
    // the counts of the atom's sub-lists, packed into its list word by lane p = 0
    const unsigned m = tpa_mask(tpa);
    int meta = tpa == 1 ? list_meta((k + 7) >> 3, 0, k) : (k << ((tpa == 4 ? 8 : 16) * p));
    if (tpa > 1) meta |= __shfl_xor_sync(m, meta, 1);
    if (tpa > 2) meta |= __shfl_xor_sync(m, meta, 2);
    if (p == 0) st_shared_v4(meta_a + 16u * (uint32_t)i, make_float4(0.f, 0.f, 0.f, __int_as_float(meta)));
  }
}

template <int APT>
__device__ void build_nlist(const Group& g, const BoxCtx& b, long long* prof = nullptr) {
  const int n = b.n;
  long long tp = prof ? clock64() : 0;
#define MDEOS_PHASE(k)                          \
  if (prof && g.tid == 0) {                     \
    const long long tn = clock64();             \
    prof[k] += tn - tp;                         \
    tp = tn;                                    \
  }
  float4* xs = g.x();
  float4* vs = g.v();
  float4* srt = g.f();  // sorted copy of the positions (forces are dead during a rebuild)
  if (b.nc > 0) {
    const int nc = b.nc, ncell = nc * nc * nc;
    int* ccount = g.cell();              // counts, then insertion cursors
    int* cstart = g.cell() + ncell + 1;  // [ncell + 1]
    for (int c = g.tid; c < ncell; c += g.nt) ccount[c] = 0;
    gbar(g.bar, g.nt);
    int mycell[APT];
#pragma unroll
    for (int a = 0; a < APT; ++a) {
      const int i = g.tid + a * g.nt;
      mycell[a] = 0;
      if (i < n) {
        mycell[a] = cell_of(xs[i], b.cinv, nc);
        atomicAdd(&ccount[mycell[a]], 1);
      }
    }
    gbar(g.bar, g.nt);
    MDEOS_PHASE(0)
    if (g.warp() == 0) {
      const int lane = g.lane();
      const int per = (ncell + 31) / 32;
      const int lo = lane * per, hi = min(lo + per, ncell);
      int sum = 0;
      for (int c = lo; c < hi; ++c) sum += ccount[c];
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      int run = incl - sum;
      for (int c = lo; c < hi; ++c) {
        const int k = ccount[c];
        cstart[c] = run;
        ccount[c] = run;
        run += k;
      }
      if (lane == 31) cstart[ncell] = incl;
    }
    gbar(g.bar, g.nt);
    MDEOS_PHASE(1)
    // scatter (position, previous slot << 16 | atom id) into the sorted copy
#pragma unroll
    for (int a = 0; a < APT; ++a) {
      const int i = g.tid + a * g.nt;
      if (i < n) {
        const int slot = atomicAdd(&ccount[mycell[a]], 1);
        const float4 xi = xs[i];
        srt[slot] = make_float4(xi.x, xi.y, xi.z,
                                __int_as_float((i << 16) | (__float_as_int(xi.w) & 0xffff)));
      }
    }
    gbar(g.bar, g.nt);
    MDEOS_PHASE(2)
    for (int c = g.tid; c < ncell; c += g.nt) {  // restore the previous order inside each cell
      const int s0 = cstart[c], s1 = cstart[c + 1];
      for (int q = s0 + 1; q < s1; ++q) {
        const float4 key = srt[q];
        const int kk = __float_as_int(key.w);
        int t = q - 1;
        while (t >= s0 && __float_as_int(srt[t].w) > kk) {
          srt[t + 1] = srt[t];
          --t;
        }
        srt[t + 1] = key;
      }
    }
    gbar(g.bar, g.nt);
    MDEOS_PHASE(3)
    // permute velocities in place: read every old slot first, then write the new ones
    float4 vnew[APT];
#pragma unroll
    for (int a = 0; a < APT; ++a) {
      const int sl = g.tid + a * g.nt;
      if (sl < n) vnew[a] = vs[__float_as_int(srt[sl].w) >> 16];
    }
    gbar(g.bar, g.nt);
#pragma unroll
    for (int a = 0; a < APT; ++a) {
      const int sl = g.tid + a * g.nt;
      if (sl < n) {
        const float4 q = srt[sl];
        vs[sl] = make_float4(vnew[a].x, vnew[a].y, vnew[a].z, 0.f);
        xs[sl] = make_float4(q.x, q.y, q.z, __int_as_float(__float_as_int(q.w) & 0xffff));
      }
    }
    gbar(g.bar, g.nt);
    MDEOS_PHASE(4)
    nl_search<APT>((uint32_t)__cvta_generic_to_shared(xs), (uint32_t)__cvta_generic_to_shared(srt),
                   (uint32_t)__cvta_generic_to_shared(cstart),
                   (uint32_t)__cvta_generic_to_shared(&g.ctrl()[CTRL_OVERFLOW]), g.nl, g.tid, g.nt,
                   g.npad, n, nc, b.L, b.cinv, b.rcs2, b.maxnb);
    gbar(g.bar, g.nt);
    MDEOS_PHASE(5)
  } else {
    gbar(g.bar, g.nt);  // positions just wrapped by their owners
    // the lists of this CTA's atoms (all of them without a cluster)
    int a0, a1;
    own_atoms(g, n, a0, a1);
    nl_search_all((uint32_t)__cvta_generic_to_shared(xs), (uint32_t)__cvta_generic_to_shared(srt),
                  (uint32_t)__cvta_generic_to_shared(&g.ctrl()[CTRL_OVERFLOW]), g.nl, g.tid, g.nt,
                  g.npad, n, b.tpa, a0 * b.tpa, a1 * b.tpa, b.L, b.invL, b.rcs2, b.maxnb);
    gbar(g.bar, g.nt);
    if (g.csize > 1) {  // a list overflow anywhere ends the box in every CTA alike
      if (g.tid == 0 && g.ctrl()[CTRL_OVERFLOW] != 0) {
        const uint32_t o_a = (uint32_t)__cvta_generic_to_shared(&g.ctrl()[CTRL_OVERFLOW]);
        for (int rk = 0; rk < g.csize; ++rk) st_cluster_s32(cluster_map(o_a, rk), 1);
      }
      cluster_sync();
    }
    MDEOS_PHASE(5)
  }
#undef MDEOS_PHASE
}

// wrap own positions into [0, L) and reset their displacement bounds (v.w)
template <int APT>
__device__ __forceinline__ void wrap_own(const Group& g, const BoxCtx& b) {
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) {
      g.v()[i].w = 0.f;
      float4 xi = g.x()[i];
      xi.x -= b.L * floorf(xi.x * b.invL);
      xi.y -= b.L * floorf(xi.y * b.invL);
      xi.z -= b.L * floorf(xi.z * b.invL);
      xi.x = fmaxf((xi.x >= b.L) ? xi.x - b.L : xi.x, 0.f);
      xi.y = fmaxf((xi.y >= b.L) ? xi.y - b.L : xi.y, 0.f);
      xi.z = fmaxf((xi.z >= b.L) ? xi.z - b.L : xi.z, 0.f);
      g.x()[i] = xi;
    }
  }
}

// Lifted FCC lattice (Eq. 6-7): first n sites of nc^3 cells in the order
// (cell z, cell y, cell x, basis), cell side L / nc.
template <int APT>
__device__ void lattice_own(const Group& g, const BoxDesc& bd) {
  const int nc = bd.nc_lat;
  const double a = bd.L / nc;
#pragma unroll
  for (int k = 0; k < APT; ++k) {
    const int i = g.tid + k * g.nt;
    if (i < bd.natoms) {
      const int c = i >> 2, bb = i & 3;
      const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
      const double bx = (bb == 1 || bb == 2) ? 0.5 : 0.0;
      const double by = (bb == 1 || bb == 3) ? 0.5 : 0.0;
      const double bz = (bb == 2 || bb == 3) ? 0.5 : 0.0;
      g.x()[i] = make_float4((float)(a * (cx + bx)), (float)(a * (cy + by)), (float)(a * (cz + bz)),
                             __int_as_float(i));  // original atom id travels with the atom
    }
  }
}

// Energy lifting, first guess (Eq. 9): Gaussian velocities at temperature T
// (Philox key = seed, counter = (atom, 0, 0, 0), Box-Muller), zero total
// momentum, exact rescale to T with N_DOF = 3N - 3.  Writes g.v().
template <int APT>
__device__ void init_velocities(const Group& g, const BoxCtx& b, unsigned long long seed, double T,
                                const RunParams& rp) {
  const uint32_t k0 = (uint32_t)(seed & 0xffffffffull), k1 = (uint32_t)(seed >> 32);
  const double sd = sqrt(T / rp.mass);
  const double two_m32 = 2.3283064365386962890625e-10;  // 2^-32
  float3 v[APT];
  long long p[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    v[a] = make_float3(0.f, 0.f, 0.f);
    if (i < b.n) {
      const uint32_t id = (uint32_t)__float_as_int(g.x()[i].w);
      uint32_t c[4] = {id, 0u, 0u, 0u};
      philox4x32_10(c, k0, k1);
      // uniforms in the open interval (0, 1); Box-Muller in FP64 (once per atom)
      const double u0 = ((double)c[0] + 0.5) * two_m32, u1 = ((double)c[1] + 0.5) * two_m32;
      const double u2 = ((double)c[2] + 0.5) * two_m32, u3 = ((double)c[3] + 0.5) * two_m32;
      const double r01 = sqrt(-2.0 * log(u0)), r23 = sqrt(-2.0 * log(u2));
      double s1, c1, s3, c3;
      sincospi(2.0 * u1, &s1, &c1);
      sincospi(2.0 * u3, &s3, &c3);
      v[a] = make_float3((float)(sd * r01 * c1), (float)(sd * r01 * s1), (float)(sd * r23 * c3));
      p[0] += fxp(v[a].x);
      p[1] += fxp(v[a].y);
      p[2] += fxp(v[a].z);
    }
  }
  double ptot[3];
  group_sum<3>(g, p, ptot);
  const float mx = (float)(ptot[0] / b.n), my = (float)(ptot[1] / b.n), mz = (float)(ptot[2] / b.n);
  long long ke[1] = {0};
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) {
      v[a].x -= mx;
      v[a].y -= my;
      v[a].z -= mz;
      ke[0] += fxp(v[a].x * v[a].x + v[a].y * v[a].y + v[a].z * v[a].z);
    }
  }
  double ketot[1];
  group_sum<1>(g, ke, ketot);
  const double Tinst = rp.mass * ketot[0] / (3.0 * b.n - 3.0);
  const float lam = (float)sqrt(T / Tinst);
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) g.v()[i] = make_float4(lam * v[a].x, lam * v[a].y, lam * v[a].z, 0.f);
  }
}

// Warm start: the element's stored final state, positions scaled affinely by
// L / L_old and wrapped into [0, L) (w keeps the atom id), velocities with the
// displacement bound (w) cleared.
template <int APT>
__device__ void load_warm(const Group& g, const BoxCtx& b, const BoxDesc& bd) {
  const float s = (float)(bd.L / bd.L_old);
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) {
      float4 xi = __ldcg(bd.warm_state + i);
      xi.x *= s;
      xi.y *= s;
      xi.z *= s;
      xi.x -= b.L * floorf(xi.x * b.invL);
      xi.y -= b.L * floorf(xi.y * b.invL);
      xi.z -= b.L * floorf(xi.z * b.invL);
      xi.x = fmaxf((xi.x >= b.L) ? xi.x - b.L : xi.x, 0.f);
      xi.y = fmaxf((xi.y >= b.L) ? xi.y - b.L : xi.y, 0.f);
      xi.z = fmaxf((xi.z >= b.L) ? xi.z - b.L : xi.z, 0.f);
      g.x()[i] = xi;
      float4 vi = __ldcg(bd.warm_state + bd.warm_cap + i);
      vi.w = 0.f;
      g.v()[i] = vi;
    }
  }
}

// Warm start velocities: remove the mean, rescale exactly to T (N_DOF = 3N - 3).
// Returns false if the state has no kinetic energy to rescale.
template <int APT>
__device__ bool warm_velocities(const Group& g, const BoxCtx& b, double T, const RunParams& rp) {
  float3 v[APT];
  long long p[3] = {0, 0, 0};
  bool bad = false;
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    v[a] = make_float3(0.f, 0.f, 0.f);
    if (i < b.n) {
      const float4 vi = g.v()[i];
      v[a] = make_float3(vi.x, vi.y, vi.z);
      bad |= !(fabsf(vi.x) + fabsf(vi.y) + fabsf(vi.z) < 1e4f);
      p[0] += fxp(vi.x);
      p[1] += fxp(vi.y);
      p[2] += fxp(vi.z);
    }
  }
  if (gbar_or(g.bar, g.nt, bad)) return false;  // stored state not usable
  double ptot[3];
  group_sum<3>(g, p, ptot);
  const float mx = (float)(ptot[0] / b.n), my = (float)(ptot[1] / b.n), mz = (float)(ptot[2] / b.n);
  long long ke[1] = {0};
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) {
      v[a].x -= mx;
      v[a].y -= my;
      v[a].z -= mz;
      ke[0] += fxp(v[a].x * v[a].x + v[a].y * v[a].y + v[a].z * v[a].z);
    }
  }
  double ketot[1];
  group_sum<1>(g, ke, ketot);
  const double Tinst = rp.mass * ketot[0] / (3.0 * b.n - 3.0);
  if (!(Tinst > 0.0) || !isfinite(Tinst)) return false;
  const float lam = (float)sqrt(T / Tinst);
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) g.v()[i] = make_float4(lam * v[a].x, lam * v[a].y, lam * v[a].z, 0.f);
  }
  return true;
}

// Store the final state into the element's slot: positions wrapped into [0, L)
// with the atom id in w, velocities with the pending thermostat factor applied.
template <int APT>
__device__ void save_warm(const Group& g, const BoxCtx& b, const BoxDesc& bd, float lam) {
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) {
      float4 xi = g.x()[i];
      xi.x -= b.L * floorf(xi.x * b.invL);
      xi.y -= b.L * floorf(xi.y * b.invL);
      xi.z -= b.L * floorf(xi.z * b.invL);
      xi.x = fmaxf((xi.x >= b.L) ? xi.x - b.L : xi.x, 0.f);
      xi.y = fmaxf((xi.y >= b.L) ? xi.y - b.L : xi.y, 0.f);
      xi.z = fmaxf((xi.z >= b.L) ? xi.z - b.L : xi.z, 0.f);
      const float4 vi = g.v()[i];
      __stcg(bd.warm_state + i, xi);
      __stcg(bd.warm_state + bd.warm_cap + i, make_float4(lam * vi.x, lam * vi.y, lam * vi.z, 0.f));
    }
  }
}

// the three force variants the step loop uses
template <int APT, int PATH>
__device__ __forceinline__ void forces_step(const Group& g, const BoxCtx& b, const RunParams& rp,
                                            bool en, bool vir, ForceAcc& acc) {
  if (vir)
    compute_forces<APT, PATH, true, true, true>(g, b, rp, acc);
  else if (en)
    compute_forces<APT, PATH, true, false, false>(g, b, rp, acc);
  else
    compute_forces<APT, PATH, false, false, false>(g, b, rp, acc);
}

// first half kick with the pending thermostat factor, then drift; returns
// whether any own atom's displacement bound passed half the skin
template <int APT>
__device__ __forceinline__ bool kick_drift(const Group& g, const BoxCtx& b, const RunParams& rp,
                                           float lam) {
  bool need = false;
#pragma unroll
  for (int a = 0; a < APT; ++a) {
    const int i = g.tid + a * g.nt;
    if (i < b.n) {
      const float4 fi = g.f()[i];
      float4 vi = g.v()[i];
      vi.x = fmaf(lam, vi.x, rp.hdtm * fi.x);
      vi.y = fmaf(lam, vi.y, rp.hdtm * fi.y);
      vi.z = fmaf(lam, vi.z, rp.hdtm * fi.z);
      // v.w: bound on the displacement since the last list build
      vi.w = fmaf(rp.dt, sqrtf(vi.x * vi.x + vi.y * vi.y + vi.z * vi.z), vi.w);
      g.v()[i] = vi;
      float4 xi = g.x()[i];
      xi.x = fmaf(rp.dt, vi.x, xi.x);
      xi.y = fmaf(rp.dt, vi.y, xi.y);
      xi.z = fmaf(rp.dt, vi.z, xi.z);
      g.x()[i] = xi;
      need = need || (vi.w > b.half_skin);
    }
  }
  return need;
}

// Warm-start lift, out of line so that its list build and force pass do not
// add to the register pressure of the step loop: the stored state scaled to
// the new box, its E_pot, the Eq. 10 temperature (or T_fixed if > 0), and the
// velocities rescaled to it.  Returns the temperature (<= 0 or NaN: failure).
template <int APT, int PATH>
__device__ __noinline__ double warm_lift(const Group& g, const BoxCtx& b, const BoxDesc& bd,
                                         const RunParams& rp, double E_tgt, double T_fixed,
                                         double ndof) {
  if (g.tid == 0) g.ctrl()[CTRL_WARM] = 1;  // read back by the restriction
  gbar(g.bar, g.nt);  // E_cold pass done before positions are replaced
  load_warm<APT>(g, b, bd);
  gbar(g.bar, g.nt);
  if (PATH == PATH_NLIST) build_nlist<APT>(g, b);
  ForceAcc f0;
  forces_step<APT, PATH>(g, b, rp, true, false, f0);
  const long long q[1] = {(long long)f0.e};
  double et[1];
  group_sum<1>(g, q, et);
  const double T = T_fixed > 0.0 ? T_fixed : 2.0 * (E_tgt - et[0]) / ndof;  // Eq. 10
  if (!(T > 0.0) || !isfinite(T)) return T;
  if (!warm_velocities<APT>(g, b, T, rp)) return -1.0;
  return T;
}

// ---------------------------------------------------------------------------
// One box, start to finish.  Every thread of the group runs the same control
// flow; branch decisions depend only on values all threads hold identically.
template <int APT, int PATH>
__device__ void run_box(const Group& g, const BoxDesc& __restrict__ bd, const RunParams& rp,
                        mdeos_result* out) {
  const BoxCtx b = make_ctx(bd, rp);
  const int n = b.n;
  const double ndof = 3.0 * n - 3.0;
  const double V = bd.L * bd.L * bd.L;
  const bool temp_mode = (bd.flags & MDEOS_REQ_TEMPERATURE) != 0;
  double* acc = g.acc();
  if (g.tid < 16) g.ctrl()[g.tid] = 0;
  for (int k = g.tid; k < kAccDoubles; k += g.nt) acc[k] = 0.0;
  for (int k = g.tid; k < kMaxSeBlocks; k += g.nt) g.bcnt()[k] = 0;
  lattice_own<APT>(g, bd);
  gbar(g.bar, g.nt);
  int builds = 0;
  for (int a = 0; a < APT; ++a) {  // zero velocities (displacement bounds) before any build
    const int i = g.tid + a * g.nt;
    if (i < n) g.v()[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (PATH == PATH_NLIST) {
    build_nlist<APT>(g, b);
    ++builds;
  }
  // E_cold: potential energy of the lifted lattice at rest (Sec. III)
  double E_cold;
  {
    ForceAcc f0;
    forces_step<APT, PATH>(g, b, rp, true, false, f0);
    const long long q[1] = {(long long)f0.e};
    double et[1];
    group_sum<1>(g, q, et);
    E_cold = et[0];
  }
  double* boxc = acc + ACC_BOX;  // FP64 box constants, read by warp 0 only
  const double E_ref = (rp.ref_mode == MDEOS_REF_FIXED) ? n * bd.e_ref : E_cold;
  const double E_tgt = n * bd.e + E_ref;
  // warm start if the element's slot holds its valid state (tag written by an
  // earlier launch; every thread reads the same value)
  double Tk;
  int status = MDEOS_OK;
  int nseg = 0;
  if (bd.warm_state != nullptr && bd.L_old > 0.0 &&
      *(volatile const unsigned long long*)bd.warm_tag == bd.element_id) {
    nseg = rp.warm_lift_iters;
    if (PATH == PATH_NLIST) ++builds;
    Tk = warm_lift<APT, PATH>(g, b, bd, rp, E_tgt, temp_mode ? bd.e : -1.0, ndof);
    if (!(Tk > 0.0) || !isfinite(Tk)) status = MDEOS_EUNPHYS;
  } else {
    nseg = rp.lift_iters;
    Tk = temp_mode ? bd.e : 2.0 * (E_tgt - E_cold) / ndof;  // Eq. 9
    if (!(Tk > 0.0) || !isfinite(Tk)) status = MDEOS_EUNPHYS;
    if (status == MDEOS_OK) init_velocities<APT>(g, b, bd.seed, Tk, rp);
  }
  if (g.tid == 0) {
    boxc[0] = E_cold;
    boxc[1] = E_ref;
    boxc[2] = E_tgt;
  }
  if (g.ctrl()[CTRL_OVERFLOW]) status = MDEOS_ENBR;
  if (bd.steps_equil == 0) nseg = 0;
  const int base = nseg > 0 ? bd.steps_equil / nseg : 0;
  int seg = 0, seg_pos = 0;
  int seg_len = (nseg == 1) ? bd.steps_equil : base;
  int nsamp = max(1, (seg_len + 9) / 10);
  const int total = bd.steps_equil + bd.steps_avg;
  const int nb = rp.se_blocks;


  const double invV = 1.0 / V, inv3V = 1.0 / (3.0 * V), inv_ndof = 1.0 / ndof;
  const int lead = (g.bar - 1) & 3 & (g.nwarps - 1);  // spreads group leaders over SMSPs
  float lam = 1.0f;
  if (g.tid == 0) boxc[3] = Tk;
  for (int step = 0; step < total && status == MDEOS_OK; ++step) {
    const bool avg = step >= bd.steps_equil;
    const int s_avg = step - bd.steps_equil;
    const bool seg_end = !avg && (seg_pos == seg_len - 1);
    const bool esamp = !avg && !temp_mode && (seg_pos >= seg_len - nsamp);
    const bool need = kick_drift<APT>(g, b, rp, lam);
    const bool rebuild = (PATH == PATH_NLIST) ? gbar_or(g.bar, g.nt, need) : (gbar(g.bar, g.nt), false);
    {
      // written by the leader warp last step (non-finite state): stop before a
      // rebuild bins such positions into cells
      const int st = g.ctrl()[CTRL_STATUS];
      if (st != 0 || g.ctrl()[CTRL_OVERFLOW] != 0) {
        status = st != 0 ? st : MDEOS_ENBR;
        break;
      }
    }
    if (PATH == PATH_NLIST && rebuild) {
      wrap_own<APT>(g, b);
      build_nlist<APT>(g, b);
      ++builds;
      if (g.ctrl()[CTRL_OVERFLOW] != 0) {
        status = MDEOS_ENBR;
        break;
      }
    }
    // forces at the new positions
    ForceAcc fa;
    forces_step<APT, PATH>(g, b, rp, avg || esamp, avg, fa);
    // second half kick; per-atom kinetic energy and kinetic stress into exact sums
    unsigned long long ke = 0, kt[6] = {0, 0, 0, 0, 0, 0};
    bool bad = fa.bad != 0;
#pragma unroll
    for (int a = 0; a < APT; ++a) {
      const int i = g.tid + a * g.nt;
      if (i < n) {
        const float4 fi = g.f()[i];
        float4 vi = g.v()[i];
        vi.x = fmaf(rp.hdtm, fi.x, vi.x);
        vi.y = fmaf(rp.hdtm, fi.y, vi.y);
        vi.z = fmaf(rp.hdtm, fi.z, vi.z);
        g.v()[i] = vi;
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
        }
      }
    }
    // per-warp partials: 0..5 stress (K + W), 6 E_pot, 7 E_kin (fxp units),
    // 8 in-cutoff pairs, 9 candidates, 10 non-finite flag
    {
      long long* red = g.red() + g.warp() * kRedSlots;
      const long long s = warp_sum_ll((long long)ke);
      const bool any_bad = __any_sync(0xffffffffu, bad);
      if (g.lane() == 0) {
        red[7] = s;
        red[10] = any_bad ? 1 : 0;
      }
      if (avg || esamp) {
        const long long se = warp_sum_ll((long long)fa.e);
        if (g.lane() == 0) red[6] = se;
      }
      if (avg) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const long long sk = warp_sum_ll((long long)(kt[k] + fa.w[k]));
          if (g.lane() == 0) red[k] = sk;
        }
        int cand = 0;
#pragma unroll
        for (int a = 0; a < APT; ++a) {
          const int i = g.tid + a * g.nt;
          if (i < n) {
            const int cw = list_entries(__float_as_int(g.f()[i].w), b.tpa);
            cand += (PATH == PATH_NLIST) ? cw
                                         : (PATH == PATH_ALLPAIRS ? n : 8 * n);
          }
        }
        const long long sp = warp_sum_ll(fa.np), sc = warp_sum_ll(cand);
        if (g.lane() == 0) {
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
    gbar(g.bar, g.nt);
    if (g.warp() == lead) {
      // Box sums of the step: the exact sums of the warp partials (lane k holds
      // quantity k); each lane then adds one quantity into its FP64 time
      // accumulator.  The thermostat's kinetic temperature comes from the same sum.
      const int lane = g.lane();
      const long long qi = warp_partials_ll(g.red(), g.nwarps, lane);
      const double q = lane < 8 ? (double)qi * kFixInv : (double)qi;
      const double s0 = __shfl_sync(0xffffffffu, q, 0), s1 = __shfl_sync(0xffffffffu, q, 1);
      const double s2 = __shfl_sync(0xffffffffu, q, 2), k7 = __shfl_sync(0xffffffffu, q, 7);
      const double Ps = (s0 + s1 + s2) * inv3V;   // Eq. 11, mean normal stress
      const double Ts = 2.0 * k7 * inv_ndof;
      if ((lane == 7 && !(Ts > 0.0)) || (lane == 10 && qi != 0))
        g.ctrl()[CTRL_STATUS] = MDEOS_EUNPHYS;
      int slot = -1;
      double val = 0.0;
      if (avg) {
        const int blk = (int)(((long long)s_avg * nb) / bd.steps_avg);
        if (lane < 6) { slot = ACC_RUN + lane; val = q * invV; }
        else if (lane < 10) { slot = ACC_RUN + lane; val = q; }
        else if (lane == 10) { slot = ACC_RUN + 10; val = Ps; }
        else if (lane == 11) { slot = ACC_RUN + 11; val = Ts; }
        else if (lane == 12) { slot = ACC_BP + blk; val = Ps; g.bcnt()[blk] += 1; }
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
        g.bc()[0] = Tn;
        acc[ACC_RUN + 12] = 0.0;
      }
      // velocity-rescale factor towards the (new) target temperature, from the
      // FP64 kinetic temperature of this step
      if (resc) {
        Tn = __shfl_sync(0xffffffffu, Tn, 6);
        if (lane == 7)
          g.bc()[5] = (Tn > 0.0 && Ts > 0.0 && isfinite(Tn) && isfinite(Ts)) ? sqrt(Tn / Ts) : -1.0;
      }
    }
    // the rescale is applied with the next first half-kick
    lam = 1.0f;
    if (resc) {
      gbar(g.bar, g.nt);
      const double lam_d = g.bc()[5];
      if (!(lam_d > 0.0)) {
        status = MDEOS_EUNPHYS;
        break;
      }
      if (seg_end) {
        Tk = g.bc()[0];
        if (g.tid == 0) boxc[3] = Tk;
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
  gbar(g.bar, g.nt);
  if (status == MDEOS_OK && g.ctrl()[CTRL_STATUS] != 0) status = g.ctrl()[CTRL_STATUS];
  if (bd.warm_state != nullptr) {
    // a list overflow leaves the stored state as it was (the host re-runs the box
    // with a larger list); any other failure invalidates it
    // (in a cluster every CTA holds the same state: the first one stores it)
    if (status == MDEOS_OK && g.crank == 0) save_warm<APT>(g, b, bd, lam);
    if (g.tid == 0 && g.crank == 0 && status != MDEOS_ENBR)
      *(volatile unsigned long long*)bd.warm_tag = (status == MDEOS_OK) ? bd.element_id : 0ull;
  }
  // restriction: time averages and block standard errors
  if (g.tid == 0 && g.crank == 0) {
    const double E_cold = boxc[0], E_ref = boxc[1], Tk = boxc[3];
    const double m = bd.steps_avg;
    mdeos_result r;
    for (int k = 0; k < 6; ++k) r.sigma[k] = acc[ACC_RUN + k] / m;
    r.P = acc[ACC_RUN + 10] / m;
    r.T = acc[ACC_RUN + 11] / m;
    r.epot = acc[ACC_RUN + 6] / m / n;
    r.ekin = acc[ACC_RUN + 7] / m / n;
    r.e_achieved = (acc[ACC_RUN + 7] / m + acc[ACC_RUN + 6] / m - E_ref) / n;
    double mP = 0.0, mT = 0.0;
    for (int k = 0; k < nb; ++k) {
      const double c = g.bcnt()[k] > 0 ? (double)g.bcnt()[k] : 1.0;
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
    r.P_se = sqrt(vP / (nb - 1) / nb);
    r.T_se = sqrt(vT / (nb - 1) / nb);
    r.T_target = Tk;
    r.e_cold = E_cold / n;
    r.L = bd.L;
    r.pairs_per_step = acc[ACC_RUN + 8] / m;
    r.cand_per_step = acc[ACC_RUN + 9] / m;
    r.element_id = bd.element_id;
    r.natoms = n;
    r.status = status;
    r.nlist_builds = builds;
    r.path = PATH;
    r.warm = g.ctrl()[CTRL_WARM];
    r.nlist_retries = 0;
    if (status != MDEOS_OK) {
      r.P = r.T = r.epot = r.ekin = r.e_achieved = r.P_se = r.T_se = 0.0;
      for (int k = 0; k < 6; ++k) r.sigma[k] = 0.0;
    }
    *out = r;
  }
  gbar(g.bar, g.nt);
}

template <int APT>
__device__ __forceinline__ void run_box_path(const Group& g, const BoxDesc& bd, const RunParams& rp,
                                             mdeos_result* out) {
  switch (bd.path) {
    case PATH_NLIST: run_box<APT, PATH_NLIST>(g, bd, rp, out); break;
    case PATH_ALLPAIRS_MI: run_box<APT, PATH_ALLPAIRS_MI>(g, bd, rp, out); break;
    default: run_box<APT, PATH_ALLPAIRS>(g, bd, rp, out); break;
  }
}

}  // namespace mdeos
