// Surrogate EOS: an ensemble of MLPs 2 -> 128 -> 128 -> 128 -> 2 (tanh) mapping
// normalised (rho, e) to normalised (P, T), trained on MD answers of this library,
// used as a gate in front of the MD path (queries on which the ensemble disagrees
// fall back to MD).
//
// Precision (BF16 weights, FP32 accumulation): weight matrices enter every product
// rounded to bfloat16; hidden activations h1..h3 and the error signals dz2, dz3 that
// feed tensor-core products are bfloat16; biases, pre-activations, outputs, gradients
// and the Adam state are FP32 (FP32 master weights).
//
// The 128x128 layers (forward Z = H W^T, backward dW = dZ^T H and dH = dZ W) run on the
// tensor cores through one GEMM kernel (mma.m16n8k16, bf16 x bf16 -> fp32), batched
// over the ensemble members on grid z; the 2-wide layers and the elementwise steps
// run on the CUDA cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "mdeos_host.h"

namespace mdeos {

constexpr int kH = 128;
// parameter offsets of one model: W1[128,2] b1 W2[128,128] b2 W3[128,128] b3 W4[2,128] b4[2]
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * 2, kOffW2 = kOffB1 + kH;
constexpr int kOffB2 = kOffW2 + kH * kH, kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH * kH;
constexpr int kOffW4 = kOffB3 + kH, kOffB4 = kOffW4 + 2 * kH, kNParam = kOffB4 + 2;

// ---------------------------------------------------------------------------
// C[z](m, n) = sum_k A[z](m, k) B[z](k, n): bf16 operands with arbitrary strides (in
// elements), fp32 result (bf16_gemm_tc_kernel below).
struct GemmArgs {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  float* C;
  int M, N, K;
  long long sa_m, sa_k, sa_z, sb_k, sb_n, sb_z, sc_m, sc_n, sc_z;
  // split of K over S CTAs per tile (kchunk elements of K each, a multiple of the
  // staged chunk): with S > 1 every CTA writes its partial tile to ws[s][z][m][n]
  // (dense), summed in the order s = 0, 1, ... by gemm_splitk_reduce
  int S, kchunk;
  float* ws;
};

// ---------------------------------------------------------------------------
// elementwise parts; index layout [model][sample][unit]

// tanh for the hidden layers, whose outputs are rounded to bf16 next (half an ulp:
// 2^-9 relative).  |x| >= 1/4: tanh|x| = 1 - 2 / (1 + e^{2|x|}) with e^{2|x|} =
// 2^{2|x| log2 e} from ex2.approx and the reciprocal from rcp.approx; |x| < 1/4, where
// that form cancels: the odd series x (1 - x^2/3 + 2x^4/15 - 17x^6/315), whose first
// omitted term is below 4e-7 relative there.  Relative error below 2e-6 everywhere
// (3.8e-7 with exact exp2 and division; the approximate instructions add at most ~5e-7,
// largest near |x| = 1/4), so a bf16 rounding differs from that of the exact tanh only
// within 2e-6 of a rounding boundary.  Saturates to +-1 for large |x|; NaN stays NaN.
__device__ __forceinline__ float tanh_act(float x) {
  const float ax = fabsf(x);
  float e, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(ax * 2.885390081777927f));  // 2 log2(e)
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + e));
  const float big = fmaf(-2.0f, r, 1.0f);
  const float x2 = x * x;
  const float small =
      ax * fmaf(x2, fmaf(x2, fmaf(x2, -17.0f / 315.0f, 2.0f / 15.0f), -1.0f / 3.0f), 1.0f);
  return copysignf(ax < 0.25f ? small : big, x);
}

// refresh the bf16 weight copies from the FP32 master parameters
__global__ void mlp_cast_weights(const float* P, __nv_bfloat16* W1b, __nv_bfloat16* W2b,
                                 __nv_bfloat16* W3b, __nv_bfloat16* W4b, int E) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)E * kH * kH;
  if (i >= n) return;
  const int e = (int)(i / (kH * kH)), r = (int)(i % (kH * kH));
  const float* p = P + (long long)e * kNParam;
  W2b[i] = __float2bfloat16_rn(p[kOffW2 + r]);
  W3b[i] = __float2bfloat16_rn(p[kOffW3 + r]);
  if (r < 2 * kH) {
    W1b[(long long)e * 2 * kH + r] = __float2bfloat16_rn(p[kOffW1 + r]);
    W4b[(long long)e * 2 * kH + r] = __float2bfloat16_rn(p[kOffW4 + r]);
  }
}

// h1 = bf16(tanh(W1 x + b1)); x [B][2] FP32 (normalised, shared by the models)
__global__ void mlp_layer1(const float* X, const float* P, const __nv_bfloat16* W1b,
                           __nv_bfloat16* H1, int B, int E) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)E * B * kH) return;
  const int j = (int)(i % kH), b = (int)((i / kH) % B), e = (int)(i / ((long long)B * kH));
  const float w0 = __bfloat162float(W1b[(long long)e * 2 * kH + 2 * j]);
  const float w1 = __bfloat162float(W1b[(long long)e * 2 * kH + 2 * j + 1]);
  const float z = X[2 * b] * w0 + X[2 * b + 1] * w1 + P[(long long)e * kNParam + kOffB1 + j];
  H1[i] = __float2bfloat16_rn(tanh_act(z));
}

// h = bf16(tanh(Z + b)) for layers 2 and 3
__global__ void mlp_bias_tanh(const float* Z, const float* P, int off_b, __nv_bfloat16* Hout,
                              int B, int E) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)E * B * kH) return;
  const int j = (int)(i % kH), e = (int)(i / ((long long)B * kH));
  Hout[i] = __float2bfloat16_rn(tanh_act(Z[i] + P[(long long)e * kNParam + off_b + j]));
}

// y = W4 h3 + b4 (FP32 accumulation); with targets: dy = 2 (y - t) / (2 B) and the
// squared-error sum (one atomic per block)
__global__ void mlp_output(const __nv_bfloat16* H3, const float* P, const __nv_bfloat16* W4b,
                           const float* T, float* Y, float* dY, float* loss, int B, int E) {
  __shared__ float s_l[8];
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < (long long)E * B * 2) {
    const int o = (int)(i % 2), b = (int)((i / 2) % B), e = (int)(i / (2LL * B));
    const __nv_bfloat16* h = H3 + ((long long)e * B + b) * kH;
    const __nv_bfloat16* w = W4b + (long long)e * 2 * kH + o * kH;
    float y = 0.f;
    for (int j = 0; j < kH; ++j) y = fmaf(__bfloat162float(w[j]), __bfloat162float(h[j]), y);
    y += P[(long long)e * kNParam + kOffB4 + o];
    Y[i] = y;
    if (T) {
      const float d = y - T[2 * b + o];
      dY[i] = d / (float)B;  // 2 (y - t) / (2 B)
      l = d * d;
    }
  }
  if (T) {
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) s_l[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_l[w];
      atomicAdd(loss, s);
    }
  }
}

// output layer backward: dW4, db4 (reductions over the batch, one thread per weight)
__global__ void mlp_back_out_w(const float* dY, const __nv_bfloat16* H3, float* G, int B, int E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E * (2 * kH + 2)) return;
  const int e = i / (2 * kH + 2), r = i % (2 * kH + 2);
  float s = 0.f;
  if (r < 2 * kH) {
    const int o = r / kH, j = r % kH;
    for (int b = 0; b < B; ++b)
      s = fmaf(dY[((long long)e * B + b) * 2 + o],
               __bfloat162float(H3[((long long)e * B + b) * kH + j]), s);
    G[(long long)e * kNParam + kOffW4 + r] = s;
  } else {
    const int o = r - 2 * kH;
    for (int b = 0; b < B; ++b) s += dY[((long long)e * B + b) * 2 + o];
    G[(long long)e * kNParam + kOffB4 + o] = s;
  }
}

// dz3 = bf16((dy W4) * (1 - h3^2))
__global__ void mlp_back_out_dz(const float* dY, const __nv_bfloat16* H3, const __nv_bfloat16* W4b,
                                __nv_bfloat16* dZ3, int B, int E) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)E * B * kH) return;
  const int j = (int)(i % kH), b = (int)((i / kH) % B), e = (int)(i / ((long long)B * kH));
  const float* dy = dY + ((long long)e * B + b) * 2;
  const __nv_bfloat16* w = W4b + (long long)e * 2 * kH;
  const float dh = dy[0] * __bfloat162float(w[j]) + dy[1] * __bfloat162float(w[kH + j]);
  const float h = __bfloat162float(H3[i]);
  dZ3[i] = __float2bfloat16_rn(dh * (1.f - h * h));
}

// dz = dH (1 - h^2), rounded to bf16 (layer 2) or kept FP32 (layer 1)
__global__ void mlp_deriv(const float* dH, const __nv_bfloat16* Hh, __nv_bfloat16* dZb, float* dZf,
                          long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h = __bfloat162float(Hh[i]);
  const float d = dH[i] * (1.f - h * h);
  if (dZb) dZb[i] = __float2bfloat16_rn(d);
  if (dZf) dZf[i] = d;
}

// bias gradient: column sums of dz over the batch
__global__ void mlp_bias_grad(const __nv_bfloat16* dZb, const float* dZf, float* G, int off_b,
                              int B, int E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E * kH) return;
  const int e = i / kH, j = i % kH;
  float s = 0.f;
  for (int b = 0; b < B; ++b) {
    const long long k = ((long long)e * B + b) * kH + j;
    s += dZb ? __bfloat162float(dZb[k]) : dZf[k];
  }
  G[(long long)e * kNParam + off_b + j] = s;
}

// first-layer weight gradient dW1 = dz1^T x (FP32)
__global__ void mlp_grad_w1(const float* dZ1, const float* X, float* G, int B, int E) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E * 2 * kH) return;
  const int e = i / (2 * kH), r = i % (2 * kH), j = r / 2, c = r % 2;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s = fmaf(dZ1[((long long)e * B + b) * kH + j], X[2 * b + c], s);
  G[(long long)e * kNParam + kOffW1 + r] = s;
}

// Adam (Kingma & Ba) on the FP32 master parameters; omb = 1 - beta and c = 1 - beta^t,
// each evaluated in FP64 on the host and rounded once
__global__ void mlp_adam(float* P, const float* G, float* Mm, float* Vv, long long n, float lr,
                         float b1, float b2, float omb1, float omb2, float eps, float c1,
                         float c2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float m = b1 * Mm[i] + omb1 * g;
  const float v = b2 * Vv[i] + omb2 * g * g;
  Mm[i] = m;
  Vv[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// normalise physical inputs (rho, e) -> x, per sample
__global__ void mlp_normalise(const double* Xp, float* X, int B, double m0, double m1, double s0,
                              double s1) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  X[2 * b] = (float)((Xp[2 * b] - m0) / s0);
  X[2 * b + 1] = (float)((Xp[2 * b + 1] - m1) / s1);
}

// ensemble mean and (population) standard deviation of the physical outputs; with
// p_asinh the networks predict asinh(P), mapped back by sinh before averaging
__global__ void mlp_ensemble(const float* Y, int B, int E, double ym0, double ym1, double ys0,
                             double ys1, int p_asinh, double* mean, double* sd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * 2) return;
  const int o = i % 2;
  const double m = o ? ym1 : ym0, s = o ? ys1 : ys0;
  double a = 0.0, q = 0.0;
  for (int e = 0; e < E; ++e) {
    double y = (double)Y[(long long)e * B * 2 + i] * s + m;
    if (o == 0 && p_asinh) y = sinh(y);
    a += y;
    q += y * y;
  }
  a /= E;
  mean[i] = a;
  sd[i] = sqrt(fmax(q / E - a * a, 0.0));
}

// ---------------------------------------------------------------------------
// Fused inference on the 5th-generation tensor cores, in tiles of 128 samples of one
// model.  Layer 1 (2 -> 128) runs on the CUDA cores and writes h1 into shared memory;
// layers 2 and 3 are tcgen05.mma (M = N = 128, K = 128 in steps of 16, bf16 x bf16 ->
// fp32) with the accumulator in tensor memory (128 columns), completion signalled on
// an mbarrier; threads read their row back (tcgen05.ld, 32 columns at a time), add
// the bias, apply tanh and write the next operand into the same tile; the 128 -> 2
// output layer reads h3 back from shared memory.
//
// Operand layout in shared memory (no swizzle, K contiguous): 8 x 8 "core matrices"
// of 128 bytes; element (r, k) at (r / 8) * SBO + (k / 8) * LBO + (r % 8) * 16 +
// (k % 8) * 2 with LBO = 128 B (next core matrix along K) and SBO = 2048 B (next
// 8-row group).  Every address an MMA can form stays inside its 32 KB tile.

constexpr int kTcRows = 128;                   // samples per tile (TMEM lanes)
constexpr int kTcThreads = 256;                // two threads per row (column halves)
constexpr uint32_t kLbo = 128, kSbo = 2048;    // bytes
constexpr int kTcTile = kH * kH * 2;           // 32 KB per operand tile
// FP32 copies of the small parameters behind the tiles and the mbarrier: W1 as
// (w_c0, w_c1) pairs, b1, b2, b3, W4 (output-major), b4
constexpr int kTcSW1 = 0, kTcSB1 = kTcSW1 + 2 * kH, kTcSB2 = kTcSB1 + kH, kTcSB3 = kTcSB2 + kH;
constexpr int kTcSW4 = kTcSB3 + kH, kTcSB4 = kTcSW4 + 2 * kH, kTcSmall = kTcSB4 + 4;
constexpr int kTcSmem = 3 * kTcTile + 1024 + 64 + kTcSmall * 4;

__device__ __forceinline__ uint32_t tc_off(int r, int k) {
  return (uint32_t)((r >> 3) * kSbo + (k >> 3) * kLbo + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, LBO, SBO (all >> 4), version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kLbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kSbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, N = M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH >> 3) << 17) |
                            ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      ::"r"(tmem), "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(mbar) : "memory");
}

__device__ __forceinline__ unsigned long long tc_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// wait on an mbarrier phase for at most ~1 s; false if it did not complete
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const unsigned long long t0 = tc_clock_ns();
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    if (done) return true;
    if ((it & 255) == 255 && tc_clock_ns() - t0 > 1000000000ull) break;
  }
  return false;
}

// 32 consecutive fp32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// bf16(tanh(z + bias)) of 8 consecutive units, packed as one 16-byte core-matrix row
__device__ __forceinline__ uint4 tanh_pack8(const float* z, const float* bias) {
  uint4 pk;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
  for (int j = 0; j < 8; j += 2)
    h[j >> 1] = __floats2bfloat162_rn(tanh_act(z[j] + bias[j]), tanh_act(z[j + 1] + bias[j + 1]));
  return pk;
}

// Persistent: grid (CTAs per model, models).  The CTA stages its model's W2 and W3
// once, then takes 128-input tiles tile = blockIdx.x, + gridDim.x, ...  Thread t
// serves row m = t % 128 (TMEM lane m) and column half t / 128: warps w and w + 4
// read the same 32 lanes, columns 0-63 and 64-127.
__global__ void __launch_bounds__(kTcThreads) mlp_infer_tc_kernel(const float* X, const float* P,
                                                                  const __nv_bfloat16* W1b,
                                                                  const __nv_bfloat16* W2b,
                                                                  const __nv_bfloat16* W3b,
                                                                  const __nv_bfloat16* W4b,
                                                                  float* Y, int B, int* err) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  const uint32_t sbase = ((uint32_t)__cvta_generic_to_shared(tsm) + 1023u) & ~1023u;
  unsigned char* gbase = tsm + (sbase - (uint32_t)__cvta_generic_to_shared(tsm));
  const uint32_t sA = sbase, sW2 = sbase + kTcTile, sW3 = sbase + 2 * kTcTile;
  const uint32_t sMbar = sbase + 3 * kTcTile, sTmem = sMbar + 8;
  unsigned char* gA = gbase;
  const int e = blockIdx.y, tid = threadIdx.x, warp = tid >> 5;
  const int m = tid & (kTcRows - 1), half = tid >> 7, c_lo = half * (kH / 2);
  const int ntiles = (B + kTcRows - 1) / kTcRows;
  const float* p = P + (long long)e * kNParam;
  float* sp = reinterpret_cast<float*>(gbase + 3 * kTcTile + 64);  // small parameters
  for (int k = tid; k < 2 * kH; k += kTcThreads) {  // the bf16-rounded weights, as FP32
    sp[kTcSW1 + k] = __bfloat162float(W1b[(long long)e * 2 * kH + k]);
    sp[kTcSW4 + k] = __bfloat162float(W4b[(long long)e * 2 * kH + k]);
  }
  for (int k = tid; k < kH; k += kTcThreads) {
    sp[kTcSB1 + k] = p[kOffB1 + k];
    sp[kTcSB2 + k] = p[kOffB2 + k];
    sp[kTcSB3 + k] = p[kOffB3 + k];
  }
  if (tid < 2) sp[kTcSB4 + tid] = p[kOffB4 + tid];
  const float* w4 = sp + kTcSW4 + half * kH;  // output unit = half
  // weights of this model into the canonical layout, 16 bytes at a time; consecutive
  // threads fill consecutive 16-byte rows of the core matrices (no bank conflicts)
  for (int q = tid; q < kH * kH / 8; q += kTcThreads) {
    const int n = (q >> 7) * 8 + (q & 7), k = ((q >> 3) & 15) * 8;
    const uint4 a2 = *reinterpret_cast<const uint4*>(W2b + (long long)e * kH * kH + n * kH + k);
    const uint4 a3 = *reinterpret_cast<const uint4*>(W3b + (long long)e * kH * kH + n * kH + k);
    *reinterpret_cast<uint4*>(gbase + kTcTile + tc_off(n, k)) = a2;
    *reinterpret_cast<uint4*>(gbase + 2 * kTcTile + tc_off(n, k)) = a3;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sMbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // 128 TMEM columns: the 128 x 128 fp32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(sTmem), "r"(kH) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(gbase + 3 * kTcTile + 8);
  // this thread's lane quarter (warp % 4) and column half
  const uint32_t tq = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c_lo;
  uint32_t commits = 0;  // MMA groups committed so far (mbarrier phase parity)
  bool ok = true;
  int tile = blockIdx.x;
  for (; tile < ntiles; tile += gridDim.x) {
    const int b = tile * kTcRows + m;
    // layer 1 on the CUDA cores: this row's units c_lo .. c_lo + 63 -> tile A
    const float x0 = b < B ? X[2 * b] : 0.f, x1 = b < B ? X[2 * b + 1] : 0.f;
#pragma unroll 1
    for (int c = c_lo; c < c_lo + kH / 2; c += 8) {
      float z[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float2 w = *reinterpret_cast<const float2*>(sp + kTcSW1 + 2 * (c + j));
        z[j] = x0 * w.x + x1 * w.y;
      }
      *reinterpret_cast<uint4*>(gA + tc_off(m, c)) = tanh_pack8(z, sp + kTcSB1 + c);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // h1 -> tensor core
    __syncthreads();
    for (int layer = 0; layer < 2; ++layer) {
      if (tid == 0) {
        const uint32_t sW = layer == 0 ? sW2 : sW3;
#pragma unroll
        for (int ks = 0; ks < kH / 16; ++ks)  // K step of 16 = two core matrices along K
          tc_mma(tmem, tc_desc(sA + ks * 2 * kLbo), tc_desc(sW + ks * 2 * kLbo), ks > 0);
        tc_commit(sMbar);
      }
      __syncwarp();
      const bool done = mbar_wait(sMbar, commits & 1u);
      ++commits;
      ok = __syncthreads_and(done) != 0;  // the same decision in every thread
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok) break;
      // epilogue: h = bf16(tanh(z + b)) of this row's 64 units -> tile A (the MMA that
      // read it has completed): h2 feeds layer 3, h3 the output layer
      const float* bias = sp + (layer == 0 ? kTcSB2 : kTcSB3) + c_lo;
#pragma unroll 1
      for (int c0 = 0; c0 < kH / 2; c0 += 32) {
        float v[32];
        tc_ld32(tq + (uint32_t)c0, v);
#pragma unroll
        for (int j8 = 0; j8 < 32; j8 += 8)
          *reinterpret_cast<uint4*>(gA + tc_off(m, c_lo + c0 + j8)) =
              tanh_pack8(v + j8, bias + c0 + j8);
      }
      if (layer == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!ok) break;
    // output unit `half` of row m: sum over the 128 units of h3 in order, FP32
    float y = 0.f;
#pragma unroll 1
    for (int c = 0; c < kH; c += 8) {
      const uint4 pk = *reinterpret_cast<const uint4*>(gA + tc_off(m, c));
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&pk);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 hf = __bfloat1622float2(h[j]);
        y = fmaf(w4[c + 2 * j], hf.x, y);
        y = fmaf(w4[c + 2 * j + 1], hf.y, y);
      }
    }
    if (b < B) Y[((long long)e * B + b) * 2 + half] = y + sp[kTcSB4 + half];
    __syncthreads();  // tile A is rewritten by the next tile's layer 1
  }
  if (!ok) {  // NaN for this CTA's unfinished tiles; let MMAs in flight finish (bounded)
    if (tid == 0) atomicExch(err, 1);
    for (; tile < ntiles; tile += gridDim.x) {
      const int b = tile * kTcRows + m;
      if (b < B) Y[((long long)e * B + b) * 2 + half] = __int_as_float(0x7fc00000);
    }
    mbar_wait(sMbar, (commits - 1u) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  __syncwarp();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kH)
                 : "memory");
}

// ---------------------------------------------------------------------------
// The training products on the 5th-generation tensor cores: C[z](m, n) =
// sum_k A[z](m, k) B[z](k, n) with arbitrary strides (GemmArgs), one 128 x 128 tile of
// C per CTA with the fp32 accumulator in
// tensor memory.  K runs in chunks of 64: the 128 threads stage A's 128 x 64 and B's
// (128 columns of C) x 64 elements into the canonical no-swizzle K-major layout (8 x 8
// core matrices of 128 B: element (r, k) at (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16
// + (k % 8) * 2; zero outside the matrices), one thread issues four tcgen05.mma of
// K = 16 and commits to an mbarrier, and every thread waits (at most ~1 s, then the
// error flag is set and the tile is left unwritten) before the next chunk overwrites the
// tiles.  Epilogue: thread t reads TMEM lane t (row m0 + t), 32 columns at a time.

constexpr int kGK = 64;                   // K per staged chunk
constexpr uint32_t kGSbo = 1024;          // bytes between 8-row groups of a chunk
constexpr int kGTile = kTcRows * kGK * 2; // 16 KB per operand chunk

__device__ __forceinline__ uint32_t gk_off(int r, int k) {
  return (uint32_t)((r >> 3) * kGSbo + (k >> 3) * kLbo + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t gk_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kLbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((kGSbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__global__ void __launch_bounds__(kTcRows) bf16_gemm_tc_kernel(GemmArgs g, int* err) {
  __shared__ __align__(1024) unsigned char gsm[2 * kGTile];
  __shared__ __align__(8) unsigned long long s_mbar;
  __shared__ uint32_t s_tmem;
  const int z = blockIdx.z / g.S, sk = blockIdx.z - z * g.S;
  const int m0 = blockIdx.y * kTcRows, n0 = blockIdx.x * kH;
  const int kbeg = sk * g.kchunk, kend = min(g.K, kbeg + g.kchunk);  // this CTA's part of K
  const __nv_bfloat16* A = g.A + (long long)z * g.sa_z;
  const __nv_bfloat16* B = g.B + (long long)z * g.sb_z;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sA = (uint32_t)__cvta_generic_to_shared(gsm), sB = sA + kGTile;
  const uint32_t mbar = (uint32_t)__cvta_generic_to_shared(&s_mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // 128 TMEM columns: the 128 x 128 fp32 accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"((uint32_t)__cvta_generic_to_shared(&s_tmem)), "r"(kH) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(&s_tmem);
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  uint32_t commits = 0;
  bool ok = true;
  // operands contiguous along K (and 16-byte aligned rows): eight elements per load,
  // one core-matrix row per store; otherwise element by element with the contiguous
  // index (M or N) running fastest across the threads
  const bool a_vec = g.sa_k == 1 && (g.sa_m & 7) == 0 && (g.sa_z & 7) == 0 &&
                     ((uintptr_t)g.A & 15) == 0 && (g.K & 7) == 0;
  const bool b_vec = g.sb_k == 1 && (g.sb_n & 7) == 0 && (g.sb_z & 7) == 0 &&
                     ((uintptr_t)g.B & 15) == 0 && (g.K & 7) == 0;
  for (int k0 = kbeg; k0 < kend; k0 += kGK) {
    if (a_vec) {
      for (int q = tid; q < kTcRows * (kGK / 8); q += kTcRows) {
        const int r = q & (kTcRows - 1), c = (q >> 7) * 8;  // consecutive threads: rows
        const int m = m0 + r, k = k0 + c;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (m < g.M && k < kend) v = *reinterpret_cast<const uint4*>(A + (long long)m * g.sa_m + k);
        *reinterpret_cast<uint4*>(gsm + gk_off(r, c)) = v;
      }
    } else {  // eight loads in flight per thread, then their stores
      for (int c0 = 0; c0 < kGK; c0 += 8) {
        const int r = tid, m = m0 + r;  // consecutive threads: rows (M)
        __nv_bfloat16 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = k0 + c0 + u;
          v[u] = (m < g.M && k < kend) ? A[(long long)m * g.sa_m + (long long)k * g.sa_k] : zero;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) *reinterpret_cast<__nv_bfloat16*>(gsm + gk_off(r, c0 + u)) = v[u];
      }
    }
    if (b_vec) {
      for (int q = tid; q < kTcRows * (kGK / 8); q += kTcRows) {
        const int r = q & (kTcRows - 1), c = (q >> 7) * 8;
        const int n = n0 + r, k = k0 + c;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (n < g.N && k < kend) v = *reinterpret_cast<const uint4*>(B + (long long)n * g.sb_n + k);
        *reinterpret_cast<uint4*>(gsm + kGTile + gk_off(r, c)) = v;
      }
    } else {
      for (int c0 = 0; c0 < kGK; c0 += 8) {
        const int r = tid, n = n0 + r;  // consecutive threads: columns (N)
        __nv_bfloat16 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int k = k0 + c0 + u;
          v[u] = (n < g.N && k < kend) ? B[(long long)k * g.sb_k + (long long)n * g.sb_n] : zero;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          *reinterpret_cast<__nv_bfloat16*>(gsm + kGTile + gk_off(r, c0 + u)) = v[u];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // tiles -> tensor core
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < kGK / 16; ++ks)  // K step of 16 = two core matrices along K
        tc_mma(tmem, gk_desc(sA + ks * 2 * kLbo), gk_desc(sB + ks * 2 * kLbo),
               (k0 > kbeg || ks > 0) ? 1u : 0u);
      tc_commit(mbar);
    }
    __syncwarp();
    const bool done = mbar_wait(mbar, commits & 1u);
    ++commits;
    ok = __syncthreads_and(done) != 0;  // the same decision in every thread
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) break;
  }
  if (ok) {
    const int m = m0 + tid;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    const int Z = gridDim.z / g.S;
    float* C = g.S > 1 ? g.ws + ((long long)sk * Z + z) * g.M * g.N : g.C + (long long)z * g.sc_z;
    const long long cm = g.S > 1 ? g.N : g.sc_m, cn = g.S > 1 ? 1 : g.sc_n;
#pragma unroll 1
    for (int c0 = 0; c0 < kH; c0 += 32) {
      float v[32];
      tc_ld32(tl + (uint32_t)c0, v);  // every lane of the warp, in or out of the matrix
      if (m < g.M)
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + c0 + j;
          if (n < g.N) C[(long long)m * cm + (long long)n * cn] = v[j];
        }
    }
  } else {  // leave the tile unwritten; let the MMAs in flight finish (bounded)
    if (tid == 0) atomicExch(err, 1);
    mbar_wait(mbar, (commits - 1u) & 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  __syncwarp();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kH)
                 : "memory");
}

// C[z](m, n) = sum over s = 0, 1, ..., S - 1 of the partial tiles ws[s][z][m][n]
__global__ void gemm_splitk_reduce(const float* ws, float* C, int M, int N, int Z, int S,
                                   long long sc_m, long long sc_n, long long sc_z) {
  const long long per = (long long)M * N, all = per * Z;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < all;
       i += (long long)gridDim.x * blockDim.x) {
    const int z = (int)(i / per);
    const long long r = i - z * per;
    const int m = (int)(r / N), n = (int)(r - (long long)m * N);
    float acc = ws[i];
    for (int s = 1; s < S; ++s) acc += ws[s * all + i];
    C[z * sc_z + m * sc_m + n * sc_n] = acc;
  }
}

__global__ void debug_tanh_kernel(const float* x, float* y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = tanh_act(x[i]);
}

}  // namespace mdeos

using namespace mdeos;

struct mdeos_surrogate {
  mdeos_handle* h = nullptr;
  int E = 4, maxB = 0;
  double norm[8] = {0, 0, 1, 1, 0, 0, 1, 1};  // x mean(2), x std(2), y mean(2), y std(2)
  int p_asinh = 0;  // 1: the networks learn asinh(P) (norm[4], norm[6] in those units)
  long long step = 0;
  float *P = nullptr, *G = nullptr, *Mm = nullptr, *Vv = nullptr;
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W4b = nullptr;
  __nv_bfloat16 *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *dZb = nullptr;
  float *Z = nullptr, *dZf = nullptr, *X = nullptr, *T = nullptr, *Y = nullptr, *dY = nullptr;
  float* loss = nullptr;
  double *Xp = nullptr, *mean = nullptr, *sd = nullptr;
  int* err = nullptr;  // set by the fused kernel when an MMA wait ran out
  float* ws = nullptr;  // partial tiles of the products whose K is split
  long long ws_elems = 0;
  int infer_path = MDEOS_SURROGATE_INFER_TC;
  bool tc_ready = false;
  int nsm = 1;
  std::vector<void*> allocs;
  // misfit map: RMS relative pressure residual of the ensemble mean per cell of a
  // bins x bins grid over the inputs it was fitted on (infinite: too few samples)
  int mis_bins = 0;
  double mis_lo[2] = {0, 0}, mis_hi[2] = {1, 1};
  std::vector<double> mis;
  double mis_threshold = INFINITY;  // gate: reject above this (infinite: map not used)
};

#define SCK(call)                                                                      \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return set_error(MDEOS_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

constexpr int kMaxSplitK = 16;  // most CTAs one tile's K is split over

// the training products: tcgen05 tiles of 128 x 128 (bf16_gemm_tc_kernel); a tensor-core
// wait that ran out sets *err (device int) and leaves its tile unwritten.  Products with
// few tiles and a long K (the weight gradients, K = batch) split K over up to
// kMaxSplitK CTAs per tile, at least two chunks each, when the workspace ws (ws_elems
// floats) holds the partial tiles; the partials are summed in a fixed order, so every
// result is the same from run to run.
static cudaError_t gemm(cudaStream_t st, int* err, float* ws, long long ws_elems,
                        const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, int M, int N,
                        int K, long long sa_m, long long sa_k, long long sa_z, long long sb_k,
                        long long sb_n, long long sb_z, long long sc_m, long long sc_n,
                        long long sc_z, int Z) {
  const int tiles = ((N + kH - 1) / kH) * ((M + kTcRows - 1) / kTcRows) * Z;
  const int nch = (K + kGK - 1) / kGK;
  int S = 1, per = nch;
  if (ws && tiles < 64 && nch >= 4) {
    const int s0 = std::min(nch / 2, kMaxSplitK);
    per = (nch + s0 - 1) / s0;
    S = (nch + per - 1) / per;  // every split holds at least one chunk
    if ((long long)S * Z * M * N > ws_elems) S = 1, per = nch;
  }
  GemmArgs g{A, B, C, M, N, K, sa_m, sa_k, sa_z, sb_k, sb_n, sb_z, sc_m, sc_n, sc_z,
             S, per * kGK, S > 1 ? ws : nullptr};
  dim3 grid((N + kH - 1) / kH, (M + kTcRows - 1) / kTcRows, Z * S);
  bf16_gemm_tc_kernel<<<grid, kTcRows, 0, st>>>(g, err);
  if (S > 1) {
    const long long all = (long long)Z * M * N;
    gemm_splitk_reduce<<<(int)std::min<long long>((all + 255) / 256, 1024), 256, 0, st>>>(
        ws, C, M, N, Z, S, sc_m, sc_n, sc_z);
  }
  return cudaGetLastError();
}

static int nblk(long long n, int t = 256) { return (int)((n + t - 1) / t); }

// forward of all models on s->X (B samples): H1..H3, Y; with targets also dY and loss
static cudaError_t forward(mdeos_surrogate* s, int B, const float* T, cudaStream_t st) {
  const int E = s->E;
  const long long EB = (long long)E * B;
  const long long sz = (long long)B * kH;
  cudaError_t e;
  mlp_layer1<<<nblk(EB * kH), 256, 0, st>>>(s->X, s->P, s->W1b, s->H1, B, E);
  // Z2 = H1 W2^T: A(m=b, k=j) = H1[b][j], B(k=j, n=o) = W2[o][j]
  e = gemm(st, s->err, s->ws, s->ws_elems, s->H1, s->W2b, s->Z, B, kH, kH, kH, 1, sz, 1, kH, kH * kH, kH, 1, sz, E);
  if (e != cudaSuccess) return e;
  mlp_bias_tanh<<<nblk(EB * kH), 256, 0, st>>>(s->Z, s->P, kOffB2, s->H2, B, E);
  e = gemm(st, s->err, s->ws, s->ws_elems, s->H2, s->W3b, s->Z, B, kH, kH, kH, 1, sz, 1, kH, kH * kH, kH, 1, sz, E);
  if (e != cudaSuccess) return e;
  mlp_bias_tanh<<<nblk(EB * kH), 256, 0, st>>>(s->Z, s->P, kOffB3, s->H3, B, E);
  mlp_output<<<nblk(EB * 2), 256, 0, st>>>(s->H3, s->P, s->W4b, T, s->Y, s->dY, s->loss, B, E);
  return cudaGetLastError();
}

// gradients of the mean-squared error of the batch into s->G
static cudaError_t backward(mdeos_surrogate* s, int B, cudaStream_t st) {
  const int E = s->E;
  const long long EB = (long long)E * B;
  const long long sz = (long long)B * kH;
  cudaError_t e;
  mlp_back_out_w<<<nblk(E * (2 * kH + 2)), 256, 0, st>>>(s->dY, s->H3, s->G, B, E);
  mlp_back_out_dz<<<nblk(EB * kH), 256, 0, st>>>(s->dY, s->H3, s->W4b, s->dZb, B, E);
  // dW3 = dZ3^T H2: A(m=o, k=b) = dZ3[b][o], B(k=b, n=j) = H2[b][j]
  e = gemm(st, s->err, s->ws, s->ws_elems, s->dZb, s->H2, s->G + kOffW3, kH, kH, B, 1, kH, sz, kH, 1, sz, kH, 1, kNParam, E);
  if (e != cudaSuccess) return e;
  mlp_bias_grad<<<nblk(E * kH), 256, 0, st>>>(s->dZb, nullptr, s->G, kOffB3, B, E);
  // dH2 = dZ3 W3: A(m=b, k=o) = dZ3[b][o], B(k=o, n=j) = W3[o][j]
  e = gemm(st, s->err, s->ws, s->ws_elems, s->dZb, s->W3b, s->Z, B, kH, kH, kH, 1, sz, kH, 1, kH * kH, kH, 1, sz, E);
  if (e != cudaSuccess) return e;
  mlp_deriv<<<nblk(EB * kH), 256, 0, st>>>(s->Z, s->H2, s->dZb, nullptr, EB * kH);
  e = gemm(st, s->err, s->ws, s->ws_elems, s->dZb, s->H1, s->G + kOffW2, kH, kH, B, 1, kH, sz, kH, 1, sz, kH, 1, kNParam, E);
  if (e != cudaSuccess) return e;
  mlp_bias_grad<<<nblk(E * kH), 256, 0, st>>>(s->dZb, nullptr, s->G, kOffB2, B, E);
  e = gemm(st, s->err, s->ws, s->ws_elems, s->dZb, s->W2b, s->Z, B, kH, kH, kH, 1, sz, kH, 1, kH * kH, kH, 1, sz, E);
  if (e != cudaSuccess) return e;
  mlp_deriv<<<nblk(EB * kH), 256, 0, st>>>(s->Z, s->H1, nullptr, s->dZf, EB * kH);
  mlp_bias_grad<<<nblk(E * kH), 256, 0, st>>>(nullptr, s->dZf, s->G, kOffB1, B, E);
  mlp_grad_w1<<<nblk(E * 2 * kH), 256, 0, st>>>(s->dZf, s->X, s->G, B, E);
  return cudaGetLastError();
}

static cudaError_t cast_weights(mdeos_surrogate* s, cudaStream_t st) {
  mlp_cast_weights<<<nblk((long long)s->E * kH * kH), 256, 0, st>>>(s->P, s->W1b, s->W2b, s->W3b,
                                                                    s->W4b, s->E);
  return cudaGetLastError();
}

extern "C" mdeos_status mdeos_surrogate_destroy(mdeos_surrogate* s);

extern "C" mdeos_status mdeos_surrogate_create(mdeos_handle* h, int32_t n_models, int32_t max_batch,
                                               uint64_t seed, mdeos_surrogate** out) {
  if (!h || !out || n_models < 1 || n_models > 16 || max_batch < 1 || max_batch > (1 << 22))
    return set_error(MDEOS_EINVAL, "bad surrogate_create arguments");
  *out = nullptr;
  mdeos_surrogate* s = new mdeos_surrogate();
  s->h = h;
  s->E = n_models;
  s->maxB = max_batch;
  const int E = n_models;
  const long long EB = (long long)E * max_batch;
  cudaError_t e = cudaSetDevice(handle_device(h));
  auto dalloc = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    if (e == cudaSuccess) s->allocs.push_back(*p);
  };
  const size_t np = (size_t)E * kNParam;
  dalloc((void**)&s->P, np * 4);
  dalloc((void**)&s->G, np * 4);
  dalloc((void**)&s->Mm, np * 4);
  dalloc((void**)&s->Vv, np * 4);
  dalloc((void**)&s->W1b, (size_t)E * 2 * kH * 2);
  dalloc((void**)&s->W2b, (size_t)E * kH * kH * 2);
  dalloc((void**)&s->W3b, (size_t)E * kH * kH * 2);
  dalloc((void**)&s->W4b, (size_t)E * 2 * kH * 2);
  dalloc((void**)&s->H1, EB * kH * 2);
  dalloc((void**)&s->H2, EB * kH * 2);
  dalloc((void**)&s->H3, EB * kH * 2);
  dalloc((void**)&s->dZb, EB * kH * 2);
  dalloc((void**)&s->Z, EB * kH * 4);
  dalloc((void**)&s->dZf, EB * kH * 4);
  dalloc((void**)&s->X, (size_t)max_batch * 2 * 4);
  dalloc((void**)&s->T, (size_t)max_batch * 2 * 4);
  dalloc((void**)&s->Y, EB * 2 * 4);
  dalloc((void**)&s->dY, EB * 2 * 4);
  dalloc((void**)&s->loss, 256);
  dalloc((void**)&s->Xp, (size_t)max_batch * 2 * 8);
  dalloc((void**)&s->mean, (size_t)max_batch * 2 * 8);
  dalloc((void**)&s->sd, (size_t)max_batch * 2 * 8);
  dalloc((void**)&s->err, 256);
  s->ws_elems = (long long)kMaxSplitK * E * kH * kH;
  dalloc((void**)&s->ws, (size_t)s->ws_elems * 4);
  if (e != cudaSuccess) {
    mdeos_surrogate_destroy(s);
    return set_error(MDEOS_ECUDA, std::string("surrogate_create: ") + cudaGetErrorString(e));
  }
  // Glorot-uniform weights, zero biases
  std::vector<float> p(np, 0.f);
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  for (int m = 0; m < E; ++m) {
    float* q = p.data() + (size_t)m * kNParam;
    const double l1 = std::sqrt(6.0 / (kH + 2)), l2 = std::sqrt(6.0 / (2 * kH));
    for (int i = 0; i < 2 * kH; ++i) q[kOffW1 + i] = (float)(l1 * u(rng));
    for (int i = 0; i < kH * kH; ++i) q[kOffW2 + i] = (float)(l2 * u(rng));
    for (int i = 0; i < kH * kH; ++i) q[kOffW3 + i] = (float)(l2 * u(rng));
    for (int i = 0; i < 2 * kH; ++i) q[kOffW4 + i] = (float)(l1 * u(rng));
  }
  cudaStream_t st = handle_stream(h);
  e = cudaMemcpyAsync(s->P, p.data(), np * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cast_weights(s, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    mdeos_surrogate_destroy(s);
    return set_error(MDEOS_ECUDA, std::string("surrogate init: ") + cudaGetErrorString(e));
  }
  *out = s;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_set_params(mdeos_surrogate* s, const float* params,
                                                   const double* norm) {
  if (!s) return set_error(MDEOS_EINVAL, "surrogate is NULL");
  cudaStream_t st = handle_stream(s->h);
  SCK(cudaSetDevice(handle_device(s->h)));
  if (params) {
    const size_t np = (size_t)s->E * kNParam;
    SCK(cudaMemcpyAsync(s->P, params, np * 4, cudaMemcpyHostToDevice, st));
    SCK(cudaMemsetAsync(s->Mm, 0, np * 4, st));
    SCK(cudaMemsetAsync(s->Vv, 0, np * 4, st));
    s->step = 0;
    SCK(cast_weights(s, st));
  }
  if (norm) std::memcpy(s->norm, norm, sizeof(s->norm));
  SCK(cudaStreamSynchronize(st));
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_get_params(mdeos_surrogate* s, float* params, double* norm) {
  if (!s) return set_error(MDEOS_EINVAL, "surrogate is NULL");
  SCK(cudaSetDevice(handle_device(s->h)));
  cudaStream_t st = handle_stream(s->h);
  if (params)
    SCK(cudaMemcpyAsync(params, s->P, (size_t)s->E * kNParam * 4, cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
  if (norm) std::memcpy(norm, s->norm, sizeof(s->norm));
  return MDEOS_OK;
}

// the tensor-core error flag of the surrogate's kernels: read and cleared (synchronous)
static mdeos_status take_tc_error(mdeos_surrogate* s, cudaStream_t st) {
  int err = 0;
  SCK(cudaMemcpyAsync(&err, s->err, 4, cudaMemcpyDeviceToHost, st));
  SCK(cudaMemsetAsync(s->err, 0, 4, st));
  SCK(cudaStreamSynchronize(st));
  if (err) return set_error(MDEOS_ETIMEDOUT, "surrogate: a tensor-core wait ran out");
  return MDEOS_OK;
}

// normalised inputs/targets of n samples into s->X / s->T (host FP64 in)
static mdeos_status load_batch(mdeos_surrogate* s, const double* xp, const double* yp, int n,
                               cudaStream_t st) {
  std::vector<float> x(2 * (size_t)n), t;
  for (int b = 0; b < n; ++b)
    for (int c = 0; c < 2; ++c)
      x[2 * b + c] = (float)((xp[2 * b + c] - s->norm[c]) / s->norm[2 + c]);
  SCK(cudaMemcpyAsync(s->X, x.data(), x.size() * 4, cudaMemcpyHostToDevice, st));
  if (yp) {
    t.resize(2 * (size_t)n);
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < 2; ++c) {
        const double y = (c == 0 && s->p_asinh) ? std::asinh(yp[2 * b]) : yp[2 * b + c];
        t[2 * b + c] = (float)((y - s->norm[4 + c]) / s->norm[6 + c]);
      }
    SCK(cudaMemcpyAsync(s->T, t.data(), t.size() * 4, cudaMemcpyHostToDevice, st));
  }
  SCK(cudaStreamSynchronize(st));  // the host vectors go out of scope
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_grads(mdeos_surrogate* s, const double* x, const double* y,
                                              int32_t n, float* grads, double* loss) {
  if (!s || !x || !y || n < 1 || n > s->maxB) return set_error(MDEOS_EINVAL, "bad grads arguments");
  SCK(cudaSetDevice(handle_device(s->h)));
  cudaStream_t st = handle_stream(s->h);
  mdeos_status ms = load_batch(s, x, y, n, st);
  if (ms != MDEOS_OK) return ms;
  SCK(cudaMemsetAsync(s->loss, 0, 4, st));
  SCK(forward(s, n, s->T, st));
  SCK(backward(s, n, st));
  count_launch(s->h, 20);
  if (grads)
    SCK(cudaMemcpyAsync(grads, s->G, (size_t)s->E * kNParam * 4, cudaMemcpyDeviceToHost, st));
  float l = 0.f;
  SCK(cudaMemcpyAsync(&l, s->loss, 4, cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
  if (loss) *loss = (double)l / (2.0 * n * s->E);
  return take_tc_error(s, st);
}

extern "C" mdeos_status mdeos_surrogate_train(mdeos_surrogate* s, const double* x, const double* y,
                                              int32_t n, int32_t epochs, int32_t batch, double lr,
                                              uint64_t seed, int32_t set_norm, double* loss_out) {
  if (!s || !x || !y || n < 1 || epochs < 0 || batch < 1 || batch > s->maxB || !(lr > 0))
    return set_error(MDEOS_EINVAL, "bad train arguments");
  if (set_norm) {  // normalisers from the training data: mean and standard deviation
    for (int c = 0; c < 4; ++c) {
      const double* a = c < 2 ? x : y;
      const int col = c % 2;
      const bool as = c == 2 && s->p_asinh;  // pressure learned as asinh(P)
      auto val = [&](int i) { return as ? std::asinh(a[2 * i + col]) : a[2 * i + col]; };
      double m = 0.0, q = 0.0;
      for (int i = 0; i < n; ++i) m += val(i);
      m /= n;
      for (int i = 0; i < n; ++i) q += (val(i) - m) * (val(i) - m);
      const double sdv = std::sqrt(q / n);
      s->norm[(c < 2 ? 0 : 4) + col] = m;
      s->norm[(c < 2 ? 2 : 6) + col] = sdv > 0 ? sdv : 1.0;
    }
  }
  SCK(cudaSetDevice(handle_device(s->h)));
  cudaStream_t st = handle_stream(s->h);
  std::mt19937_64 rng(seed);
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  std::vector<double> bx(2 * (size_t)batch), by(2 * (size_t)batch);
  const long long np = (long long)s->E * kNParam;
  const float b1 = 0.9f, b2 = 0.999f;
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(perm.begin(), perm.end(), rng);
    double lsum = 0.0;
    int nb = 0;
    for (int off = 0; off + batch <= n; off += batch) {  // full batches only
      for (int k = 0; k < batch; ++k) {
        const int i = perm[off + k];
        bx[2 * k] = x[2 * i];
        bx[2 * k + 1] = x[2 * i + 1];
        by[2 * k] = y[2 * i];
        by[2 * k + 1] = y[2 * i + 1];
      }
      mdeos_status ms = load_batch(s, bx.data(), by.data(), batch, st);
      if (ms != MDEOS_OK) return ms;
      SCK(cudaMemsetAsync(s->loss, 0, 4, st));
      SCK(forward(s, batch, s->T, st));
      SCK(backward(s, batch, st));
      ++s->step;
      const float c1 = (float)(1.0 - std::pow(0.9, (double)s->step));
      const float c2 = (float)(1.0 - std::pow(0.999, (double)s->step));
      mlp_adam<<<nblk(np), 256, 0, st>>>(s->P, s->G, s->Mm, s->Vv, np, (float)lr, b1, b2,
                                         (float)(1.0 - 0.9), (float)(1.0 - 0.999), 1e-8f, c1, c2);
      SCK(cudaGetLastError());
      SCK(cast_weights(s, st));
      count_launch(s->h, 22);
      float l = 0.f;
      SCK(cudaMemcpyAsync(&l, s->loss, 4, cudaMemcpyDeviceToHost, st));
      SCK(cudaStreamSynchronize(st));
      lsum += (double)l / (2.0 * batch * s->E);
      ++nb;
    }
    if (loss_out) loss_out[ep] = nb ? lsum / nb : 0.0;
  }
  return take_tc_error(s, st);
}

// inference of B <= maxB inputs (device FP64 [B][2]) -> per-model s->Y and the ensemble
// mean / sd (device FP64 [B][2]) on stream st
static cudaError_t infer(mdeos_surrogate* s, const double* dx, int B, double* dmean, double* dsd,
                         int path, cudaStream_t st) {
  mlp_normalise<<<nblk(B), 256, 0, st>>>(dx, s->X, B, s->norm[0], s->norm[1], s->norm[2],
                                         s->norm[3]);
  cudaError_t e;
  if (path == MDEOS_SURROGATE_INFER_MMA) {
    e = forward(s, B, nullptr, st);
    count_launch(s->h, 9);
  } else {
    if (!s->tc_ready) {
      e = cudaFuncSetAttribute(mlp_infer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kTcSmem);
      if (e != cudaSuccess) return e;
      int dev = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      s->tc_ready = true;
    }
    // two resident CTAs per SM in all (shared memory bounds it at two)
    const int tiles = (B + kTcRows - 1) / kTcRows;
    const int per_model = std::max(1, std::min(tiles, (2 * s->nsm + s->E - 1) / s->E));
    dim3 grid(per_model, s->E);
    mlp_infer_tc_kernel<<<grid, kTcThreads, kTcSmem, st>>>(s->X, s->P, s->W1b, s->W2b, s->W3b,
                                                          s->W4b, s->Y, B, s->err);
    e = cudaGetLastError();
    count_launch(s->h, 3);
  }
  if (e != cudaSuccess) return e;
  mlp_ensemble<<<nblk(2 * B), 256, 0, st>>>(s->Y, B, s->E, s->norm[4], s->norm[5], s->norm[6],
                                            s->norm[7], s->p_asinh, dmean, dsd);
  return cudaGetLastError();
}

extern "C" mdeos_status mdeos_surrogate_set_output_transform(mdeos_surrogate* s, int32_t mode) {
  if (!s || (mode != MDEOS_SURROGATE_P_LINEAR && mode != MDEOS_SURROGATE_P_ASINH))
    return set_error(MDEOS_EINVAL, "bad output transform");
  s->p_asinh = mode == MDEOS_SURROGATE_P_ASINH ? 1 : 0;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_set_infer_path(mdeos_surrogate* s, int32_t path) {
  if (!s || (path != MDEOS_SURROGATE_INFER_TC && path != MDEOS_SURROGATE_INFER_MMA))
    return set_error(MDEOS_EINVAL, "bad inference path");
  s->infer_path = path;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_infer_device(mdeos_surrogate* s, const double* d_x,
                                                     int32_t n, double* d_mean, double* d_sd,
                                                     void* stream) {
  if (!s || (n > 0 && (!d_x || !d_mean || !d_sd)) || n < 0)
    return set_error(MDEOS_EINVAL, "bad infer_device arguments");
  SCK(cudaSetDevice(handle_device(s->h)));
  cudaStream_t st = stream ? (cudaStream_t)stream : handle_stream(s->h);
  for (int off = 0; off < n; off += s->maxB) {
    const int B = std::min(s->maxB, n - off);
    SCK(infer(s, d_x + 2 * (size_t)off, B, d_mean + 2 * (size_t)off, d_sd + 2 * (size_t)off,
              s->infer_path, st));
  }
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_predict(mdeos_surrogate* s, const double* x, int32_t n,
                                                double* mean, double* sd, float* per_model) {
  if (!s || !x || n < 0) return set_error(MDEOS_EINVAL, "bad predict arguments");
  SCK(cudaSetDevice(handle_device(s->h)));
  cudaStream_t st = handle_stream(s->h);
  for (int off = 0; off < n; off += s->maxB) {
    const int B = std::min(s->maxB, n - off);
    SCK(cudaMemcpyAsync(s->Xp, x + 2 * (size_t)off, (size_t)B * 16, cudaMemcpyHostToDevice, st));
    SCK(infer(s, s->Xp, B, s->mean, s->sd, s->infer_path, st));
    if (mean)
      SCK(cudaMemcpyAsync(mean + 2 * (size_t)off, s->mean, (size_t)B * 16, cudaMemcpyDeviceToHost, st));
    if (sd)
      SCK(cudaMemcpyAsync(sd + 2 * (size_t)off, s->sd, (size_t)B * 16, cudaMemcpyDeviceToHost, st));
    if (per_model)
      for (int m = 0; m < s->E; ++m)
        SCK(cudaMemcpyAsync(per_model + ((size_t)m * n + off) * 2, s->Y + (size_t)m * B * 2,
                            (size_t)B * 8, cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));
  }
  int err = 0;
  SCK(cudaMemcpyAsync(&err, s->err, 4, cudaMemcpyDeviceToHost, st));
  SCK(cudaMemsetAsync(s->err, 0, 4, st));
  SCK(cudaStreamSynchronize(st));
  if (err) return set_error(MDEOS_ETIMEDOUT, "surrogate: a tensor-core wait ran out");
  return MDEOS_OK;
}

// Surrogate answer where the ensemble agrees (sd_P <= threshold * max(|P|, 1)),
// the MD path (requests evaluated with natoms = md_natoms) elsewhere.
// cell of the misfit grid holding input (rho, e); -1 outside the fitted range
static int misfit_cell(const mdeos_surrogate* s, double rho, double e) {
  if (s->mis_bins < 1) return -1;
  const double in[2] = {rho, e};
  int c[2];
  for (int k = 0; k < 2; ++k) {
    const double t = (in[k] - s->mis_lo[k]) / (s->mis_hi[k] - s->mis_lo[k]);
    if (!(t >= 0.0 && t <= 1.0)) return -1;
    c[k] = std::min((int)(t * s->mis_bins), s->mis_bins - 1);
  }
  return c[0] * s->mis_bins + c[1];
}

static double misfit_at(const mdeos_surrogate* s, double rho, double e) {
  const int c = misfit_cell(s, rho, e);
  return c < 0 ? INFINITY : s->mis[c];
}

extern "C" mdeos_status mdeos_surrogate_fit_misfit(mdeos_surrogate* s, const double* x,
                                                   const double* y, int32_t n, int32_t bins,
                                                   int32_t min_count) {
  if (!s || !x || !y || n < 1 || bins < 1 || bins > 1024 || min_count < 1)
    return set_error(MDEOS_EINVAL, "bad fit_misfit arguments");
  std::vector<double> mean(2 * (size_t)n), sd(2 * (size_t)n);
  mdeos_status ms = mdeos_surrogate_predict(s, x, n, mean.data(), sd.data(), nullptr);
  if (ms != MDEOS_OK) return ms;
  for (int k = 0; k < 2; ++k) {
    s->mis_lo[k] = INFINITY;
    s->mis_hi[k] = -INFINITY;
    for (int i = 0; i < n; ++i) {
      s->mis_lo[k] = std::min(s->mis_lo[k], x[2 * i + k]);
      s->mis_hi[k] = std::max(s->mis_hi[k], x[2 * i + k]);
    }
    if (!(s->mis_hi[k] > s->mis_lo[k])) s->mis_hi[k] = s->mis_lo[k] + 1.0;
  }
  s->mis_bins = bins;
  std::vector<double> sum((size_t)bins * bins, 0.0);
  std::vector<int> cnt((size_t)bins * bins, 0);
  for (int i = 0; i < n; ++i) {
    const int c = misfit_cell(s, x[2 * i], x[2 * i + 1]);
    if (c < 0) continue;
    const double r = (mean[2 * i] - y[2 * i]) / std::max(std::fabs(y[2 * i]), 1.0);
    sum[c] += r * r;
    ++cnt[c];
  }
  s->mis.assign((size_t)bins * bins, INFINITY);
  for (size_t c = 0; c < s->mis.size(); ++c)
    if (cnt[c] >= min_count) s->mis[c] = std::sqrt(sum[c] / cnt[c]);
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_misfit(const mdeos_surrogate* s, const double* x,
                                               int32_t n, double* out) {
  if (!s || !x || !out || n < 0) return set_error(MDEOS_EINVAL, "bad misfit arguments");
  if (s->mis_bins < 1) return set_error(MDEOS_EINVAL, "no misfit map fitted");
  for (int i = 0; i < n; ++i) out[i] = misfit_at(s, x[2 * i], x[2 * i + 1]);
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_set_misfit_threshold(mdeos_surrogate* s,
                                                             double threshold) {
  if (!s || !(threshold >= 0.0)) return set_error(MDEOS_EINVAL, "bad misfit threshold");
  if (std::isfinite(threshold) && s->mis_bins < 1)
    return set_error(MDEOS_EINVAL, "no misfit map fitted");
  s->mis_threshold = threshold;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_gated_eval(mdeos_surrogate* s, const mdeos_request* reqs,
                                                   int32_t n, double threshold, int32_t md_natoms,
                                                   mdeos_result* out, int32_t* used_md) {
  if (!s || !reqs || !out || n < 0 || !(threshold >= 0))
    return set_error(MDEOS_EINVAL, "bad gated_eval arguments");
  std::vector<double> x(2 * (size_t)n), mean(2 * (size_t)n), sd(2 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    x[2 * i] = reqs[i].rho;
    x[2 * i + 1] = reqs[i].e;
  }
  mdeos_status ms = mdeos_surrogate_predict(s, x.data(), n, mean.data(), sd.data(), nullptr);
  if (ms != MDEOS_OK) return ms;
  std::vector<mdeos_request> md;
  std::vector<int> idx;
  for (int i = 0; i < n; ++i) {
    const bool ok = sd[2 * i] <= threshold * std::max(std::fabs(mean[2 * i]), 1.0) &&
                    (reqs[i].flags & MDEOS_REQ_TEMPERATURE) == 0 &&
                    (!std::isfinite(s->mis_threshold) ||
                     misfit_at(s, reqs[i].rho, reqs[i].e) <= s->mis_threshold);
    if (used_md) used_md[i] = ok ? 0 : 1;
    if (ok) {
      mdeos_result& r = out[i];
      std::memset(&r, 0, sizeof(r));
      r.P = mean[2 * i];
      r.T = mean[2 * i + 1];
      r.P_se = sd[2 * i];
      r.T_se = sd[2 * i + 1];
      r.sigma[0] = r.sigma[1] = r.sigma[2] = r.P;
      r.element_id = reqs[i].element_id;
      r.natoms = 0;
      r.status = MDEOS_OK;
      r.path = -2;  // answered by the surrogate
    } else {
      mdeos_request q = reqs[i];
      if (md_natoms > 0) q.natoms = md_natoms;
      md.push_back(q);
      idx.push_back(i);
    }
  }
  if (!md.empty()) {
    uint64_t t = 0;
    ms = mdeos_submit(s->h, md.data(), (int)md.size(), &t);
    if (ms != MDEOS_OK) return ms;
    std::vector<mdeos_result> r(md.size());
    ms = mdeos_poll(s->h, t, r.data(), -1);
    if (ms != MDEOS_OK) return ms;
    for (size_t k = 0; k < md.size(); ++k) out[idx[k]] = r[k];
  }
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_surrogate_destroy(mdeos_surrogate* s) {
  if (!s) return MDEOS_OK;
  if (s->h) {
    cudaSetDevice(handle_device(s->h));
    cudaStreamSynchronize(handle_stream(s->h));
  }
  for (void* p : s->allocs) cudaFree(p);
  delete s;
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_debug_gemm_bf16(const uint16_t* A, const uint16_t* B, float* C,
                                              int32_t M, int32_t N, int32_t K, int64_t sa_m,
                                              int64_t sa_k, int64_t sb_k, int64_t sb_n,
                                              int64_t sc_m, int64_t sc_n, void* stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1)
    return set_error(MDEOS_EINVAL, "bad gemm arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int* err = nullptr;
  float* ws = nullptr;
  const long long ws_elems = (long long)kMaxSplitK * M * N;
  SCK(cudaMallocAsync(&err, sizeof(int), st));
  SCK(cudaMemsetAsync(err, 0, sizeof(int), st));
  SCK(cudaMallocAsync(&ws, (size_t)ws_elems * 4, st));
  cudaError_t e = gemm(st, err, ws, ws_elems, reinterpret_cast<const __nv_bfloat16*>(A),
                       reinterpret_cast<const __nv_bfloat16*>(B), C, M, N, K, sa_m, sa_k, 0, sb_k,
                       sb_n, 0, sc_m, sc_n, 0, 1);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(err, st);
  cudaFreeAsync(ws, st);
  if (e != cudaSuccess) return set_error(MDEOS_ECUDA, cudaGetErrorString(e));
  if (herr) return set_error(MDEOS_ETIMEDOUT, "gemm: a tensor-core wait ran out");
  return MDEOS_OK;
}

extern "C" mdeos_status mdeos_debug_tanh(const float* x, float* y, int32_t n, void* stream) {
  if (!x || !y || n < 1) return set_error(MDEOS_EINVAL, "bad tanh arguments");
  cudaStream_t st = (cudaStream_t)stream;
  debug_tanh_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, y, n);
  SCK(cudaGetLastError());
  SCK(cudaStreamSynchronize(st));
  return MDEOS_OK;
}
