// The learned leap of include/lbnop.h: a periodic convolutional U-Net whose 3 x 3
// convolutions are implicit GEMMs on BF16 tensor-core operands (mma.sync m16n8k16, FP32
// accumulation), with its backward pass, Adam, and the leap/LBM alternation.
//
// GEMM views of one layer (p: pixel, t: tap of the 3 x 3 stencil, off(t) its offset):
//   forward      y[p][n]  = sum_{t, k} x[p + off(t)][k] W[t][n][k]        M = pixels, K = 9 c_in
//   data grad    dx[p][n] = sum_{t, k} dy[p + off(t)][k] W[8 - t][k][n]   the same kernel on a
//                                                                         flipped, transposed copy
//   weight grad  dW[t][m][n] = sum_p dy[p][m] x[p + off(t)][n]            K = pixels (split-K)
// Activations are channels-last BF16; every tensor lives in the caller's workspace.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "lbnop.h"

namespace nop {

using bf16 = __nv_bfloat16;

constexpr int NL = 16;
struct LayerSpec {
  int ci, co, level;
  bool act;
};
// The table of include/lbnop.h.
constexpr LayerSpec kL[NL] = {{16, 96, 0, true},  {96, 96, 0, true},  {96, 64, 1, true},  {64, 64, 1, true},
                              {64, 96, 2, true},  {96, 96, 2, true},  {96, 96, 3, true},  {96, 96, 3, true},
                              {96, 96, 2, true},  {96, 64, 2, false}, {64, 64, 1, true},  {64, 96, 1, false},
                              {96, 96, 0, true},  {96, 16, 0, false}, {16, 16, 0, false}, {16, 16, 0, false}};
enum { E0A, E0B, E1A, E1B, E2A, E2B, M3A, M3B, D2A, D2B, D1A, D1B, D0A, OUT, LIN, LINA };
// Channels of the skip tensors h0..h3 at levels 0..3 (and of every tensor summed with them).
constexpr int CH[4] = {kL[E0B].co, kL[E1B].co, kL[E2B].co, kL[M3B].co};
static_assert(kL[D1B].co == CH[0] && kL[D2B].co == CH[1] && kL[D2A].ci == CH[3] && kL[D2A].ci == CH[2],
              "skip additions need equal channel counts");

struct LayerTab {
  int off_w[NL], ci[NL], co[NL], woff[NL];
};

// ---------------------------------------------------------------- small helpers

// The logistic function with the fast exponential and division intrinsics: a few ulp of FP32,
// far below the BF16 rounding every activation gets next; exp(-z) = inf gives 0 exactly.
__device__ __forceinline__ float sigmoid_f(float z) { return __fdividef(1.0f, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_f(float z) { return z * sigmoid_f(z); }
__device__ __forceinline__ float silu_grad_f(float z) {
  const float s = sigmoid_f(z);
  return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D += A B for one m16n8k16 tile: A row-major 16 x 16, B column-major 16 x 8, BF16 in,
// FP32 accumulate. Fragment of lane l (g = l / 4, q = l % 4): a = {A[g][2q..], A[g+8][2q..],
// A[g][2q+8..], A[g+8][2q+8..]}, b = {B[2q..][g], B[2q+8..][g]}, d = {D[g][2q..], D[g+8][2q..]}.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const bf16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t& r0, uint32_t& r1, const bf16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(a));
}

// ---------------------------------------------------------------- convolution (forward, data grad)

struct ConvArgs {
  const bf16* x;   // [B][H][W][CI]
  const bf16* x2;  // or null: a second input of the same shape, multiplied by the same weights
  const bf16* w;  // TW = false: [9][CO][CI]; TW = true: [9][CI][CO], read at tap 8 - t
  const bf16* w2;  // or null: the BF16 remainder of the weights (w + w2 ~ 16 bits), applied to x
  const unsigned char* wpk;  // or null: w packed for the tensor-core path (tc_pack_kernel)
  int B, H, W;
  const float* bias;  // [CO] or null
  const float* film;  // [CO] or null: adds alpha[b] film[n]
  bf16* z;            // BF16 pre-activation out, or null
  bf16* a;            // BF16 SiLU(z) out, or null
  float* yf;          // FP32 out, or null
  int accumulate;     // yf += instead of yf =
  int scale_alpha;    // multiply the result (after bias) by alpha[b]
  float alpha[LBNOP_MAX_BATCH];
};

// Bias, conditioning, alpha scaling and the stores for the lane's two pixel rows (pixels
// base + g and base + g + 8, ok[r] false past the end) and its NT pairs of channels
// n0 + 8 j + 2 q, from the m16n8 accumulator layout.
template <int CO, int NT>
__device__ __forceinline__ void conv_epilogue(const ConvArgs& p, const float (&acc)[NT][4], int base, int n0,
                                              int g, int q, const bool (&ok)[2], const int (&bi)[2]) {
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    if (!ok[r]) continue;
    const int pix = base + g + 8 * r;
    const float al = p.film ? p.alpha[bi[r]] : 0.0f;  // bi[r] is the row's sample
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int n = n0 + 8 * j + 2 * q;
      float v0 = acc[j][2 * r], v1 = acc[j][2 * r + 1];
      if (p.bias) {
        v0 += p.bias[n];
        v1 += p.bias[n + 1];
      }
      if (p.film) {
        v0 = fmaf(al, p.film[n], v0);
        v1 = fmaf(al, p.film[n + 1], v1);
      }
      if (p.scale_alpha) {
        v0 *= p.alpha[bi[r]];
        v1 *= p.alpha[bi[r]];
      }
      const size_t o = (size_t)pix * CO + n;
      if (p.yf) {
        float2* y = reinterpret_cast<float2*>(p.yf + o);
        if (p.accumulate) {
          const float2 old = *y;
          *y = make_float2(old.x + v0, old.y + v1);
        } else {
          *y = make_float2(v0, v1);
        }
      }
      if (p.z) *reinterpret_cast<__nv_bfloat162*>(p.z + o) = __floats2bfloat162_rn(v0, v1);
      if (p.a) *reinterpret_cast<__nv_bfloat162*>(p.a + o) = __floats2bfloat162_rn(silu_f(v0), silu_f(v1));
    }
  }
}

constexpr int CONV_THREADS = 128;  // four warps, 16 pixels each

// Each warp computes 16 consecutive pixels x BN output channels (the block's channel
// slice blockIdx.y); A fragments come straight from the channels-last input (32-bit
// pairs of channels), B fragments from the weights (L1-resident). The K loop (9 taps x
// CI / 16) is unrolled with the fragments of step k + 1 loaded while step k multiplies.
template <int CI, int CO, int BN, bool TW, bool DUAL, bool WLO = false>
__global__ void __launch_bounds__(CONV_THREADS) conv_kernel(const ConvArgs p) {
  constexpr int NT = BN / 8, CPT = CI / 16, KS = 9 * CPT, KT = KS * (1 + (DUAL ? 1 : 0) + (WLO ? 1 : 0));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
  const int HW = p.H * p.W, npix = p.B * HW;
  const int base = (blockIdx.x * 4 + warp) * 16;
  const int n0 = blockIdx.y * BN;
  if (base >= npix) return;
  int bi[2];
  int off[2][9];  // element offset of (row r's pixel + tap offset, channel 2q)
  bool ok[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    int pix = base + g + 8 * r;
    ok[r] = pix < npix;
    pix = ok[r] ? pix : base;  // out-of-range rows load a valid pixel; their results are dropped
    bi[r] = pix / HW;
    const int rem = pix - bi[r] * HW, h = rem / p.W, w = rem - h * p.W;
#pragma unroll
    for (int t = 0; t < 9; ++t)
      off[r][t] = ((bi[r] * p.H + wrap1(h + t / 3 - 1, p.H)) * p.W + wrap1(w + t % 3 - 1, p.W)) * CI + 2 * q;
  }
  // passes of KS steps: (x, w), then (x2, w) if DUAL, then (x, w2) if WLO
  auto load = [&](int kk, uint32_t (&a)[4], uint32_t (&b)[NT][2]) {
    const int pass = kk / KS, ks = kk % KS;
    const bool second_x = DUAL && pass == 1;
    const bool second_w = WLO && pass == (DUAL ? 2 : 1);
    const bf16* x = second_x ? p.x2 : p.x;
    const bf16* wbase = second_w ? p.w2 : p.w;
    const int t = ks / CPT, c0 = (ks % CPT) * 16;
    a[0] = ld32(x + off[0][t] + c0);
    a[1] = ld32(x + off[1][t] + c0);
    a[2] = ld32(x + off[0][t] + c0 + 8);
    a[3] = ld32(x + off[1][t] + c0 + 8);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      if constexpr (!TW) {
        const bf16* wr = wbase + ((size_t)t * CO + n0 + 8 * j + g) * CI + c0 + 2 * q;
        b[j][0] = ld32(wr);
        b[j][1] = ld32(wr + 8);
      } else {
        const bf16* wr = p.w + ((size_t)(8 - t) * CI + c0 + 2 * q) * CO + n0 + 8 * j + g;
        b[j][0] = pack2(wr[0], wr[CO]);
        b[j][1] = pack2(wr[8 * CO], wr[9 * CO]);
      }
    }
  };
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
  uint32_t a[2][4], b[2][NT][2];
  load(0, a[0], b[0]);
#pragma unroll
  for (int kk = 0; kk < KT; ++kk) {
    if (kk + 1 < KT) load(kk + 1, a[(kk + 1) & 1], b[(kk + 1) & 1]);
#pragma unroll
    for (int j = 0; j < NT; ++j) mma_bf16(acc[j], a[kk & 1], b[kk & 1][j][0], b[kk & 1][j][1]);
  }

  conv_epilogue<CO, NT>(p, acc, base, n0, g, q, ok, bi);
}

constexpr int SPLITK_THREADS = 9 * 32;  // one warp per tap

// The same convolution for layers with few pixels: one block per 16 pixels x 16 output
// channels, warp t multiplies tap t only (CI / 16 k-steps instead of 9 CI / 16), and the
// nine partial tiles are added in shared memory in tap order before the epilogue. The
// chain of dependent steps per warp is nine times shorter, so the coarse levels, which have
// too few pixels to fill the GPU, stop waiting on it.
template <int CI, int CO>
__global__ void __launch_bounds__(SPLITK_THREADS) conv_splitk_kernel(const ConvArgs p) {
  constexpr int CPT = CI / 16;
  __shared__ float red[9][8][32];
  const int lane = threadIdx.x & 31, t = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
  const int HW = p.H * p.W, npix = p.B * HW;
  const int base = blockIdx.x * 16, n0 = blockIdx.y * 16;
  int bi[2], off[2];
  bool ok[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    int pix = base + g + 8 * r;
    ok[r] = pix < npix;
    pix = ok[r] ? pix : base;  // out-of-range rows load a valid pixel; their results are dropped
    bi[r] = pix / HW;
    const int rem = pix - bi[r] * HW, h = rem / p.W, w = rem - h * p.W;
    off[r] = ((bi[r] * p.H + wrap1(h + t / 3 - 1, p.H)) * p.W + wrap1(w + t % 3 - 1, p.W)) * CI + 2 * q;
  }
  float acc[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
  for (int cc = 0; cc < CPT; ++cc) {
    const int c0 = cc * 16;
    const uint32_t a[4] = {ld32(p.x + off[0] + c0), ld32(p.x + off[1] + c0), ld32(p.x + off[0] + c0 + 8),
                           ld32(p.x + off[1] + c0 + 8)};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const bf16* wr = p.w + ((size_t)t * CO + n0 + 8 * j + g) * CI + c0 + 2 * q;
      mma_bf16(acc[j], a, ld32(wr), ld32(wr + 8));
    }
  }
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) red[t][4 * j + e][lane] = acc[j][e];
  __syncthreads();
  if (t != 0) return;
  float sum[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float v = red[0][4 * j + e][lane];
#pragma unroll
      for (int tt = 1; tt < 9; ++tt) v += red[tt][4 * j + e][lane];
      sum[j][e] = v;
    }
  conv_epilogue<CO, 2>(p, sum, base, n0, g, q, ok, bi);
}

// ---------------------------------------------------------------- convolution, shared-memory staged

__device__ __forceinline__ void cp_async16_cg(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16* p) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

template <int CI, int BN>
constexpr int conv_smem_bytes() {
  return 2 * (64 + BN) * (CI + 8) * 2 + 64 * 16;
}

// The convolution with its operands staged through shared memory: a block computes 64
// pixels x BN output channels (slice blockIdx.y). For each tap it copies the 64 shifted
// input rows (CI channels each) and the tap's BN x CI weights with 16-byte cp.async into a
// two-stage ring (the next tap lands while this one multiplies), and each warp reads its
// fragments with ldmatrix: A (16 pixels x 16 channels) once per k-step, B in pairs of
// 8-channel tiles. Rows are padded by 16 bytes so that ldmatrix rows hit distinct banks.
template <int CI, int CO, int BN>
__global__ void __launch_bounds__(CONV_THREADS) conv_smem_kernel(const ConvArgs p) {
  constexpr int PA = CI + 8, NT = BN / 8, CPT = CI / 16, CH = CI / 8;
  static_assert(NT % 2 == 0, "n-tiles come in pairs");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16* stage_base = reinterpret_cast<bf16*>(smem_raw);
  int4* spix = reinterpret_cast<int4*>(smem_raw + 2 * (64 + BN) * PA * 2);  // (b, h, w, ok) per tile pixel
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, q = lane & 3;
  const int HW = p.H * p.W, npix = p.B * HW;
  const int base0 = blockIdx.x * 64, n0 = blockIdx.y * BN;
  if (tid < 64) {
    int pix = base0 + tid;
    const int ok = pix < npix;
    pix = ok ? pix : base0;  // rows past the end copy a valid pixel; their results are dropped
    const int b = pix / HW, rem = pix - b * HW, h = rem / p.W;
    spix[tid] = make_int4(b, h, rem - h * p.W, ok);
  }
  __syncthreads();
  auto stage = [&](int t, int buf) {
    bf16* sA = stage_base + buf * (64 + BN) * PA;
    bf16* sB = sA + 64 * PA;
    const int dy = t / 3 - 1, dx = t % 3 - 1;
    for (int v = tid; v < 64 * CH; v += CONV_THREADS) {
      const int r = v / CH, c = v - r * CH;
      const int4 pb = spix[r];
      cp_async16_cg(sA + r * PA + 8 * c,
                    p.x + ((size_t)(pb.x * p.H + wrap1(pb.y + dy, p.H)) * p.W + wrap1(pb.z + dx, p.W)) * CI + 8 * c);
    }
    for (int v = tid; v < BN * CH; v += CONV_THREADS) {
      const int n = v / CH, c = v - n * CH;
      cp_async16_cg(sB + n * PA + 8 * c, p.w + ((size_t)t * CO + n0 + n) * CI + 8 * c);
    }
  };
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
  stage(0, 0);
  cp_async_commit_group();
#pragma unroll 1
  for (int t = 0; t < 9; ++t) {
    if (t + 1 < 9) stage(t + 1, (t + 1) & 1);
    cp_async_commit_group();  // (empty after the last tap)
    cp_async_wait_group<1>();  // tap t has landed for this thread
    __syncthreads();           // and for everyone
    const bf16* sA = stage_base + (t & 1) * (64 + BN) * PA + (warp * 16) * PA;
    const bf16* sB = stage_base + (t & 1) * (64 + BN) * PA + 64 * PA;
#pragma unroll
    for (int kk = 0; kk < CPT; ++kk) {
      uint32_t a[4];
      ldsm_x4(a, sA + (lane & 15) * PA + kk * 16 + (lane >> 4) * 8);
#pragma unroll
      for (int jp = 0; jp < NT / 2; ++jp) {
        uint32_t b[4];  // {b0, b1} of n-tile 2 jp, then of n-tile 2 jp + 1
        ldsm_x4(b, sB + (jp * 16 + (lane >> 4) * 8 + (lane & 7)) * PA + kk * 16 + ((lane >> 3) & 1) * 8);
        mma_bf16(acc[2 * jp], a, b[0], b[1]);
        mma_bf16(acc[2 * jp + 1], a, b[2], b[3]);
      }
    }
    __syncthreads();  // the buffer of tap t is refilled with tap t + 2 next
  }
  const int base = base0 + warp * 16;
  int bi[2];
  bool ok[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int4 pb = spix[warp * 16 + g + 8 * r];
    bi[r] = pb.x;
    ok[r] = pb.w != 0;
  }
  conv_epilogue<CO, NT>(p, acc, base, n0, g, q, ok, bi);
}

// ---------------------------------------------------------------- weight gradient

struct WgradArgs {
  const bf16* x;   // [B][H][W][CI]
  const bf16* dz;  // [B][H][W][CO]
  int B, H, W;
  int chunk;  // pixels per block (multiple of 32)
  float* dw;  // [9][CO][CI], accumulated with atomicAdd
};

// Block (chunk, tap): stages 32 pixels of dz and of the shifted x in shared memory, then
// ldmatrix.trans gives fragments whose K index runs over pixels. Warps share the
// (CO / 16) x (CI / 8) output tiles.
template <int CI, int CO>
__global__ void __launch_bounds__(128) wgrad_kernel(const WgradArgs p) {
  constexpr int MT = CO / 16, NT = CI / 8, TILES = MT * NT, PER = (TILES + 3) / 4;
  constexpr int PZ = CO + 8, PX = CI + 8;  // padded pitches: conflict-free ldmatrix rows
  __shared__ __align__(16) bf16 sz[32 * PZ];
  __shared__ __align__(16) bf16 sx[32 * PX];
  const int t = blockIdx.y, dy = t / 3 - 1, dx = t % 3 - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, q = lane & 3;
  const int HW = p.H * p.W, npix = p.B * HW;
  const int p0 = blockIdx.x * p.chunk, p1 = min(npix, p0 + p.chunk);
  float acc[PER][4];
#pragma unroll
  for (int i = 0; i < PER; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0f;

  for (int pb = p0; pb < p1; pb += 32) {
    constexpr int VZ = CO / 8, VX = CI / 8;
    for (int v = threadIdx.x; v < 32 * VZ; v += 128) {
      const int r = v / VZ, c = v - r * VZ, pix = pb + r;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (pix < p1) val = *reinterpret_cast<const uint4*>(p.dz + (size_t)pix * CO + 8 * c);
      *reinterpret_cast<uint4*>(sz + r * PZ + 8 * c) = val;
    }
    for (int v = threadIdx.x; v < 32 * VX; v += 128) {
      const int r = v / VX, c = v - r * VX, pix = pb + r;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (pix < p1) {
        const int b = pix / HW, rem = pix - b * HW, h = rem / p.W, w = rem - h * p.W;
        val = *reinterpret_cast<const uint4*>(
            p.x + ((size_t)(b * p.H + wrap1(h + dy, p.H)) * p.W + wrap1(w + dx, p.W)) * CI + 8 * c);
      }
      *reinterpret_cast<uint4*>(sx + r * PX + 8 * c) = val;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 32; ks += 16) {
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        const int tile = warp + 4 * i;
        if (tile < TILES) {
          const int mt = tile / NT, nt = tile - mt * NT;
          uint32_t a[4], b0, b1;
          // matrix l/8 = (m block (l/8)&1, k block (l/8)>>1): a = {A00, A10, A01, A11}
          ldsm_x4_t(a, sz + (ks + ((lane >> 4) << 3) + (lane & 7)) * PZ + 16 * mt + (((lane >> 3) & 1) << 3));
          ldsm_x2_t(b0, b1, sx + (ks + (lane & 15)) * PX + 8 * nt);
          mma_bf16(acc[i], a, b0, b1);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int tile = warp + 4 * i;
    if (tile < TILES) {
      const int mt = tile / NT, nt = tile - mt * NT;
      float* d = p.dw + ((size_t)t * CO + 16 * mt + g) * CI + 8 * nt + 2 * q;
      atomicAdd(d, acc[i][0]);
      atomicAdd(d + 1, acc[i][1]);
      atomicAdd(d + 8 * CI, acc[i][2]);
      atomicAdd(d + 8 * CI + 1, acc[i][3]);
    }
  }
}

// ---------------------------------------------------------------- elementwise and reductions

constexpr int HEAD_BLOCKS = 128;  // partial sums per sample (fixed order: deterministic)

// sig[b] = root mean square of field b from its sum of squares (1 for a zero field).
// Sum of one sample's HEAD_BLOCKS partial sums by one warp, in a fixed order (valid in lane 0).
__device__ __forceinline__ double warp_partials(const double* __restrict__ part, int lane) {
  double v = 0.0;
  for (int k = lane; k < HEAD_BLOCKS; k += 32) v += part[k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// One warp per sample (grid B, 32 threads).
__global__ void rms_kernel(const double* __restrict__ partial2, int B, long long n, double* __restrict__ sig) {
  const int b = blockIdx.x, lane = threadIdx.x;
  if (b >= B) return;
  const double s = warp_partials(partial2 + (size_t)b * HEAD_BLOCKS, lane);
  if (lane == 0) {
    const double r = sqrt(s / (double)n);
    sig[b] = r > 1e-30 ? r : 1.0;
  }
}

// x = phi / sig[b] ([B][H][W] FP32) -> [B][H/4][W/4][16], channel 4 di + dj = x[4 i + di][4 j + dj],
// as two BF16 tensors: x0 = bf16(x) and x0l = bf16(x - x0) (together about 16 bits).
__global__ void s2d_kernel(const float* __restrict__ phi, const double* __restrict__ sig, int B, int H, int W,
                           bf16* __restrict__ x0, bf16* __restrict__ x0l) {
  const int h = H / 4, w = W / 4, n = B * h * w;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int b = k / (h * w), rem = k - b * h * w, i = rem / w, j = rem - i * w;
    const float inv = (float)(1.0 / sig[b]);
    __align__(16) bf16 v[16];
    __align__(16) bf16 lo[16];
#pragma unroll
    for (int di = 0; di < 4; ++di) {
      const float4 r = *reinterpret_cast<const float4*>(phi + ((size_t)b * H + 4 * i + di) * W + 4 * j);
      const float e[4] = {r.x * inv, r.y * inv, r.z * inv, r.w * inv};
#pragma unroll
      for (int dj = 0; dj < 4; ++dj) {
        v[4 * di + dj] = __float2bfloat16_rn(e[dj]);
        lo[4 * di + dj] = __float2bfloat16_rn(e[dj] - __bfloat162float(v[4 * di + dj]));
      }
    }
    uint4* dst = reinterpret_cast<uint4*>(x0 + (size_t)k * 16);
    dst[0] = reinterpret_cast<const uint4*>(v)[0];
    dst[1] = reinterpret_cast<const uint4*>(v)[1];
    uint4* dl = reinterpret_cast<uint4*>(x0l + (size_t)k * 16);
    dl[0] = reinterpret_cast<const uint4*>(lo)[0];
    dl[1] = reinterpret_cast<const uint4*>(lo)[1];
  }
}

// Eight BF16 channels of one pixel in one 16-byte word. The elementwise kernels below give
// each thread 8 channels of one pixel (every channel count here is a multiple of 8) and index
// in 32 bits (B H W C < 2^31 for every tensor of a context).
union BF8 {
  uint4 u;
  bf16 h[8];
};

__device__ __forceinline__ BF8 ld8(const bf16* p) {
  BF8 v;
  v.u = *reinterpret_cast<const uint4*>(p);
  return v;
}

// 2 x 2 average: x [B][2h][2w][C] -> y [B][h][w][C].
__global__ void pool_kernel(const bf16* __restrict__ x, int B, int h, int w, int C, bf16* __restrict__ y) {
  const int cv = C >> 3, n = B * h * w * cv;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int c8 = k % cv, pix = k / cv, j = pix % w, t = pix / w;  // t = b h + i: input row 2 t
    const size_t r0 = ((size_t)(2 * t) * (2 * w) + 2 * j) * C + 8 * c8, r1 = r0 + (size_t)2 * w * C;
    const BF8 a = ld8(x + r0), b = ld8(x + r0 + C), c = ld8(x + r1), d = ld8(x + r1 + C);
    BF8 o;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const float s = (__bfloat162float(a.h[e]) + __bfloat162float(b.h[e])) +
                      (__bfloat162float(c.h[e]) + __bfloat162float(d.h[e]));
      o.h[e] = __float2bfloat16_rn(0.25f * s);
    }
    *reinterpret_cast<uint4*>(y + (size_t)k * 8) = o.u;
  }
}

// y [B][h][w][C] = nearest 2x upsampling of xc [B][h/2][w/2][C] plus skip [B][h][w][C].
__global__ void up_add_kernel(const bf16* __restrict__ xc, const bf16* __restrict__ skip, int B, int h, int w, int C,
                              bf16* __restrict__ y) {
  const int cv = C >> 3, n = B * h * w * cv;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int c8 = k % cv, pix = k / cv, j = pix % w, t = pix / w, i = t % h, b = t / h;
    const size_t src = ((size_t)(b * (h / 2) + i / 2) * (w / 2) + j / 2) * C + 8 * c8;
    const BF8 u = ld8(xc + src), v = ld8(skip + (size_t)k * 8);
    BF8 o;
#pragma unroll
    for (int e = 0; e < 8; ++e) o.h[e] = __float2bfloat16_rn(__bfloat162float(u.h[e]) + __bfloat162float(v.h[e]));
    *reinterpret_cast<uint4*>(y + (size_t)k * 8) = o.u;
  }
}

// dz [B][h][w][C] (BF16) from FP32 gradients: g at the same level, or the 2 x 2 sums of gf
// (the adjoint of nearest upsampling) when gf is given; times SiLU'(z) when z is given.
__global__ void dz_kernel(const float* __restrict__ g, const float* __restrict__ gf, const bf16* __restrict__ z, int B,
                          int h, int w, int C, bf16* __restrict__ dz) {
  const int cv = C >> 3, n = B * h * w * cv;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    float v[8];
    if (gf) {
      const int c8 = k % cv, pix = k / cv, j = pix % w, t = pix / w;
      const size_t r0 = ((size_t)(2 * t) * (2 * w) + 2 * j) * C + 8 * c8, r1 = r0 + (size_t)2 * w * C;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float4 a = *reinterpret_cast<const float4*>(gf + r0 + 4 * q);
        const float4 b = *reinterpret_cast<const float4*>(gf + r0 + C + 4 * q);
        const float4 c = *reinterpret_cast<const float4*>(gf + r1 + 4 * q);
        const float4 d = *reinterpret_cast<const float4*>(gf + r1 + C + 4 * q);
        v[4 * q + 0] = (a.x + b.x) + (c.x + d.x);
        v[4 * q + 1] = (a.y + b.y) + (c.y + d.y);
        v[4 * q + 2] = (a.z + b.z) + (c.z + d.z);
        v[4 * q + 3] = (a.w + b.w) + (c.w + d.w);
      }
    } else {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float4 a = *reinterpret_cast<const float4*>(g + (size_t)k * 8 + 4 * q);
        v[4 * q + 0] = a.x;
        v[4 * q + 1] = a.y;
        v[4 * q + 2] = a.z;
        v[4 * q + 3] = a.w;
      }
    }
    if (z) {
      const BF8 zz = ld8(z + (size_t)k * 8);
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] *= silu_grad_f(__bfloat162float(zz.h[e]));
    }
    BF8 o;
#pragma unroll
    for (int e = 0; e < 8; ++e) o.h[e] = __float2bfloat16_rn(v[e]);
    *reinterpret_cast<uint4*>(dz + (size_t)k * 8) = o.u;
  }
}

// gf [B][2h][2w][C] += the adjoint of 2 x 2 averaging of gc [B][h][w][C] (FP32), four channels
// per thread.
__global__ void pool_bwd_kernel(const float* __restrict__ gc, int B, int h, int w, int C, float* __restrict__ gf) {
  const int cv = C >> 2, n = B * 4 * h * w * cv;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int c4 = k % cv, pix = k / cv, j = pix % (2 * w), t = pix / (2 * w), i = t % (2 * h), b = t / (2 * h);
    const float4 s = *reinterpret_cast<const float4*>(gc + ((size_t)(b * h + i / 2) * w + j / 2) * C + 4 * c4);
    float4* d = reinterpret_cast<float4*>(gf + (size_t)k * 4);
    float4 v = *d;
    v.x += 0.25f * s.x;
    v.y += 0.25f * s.y;
    v.z += 0.25f * s.z;
    v.w += 0.25f * s.w;
    *d = v;
  }
}

// Bias gradient sum_p dz[p][c] and conditioning gradient sum_p alpha[b(p)] dz[p][c].
struct ColsumArgs {
  const bf16* dz;
  int P, B, C;  // P pixels per sample
  float* db;
  float* dv;  // or null
  float alpha[LBNOP_MAX_BATCH];
};
__global__ void colsum_kernel(const ColsumArgs a) {
  __shared__ float s_b[256], s_v[256];
  const int rows = blockDim.x / a.C, c = threadIdx.x % a.C, r = threadIdx.x / a.C;
  const long long n = (long long)a.P * a.B;
  float sb = 0.0f, sv = 0.0f;
  if (r < rows)
    for (long long pix = (long long)blockIdx.x * rows + r; pix < n; pix += (long long)gridDim.x * rows) {
      const float v = __bfloat162float(a.dz[pix * a.C + c]);
      sb += v;
      if (a.dv) sv = fmaf(a.alpha[pix / a.P], v, sv);
    }
  s_b[threadIdx.x] = sb;
  s_v[threadIdx.x] = sv;
  __syncthreads();
  if (r == 0) {
    for (int k = 1; k < rows; ++k) {
      sb += s_b[k * a.C + c];
      sv += s_v[k * a.C + c];
    }
    atomicAdd(a.db + c, sb);
    if (a.dv) atomicAdd(a.dv + c, sv);
  }
}


__device__ __forceinline__ double block_sum_d(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

// partial[b][blk] = sums over slices of sample b of v (n values per sample); with
// target, of (v - target) and of (v - target)^2 (partial2).
__global__ void sample_sums_kernel(const float* __restrict__ v, const float* __restrict__ target, long long n,
                                   double* __restrict__ partial, double* __restrict__ partial2) {
  __shared__ double sh[32];
  const int b = blockIdx.y;
  const float* vb = v + (size_t)b * n;
  const float* tb = target ? target + (size_t)b * n : nullptr;
  double s = 0.0, s2 = 0.0;
  // four values per load where every sample starts on a 16-byte boundary, then the tail
  const long long n4 = (n & 3) == 0 ? n >> 2 : 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n4; k += stride) {
    const float4 a = reinterpret_cast<const float4*>(vb)[k];
    double d[4] = {a.x, a.y, a.z, a.w};
    if (tb) {
      const float4 t = reinterpret_cast<const float4*>(tb)[k];
      d[0] -= (double)t.x;
      d[1] -= (double)t.y;
      d[2] -= (double)t.z;
      d[3] -= (double)t.w;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      s += d[e];
      s2 += d[e] * d[e];
    }
  }
  for (long long k = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride) {
    const double d = tb ? (double)vb[k] - (double)tb[k] : (double)vb[k];
    s += d;
    s2 += d * d;
  }
  s = block_sum_d(s, sh);
  if (partial2) s2 = block_sum_d(s2, sh);
  if (threadIdx.x == 0) {
    partial[b * gridDim.x + blockIdx.x] = s;
    if (partial2) partial2[b * gridDim.x + blockIdx.x] = s2;
  }
}

struct SampleWeights {
  float v[LBNOP_MAX_BATCH];
};

// y[b][k] = bf16(w[b] x[b][k]) for `per` values per sample.
__global__ void scale_rows_kernel(const bf16* __restrict__ x, long long per, int B, const SampleWeights w,
                                  bf16* __restrict__ y) {
  const long long n = per * B;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    y[k] = __float2bfloat16_rn(w.v[k / per] * __bfloat162float(x[k]));
}

// mean[b] = sum of partial[b][*] / n; with partial2, loss = sum_b w[b] partial2[b][*] / (B n).
__global__ void finish_sums_kernel(const double* __restrict__ partial, const double* __restrict__ partial2, int B,
                                   long long n, const SampleWeights w, double* __restrict__ mean,
                                   double* __restrict__ loss) {
  // one block of 32 warps; warp k handles samples k and k + 32 (B <= 64)
  __shared__ double s2s[LBNOP_MAX_BATCH];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int b = wid; b < B; b += 32) {
    const double sm = warp_partials(partial + (size_t)b * HEAD_BLOCKS, lane);
    const double s2 = partial2 ? warp_partials(partial2 + (size_t)b * HEAD_BLOCKS, lane) : 0.0;
    if (lane == 0) {
      mean[b] = sm / (double)n;
      s2s[b] = s2;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && partial2) {
    double tot2 = 0.0;
    for (int b = 0; b < B; ++b) tot2 += (double)w.v[b] * s2s[b];
    *loss = tot2 / ((double)B * (double)n);
  }
}

// phi_out = phi + scale sig[b] (D - mean D), D = depth-to-space of zout [B][H/4][W/4][16].
__global__ void head_kernel(const float* __restrict__ phi, const float* __restrict__ zout,
                            const double* __restrict__ mean, const double* __restrict__ sig, int B, int H, int W,
                            float scale, float* __restrict__ phi_out) {
  const long long n = (long long)B * H * W;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % W), y = (int)((k / W) % H), b = (int)(k / ((long long)W * H));
    const float D = zout[((size_t)(b * (H / 4) + y / 4) * (W / 4) + x / 4) * 16 + 4 * (y & 3) + (x & 3)];
    phi_out[k] = phi[k] + scale * (float)sig[b] * (D - (float)mean[b]);
  }
}

// dz_out = space-to-depth of scale sig[b] (g - mean g), g = 2 w[b] (phi_out - target) / (B H W)
// the gradient of the weighted mean squared error; mean_d[b] is the mean of
// (phi_out - target) and coef[b] = 2 scale w[b] / (B H W).
__global__ void head_bwd_kernel(const float* __restrict__ phi_out, const float* __restrict__ target,
                                const double* __restrict__ mean_d, const double* __restrict__ sig, int B, int H,
                                int W, const SampleWeights coef, bf16* __restrict__ dz) {
  const long long n = (long long)B * H * W;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(k % W), y = (int)((k / W) % H), b = (int)(k / ((long long)W * H));
    const float d = (float)((double)phi_out[k] - (double)target[k] - mean_d[b]);
    dz[((size_t)(b * (H / 4) + y / 4) * (W / 4) + x / 4) * 16 + 4 * (y & 3) + (x & 3)] =
        __float2bfloat16_rn(coef.v[b] * (float)sig[b] * d);
  }
}

// The global L2 norm of the gradient, in FP64 and a fixed order: grad_sq_kernel (grid of
// HEAD_BLOCKS) leaves one partial sum of grad^2 per block (FP64 runs at a small fraction of
// the FP32 rate, so the sum is spread over the SMs), then grad_norm_kernel (one warp) adds the
// partials and takes the square root.
__global__ void grad_sq_kernel(const float* __restrict__ grad, long long n, double* __restrict__ partial) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const double g = grad[k];
    s = fma(g, g, s);
  }
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}
__global__ void grad_norm_kernel(const double* __restrict__ partial, double* __restrict__ norm) {
  const double s = warp_partials(partial, threadIdx.x);
  if (threadIdx.x == 0) *norm = sqrt(s);
}

// Audit of a judged leap: sum (a - b)^2 and sum b^2 over n values in FP64 and a fixed
// order; diff_norm_kernel (grid of HEAD_BLOCKS) leaves the two partial sums of each block in
// partial[2 blk], partial[2 blk + 1]; diff_norm_final (one warp) writes out[0] = sum (a - b)^2
// and out[1] = sum b^2.
__global__ void diff_norm_kernel(const float* __restrict__ a, const float* __restrict__ b, long long n,
                                 double* __restrict__ partial) {
  __shared__ double sh[32];
  double d2 = 0.0, b2 = 0.0;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const double bv = b[k], dv = (double)a[k] - bv;
    d2 = fma(dv, dv, d2);
    b2 = fma(bv, bv, b2);
  }
  d2 = block_sum_d(d2, sh);
  __syncthreads();
  b2 = block_sum_d(b2, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = d2;
    partial[2 * blockIdx.x + 1] = b2;
  }
}
__global__ void diff_norm_final(const double* __restrict__ partial, int blocks, double* __restrict__ out) {
  double d2 = 0.0, b2 = 0.0;
  for (int k = threadIdx.x; k < blocks; k += 32) {
    d2 += partial[2 * k];
    b2 += partial[2 * k + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2 += __shfl_down_sync(0xffffffffu, d2, o);
    b2 += __shfl_down_sync(0xffffffffu, b2, o);
  }
  if (threadIdx.x == 0) {
    out[0] = d2;
    out[1] = b2;
  }
}

// The four quarter turns of an n x n field into out[k] (k = 0..3, n^2 values each), row i and
// column j: turn_k(phi)[i][j] = phi[src_k(i, j)] with src_1 = (j, n-1-i), src_2 = (n-1-i,
// n-1-j), src_3 = (n-1-j, i) (k = 1 a counter-clockwise quarter turn about the centre).
__global__ void turns_kernel(const float* __restrict__ phi, int n, float* __restrict__ out) {
  const long long nn = (long long)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nn; idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
    out[idx] = phi[idx];
    out[nn + idx] = phi[(long long)j * n + (n - 1 - i)];
    out[2 * nn + idx] = phi[(long long)(n - 1 - i) * n + (n - 1 - j)];
    out[3 * nn + idx] = phi[(long long)(n - 1 - j) * n + i];
  }
}
// The mean of four predictions y[k] of the turned fields, each turned back (turn_{4-k}).
__global__ void turns_back_kernel(const float* __restrict__ y, int n, float* __restrict__ out) {
  const long long nn = (long long)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nn; idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
    const float y0 = y[idx];
    const float y1 = y[nn + (long long)(n - 1 - j) * n + i];
    const float y2 = y[2 * nn + (long long)(n - 1 - i) * n + (n - 1 - j)];
    const float y3 = y[3 * nn + (long long)j * n + (n - 1 - i)];
    out[idx] = (((y0 + y1) + y2) + y3) * 0.25f;
  }
}

// Adam (Kingma and Ba 2015, Algorithm 1; c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)) on
// the gradient scaled by min(1, clip / |grad|) when clip > 0 (global-norm clipping), then the
// BF16 copies of every weight: wf[t][co][ci] and wb[t][ci][co] = W[8 - t][co][ci].
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ grad, long long n, float lr, float c1, float c2, int update,
                            const double* __restrict__ gnorm, double clip, const LayerTab tab,
                            bf16* __restrict__ wf, bf16* __restrict__ wb, bf16* __restrict__ wlo) {
  float gscale = 1.0f;
  if (update && clip > 0.0) {
    const double nrm = *gnorm;
    if (nrm > clip) gscale = (float)(clip / nrm);
  }
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    float th = theta[k];
    if (update) {
      const float gk = grad[k] * gscale;
      const float mk = fmaf(0.9f, m[k], 0.1f * gk);
      const float vk = fmaf(0.999f, v[k], 0.001f * gk * gk);
      m[k] = mk;
      v[k] = vk;
      th -= lr * (mk * c1) / (sqrtf(vk * c2) + 1e-8f);
      theta[k] = th;
    }
    for (int l = 0; l < NL; ++l) {
      const long long rel = k - tab.off_w[l];
      const int ci = tab.ci[l], co = tab.co[l];
      if (rel >= 0 && rel < 9LL * co * ci) {
        const int t = (int)(rel / ((long long)co * ci)), r2 = (int)(rel % ((long long)co * ci));
        const int o = r2 / ci, i = r2 - o * ci;
        const bf16 hv = __float2bfloat16_rn(th);
        wf[tab.woff[l] + rel] = hv;
        wlo[tab.woff[l] + rel] = __float2bfloat16_rn(th - __bfloat162float(hv));
        wb[tab.woff[l] + ((size_t)(8 - t) * ci + i) * co + o] = hv;
        break;
      }
    }
  }
}

__global__ void finite_kernel(const float* __restrict__ v, long long n, int* bad) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    if (!isfinite(v[k])) atomicOr(bad, 1);
}

// ---------------------------------------------------------------- launch helpers

// Multiprocessor count of the current device, queried once per device.
int device_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

// Fields with few pixels (coarse levels, small batches) split the output channels over
// blocks in slices of 16, so that enough warps run; large ones keep all channels per warp
// and load each A fragment once.
// conv_smem_kernel with its dynamic shared memory (opted in once per device above 48 KB).
template <int CI, int CO, int BN>
void launch_smem(const ConvArgs& a, dim3 grid, cudaStream_t s) {
  constexpr int bytes = conv_smem_bytes<CI, BN>();
  if constexpr (bytes > 48 * 1024) {
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load(std::memory_order_relaxed) & bit)) {
      cudaFuncSetAttribute(conv_smem_kernel<CI, CO, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      done.fetch_or(bit, std::memory_order_relaxed);
    }
  }
  conv_smem_kernel<CI, CO, BN><<<grid, CONV_THREADS, bytes, s>>>(a);
}

}  // namespace nop

#include "lbnop_tc.cuh"

namespace nop {

template <int CI, int CO, bool TW>
void conv_t(const ConvArgs& a, cudaStream_t s) {
  const int npix = a.B * a.H * a.W;
  // rows of 128 pixels or more: the tcgen05 path (operands by TMA, accumulators in TMEM)
  if constexpr (!TW) {
    if (tc_applies(a, CI, CO) && launch_tc<CI, CO>(a, nullptr, device_sms(), s)) return;
  }
  const int tiles = (npix + 63) / 64;
  const long long want_warps = (long long)device_sms() * 16;  // below this, slice the channels
  if constexpr (TW) {  // the operator entry point on forward-layout weights (register-fed)
    conv_kernel<CI, CO, CO, true, false><<<dim3(tiles, 1), CONV_THREADS, 0, s>>>(a);
  } else {
    if constexpr (CI == 16) {  // layers reading phi: low halves of the input (and weights)
      if (a.x2 && a.w2) {
        if constexpr (CO == 16) {
          if ((long long)tiles * 4 < want_warps)
            conv_kernel<CI, CO, 16, false, true, true><<<dim3(tiles, 1), CONV_THREADS, 0, s>>>(a);
          else
            conv_kernel<CI, CO, CO, false, true, true><<<dim3(tiles, 1), CONV_THREADS, 0, s>>>(a);
        }
        return;
      }
      if (a.x2) {
        if ((long long)tiles * 4 < want_warps)
          conv_kernel<CI, CO, 16, false, true><<<dim3(tiles, CO / 16), CONV_THREADS, 0, s>>>(a);
        else
          conv_kernel<CI, CO, CO, false, true><<<dim3(tiles, 1), CONV_THREADS, 0, s>>>(a);
        return;
      }
    }
    // few enough blocks of 16 x 16 that about five per SM cover the layer: the coarse levels
    if ((long long)((npix + 15) / 16) * (CO / 16) <= (long long)device_sms() * 5) {
      conv_splitk_kernel<CI, CO><<<dim3((npix + 15) / 16, CO / 16), SPLITK_THREADS, 0, s>>>(a);
      return;
    }
    // operands staged through shared memory; mid-size layers split the output channels into
    // slices of 32 so that enough blocks run
    if constexpr (CO > 16) {
      if ((long long)tiles * 4 < want_warps) {
        launch_smem<CI, CO, 32>(a, dim3(tiles, CO / 32), s);
        return;
      }
    }
    launch_smem<CI, CO, CO>(a, dim3(tiles, 1), s);
  }
}

template <int CI, int CO>
void wgrad_t(const WgradArgs& a, cudaStream_t s) {
  // rows of 128 pixels or more: the tcgen05 path (pixels as the contraction, accumulators in TMEM)
  if (wgrad_tc_applies(a)) {
    launch_wgrad_tc<CI, CO>(a, nullptr, device_sms(), s);
    return;
  }
  const int npix = a.B * a.H * a.W;
  wgrad_kernel<CI, CO><<<dim3((npix + a.chunk - 1) / a.chunk, 9), 128, 0, s>>>(a);
}

bool channels_ok(int c) { return c == 16 || c == 64 || c == 96; }

#define NOP_CH_SWITCH(CI, CO, CALL) \
  switch (CI * 1000 + CO) {          \
    case 16016: CALL(16, 16); break; \
    case 16064: CALL(16, 64); break; \
    case 16096: CALL(16, 96); break; \
    case 64016: CALL(64, 16); break; \
    case 64064: CALL(64, 64); break; \
    case 64096: CALL(64, 96); break; \
    case 96016: CALL(96, 16); break; \
    case 96064: CALL(96, 64); break; \
    case 96096: CALL(96, 96); break; \
    default: break;                  \
  }

void conv_launch(int ci, int co, bool tw, const ConvArgs& a, cudaStream_t s) {
#define NOP_CONV_F(I, O) conv_t<I, O, false>(a, s)
#define NOP_CONV_T(I, O) conv_t<I, O, true>(a, s)
  if (tw) {
    NOP_CH_SWITCH(ci, co, NOP_CONV_T)
  } else {
    NOP_CH_SWITCH(ci, co, NOP_CONV_F)
  }
#undef NOP_CONV_F
#undef NOP_CONV_T
}

int wgrad_chunk(int npix) {
  int c = (npix + 63) / 64;
  c = (c + 31) / 32 * 32;
  return c < 512 ? 512 : c;
}

void wgrad_launch(int ci, int co, const WgradArgs& a, cudaStream_t s) {
#define NOP_WG(I, O) wgrad_t<I, O>(a, s)
  NOP_CH_SWITCH(ci, co, NOP_WG)
#undef NOP_WG
}

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  const long long cap = (long long)device_sms() * 16;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

}  // namespace nop

using namespace nop;

// ---------------------------------------------------------------- context

struct lbnop_ctx {
  lbnop_params p;
  cudaStream_t stream;
  LayerTab tab;
  long long n_params, n_w;
  int off_b[NL], off_v;
  int h0, w0;  // level-0 size (H/4, W/4)
  float *theta, *m, *v, *grad;
  bf16 *wf, *wb, *wlo;
  unsigned char* wpk;       // weights of the tensor-core layers in that path's layout
  long long wpk_off[NL];    // byte offset of layer l's packed weights, or -1 (mma.sync path)
  long long wpkb_off[NL];   // the same for its data-gradient convolution (weights wb), or -1
  long long wver, wpk_ver;  // refreshes of the BF16 weights; the one the packed copy is of
  // activations (BF16), by level; z_* pre-activations, a_* SiLU outputs
  bf16 *x0, *x0l, *z[NL], *a[NL], *p1, *p2, *p3, *in_d2a, *in_d1a, *in_d0a;
  bf16* dz[4];
  bf16* dz_lina;  // alpha times the output layer's dz (level 0, 16 channels)
  float *g0a, *g0b, *g1a, *g1b, *g2a, *g2b, *g3a;
  float* zout;
  double *partial, *partial2, *mean, *loss, *sig;
  double* gnorm;  // global L2 norm of the last gradient
  double clip;    // Adam clips the gradient to this global norm; 0: off
  float *leap0, *leap1;
  float* phi_out;  // [max_batch][H][W], the training forward's output
  int* flags;
  int leap_turns;           // quarter turns a leap averages the network over (1 or 4)
  char* judge_state;        // two saved lbch states of an H x W FP32 field (judged leap runs)
  size_t judge_state_bytes; // bytes of one of them
  double* judge_vals;       // 16 doubles: two slots of mass / energy readings and audit sums
  cudaStream_t side;        // judged runs read their readings back on this stream (made on first use)
  cudaEvent_t ready[2];     // recorded after each cycle's first reading
  bool side_made;
  long long adam_t;
  int last_batch;
  bool failed;
  char err[512];
};

namespace {

constexpr size_t NOP_ALIGN = 256;
size_t al(size_t b) { return (b + NOP_ALIGN - 1) / NOP_ALIGN * NOP_ALIGN; }

const char* check_params(const lbnop_params* p) {
  if (!p) return "params is NULL";
  if (p->H < 32 || p->W < 32 || p->H > 8192 || p->W > 8192 || p->H % 32 || p->W % 32)
    return "H and W must be multiples of 32 in [32, 8192]";
  if (p->max_batch < 1 || p->max_batch > LBNOP_MAX_BATCH) return "max_batch must be in [1, 64]";
  if (!(p->scale > 0.0) || !std::isfinite(p->scale)) return "scale must be finite and > 0";
  return nullptr;
}

long long level_pixels(const lbnop_params* p, int level) {
  return (long long)p->max_batch * ((p->H / 4) >> level) * ((p->W / 4) >> level);
}

// Bytes of the lbch state of an H x W field in FP32 storage (the leap runs' lbm context).
size_t judge_state_size(const lbnop_params* p) {
  lbch_params q{};
  q.nx = p->W;
  q.ny = p->H;
  q.M = 0.1;
  q.sigma = 0.01;
  q.D = 5.0;
  q.eps = 0.03;
  for (int i = 0; i < 9; ++i) q.s[i] = 1.0;
  q.storage = LBCH_STORE_F32;
  q.regularization = LBCH_REG_WILLMORE;
  return lbch_state_bytes(&q);
}

// Walks the workspace layout; with c == nullptr only measures it.
size_t layout(const lbnop_params* p, lbnop_ctx* c, char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* r = base ? base + off : nullptr;
    off += al(bytes);
    return r;
  };
  long long n_params = 0, n_w = 0;
  for (int l = 0; l < NL; ++l) {
    n_params += 9LL * kL[l].co * kL[l].ci + kL[l].co + (l == E0A ? kL[l].co : 0);
    n_w += 9LL * kL[l].co * kL[l].ci;
  }
  const long long P[4] = {level_pixels(p, 0), level_pixels(p, 1), level_pixels(p, 2), level_pixels(p, 3)};
  char* theta = take(n_params * 4);
  char* m = take(n_params * 4);
  char* v = take(n_params * 4);
  char* grad = take(n_params * 4);
  char* wf = take(n_w * 2);
  char* wb = take(n_w * 2);
  char* wlo = take(n_w * 2);
  long long wpk_off[NL], wpkb_off[NL], wpk_bytes = 0;
  for (int l = 0; l < NL; ++l) {
    const int lv = kL[l].level, kc = (l == E0A ? 2 : 1) * kL[l].ci / 8;
    // the layers whose level rows the tensor-core path takes (tc_applies, at the level's size):
    // their forward weights and, but for the layers reading phi (no input gradient), the
    // transposed weights of their data gradient (c_in and c_out swapped)
    const bool tc = l != LIN && l != LINA && ((p->W / 4) >> lv) % 128 == 0 && ((p->H / 4) >> lv) % 4 == 0;
    wpk_off[l] = tc ? wpk_bytes : -1;
    if (tc) wpk_bytes += 9LL * kc * (kL[l].co * 16 + 16);
    wpkb_off[l] = tc && l != E0A ? wpk_bytes : -1;
    if (tc && l != E0A) wpk_bytes += 9LL * (kL[l].co / 8) * (kL[l].ci * 16 + 16);
  }
  char* wpk = take(wpk_bytes > 0 ? (size_t)wpk_bytes : 16);
  char* x0 = take(P[0] * 16 * 2);
  char* x0l = take(P[0] * 16 * 2);
  char *zz[NL], *aa[NL];
  for (int l = 0; l < NL; ++l) {
    zz[l] = take(P[kL[l].level] * kL[l].co * 2);
    aa[l] = kL[l].act ? take(P[kL[l].level] * kL[l].co * 2) : nullptr;
  }
  // widest tensor per level (the dz and gradient buffers serve every layer of their level)
  int wide[4] = {16, 0, 0, 0};
  for (int l = 0; l < NL; ++l) {
    wide[kL[l].level] = wide[kL[l].level] > kL[l].co ? wide[kL[l].level] : kL[l].co;
    wide[kL[l].level] = wide[kL[l].level] > kL[l].ci ? wide[kL[l].level] : kL[l].ci;
  }
  char* p1 = take(P[1] * CH[0] * 2);
  char* p2 = take(P[2] * CH[1] * 2);
  char* p3 = take(P[3] * CH[2] * 2);
  char* in2 = take(P[2] * CH[2] * 2);
  char* in1 = take(P[1] * CH[1] * 2);
  char* in0 = take(P[0] * CH[0] * 2);
  char* dz[4] = {take(P[0] * wide[0] * 2), take(P[1] * wide[1] * 2), take(P[2] * wide[2] * 2),
                 take(P[3] * wide[3] * 2)};
  char* dz_lina = take(P[0] * 16 * 2);
  char* g0a = take(P[0] * wide[0] * 4);
  char* g0b = take(P[0] * wide[0] * 4);
  char* g1a = take(P[1] * wide[1] * 4);
  char* g1b = take(P[1] * wide[1] * 4);
  char* g2a = take(P[2] * wide[2] * 4);
  char* g2b = take(P[2] * wide[2] * 4);
  char* g3a = take(P[3] * wide[3] * 4);
  char* zout = take(P[0] * 16 * 4);
  char* partial = take((size_t)LBNOP_MAX_BATCH * HEAD_BLOCKS * 8);
  char* partial2 = take((size_t)LBNOP_MAX_BATCH * HEAD_BLOCKS * 8);
  char* mean = take(LBNOP_MAX_BATCH * 8);
  char* sig = take(LBNOP_MAX_BATCH * 8);
  char* loss = take(8);
  char* gnorm = take(8);
  char* leap0 = take((size_t)p->H * p->W * 4);
  char* leap1 = take((size_t)p->H * p->W * 4);
  char* phi_out = take((size_t)p->max_batch * p->H * p->W * 4);
  char* flags = take(16);
  const size_t jsb = judge_state_size(p);
  char* judge_state = take(2 * jsb);
  char* judge_vals = take(16 * 8);
  if (c) {
    c->n_params = n_params;
    c->n_w = n_w;
    c->theta = (float*)theta;
    c->m = (float*)m;
    c->v = (float*)v;
    c->grad = (float*)grad;
    c->wf = (bf16*)wf;
    c->wb = (bf16*)wb;
    c->wlo = (bf16*)wlo;
    c->wpk = (unsigned char*)wpk;
    for (int l = 0; l < NL; ++l) {
      c->wpk_off[l] = wpk_off[l];
      c->wpkb_off[l] = wpkb_off[l];
    }
    c->x0 = (bf16*)x0;
    c->x0l = (bf16*)x0l;
    for (int l = 0; l < NL; ++l) {
      c->z[l] = (bf16*)zz[l];
      c->a[l] = (bf16*)aa[l];
    }
    c->p1 = (bf16*)p1;
    c->p2 = (bf16*)p2;
    c->p3 = (bf16*)p3;
    c->in_d2a = (bf16*)in2;
    c->in_d1a = (bf16*)in1;
    c->in_d0a = (bf16*)in0;
    for (int k = 0; k < 4; ++k) c->dz[k] = (bf16*)dz[k];
    c->dz_lina = (bf16*)dz_lina;
    c->g0a = (float*)g0a;
    c->g0b = (float*)g0b;
    c->g1a = (float*)g1a;
    c->g1b = (float*)g1b;
    c->g2a = (float*)g2a;
    c->g2b = (float*)g2b;
    c->g3a = (float*)g3a;
    c->zout = (float*)zout;
    c->partial = (double*)partial;
    c->partial2 = (double*)partial2;
    c->mean = (double*)mean;
    c->sig = (double*)sig;
    c->loss = (double*)loss;
    c->gnorm = (double*)gnorm;
    c->leap0 = (float*)leap0;
    c->leap1 = (float*)leap1;
    c->phi_out = (float*)phi_out;
    c->flags = (int*)flags;
    c->judge_state = judge_state;
    c->judge_state_bytes = jsb;
    c->judge_vals = (double*)judge_vals;
  }
  return off;
}

void set_err(lbnop_ctx* c, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof(c->err), fmt, ap);
  va_end(ap);
}

bool cuda_bad(lbnop_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return false;
  c->failed = true;
  set_err(c, "%s: %s", what, cudaGetErrorString(e));
  return true;
}

lbch_status pre(lbnop_ctx* c) {
  if (!c) return LBCH_EINVAL;
  return c->failed ? LBCH_ESTATE : LBCH_OK;
}

lbch_status done(lbnop_ctx* c, const char* what) {
  return cuda_bad(c, cudaGetLastError(), what) ? LBCH_ECUDA : LBCH_OK;
}

// After a synchronisation that covers this context's convolutions: true (and the context
// failed) if a tensor-core convolution of this process gave up a bounded wait (its outputs are
// invalid; tc_fault_flag), or if the flag cannot be read.
bool tc_faulted(lbnop_ctx* c, const char* what) {
  int v = 0;
  if (cuda_bad(c, cudaMemcpyFromSymbol(&v, tc_fault_flag, sizeof(int)), what)) return true;
  if (!v) return false;
  c->failed = true;
  set_err(c, "%s: a tensor-core convolution gave up a bounded wait; its results are invalid", what);
  return true;
}

// Level dimensions for `batch` fields.
struct Dims {
  int B, h[4], w[4];
};
Dims dims(const lbnop_ctx* c, int batch) {
  Dims d;
  d.B = batch;
  for (int l = 0; l < 4; ++l) {
    d.h[l] = c->h0 >> l;
    d.w[l] = c->w0 >> l;
  }
  return d;
}

const bf16* wf_of(const lbnop_ctx* c, int l) { return c->wf + c->tab.woff[l]; }
const bf16* wb_of(const lbnop_ctx* c, int l) { return c->wb + c->tab.woff[l]; }
const float* bias_of(const lbnop_ctx* c, int l) { return c->theta + c->off_b[l]; }

// One layer forward: x -> z (kept when training or when the layer is linear) and a.
void layer_fwd(lbnop_ctx* c, int l, const Dims& d, const bf16* x, bool training, const double* alpha) {
  ConvArgs a{};
  a.x = x;
  a.x2 = (l == E0A || l == LIN || l == LINA) ? c->x0l : nullptr;
  a.w2 = (l == LIN || l == LINA) ? c->wlo + c->tab.woff[l] : nullptr;
  a.w = wf_of(c, l);
  a.wpk = c->wpk_off[l] >= 0 ? c->wpk + c->wpk_off[l] : nullptr;
  a.B = d.B;
  a.H = d.h[kL[l].level];
  a.W = d.w[kL[l].level];
  a.bias = bias_of(c, l);
  a.film = l == E0A ? c->theta + c->off_v : nullptr;
  for (int b = 0; b < d.B; ++b) a.alpha[b] = (float)alpha[b];
  if (l == OUT || l == LIN || l == LINA) {  // the three terms of D sum into zout
    a.yf = c->zout;
    a.accumulate = l != OUT;
    a.scale_alpha = l == LINA;
  } else {
    a.z = (training || !kL[l].act) ? c->z[l] : nullptr;
    a.a = kL[l].act ? c->a[l] : nullptr;
  }
  conv_launch(kL[l].ci, kL[l].co, false, a, c->stream);
}

// The tensor-core layers' weights in that path's layout, once per refresh of the BF16 weights.
void pack_weights(lbnop_ctx* c) {
  if (c->wpk_ver == c->wver) return;
  for (int l = 0; l < NL; ++l) {
    if (c->wpk_off[l] < 0) continue;
    const int kc = (l == E0A ? 2 : 1) * kL[l].ci / 8;
    tc_pack_kernel<<<grid_for(9LL * kc * (kL[l].co + 1), 256), 256, 0, c->stream>>>(
        wf_of(c, l), kL[l].ci, kL[l].co, kc, c->wpk + c->wpk_off[l]);
    if (c->wpkb_off[l] >= 0)
      tc_pack_kernel<<<grid_for(9LL * (kL[l].co / 8) * (kL[l].ci + 1), 256), 256, 0, c->stream>>>(
          wb_of(c, l), kL[l].co, kL[l].ci, kL[l].co / 8, c->wpk + c->wpkb_off[l]);
  }
  c->wpk_ver = c->wver;
}

void forward_impl(lbnop_ctx* c, const float* d_phi, const double* alpha, int batch, float* d_out, bool training) {
  const Dims d = dims(c, batch);
  cudaStream_t s = c->stream;
  pack_weights(c);
  const long long P0 = (long long)batch * d.h[0] * d.w[0];
  const long long hw = (long long)c->p.H * c->p.W;
  sample_sums_kernel<<<dim3(HEAD_BLOCKS, batch), 256, 0, s>>>(d_phi, nullptr, hw, c->partial, c->partial2);
  rms_kernel<<<batch, 32, 0, s>>>(c->partial2, batch, hw, c->sig);
  s2d_kernel<<<grid_for(P0, 256), 256, 0, s>>>(d_phi, c->sig, batch, c->p.H, c->p.W, c->x0, c->x0l);
  layer_fwd(c, E0A, d, c->x0, training, alpha);
  layer_fwd(c, E0B, d, c->a[E0A], training, alpha);
  auto pool = [&](const bf16* x, int lvl, int C, bf16* y) {
    const long long n = (long long)batch * d.h[lvl] * d.w[lvl] * (C / 8);
    pool_kernel<<<grid_for(n, 256), 256, 0, s>>>(x, batch, d.h[lvl], d.w[lvl], C, y);
  };
  auto up_add = [&](const bf16* xc, const bf16* skip, int lvl, int C, bf16* y) {
    const long long n = (long long)batch * d.h[lvl] * d.w[lvl] * (C / 8);
    up_add_kernel<<<grid_for(n, 256), 256, 0, s>>>(xc, skip, batch, d.h[lvl], d.w[lvl], C, y);
  };
  pool(c->a[E0B], 1, CH[0], c->p1);
  layer_fwd(c, E1A, d, c->p1, training, alpha);
  layer_fwd(c, E1B, d, c->a[E1A], training, alpha);
  pool(c->a[E1B], 2, CH[1], c->p2);
  layer_fwd(c, E2A, d, c->p2, training, alpha);
  layer_fwd(c, E2B, d, c->a[E2A], training, alpha);
  pool(c->a[E2B], 3, CH[2], c->p3);
  layer_fwd(c, M3A, d, c->p3, training, alpha);
  layer_fwd(c, M3B, d, c->a[M3A], training, alpha);
  up_add(c->a[M3B], c->a[E2B], 2, CH[2], c->in_d2a);
  layer_fwd(c, D2A, d, c->in_d2a, training, alpha);
  layer_fwd(c, D2B, d, c->a[D2A], training, alpha);
  up_add(c->z[D2B], c->a[E1B], 1, CH[1], c->in_d1a);
  layer_fwd(c, D1A, d, c->in_d1a, training, alpha);
  layer_fwd(c, D1B, d, c->a[D1A], training, alpha);
  up_add(c->z[D1B], c->a[E0B], 0, CH[0], c->in_d0a);
  layer_fwd(c, D0A, d, c->in_d0a, training, alpha);
  layer_fwd(c, OUT, d, c->a[D0A], training, alpha);
  layer_fwd(c, LIN, d, c->x0, training, alpha);
  layer_fwd(c, LINA, d, c->x0, training, alpha);
  // head: D - mean D per field
  const long long nz = (long long)d.h[0] * d.w[0] * 16;
  sample_sums_kernel<<<dim3(HEAD_BLOCKS, batch), 256, 0, s>>>(c->zout, nullptr, nz, c->partial, nullptr);
  finish_sums_kernel<<<1, 1024, 0, s>>>(c->partial, nullptr, batch, (long long)c->p.H * c->p.W, SampleWeights{},
                                      c->mean, nullptr);
  const long long n = (long long)batch * c->p.H * c->p.W;
  head_kernel<<<grid_for(n, 256), 256, 0, s>>>(d_phi, c->zout, c->mean, c->sig, batch, c->p.H, c->p.W,
                                               (float)c->p.scale,
                                               d_out);
}

// Backward of layer l given dz (its pre-activation gradient, BF16, in c->dz[level]):
// weight and bias gradients, and the input gradient into gin (FP32) unless gin is null.
void layer_bwd(lbnop_ctx* c, int l, const Dims& d, const bf16* x_in, float* gin, const double* alpha,
               const bf16* dz_in = nullptr) {
  cudaStream_t s = c->stream;
  const int lvl = kL[l].level, ci = kL[l].ci, co = kL[l].co;
  const bf16* dz = dz_in ? dz_in : c->dz[lvl];
  ColsumArgs cs{};
  cs.dz = dz;
  cs.P = d.h[lvl] * d.w[lvl];
  cs.B = d.B;
  cs.C = co;
  cs.db = c->grad + c->off_b[l];
  cs.dv = l == E0A ? c->grad + c->off_v : nullptr;
  for (int b = 0; b < d.B; ++b) cs.alpha[b] = (float)alpha[b];
  const long long npix = (long long)d.B * cs.P;
  const int rows = 256 / co;
  int blocks = (int)((npix + rows * 64 - 1) / (rows * 64));
  blocks = blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks);
  colsum_kernel<<<blocks, rows * co, 0, s>>>(cs);
  WgradArgs wg{};
  wg.x = x_in;
  wg.dz = dz;
  wg.B = d.B;
  wg.H = d.h[lvl];
  wg.W = d.w[lvl];
  wg.chunk = wgrad_chunk((int)npix);
  wg.dw = c->grad + c->tab.off_w[l];
  wgrad_launch(ci, co, wg, s);
  if (x_in == c->x0) {  // the low half of the input shares the weights
    wg.x = c->x0l;
    wgrad_launch(ci, co, wg, s);
  }
  if (gin) {
    ConvArgs a{};
    a.x = dz;
    a.w = wb_of(c, l);
    a.wpk = c->wpkb_off[l] >= 0 ? c->wpk + c->wpkb_off[l] : nullptr;
    a.B = d.B;
    a.H = d.h[lvl];
    a.W = d.w[lvl];
    a.yf = gin;
    conv_launch(co, ci, false, a, s);
  }
}

// dz[level] = g (or up-adjoint of gf) times SiLU'(z) where z is given.
void make_dz(lbnop_ctx* c, const Dims& d, int lvl, int C, const float* g, const float* gf, const bf16* z) {
  const long long n = (long long)d.B * d.h[lvl] * d.w[lvl] * (C / 8);
  dz_kernel<<<grid_for(n, 256), 256, 0, c->stream>>>(g, gf, z, d.B, d.h[lvl], d.w[lvl], C, c->dz[lvl]);
}

void pool_bwd(lbnop_ctx* c, const Dims& d, int lvl_coarse, int C, const float* gc, float* gf) {
  const long long n = (long long)d.B * 4 * d.h[lvl_coarse] * d.w[lvl_coarse] * (C / 4);
  pool_bwd_kernel<<<grid_for(n, 256), 256, 0, c->stream>>>(gc, d.B, d.h[lvl_coarse], d.w[lvl_coarse], C, gf);
}

void backward_impl(lbnop_ctx* c, const float* d_phi, const double* alpha, const float* d_target,
                   const double* weight, int batch) {
  cudaStream_t s = c->stream;
  const Dims d = dims(c, batch);
  float* phi_out = c->phi_out;
  forward_impl(c, d_phi, alpha, batch, phi_out, true);
  const long long hw = (long long)c->p.H * c->p.W, n = batch * hw;
  sample_sums_kernel<<<dim3(HEAD_BLOCKS, batch), 256, 0, s>>>(phi_out, d_target, hw, c->partial, c->partial2);
  SampleWeights w{}, coef{};
  for (int b = 0; b < batch; ++b) {
    w.v[b] = weight ? (float)weight[b] : 1.0f;
    coef.v[b] = (float)(c->p.scale * 2.0 * (weight ? weight[b] : 1.0) / (double)n);
  }
  finish_sums_kernel<<<1, 1024, 0, s>>>(c->partial, c->partial2, batch, hw, w, c->mean, c->loss);
  cudaMemsetAsync(c->grad, 0, c->n_params * sizeof(float), s);
  head_bwd_kernel<<<grid_for(n, 256), 256, 0, s>>>(phi_out, d_target, c->mean, c->sig, batch, c->p.H, c->p.W, coef,
                                                   c->dz[0]);
  // the linear path: D gets lin(x) + alpha lina(x), so lin's dz is dz_out and lina's is alpha dz_out
  layer_bwd(c, LIN, d, c->x0, nullptr, alpha);
  {
    const long long nz = (long long)batch * d.h[0] * d.w[0] * 16;
    SampleWeights al{};
    for (int b = 0; b < batch; ++b) al.v[b] = (float)alpha[b];
    scale_rows_kernel<<<grid_for(nz, 256), 256, 0, s>>>(c->dz[0], (long long)d.h[0] * d.w[0] * 16, batch, al,
                                                        c->dz_lina);
  }
  layer_bwd(c, LINA, d, c->x0, nullptr, alpha, c->dz_lina);
  layer_bwd(c, OUT, d, c->a[D0A], c->g0a, alpha);
  make_dz(c, d, 0, kL[D0A].co, c->g0a, nullptr, c->z[D0A]);
  layer_bwd(c, D0A, d, c->in_d0a, c->g0b, alpha);  // g0b: gradient in h0 from here on
  make_dz(c, d, 1, kL[D1B].co, nullptr, c->g0b, nullptr);
  layer_bwd(c, D1B, d, c->a[D1A], c->g1a, alpha);
  make_dz(c, d, 1, kL[D1A].co, c->g1a, nullptr, c->z[D1A]);
  layer_bwd(c, D1A, d, c->in_d1a, c->g1b, alpha);  // g1b: gradient in h1
  make_dz(c, d, 2, kL[D2B].co, nullptr, c->g1b, nullptr);
  layer_bwd(c, D2B, d, c->a[D2A], c->g2a, alpha);
  make_dz(c, d, 2, kL[D2A].co, c->g2a, nullptr, c->z[D2A]);
  layer_bwd(c, D2A, d, c->in_d2a, c->g2b, alpha);  // g2b: gradient in h2
  make_dz(c, d, 3, kL[M3B].co, nullptr, c->g2b, c->z[M3B]);
  layer_bwd(c, M3B, d, c->a[M3A], c->g3a, alpha);
  make_dz(c, d, 3, kL[M3A].co, c->g3a, nullptr, c->z[M3A]);
  layer_bwd(c, M3A, d, c->p3, c->g3a, alpha);
  pool_bwd(c, d, 3, kL[M3A].ci, c->g3a, c->g2b);
  make_dz(c, d, 2, kL[E2B].co, c->g2b, nullptr, c->z[E2B]);
  layer_bwd(c, E2B, d, c->a[E2A], c->g2a, alpha);
  make_dz(c, d, 2, kL[E2A].co, c->g2a, nullptr, c->z[E2A]);
  layer_bwd(c, E2A, d, c->p2, c->g2a, alpha);
  pool_bwd(c, d, 2, kL[E2A].ci, c->g2a, c->g1b);
  make_dz(c, d, 1, kL[E1B].co, c->g1b, nullptr, c->z[E1B]);
  layer_bwd(c, E1B, d, c->a[E1A], c->g1a, alpha);
  make_dz(c, d, 1, kL[E1A].co, c->g1a, nullptr, c->z[E1A]);
  layer_bwd(c, E1A, d, c->p1, c->g1a, alpha);
  pool_bwd(c, d, 1, kL[E1A].ci, c->g1a, c->g0b);
  make_dz(c, d, 0, kL[E0B].co, c->g0b, nullptr, c->z[E0B]);
  layer_bwd(c, E0B, d, c->a[E0A], c->g0a, alpha);
  make_dz(c, d, 0, kL[E0A].co, c->g0a, nullptr, c->z[E0A]);
  layer_bwd(c, E0A, d, c->x0, nullptr, alpha);
  grad_sq_kernel<<<HEAD_BLOCKS, 256, 0, s>>>(c->grad, c->n_params, c->partial);
  grad_norm_kernel<<<1, 32, 0, s>>>(c->partial, c->gnorm);
  c->last_batch = batch;
}

void refresh_or_update(lbnop_ctx* c, bool update, double lr) {
  float c1 = 1.0f, c2 = 1.0f;
  if (update) {
    c->adam_t += 1;
    c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)c->adam_t)));
    c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)c->adam_t)));
  }
  adam_kernel<<<grid_for(c->n_params, 256), 256, 0, c->stream>>>(c->theta, c->m, c->v, c->grad, c->n_params,
                                                                 (float)lr, c1, c2, update ? 1 : 0, c->gnorm,
                                                                 c->clip, c->tab, c->wf, c->wb, c->wlo);
  ++c->wver;  // the packed tensor-core weights are stale until the next forward repacks them
}

lbch_status check_batch(lbnop_ctx* c, int batch, const double* h_alpha) {
  if (batch < 1 || batch > c->p.max_batch) {
    set_err(c, "batch must be in [1, max_batch = %d]", c->p.max_batch);
    return LBCH_EINVAL;
  }
  if (!h_alpha) {
    set_err(c, "h_alpha is NULL");
    return LBCH_EINVAL;
  }
  return LBCH_OK;
}

}  // namespace

extern "C" {

int64_t lbnop_param_count(void) {
  int64_t n = 0;
  for (int l = 0; l < NL; ++l) n += 9LL * kL[l].co * kL[l].ci + kL[l].co + (l == E0A ? kL[l].co : 0);
  return n;
}

size_t lbnop_workspace_bytes(const lbnop_params* p) {
  if (check_params(p)) return 0;
  return layout(p, nullptr, nullptr);
}

lbch_status lbnop_create(const lbnop_params* p, void* d_workspace, size_t bytes, void* cuda_stream, lbnop_ctx** out) {
  if (!out || check_params(p)) return LBCH_EINVAL;
  if (!d_workspace || bytes < lbnop_workspace_bytes(p) || ((uintptr_t)d_workspace % NOP_ALIGN) != 0)
    return LBCH_ENOMEM;
  lbnop_ctx* c = new (std::nothrow) lbnop_ctx();
  if (!c) return LBCH_ENOMEM;
  c->p = *p;
  c->stream = (cudaStream_t)cuda_stream;
  c->h0 = p->H / 4;
  c->w0 = p->W / 4;
  layout(p, c, (char*)d_workspace);
  int off = 0, woff = 0;
  for (int l = 0; l < NL; ++l) {
    c->tab.off_w[l] = off;
    c->tab.ci[l] = kL[l].ci;
    c->tab.co[l] = kL[l].co;
    c->tab.woff[l] = woff;
    off += 9 * kL[l].co * kL[l].ci;
    woff += 9 * kL[l].co * kL[l].ci;
    c->off_b[l] = off;
    off += kL[l].co;
    if (l == E0A) {
      c->off_v = off;
      off += kL[l].co;
    }
  }
  c->adam_t = 0;
  c->wver = 0;
  c->wpk_ver = -1;  // the first forward packs
  c->last_batch = 0;
  c->leap_turns = 1;
  c->failed = false;
  c->err[0] = 0;
  *out = c;
  return LBCH_OK;
}

lbch_status lbnop_set_params(lbnop_ctx* c, const float* h_theta) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!h_theta) return LBCH_EINVAL;
  const size_t nb = c->n_params * sizeof(float);
  if (cuda_bad(c, cudaMemcpyAsync(c->theta, h_theta, nb, cudaMemcpyHostToDevice, c->stream), "set_params: copy") ||
      cuda_bad(c, cudaMemsetAsync(c->m, 0, nb, c->stream), "set_params: clear") ||
      cuda_bad(c, cudaMemsetAsync(c->v, 0, nb, c->stream), "set_params: clear") ||
      cuda_bad(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "set_params: clear"))
    return LBCH_ECUDA;
  finite_kernel<<<grid_for(c->n_params, 256), 256, 0, c->stream>>>(c->theta, c->n_params, c->flags);
  refresh_or_update(c, false, 0.0);
  c->adam_t = 0;
  int bad = 0;
  if (cuda_bad(c, cudaMemcpyAsync(&bad, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "set_params") ||
      cuda_bad(c, cudaStreamSynchronize(c->stream), "set_params: sync") || tc_faulted(c, "set_params"))
    return LBCH_ECUDA;
  if (bad) {
    set_err(c, "set_params: NaN or Inf in the parameters");
    return LBCH_ENONFINITE;
  }
  return done(c, "set_params");
}

lbch_status lbnop_get_params(lbnop_ctx* c, float* h_theta) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!h_theta) return LBCH_EINVAL;
  if (cuda_bad(c, cudaMemcpyAsync(h_theta, c->theta, c->n_params * 4, cudaMemcpyDeviceToHost, c->stream), "get") ||
      cuda_bad(c, cudaStreamSynchronize(c->stream), "get_params: sync"))
    return LBCH_ECUDA;
  return LBCH_OK;
}

lbch_status lbnop_forward(lbnop_ctx* c, const float* d_phi, const double* h_alpha, int32_t batch, float* d_phi_out) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!d_phi || !d_phi_out) return LBCH_EINVAL;
  if ((st = check_batch(c, batch, h_alpha)) != LBCH_OK) return st;
  forward_impl(c, d_phi, h_alpha, batch, d_phi_out, false);
  return done(c, "forward: launch");
}

lbch_status lbnop_backward(lbnop_ctx* c, const float* d_phi, const double* h_alpha, const float* d_target,
                           const double* h_weight, int32_t batch, double* h_loss) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!d_phi || !d_target) return LBCH_EINVAL;
  if ((st = check_batch(c, batch, h_alpha)) != LBCH_OK) return st;
  if (h_weight)
    for (int b = 0; b < batch; ++b)
      if (!(h_weight[b] >= 0.0) || !std::isfinite(h_weight[b])) {
        set_err(c, "backward: weights must be finite and >= 0");
        return LBCH_EINVAL;
      }
  backward_impl(c, d_phi, h_alpha, d_target, h_weight, batch);
  if ((st = done(c, "backward: launch")) != LBCH_OK) return st;
  if (h_loss) {
    if (cuda_bad(c, cudaMemcpyAsync(h_loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "loss") ||
        cuda_bad(c, cudaStreamSynchronize(c->stream), "backward: sync") || tc_faulted(c, "backward"))
      return LBCH_ECUDA;
  }
  return LBCH_OK;
}

lbch_status lbnop_get_grads(lbnop_ctx* c, float* h_grad) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!h_grad) return LBCH_EINVAL;
  if (cuda_bad(c, cudaMemcpyAsync(h_grad, c->grad, c->n_params * 4, cudaMemcpyDeviceToHost, c->stream), "grads") ||
      cuda_bad(c, cudaStreamSynchronize(c->stream), "get_grads: sync") || tc_faulted(c, "get_grads"))
    return LBCH_ECUDA;
  return LBCH_OK;
}

lbch_status lbnop_adam(lbnop_ctx* c, double lr) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!(lr >= 0.0) || !std::isfinite(lr)) return LBCH_EINVAL;
  if (c->last_batch == 0) {
    set_err(c, "adam: no gradient yet (call lbnop_backward first)");
    return LBCH_EINVAL;
  }
  refresh_or_update(c, true, lr);
  return done(c, "adam: launch");
}

lbch_status lbnop_set_clip(lbnop_ctx* c, double max_norm) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!(max_norm >= 0.0) || !std::isfinite(max_norm)) {
    set_err(c, "set_clip: max_norm must be finite and >= 0");
    return LBCH_EINVAL;
  }
  c->clip = max_norm;
  return LBCH_OK;
}

lbch_status lbnop_grad_norm(lbnop_ctx* c, double* h_norm) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!h_norm) return LBCH_EINVAL;
  if (c->last_batch == 0) {
    set_err(c, "grad_norm: no gradient yet (call lbnop_backward first)");
    return LBCH_EINVAL;
  }
  if (cuda_bad(c, cudaMemcpyAsync(h_norm, c->gnorm, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "gnorm") ||
      cuda_bad(c, cudaStreamSynchronize(c->stream), "grad_norm: sync") || tc_faulted(c, "grad_norm"))
    return LBCH_ECUDA;
  return LBCH_OK;
}

lbch_status lbnop_train_step(lbnop_ctx* c, const float* d_phi, const double* h_alpha, const float* d_target,
                             const double* h_weight, int32_t batch, double lr, double* h_loss) {
  lbch_status st = lbnop_backward(c, d_phi, h_alpha, d_target, h_weight, batch, nullptr);
  if (st != LBCH_OK) return st;
  if ((st = lbnop_adam(c, lr)) != LBCH_OK) return st;
  if (h_loss) {
    if (cuda_bad(c, cudaMemcpyAsync(h_loss, c->loss, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "loss") ||
        cuda_bad(c, cudaStreamSynchronize(c->stream), "train_step: sync") || tc_faulted(c, "train_step"))
      return LBCH_ECUDA;
  }
  return LBCH_OK;
}

// One leap of the field in leap0, in place: the network, or the mean over the field's four
// quarter turns of the network's predictions turned back (lbnop_set_leap_turns).
static void leap_forward(lbnop_ctx* c, double alpha) {
  if (c->leap_turns == 4) {
    const int n = c->p.H;
    const double a4[4] = {alpha, alpha, alpha, alpha};
    turns_kernel<<<grid_for((long long)n * n, 256), 256, 0, c->stream>>>(c->leap0, n, c->phi_out);
    forward_impl(c, c->phi_out, a4, 4, c->phi_out, false);
    turns_back_kernel<<<grid_for((long long)n * n, 256), 256, 0, c->stream>>>(c->phi_out, n, c->leap0);
  } else {
    forward_impl(c, c->leap0, &alpha, 1, c->leap0, false);
  }
}

lbch_status lbnop_set_leap_turns(lbnop_ctx* c, int32_t turns) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (turns != 1 && turns != 4) {
    set_err(c, "set_leap_turns: turns must be 1 or 4");
    return LBCH_EINVAL;
  }
  if (turns == 4 && (c->p.H != c->p.W || c->p.max_batch < 4)) {
    set_err(c, "set_leap_turns: 4 turns need a square field and max_batch >= 4");
    return LBCH_EINVAL;
  }
  c->leap_turns = turns;
  return LBCH_OK;
}

lbch_status lbnop_leap_run(lbnop_ctx* c, lbch_ctx* lbm, double alpha, int64_t cycles, int64_t lbm_steps) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!lbm || cycles < 0 || lbm_steps < 0) return LBCH_EINVAL;
  for (int64_t k = 0; k < cycles; ++k) {
    if ((st = lbch_get_phi_device(lbm, c->leap0)) != LBCH_OK) {
      set_err(c, "leap_run: lbch_get_phi_device: %s", lbch_last_error(lbm));
      return st;
    }
    leap_forward(c, alpha);
    if ((st = lbch_init_field_device(lbm, c->leap0)) != LBCH_OK ||
        (st = lbch_step(lbm, lbm_steps)) != LBCH_OK) {
      set_err(c, "leap_run: %s", lbch_last_error(lbm));
      return st;
    }
  }
  return done(c, "leap_run: launch");
}

lbch_status lbnop_leap_run_judged(lbnop_ctx* c, lbch_ctx* lbm, double alpha, int64_t cycles, int64_t lbm_steps,
                                  const lbnop_judge* judge, lbnop_judge_stats* stats) {
  lbch_status st = pre(c);
  if (st != LBCH_OK) return st;
  if (!lbm || !judge || cycles < 0 || lbm_steps < 0) return LBCH_EINVAL;
  const lbnop_judge& J = *judge;
  if (J.leap_steps < 1 || J.audit_every < 0 || !(J.energy_rtol >= 0.0) || !std::isfinite(J.energy_rtol) ||
      !(J.mass_atol >= 0.0) || !std::isfinite(J.mass_atol) || !(J.phi_rtol >= 0.0) || !std::isfinite(J.phi_rtol)) {
    set_err(c, "leap_run_judged: invalid judge (leap_steps >= 1, tolerances finite and >= 0)");
    return LBCH_EINVAL;
  }
  if (!c->side_made) {  // the read-back stream and its events, made once per context
    cudaStream_t side = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e0, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e1, cudaEventDisableTiming) != cudaSuccess) {
      if (e0) cudaEventDestroy(e0);
      if (side) cudaStreamDestroy(side);
      cuda_bad(c, cudaGetLastError(), "leap_run_judged: stream and events");
      return LBCH_ECUDA;
    }
    c->side = side;
    c->ready[0] = e0;
    c->ready[1] = e1;
    c->side_made = true;
  }
  lbnop_judge_stats S{};
  S.max_leap_rise = -INFINITY;
  S.max_corr_rise = -INFINITY;
  const double nodes = (double)c->p.H * c->p.W;
  const int64_t t0 = lbch_steps_taken(lbm);
  // Readings of cycle k in slot k % 2 (8 doubles): mass and energy of phi when the cycle starts,
  // then after its leap, then the audit sums. The reading at the start of cycle k + 1 is also
  // the one after cycle k's correction steps.
  double* dv = c->judge_vals;
  double hv[16];
  auto backup = [&](int s) { return c->judge_state + (size_t)s * c->judge_state_bytes; };
  auto audited = [&](int64_t k) { return J.audit_every > 0 && (k + 1) % J.audit_every == 0; };
  auto lbm_fail = [&](lbch_status s) {
    set_err(c, "leap_run_judged: %s", lbch_last_error(lbm));
    return s;
  };
  // Enqueues cycle k (k == cycles: only the readings after the last cycle); asynchronous.
  auto enqueue = [&](int64_t k) -> lbch_status {
    const int s = (int)(k & 1);
    double* v = dv + 8 * s;
    lbch_status r;
    if ((r = lbch_get_phi_device(lbm, c->leap0)) != LBCH_OK ||
        (r = lbch_field_diagnostics_device(lbm, c->leap0, v)) != LBCH_OK)
      return lbm_fail(r);
    if (cuda_bad(c, cudaEventRecord(c->ready[s], c->stream), "leap_run_judged: event")) return LBCH_ECUDA;
    if (k >= cycles) return LBCH_OK;
    if (audited(k)) {  // the plain K steps from this state beside the network's prediction
      leap_forward(c, alpha);
      if ((r = lbch_step(lbm, J.leap_steps)) != LBCH_OK || (r = lbch_get_phi_device(lbm, c->leap1)) != LBCH_OK)
        return lbm_fail(r);
      diff_norm_kernel<<<HEAD_BLOCKS, 256, 0, c->stream>>>(c->leap0, c->leap1, (long long)c->p.H * c->p.W,
                                                           c->partial);
      diff_norm_final<<<1, 32, 0, c->stream>>>(c->partial, HEAD_BLOCKS, v + 4);
    } else {
      if ((r = lbch_save_state_device(lbm, backup(s), c->judge_state_bytes)) != LBCH_OK) return lbm_fail(r);
      leap_forward(c, alpha);
      if ((r = lbch_field_diagnostics_device(lbm, c->leap0, v + 2)) != LBCH_OK ||
          (r = lbch_init_field_device(lbm, c->leap0)) != LBCH_OK)
        return lbm_fail(r);
    }
    if ((r = lbch_step(lbm, lbm_steps)) != LBCH_OK) return lbm_fail(r);
    return cuda_bad(c, cudaGetLastError(), "leap_run_judged: launch") ? LBCH_ECUDA : LBCH_OK;
  };
  // Both slots, once the reading at the start of cycle k + 1 (slot s) is done; the stream of
  // the run keeps working meanwhile.
  auto fetch = [&](int s) {
    return !cuda_bad(c, cudaStreamWaitEvent(c->side, c->ready[s], 0), "leap_run_judged: wait") &&
           !cuda_bad(c, cudaMemcpyAsync(hv, dv, sizeof(hv), cudaMemcpyDeviceToHost, c->side), "leap_run_judged: read") &&
           !cuda_bad(c, cudaStreamSynchronize(c->side), "leap_run_judged: read");
  };
  if (cycles > 0 && (st = enqueue(0)) != LBCH_OK) return st;
  for (int64_t k = 0; k < cycles; ++k) {
    // Cycle k + 1 goes on the stream before cycle k is judged; if cycle k is rejected it is
    // discarded and enqueued again after the plain steps that replace cycle k.
    if ((st = enqueue(k + 1)) != LBCH_OK) return st;
    if (!fetch((int)((k + 1) & 1))) return LBCH_ECUDA;
    const double* a = hv + 8 * (k & 1);
    const double* b = hv + 8 * ((k + 1) & 1);
    const double m_pre = a[0], e_pre = a[1], m_leap = a[2], e_leap = a[3], e_corr = b[1];
    if (audited(k)) {
      const double err = std::sqrt(a[4] / a[5]);
      ++S.audits;
      S.lbm_steps += J.leap_steps + lbm_steps;
      if (std::isfinite(err) && err <= J.phi_rtol) {
        ++S.accepted;
      } else {
        ++S.rejected;
        ++S.rejected_audit;
      }
      S.max_audit_err = std::isfinite(err) ? std::max(S.max_audit_err, err) : INFINITY;
      continue;
    }
    const bool finite = std::isfinite(m_pre) && std::isfinite(e_pre) && std::isfinite(m_leap) &&
                        std::isfinite(e_leap) && std::isfinite(b[0]) && std::isfinite(e_corr);
    bool ok = finite;
    if (!finite) {
      ++S.rejected_nonfinite;
    } else {
      const double rise_leap = (e_leap - e_pre) / std::fabs(e_pre);
      const double rise_corr = (e_corr - e_leap) / std::fabs(e_leap);
      S.max_leap_rise = std::max(S.max_leap_rise, rise_leap);
      S.max_corr_rise = std::max(S.max_corr_rise, rise_corr);
      if (std::fabs(m_leap - m_pre) > J.mass_atol * nodes) {
        ok = false;
        ++S.rejected_mass;
      } else if (e_leap > e_pre + J.energy_rtol * std::fabs(e_pre) ||
                 e_corr > e_leap + J.energy_rtol * std::fabs(e_leap)) {
        ok = false;
        ++S.rejected_energy;
      }
    }
    if (ok) {
      ++S.accepted;
      S.lbm_steps += lbm_steps;
      continue;
    }
    // Rejected: the plain scheme over the same simulated time from the state saved before the
    // leap, then cycle k + 1 (or the last readings) again on top of it.
    ++S.rejected;
    S.lbm_steps += J.leap_steps + lbm_steps;
    if ((st = lbch_restore_state_device(lbm, backup((int)(k & 1)), c->judge_state_bytes)) != LBCH_OK ||
        (st = lbch_step(lbm, J.leap_steps + lbm_steps)) != LBCH_OK)
      return lbm_fail(st);
    if ((st = enqueue(k + 1)) != LBCH_OK) return st;
  }
  if ((st = lbch_set_steps_taken(lbm, t0 + cycles * (J.leap_steps + lbm_steps))) != LBCH_OK) return lbm_fail(st);
  // every leap's forward pass completed before the last readings were copied back
  if (cycles > 0 && tc_faulted(c, "leap_run_judged")) return LBCH_ECUDA;
  if (stats) *stats = S;
  return done(c, "leap_run_judged: launch");
}

static lbch_status op_check(int32_t B, int32_t H, int32_t W, int32_t ci, int32_t co) {
  if (B < 1 || H < 1 || W < 1 || (long long)B * H * W >= (1LL << 31) / 96) return LBCH_EINVAL;
  if (!channels_ok(ci) || !channels_ok(co)) return LBCH_EINVAL;
  return LBCH_OK;
}

size_t lbnop_conv3x3_packed_bytes(int32_t c_in, int32_t c_out) {
  if (!channels_ok(c_in) || !channels_ok(c_out)) return 0;
  return tc_pack_bytes(c_in, c_out, false);
}

lbch_status lbnop_conv3x3_pack(const uint16_t* d_w, int32_t c_in, int32_t c_out, void* d_packed, void* cuda_stream) {
  if (!d_w || !d_packed || !channels_ok(c_in) || !channels_ok(c_out) || ((uintptr_t)d_w % 16) != 0 ||
      ((uintptr_t)d_packed % 16) != 0)
    return LBCH_EINVAL;
  if (cudaPeekAtLastError() != cudaSuccess) return LBCH_ECUDA;  // an earlier error stays the caller's
  const int kc = tc_kc(c_in, false);
  tc_pack_kernel<<<grid_for(9LL * kc * (c_out + 1), 256), 256, 0, (cudaStream_t)cuda_stream>>>(
      (const bf16*)d_w, c_in, c_out, kc, (unsigned char*)d_packed);
  return cudaGetLastError() == cudaSuccess ? LBCH_OK : LBCH_ECUDA;
}

lbch_status lbnop_conv3x3_packed(const uint16_t* d_x, const uint16_t* d_w, const void* d_packed, const float* d_bias,
                                 int32_t B, int32_t H, int32_t W, int32_t c_in, int32_t c_out, float* d_y,
                                 void* cuda_stream) {
  if (!d_x || !d_w || !d_y || op_check(B, H, W, c_in, c_out) != LBCH_OK) return LBCH_EINVAL;
  if (cudaPeekAtLastError() != cudaSuccess) return LBCH_ECUDA;
  ConvArgs a{};
  a.x = (const bf16*)d_x;
  a.w = (const bf16*)d_w;
  a.wpk = (const unsigned char*)d_packed;
  a.B = B;
  a.H = H;
  a.W = W;
  a.bias = d_bias;
  a.yf = d_y;
  conv_launch(c_in, c_out, false, a, (cudaStream_t)cuda_stream);
  return cudaGetLastError() == cudaSuccess ? LBCH_OK : LBCH_ECUDA;
}

lbch_status lbnop_conv3x3(const uint16_t* d_x, const uint16_t* d_w, const float* d_bias, int32_t B, int32_t H,
                          int32_t W, int32_t c_in, int32_t c_out, float* d_y, void* cuda_stream) {
  // no packed weights: the mma.sync kernels for every shape (the library allocates nothing)
  return lbnop_conv3x3_packed(d_x, d_w, nullptr, d_bias, B, H, W, c_in, c_out, d_y, cuda_stream);
}

lbch_status lbnop_conv3x3_bwd_data(const uint16_t* d_dy, const uint16_t* d_w, int32_t B, int32_t H, int32_t W,
                                   int32_t c_in, int32_t c_out, float* d_dx, void* cuda_stream) {
  if (!d_dy || !d_w || !d_dx || op_check(B, H, W, c_in, c_out) != LBCH_OK) return LBCH_EINVAL;
  if (cudaPeekAtLastError() != cudaSuccess) return LBCH_ECUDA;
  ConvArgs a{};
  a.x = (const bf16*)d_dy;
  a.w = (const bf16*)d_w;
  a.B = B;
  a.H = H;
  a.W = W;
  a.yf = d_dx;
  conv_launch(c_out, c_in, true, a, (cudaStream_t)cuda_stream);
  return cudaGetLastError() == cudaSuccess ? LBCH_OK : LBCH_ECUDA;
}

lbch_status lbnop_conv3x3_bwd_weight(const uint16_t* d_x, const uint16_t* d_dy, int32_t B, int32_t H, int32_t W,
                                     int32_t c_in, int32_t c_out, float* d_dw, void* cuda_stream) {
  if (!d_x || !d_dy || !d_dw || op_check(B, H, W, c_in, c_out) != LBCH_OK) return LBCH_EINVAL;
  if (cudaPeekAtLastError() != cudaSuccess) return LBCH_ECUDA;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(d_dw, 0, (size_t)9 * c_in * c_out * sizeof(float), s) != cudaSuccess) return LBCH_ECUDA;
  WgradArgs a{};
  a.x = (const bf16*)d_x;
  a.dz = (const bf16*)d_dy;
  a.B = B;
  a.H = H;
  a.W = W;
  a.chunk = wgrad_chunk(B * H * W);
  a.dw = d_dw;
  wgrad_launch(c_in, c_out, a, s);
  return cudaGetLastError() == cudaSuccess ? LBCH_OK : LBCH_ECUDA;
}

int64_t lbnop_tc_launches(void) { return tc_counter().load(std::memory_order_relaxed); }

int32_t lbnop_tc_fault(void) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, tc_fault_flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return v ? 1 : 0;
}

const char* lbnop_last_error(const lbnop_ctx* c) { return c ? c->err : "context is NULL"; }

void lbnop_destroy(lbnop_ctx* c) {
  if (c && c->side_made) {
    cudaEventDestroy(c->ready[0]);
    cudaEventDestroy(c->ready[1]);
    cudaStreamDestroy(c->side);
  }
  delete c;
}

}  // extern "C"
