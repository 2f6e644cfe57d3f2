// The periodic 3 x 3 convolution of lbnop.cu on the 5th-generation tensor cores (tcgen05):
// operands staged in shared memory by the Tensor Memory Accelerator (cp.async.bulk.tensor),
// FP32 accumulators in tensor memory (TMEM), one elected thread issuing the MMAs.
//
// Scope: rows of a multiple of 128 pixels (W % 128 == 0), H a multiple of 4, c_in and c_out
// in {16, 64, 96}, one input tensor (no second BF16 half). That covers the finest level of the
// learned leap on 512 x 512 and larger fields, where most of its convolution work is; every
// other layer keeps the mma.sync kernels.
//
// A CTA computes R (1, 2 or 4) consecutive rows (same sample) x 128 pixels x all c_out channels:
//   - the R + 2 input rows it needs (rows h - 1 .. h + R, periodic in h) land by one TMA
//     load each, as [c_in / 8 chunks][136 pixel slots][8 channels]: pixel x0 - 4 + s in slot s,
//     out-of-range slots zero-filled, then the two slots that periodic wrap needs (x0 - 1 at
//     the row's start, x0 + 128 at its end) copied from global memory by the threads. This is
//     the K-major, no-swizzle canonical layout of the MMA's A operand: 16-byte rows (one pixel's
//     8 channels) 16 bytes apart within a chunk, chunks 136 x 16 bytes apart. The operand of tap
//     (dy, dx) for output row r is input row r + 1 + dy read from slot 4 + dx on: a shift of
//     the descriptor's start address, no copy.
//   - the weights of one tap, W[t] = [c_out][c_in] (K-major B operand), land by one TMA load per
//     tap into a three-stage ring, refilled as soon as the MMAs of the tap they held complete.
//   - accumulators: R x c_out FP32 columns of TMEM (lane = pixel), D += A_t B_t^T over the
//     9 taps and c_in / 16 K-steps of 16.
//   - epilogue: each thread owns one pixel (TMEM lane), reads its c_out accumulators per row
//     with tcgen05.ld and applies bias, conditioning, alpha scaling and the stores of
//     conv_epilogue.
// Every wait on an mbarrier is bounded; on timeout the kernel sets *err and stops issuing.
#pragma once

#include <cuda.h>

namespace nop {

constexpr int TC_SLOTS = 136;      // pixel slots per chunk block (4 + 128 + 4)
constexpr int TC_OFF = 4;          // slot of the tile's first pixel
constexpr int TC_THREADS = 128;    // four warps: one TMEM lane quarter each
constexpr int TC_BSTAGES = 3;
constexpr unsigned TC_SPIN_LIMIT = 1u << 20;  // bounded mbarrier waits (about a second at most)

// Set by a CTA whose wait gave up; every later CTA of the path then returns at once.
__device__ int tc_fault_flag;

template <int CI>
__host__ __device__ constexpr int tc_row_bytes() { return (CI / 8) * TC_SLOTS * 16; }
template <int CI, int CO, int R>
__host__ __device__ constexpr int tc_smem_bytes() {
  return (R + 2) * tc_row_bytes<CI>() + TC_BSTAGES * CO * CI * 2 + 128 /* barriers, TMEM address */ +
         128 /* alignment */;
}
// TMEM columns: a power of two >= 32 that holds R accumulators of CO columns.
template <int CO, int R>
__host__ __device__ constexpr int tc_tmem_cols() {
  return R * CO <= 32 ? 32 : (R * CO <= 64 ? 64 : (R * CO <= 128 ? 128 : (R * CO <= 256 ? 256 : 512)));
}

struct TcArgs {
  CUtensorMap xmap;  // input activations, 4D {8, W, CI / 8, B H}
  CUtensorMap wmap;  // weights, 4D {8, CO, CI / 8, 9}
  int* err;          // also set to 1 if a wait gave up (may be null)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Waits for the phase with the given parity to complete; false if it did not within the limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (unsigned i = 0; i < TC_SPIN_LIMIT; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand without swizzling: 8-row x 16-byte
// core matrices, rows 16 bytes apart; lbo = bytes between K-adjacent core matrices, sbo =
// bytes between core matrices adjacent in M (or N); bits 46-47 hold the descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits
// 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits
// 24-28.
template <int M, int N>
__host__ __device__ constexpr uint32_t umma_idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (shape 32x32b, 32 repetitions).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// 16 columns (shape 32x32b, 16 repetitions).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[32]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Bias, conditioning, alpha scaling and the stores of conv_epilogue for `cnt` consecutive
// channels n0 .. n0 + cnt - 1 of one pixel.
template <int CO, int CNT>
__device__ __forceinline__ void tc_epilogue(const ConvArgs& p, size_t pix, int b, int n0, float (&v)[32]) {
  const float al = p.film ? p.alpha[b] : 0.0f;
  const float sc = p.scale_alpha ? p.alpha[b] : 1.0f;
#pragma unroll
  for (int j = 0; j < CNT; ++j) {
    float x = v[j];
    if (p.bias) x += p.bias[n0 + j];
    if (p.film) x = fmaf(al, p.film[n0 + j], x);
    if (p.scale_alpha) x *= sc;
    v[j] = x;
  }
  const size_t o = pix * CO + n0;
  if (p.yf) {
#pragma unroll
    for (int j = 0; j < CNT; j += 4) {
      float4* y = reinterpret_cast<float4*>(p.yf + o + j);
      float4 w = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      if (p.accumulate) {
        const float4 old = *y;
        w = make_float4(old.x + w.x, old.y + w.y, old.z + w.z, old.w + w.w);
      }
      *y = w;
    }
  }
  if (p.z) {
#pragma unroll
    for (int j = 0; j < CNT; j += 8) {
      uint4 u;
      u.x = pack2(__float2bfloat16_rn(v[j]), __float2bfloat16_rn(v[j + 1]));
      u.y = pack2(__float2bfloat16_rn(v[j + 2]), __float2bfloat16_rn(v[j + 3]));
      u.z = pack2(__float2bfloat16_rn(v[j + 4]), __float2bfloat16_rn(v[j + 5]));
      u.w = pack2(__float2bfloat16_rn(v[j + 6]), __float2bfloat16_rn(v[j + 7]));
      *reinterpret_cast<uint4*>(p.z + o + j) = u;
    }
  }
  if (p.a) {
#pragma unroll
    for (int j = 0; j < CNT; j += 8) {
      uint4 u;
      u.x = pack2(__float2bfloat16_rn(silu_f(v[j])), __float2bfloat16_rn(silu_f(v[j + 1])));
      u.y = pack2(__float2bfloat16_rn(silu_f(v[j + 2])), __float2bfloat16_rn(silu_f(v[j + 3])));
      u.z = pack2(__float2bfloat16_rn(silu_f(v[j + 4])), __float2bfloat16_rn(silu_f(v[j + 5])));
      u.w = pack2(__float2bfloat16_rn(silu_f(v[j + 6])), __float2bfloat16_rn(silu_f(v[j + 7])));
      *reinterpret_cast<uint4*>(p.a + o + j) = u;
    }
  }
}

// Grid: (W / 128) x (B H / R) CTAs of TC_THREADS; R output rows per CTA.
template <int CI, int CO, int R>
__global__ void __launch_bounds__(TC_THREADS, 1) conv_tc_kernel(const __grid_constant__ TcArgs ta,
                                                                 const __grid_constant__ ConvArgs p) {
  static_assert(CI % 16 == 0 && CO % 16 == 0 && CO <= 256, "UMMA shape: K steps of 16, N a multiple of 16");
  static_assert(R * CO <= 512, "accumulators fit in TMEM");
  constexpr int TC_R = R, TC_IN = R + 2;
  constexpr int KC = CI / 8;                          // 8-channel chunks of the input
  constexpr int ROW = tc_row_bytes<CI>();             // bytes per staged input row
  constexpr uint32_t LBO_A = TC_SLOTS * 16, LBO_B = CO * 16, SBO = 128;
  constexpr int BBYTES = CO * CI * 2;
  constexpr int COLS = tc_tmem_cols<CO, R>();
  constexpr uint32_t IDESC = umma_idesc_bf16<128, CO>();
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  // 128-byte aligned base for the TMA destinations
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 127) & ~(uintptr_t)127);
  unsigned char* sA = base;
  unsigned char* sB = base + TC_IN * ROW;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + TC_BSTAGES * BBYTES);  // a_full, b_full[3], b_empty[3], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);
  const uint32_t a_full = smem_u32(&bars[0]), done_bar = smem_u32(&bars[7]);
  auto b_full = [&](int s) { return smem_u32(&bars[1 + s]); };
  auto b_empty = [&](int s) { return smem_u32(&bars[4 + s]); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (*(volatile int*)&tc_fault_flag) return;  // an earlier CTA's wait gave up: do nothing
  const int x0 = blockIdx.x * 128;
  const int row0 = blockIdx.y * TC_R;  // first output row in the flattened (b, h) order
  const int b = row0 / p.H, h0 = row0 - b * p.H;

  if (tid == 0) {
    for (int i = 0; i < 8; ++i) mbar_init(smem_u32(&bars[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // Input rows h0 - 1 .. h0 + TC_R of sample b (periodic in h), and the first taps' weights.
  if (tid == 0) {
    mbar_expect_tx(a_full, TC_IN * ROW);
    for (int i = 0; i < TC_IN; ++i) {
      const int h = wrap1(h0 - 1 + i, p.H);
      tma_load_4d(smem_u32(sA + i * ROW), &ta.xmap, 0, x0 - TC_OFF, 0, b * p.H + h, a_full);
    }
    for (int s = 0; s < TC_BSTAGES; ++s) {
      mbar_expect_tx(b_full(s), BBYTES);
      tma_load_4d(smem_u32(sB + s * BBYTES), &ta.wmap, 0, 0, 0, s, b_full(s));
    }
  }
  bool ok = mbar_wait(a_full, 0);
  // Periodic wrap: slot TC_OFF - 1 holds pixel W - 1 at a row's start, slot TC_OFF + 128 pixel 0
  // at its end (inside a row the TMA load brought the true neighbours).
  if (ok) {
    const bool first = x0 == 0, last = x0 + 128 == p.W;
    for (int v = tid; v < TC_IN * KC * 2; v += TC_THREADS) {
      const int side = v & 1, c = (v >> 1) % KC, i = (v >> 1) / KC;
      if (side == 0 ? !first : !last) continue;
      const int h = wrap1(h0 - 1 + i, p.H);
      const int src_x = side == 0 ? p.W - 1 : 0;
      const uint4 val = *reinterpret_cast<const uint4*>(p.x + ((size_t)(b * p.H + h) * p.W + src_x) * CI + 8 * c);
      const int slot = side == 0 ? TC_OFF - 1 : TC_OFF + 128;
      *reinterpret_cast<uint4*>(sA + i * ROW + c * (TC_SLOTS * 16) + slot * 16) = val;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> MMA reads
  }
  __syncthreads();

  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    for (int t = 0; t < 9 && ok; ++t) {
      const int s = t % TC_BSTAGES;
      if (!mbar_wait(b_full(s), (t / TC_BSTAGES) & 1)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int dy = t / 3 - 1, dx = t % 3 - 1;
      const uint32_t bbase = smem_u32(sB + s * BBYTES);
#pragma unroll
      for (int r = 0; r < TC_R; ++r) {
        const uint32_t abase = smem_u32(sA + (r + 1 + dy) * ROW) + (uint32_t)((TC_OFF + dx) * 16);
#pragma unroll
        for (int kk = 0; kk < CI / 16; ++kk) {
          const uint64_t ad = umma_desc(abase + kk * 2 * LBO_A, LBO_A, SBO);
          const uint64_t bd = umma_desc(bbase + kk * 2 * LBO_B, LBO_B, SBO);
          umma_bf16(tmem + (uint32_t)(r * CO), ad, bd, IDESC, (t > 0 || kk > 0) ? 1u : 0u);
        }
      }
      umma_commit(b_empty(s));  // this stage is free once these MMAs have read it
      // Refill the stage of the previous tap (its MMAs ran while this tap's were queued), so
      // that the tensor cores always have a tap's MMAs waiting.
      const int tp = t - 1, np = tp + TC_BSTAGES;
      if (tp >= 0 && np < 9) {
        const int sp = tp % TC_BSTAGES;
        if (!mbar_wait(b_empty(sp), (tp / TC_BSTAGES) & 1)) {
          ok = false;
          break;
        }
        mbar_expect_tx(b_full(sp), BBYTES);
        tma_load_4d(smem_u32(sB + sp * BBYTES), &ta.wmap, 0, 0, 0, np, b_full(sp));
      }
    }
    umma_commit(done_bar);  // arrives once every MMA issued above has completed
  }
  const bool issued = __syncthreads_and(ok ? 1 : 0) != 0;
  // Wait for the accumulators (on the failure path, for whatever was issued).
  const bool fin = mbar_wait(done_bar, 0);
  const bool good = __syncthreads_and((issued && fin) ? 1 : 0) != 0;  // uniform over the CTA
  if (!good && tid == 0) {
    atomicExch(&tc_fault_flag, 1);
    if (ta.err) atomicExch(ta.err, 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  if (good) {
    const int x = x0 + 32 * warp + lane;
#pragma unroll 1
    for (int r = 0; r < TC_R; ++r) {
      const size_t pix = (size_t)(row0 + r) * p.W + x;
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(r * CO);
#pragma unroll
      for (int c = 0; c < CO / 32; ++c) {
        float v[32];
        tmem_ld32(lane_addr + 32 * c, v);
        tc_epilogue<CO, 32>(p, pix, b, 32 * c, v);
      }
      if constexpr (CO % 32 == 16) {
        float v[32];
        tmem_ld16(lane_addr + 32 * (CO / 32), v);
        tc_epilogue<CO, 16>(p, pix, b, 32 * (CO / 32), v);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
}

// ---------------------------------------------------------------- host side

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline EncodeTiledFn encode_tiled() {
  static std::atomic<EncodeTiledFn> fn{nullptr};
  EncodeTiledFn f = fn.load(std::memory_order_acquire);
  if (!f) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f = reinterpret_cast<EncodeTiledFn>(p);
    fn.store(f, std::memory_order_release);
  }
  return f;
}

// 4D map {8, d1, d2, d3} of BF16 with strides s1, s2, s3 (bytes) and box {8, b1, b2, 1}.
inline bool make_map_4d(CUtensorMap* m, const void* base, uint64_t d1, uint64_t d2, uint64_t d3, uint64_t s1,
                        uint64_t s2, uint64_t s3, uint32_t b1, uint32_t b2) {
  EncodeTiledFn f = encode_tiled();
  if (!f) return false;
  const cuuint64_t dims[4] = {8, d1, d2, d3};
  const cuuint64_t strides[3] = {s1, s2, s3};
  const cuuint32_t box[4] = {8, b1, b2, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return f(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Whether the tensor-core path takes this convolution.
inline bool tc_applies(const ConvArgs& a, int ci, int co) {
  return a.x2 == nullptr && a.w2 == nullptr && a.W % 128 == 0 && a.H % 4 == 0 && a.W <= 8192 &&
         (ci == 16 || ci == 64 || ci == 96) && (co == 16 || co == 64 || co == 96) &&
         ((uintptr_t)a.x % 16) == 0 && ((uintptr_t)a.w % 16) == 0;
}

inline std::atomic<long long>& tc_counter() {
  static std::atomic<long long> n{0};
  return n;
}

template <int CI, int CO, int R>
void launch_tc_rows(const TcArgs& ta, const ConvArgs& a, cudaStream_t s) {
  constexpr int bytes = tc_smem_bytes<CI, CO, R>();
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_relaxed) & bit)) {
    cudaFuncSetAttribute(conv_tc_kernel<CI, CO, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done.fetch_or(bit, std::memory_order_relaxed);
  }
  conv_tc_kernel<CI, CO, R><<<dim3(a.W / 128, a.B * a.H / R), TC_THREADS, bytes, s>>>(ta, a);
}

// Launches conv_tc_kernel for this convolution; false if the tensor maps could not be made
// (the caller then runs the mma.sync path). Rows per CTA: 4 when that still gives two waves
// of CTAs over the SMs (operands reused by four rows), else fewer (more CTAs).
template <int CI, int CO>
bool launch_tc(const ConvArgs& a, int* err, int sms, cudaStream_t s) {
  TcArgs ta;
  ta.err = err;
  const uint64_t W = a.W, rows = (uint64_t)a.B * a.H;
  if (!make_map_4d(&ta.xmap, a.x, W, CI / 8, rows, CI * 2, 16, W * CI * 2, TC_SLOTS, CI / 8)) return false;
  if (!make_map_4d(&ta.wmap, a.w, CO, CI / 8, 9, CI * 2, 16, (uint64_t)CO * CI * 2, CO, CI / 8)) return false;
  const long long ctas4 = (long long)(a.W / 128) * (long long)rows / 4;
  if (ctas4 >= 2LL * sms)
    launch_tc_rows<CI, CO, 4>(ta, a, s);
  else if (ctas4 * 2 >= sms)
    launch_tc_rows<CI, CO, 2>(ta, a, s);
  else
    launch_tc_rows<CI, CO, 1>(ta, a, s);
  tc_counter().fetch_add(1, std::memory_order_relaxed);
  return true;
}

}  // namespace nop
