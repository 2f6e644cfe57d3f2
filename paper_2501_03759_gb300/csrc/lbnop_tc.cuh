// The periodic 3 x 3 convolution of lbnop.cu on the 5th-generation tensor cores (tcgen05):
// operands in shared memory in the MMA's canonical K-major layout, FP32 accumulators in
// tensor memory (TMEM), one thread issuing the MMAs, producer warps refilling a ring of
// weight taps under mbarriers.
//
// Scope: rows of a multiple of 128 pixels (W % 128 == 0), H a multiple of 4, c_in and c_out
// in {16, 64, 96}, one input tensor (no second BF16 half). That covers the finest level of the
// learned leap on 512 x 512 and larger fields, where most of its convolution work is; every
// other layer keeps the mma.sync kernels.
//
// A CTA computes R (1, 2 or 4) consecutive rows (same sample) x 128 pixels x all c_out channels:
//   - the R + 2 input rows it needs (rows h - 1 .. h + R, periodic in h) are copied once, 16
//     bytes (8 channels of one pixel) per cp.async, consecutive threads reading consecutive
//     bytes, into [c_in / 8 chunks][130 pixel slots][8 channels]: pixel x0 - 1 + s (periodic in
//     x) in slot s. That is the K-major, no-swizzle canonical layout of the MMA's A operand:
//     16-byte rows (one pixel's 8 channels) 16 bytes apart within a chunk block, chunk blocks
//     131 x 16 bytes apart (one spare row shifts consecutive chunks to different bank groups).
//     The operand of tap (dy, dx) for output row r is input row r + 1 + dy from slot 1 + dx on:
//     a shift of the descriptor's start address, no copy.
//   - the weights of one tap, W[t] = [c_out][c_in] (the K-major B operand), land in a
//     three-stage ring: three producer warps copy a tap as soon as the MMAs that read the
//     previous contents of its stage have completed, and arrive on the stage's mbarrier.
//   - accumulators: R x c_out FP32 columns of TMEM (lane = pixel), D += A_t B_t^T over the
//     9 taps and c_in / 16 K-steps of 16.
//   - epilogue: each thread owns one pixel (TMEM lane); it reads its c_out accumulators of a
//     row with tcgen05.ld, adds bias and conditioning, scales, and stages the row in shared
//     memory, from where all threads write it out coalesced (conv_epilogue's outputs).
// Staging through TMA was measured first: tensor-map boxes whose innermost extent is one
// 8-channel chunk (16 bytes) move each pixel's chunk as a separate request, and operand
// staging then took most of a CTA's time (a c_out = 16 layer ran 80 us against 115 us for
// c_out = 96 at batch 16). Coalesced 16-byte copies land the same layout at full rate.
// Every wait on an mbarrier is bounded; on timeout the kernel sets an error flag and stops.
#pragma once

namespace nop {

constexpr int TC_SLOTS = 130;                  // pixel slots per chunk block: x0 - 1 .. x0 + 128
constexpr int TC_CHUNK_A = (TC_SLOTS + 1) * 16;  // bytes between chunk blocks of an input row
constexpr int TC_THREADS = 128;                // four warps: one TMEM lane quarter each
constexpr int TC_LOADERS = 96;                 // warps 1-3 copy weight taps
constexpr int TC_MAX_BSTAGES = 4;
constexpr unsigned TC_SPIN_LIMIT = 1u << 20;   // bounded mbarrier waits (about a second at most)

// Set by a CTA whose wait gave up; every later CTA of the path then returns at once.
__device__ int tc_fault_flag;

template <int CI>
__host__ __device__ constexpr int tc_row_bytes() { return (CI / 8) * TC_CHUNK_A; }
template <int CO>
__host__ __device__ constexpr int tc_chunk_b() { return CO * 16 + 16; }  // bytes between chunk blocks of a tap
template <int CI, int CO>
__host__ __device__ constexpr int tc_tap_bytes() { return (CI / 8) * tc_chunk_b<CO>(); }
template <int CO>
__host__ __device__ constexpr int tc_stage_pitch() { return CO + 4; }
// Weight-ring stages: four where they fit beside the input rows in one CTA's shared memory
// (more taps in flight hide the copy latency behind the MMAs), else three.
template <int CI, int CO, int R>
__host__ __device__ constexpr int tc_bstages() {
  return (R + 2) * tc_row_bytes<CI>() + 4 * tc_tap_bytes<CI, CO>() + 512 <= 227 * 1024 ? 4 : 3;
}
template <int CI, int CO, int R>
__host__ __device__ constexpr int tc_operand_bytes() {
  return (R + 2) * tc_row_bytes<CI>() + tc_bstages<CI, CO, R>() * tc_tap_bytes<CI, CO>();
}
template <int CO>
__host__ __device__ constexpr int tc_staged_bytes() { return 128 * tc_stage_pitch<CO>() * 4 + 2 * CO * 4; }
// The operand buffers, reused for the staged output rows, then 9 mbarriers and the TMEM address.
template <int CI, int CO, int R>
__host__ __device__ constexpr int tc_main_bytes() {
  return tc_operand_bytes<CI, CO, R>() > tc_staged_bytes<CO>() ? tc_operand_bytes<CI, CO, R>() : tc_staged_bytes<CO>();
}
template <int CI, int CO, int R>
__host__ __device__ constexpr int tc_smem_bytes() { return tc_main_bytes<CI, CO, R>() + 128 + 128 /* alignment */; }
// TMEM columns: a power of two >= 32 that holds R accumulators of CO columns.
template <int CO, int R>
__host__ __device__ constexpr int tc_tmem_cols() {
  return R * CO <= 32 ? 32 : (R * CO <= 64 ? 64 : (R * CO <= 128 ? 128 : (R * CO <= 256 ? 256 : 512)));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
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
__device__ __forceinline__ void tc_cp16(uint32_t smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem), "l"(gmem) : "memory");
}
// This thread's copies have landed and are visible to the tensor cores (async proxy).
__device__ __forceinline__ void tc_cp_done() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

// The CO accumulator columns of this thread's TMEM lane: loads of 32 (and one of 16) columns,
// then one wait for all of them.
template <int CO>
__device__ __forceinline__ void tmem_ld_row(uint32_t taddr, float (&v)[CO]) {
  uint32_t r[CO];
#pragma unroll
  for (int c = 0; c < CO / 32; ++c)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[32 * c + 0]), "=r"(r[32 * c + 1]), "=r"(r[32 * c + 2]), "=r"(r[32 * c + 3]), "=r"(r[32 * c + 4]),
          "=r"(r[32 * c + 5]), "=r"(r[32 * c + 6]), "=r"(r[32 * c + 7]), "=r"(r[32 * c + 8]), "=r"(r[32 * c + 9]),
          "=r"(r[32 * c + 10]), "=r"(r[32 * c + 11]), "=r"(r[32 * c + 12]), "=r"(r[32 * c + 13]),
          "=r"(r[32 * c + 14]), "=r"(r[32 * c + 15]), "=r"(r[32 * c + 16]), "=r"(r[32 * c + 17]),
          "=r"(r[32 * c + 18]), "=r"(r[32 * c + 19]), "=r"(r[32 * c + 20]), "=r"(r[32 * c + 21]),
          "=r"(r[32 * c + 22]), "=r"(r[32 * c + 23]), "=r"(r[32 * c + 24]), "=r"(r[32 * c + 25]),
          "=r"(r[32 * c + 26]), "=r"(r[32 * c + 27]), "=r"(r[32 * c + 28]), "=r"(r[32 * c + 29]),
          "=r"(r[32 * c + 30]), "=r"(r[32 * c + 31])
        : "r"(taddr + 32 * c));
  if constexpr (CO % 32 == 16) {
    constexpr int o = CO - 16;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[o + 0]), "=r"(r[o + 1]), "=r"(r[o + 2]), "=r"(r[o + 3]), "=r"(r[o + 4]), "=r"(r[o + 5]),
          "=r"(r[o + 6]), "=r"(r[o + 7]), "=r"(r[o + 8]), "=r"(r[o + 9]), "=r"(r[o + 10]), "=r"(r[o + 11]),
          "=r"(r[o + 12]), "=r"(r[o + 13]), "=r"(r[o + 14]), "=r"(r[o + 15])
        : "r"(taddr + (uint32_t)o));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < CO; ++i) v[i] = __uint_as_float(r[i]);
}

// The epilogue stages one output row (128 pixels x CO channels, FP32) in shared memory with
// rows TC_STAGE(CO) floats apart: 16-byte aligned, and 8 consecutive pixels (one phase of a
// 16-byte store) fall in distinct bank groups. It is then written out in 16-byte pieces that
// consecutive threads take from consecutive addresses (coalesced).
// Stores of one staged output row: the FP32 result (added to what is there with accumulate),
// its BF16 rounding and its SiLU in BF16, as conv_epilogue does.
template <int CO>
__device__ __forceinline__ void tc_store_row(const ConvArgs& p, const float* stage, size_t pix0, int tid) {
  constexpr int Q = CO / 4, PITCH = tc_stage_pitch<CO>();
  for (int idx = tid; idx < 128 * Q; idx += TC_THREADS) {
    const int px = idx / Q, c4 = idx - px * Q;
    float4 v = *reinterpret_cast<const float4*>(stage + px * PITCH + 4 * c4);
    const size_t o = (pix0 + px) * CO + 4 * c4;
    if (p.yf) {
      float4* y = reinterpret_cast<float4*>(p.yf + o);
      if (p.accumulate) {
        const float4 old = *y;
        *y = make_float4(old.x + v.x, old.y + v.y, old.z + v.z, old.w + v.w);
      } else {
        *y = v;
      }
    }
    if (p.z)
      *reinterpret_cast<uint2*>(p.z + o) = make_uint2(pack2(__float2bfloat16_rn(v.x), __float2bfloat16_rn(v.y)),
                                                      pack2(__float2bfloat16_rn(v.z), __float2bfloat16_rn(v.w)));
    if (p.a)
      *reinterpret_cast<uint2*>(p.a + o) =
          make_uint2(pack2(__float2bfloat16_rn(silu_f(v.x)), __float2bfloat16_rn(silu_f(v.y))),
                     pack2(__float2bfloat16_rn(silu_f(v.z)), __float2bfloat16_rn(silu_f(v.w))));
  }
}

// Grid: (W / 128) x (B H / R) CTAs of TC_THREADS; R output rows per CTA.
template <int CI, int CO, int R>
__global__ void __launch_bounds__(TC_THREADS, 1) conv_tc_kernel(const __grid_constant__ ConvArgs p, int* err) {
  static_assert(CI % 16 == 0 && CO % 16 == 0 && CO <= 256, "UMMA shape: K steps of 16, N a multiple of 16");
  static_assert(R * CO <= 512, "accumulators fit in TMEM");
  constexpr int KC = CI / 8;                    // 8-channel chunks of the input
  constexpr int ROW = tc_row_bytes<CI>();       // bytes per staged input row
  constexpr int TAP = tc_tap_bytes<CI, CO>();   // bytes per staged weight tap
  constexpr uint32_t LBO_A = TC_CHUNK_A, LBO_B = tc_chunk_b<CO>(), SBO = 128;
  constexpr int COLS = tc_tmem_cols<CO, R>();
  constexpr uint32_t IDESC = umma_idesc_bf16<128, CO>();
  constexpr int TC_BSTAGES = tc_bstages<CI, CO, R>();
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 127) & ~(uintptr_t)127);
  unsigned char* sA = base;
  unsigned char* sB = base + (R + 2) * ROW;
  // b_full[stages], b_empty[stages], done (9 at most), then the TMEM address
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + tc_main_bytes<CI, CO, R>());
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_MAX_BSTAGES + 1);
  const uint32_t done_bar = smem_u32(&bars[2 * TC_BSTAGES]);
  auto b_full = [&](int s) { return smem_u32(&bars[s]); };
  auto b_empty = [&](int s) { return smem_u32(&bars[TC_BSTAGES + s]); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (*(volatile int*)&tc_fault_flag) return;  // an earlier CTA's wait gave up: do nothing
  const int x0 = blockIdx.x * 128;
  const int row0 = blockIdx.y * R;  // first output row in the flattened (b, h) order
  const int b = row0 / p.H, h0 = row0 - b * p.H;

  if (tid == 0) {
    for (int s = 0; s < TC_BSTAGES; ++s) {
      mbar_init(b_full(s), TC_LOADERS);
      mbar_init(b_empty(s), 1);
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // Warps 1-3 issue the first weight taps (one per stage) before the input rows, so that
  // both sets of copies are in flight together; they arrive on the taps' barriers below.
  auto copy_tap = [&](int t) {
    const int s = t % TC_BSTAGES;
    for (int idx = tid - 32; idx < CO * KC; idx += TC_LOADERS) {
      const int n = idx / KC, c = idx - n * KC;
      tc_cp16(smem_u32(sB + s * TAP + c * LBO_B + n * 16), p.w + ((size_t)t * CO + n) * CI + 8 * c);
    }
  };
  if (warp != 0)
    for (int t = 0; t < TC_BSTAGES; ++t) copy_tap(t);
  // The R + 2 input rows, by every thread: periodic in h and in x.
  for (int idx = tid; idx < (R + 2) * TC_SLOTS * KC; idx += TC_THREADS) {
    const int i = idx / (TC_SLOTS * KC), rem = idx - i * (TC_SLOTS * KC);
    const int s = rem / KC, c = rem - s * KC;
    const int h = wrap1(h0 - 1 + i, p.H), x = wrap1(x0 - 1 + s, p.W);
    tc_cp16(smem_u32(sA + i * ROW + c * TC_CHUNK_A + s * 16), p.x + ((size_t)(b * p.H + h) * p.W + x) * CI + 8 * c);
  }
  tc_cp_done();  // this thread's input rows (and first taps) have landed
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();  // after it: the barriers are initialised and every input row is in place
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (warp != 0)
    for (int t = 0; t < TC_BSTAGES; ++t) mbar_arrive(b_full(t));

  bool ok = true;
  if (warp == 0) {
    if (lane == 0) {  // the MMA issuer
      for (int t = 0; t < 9 && ok; ++t) {
        const int s = t % TC_BSTAGES;
        if (!mbar_wait(b_full(s), (t / TC_BSTAGES) & 1)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int dy = t / 3 - 1, dx = t % 3 - 1;
        const uint32_t bbase = smem_u32(sB + s * TAP);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const uint32_t abase = smem_u32(sA + (r + 1 + dy) * ROW) + (uint32_t)((1 + dx) * 16);
#pragma unroll
          for (int kk = 0; kk < CI / 16; ++kk) {
            const uint64_t ad = umma_desc(abase + kk * 2 * LBO_A, LBO_A, SBO);
            const uint64_t bd = umma_desc(bbase + kk * 2 * LBO_B, LBO_B, SBO);
            umma_bf16(tmem + (uint32_t)(r * CO), ad, bd, IDESC, (t > 0 || kk > 0) ? 1u : 0u);
          }
        }
        umma_commit(b_empty(s));  // the stage is free once these MMAs have read it
      }
      umma_commit(done_bar);  // arrives once every MMA issued above has completed
    }
  } else {  // warps 1-3: the remaining weight taps, each into the stage its tap - stages left
    for (int t = TC_BSTAGES; t < 9; ++t) {
      const int s = t % TC_BSTAGES;
      if (!mbar_wait(b_empty(s), ((t - TC_BSTAGES) / TC_BSTAGES) & 1)) {
        ok = false;
        break;
      }
      copy_tap(t);
      tc_cp_done();
      mbar_arrive(b_full(s));
    }
  }
  __syncwarp();
  const bool issued = __syncthreads_and(ok ? 1 : 0) != 0;
  // Wait for the accumulators (on the failure path, for whatever was issued).
  const bool fin = mbar_wait(done_bar, 0);
  const bool good = __syncthreads_and((issued && fin) ? 1 : 0) != 0;  // uniform over the CTA
  if (!good && tid == 0) {
    atomicExch(&tc_fault_flag, 1);
    if (err) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (good) {
    // The MMAs have completed: the operand buffers are free and hold the staged rows now.
    constexpr int PITCH = tc_stage_pitch<CO>();
    float* stage = reinterpret_cast<float*>(base);
    float* sbias = stage + 128 * PITCH;  // bias (0 if none), then the conditioning times alpha
    float* sfilm = sbias + CO;
    const float al = p.film ? p.alpha[b] : 0.0f;
    const float sc = p.scale_alpha ? p.alpha[b] : 1.0f;
    for (int n = tid; n < CO; n += TC_THREADS) {
      sbias[n] = p.bias ? p.bias[n] : 0.0f;
      sfilm[n] = p.film ? al * p.film[n] : 0.0f;
    }
    __syncthreads();
    const int px = 32 * warp + lane;  // this thread's TMEM lane: pixel x0 + px
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(r * CO);
      float v[CO];
      tmem_ld_row<CO>(lane_addr, v);
#pragma unroll
      for (int j = 0; j < CO; j += 4) {
        float4 o;
        o.x = (v[j] + sbias[j] + sfilm[j]) * sc;
        o.y = (v[j + 1] + sbias[j + 1] + sfilm[j + 1]) * sc;
        o.z = (v[j + 2] + sbias[j + 2] + sfilm[j + 2]) * sc;
        o.w = (v[j + 3] + sbias[j + 3] + sfilm[j + 3]) * sc;
        *reinterpret_cast<float4*>(stage + px * PITCH + j) = o;
      }
      __syncthreads();
      tc_store_row<CO>(p, stage, (size_t)(row0 + r) * p.W + x0, tid);
      __syncthreads();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
}

// ---------------------------------------------------------------- host side

// Whether the tensor-core path takes this convolution.
inline bool tc_applies(const ConvArgs& a, int ci, int co) {
  return a.x2 == nullptr && a.w2 == nullptr && a.W % 128 == 0 && a.H % 4 == 0 && (ci == 16 || ci == 64 || ci == 96) &&
         (co == 16 || co == 64 || co == 96) && ((uintptr_t)a.x % 16) == 0 && ((uintptr_t)a.w % 16) == 0;
}

inline std::atomic<long long>& tc_counter() {
  static std::atomic<long long> n{0};
  return n;
}

template <int CI, int CO, int R>
void launch_tc_rows(const ConvArgs& a, int* err, cudaStream_t s) {
  constexpr int bytes = tc_smem_bytes<CI, CO, R>();
  static_assert(bytes <= 227 * 1024, "fits in one CTA's shared memory");
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_relaxed) & bit)) {
    cudaFuncSetAttribute(conv_tc_kernel<CI, CO, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done.fetch_or(bit, std::memory_order_relaxed);
  }
  conv_tc_kernel<CI, CO, R><<<dim3(a.W / 128, a.B * a.H / R), TC_THREADS, bytes, s>>>(a, err);
}

// Launches conv_tc_kernel for this convolution. Rows per CTA: 4 when that still gives two
// waves of CTAs over the SMs (operands reused by four rows), else fewer (more CTAs).
template <int CI, int CO>
bool launch_tc(const ConvArgs& a, int* err, int sms, cudaStream_t s) {
  const long long ctas4 = (long long)(a.W / 128) * ((long long)a.B * a.H) / 4;
  if (ctas4 >= 2LL * sms)
    launch_tc_rows<CI, CO, 4>(a, err, s);
  else if (ctas4 * 2 >= sms)
    launch_tc_rows<CI, CO, 2>(a, err, s);
  else
    launch_tc_rows<CI, CO, 1>(a, err, s);
  tc_counter().fetch_add(1, std::memory_order_relaxed);
  return true;
}

}  // namespace nop
