// The periodic 3 x 3 convolution of lbnop.cu on the 5th-generation tensor cores (tcgen05):
// operands in shared memory in the MMA's canonical K-major layout, FP32 accumulators in
// tensor memory (TMEM), one thread issuing the MMAs, one thread refilling a ring of weight
// taps by bulk asynchronous copies under mbarriers.
//
// Scope: rows of a multiple of 128 pixels (W % 128 == 0), H a multiple of 4, c_in and c_out
// in {16, 64, 96}; with X2, c_in = 16 and a second input tensor x2 (the BF16 remainder of
// the first), multiplied by the same weights: the contraction then runs over K = 32, the
// chunks of x followed by those of x2. That covers the finest level of the learned leap on
// 512 x 512 and larger fields, where most of its convolution work is; every other layer keeps
// the mma.sync kernels.
//
// A CTA (8 warps) computes R (1, 2 or 4) consecutive rows (same sample) x 128 pixels x all
// c_out channels:
//   - the R + 2 input rows it needs (rows h - 1 .. h + R, periodic in h) are copied once, 16
//     bytes (8 channels of one pixel) per cp.async, consecutive threads reading consecutive
//     bytes, into [K / 8 chunks][130 pixel slots][8 channels]: pixel x0 - 1 + s (periodic in
//     x) in slot s. That is the K-major, no-swizzle canonical layout of the MMA's A operand:
//     16-byte rows (one pixel's 8 channels) 16 bytes apart within a chunk block, chunk blocks
//     131 x 16 bytes apart (one spare row shifts consecutive chunks to different bank groups).
//     The operand of tap (dy, dx) for output row r is input row r + 1 + dy from slot 1 + dx on:
//     a shift of the descriptor's start address, no copy.
//   - the weights of one tap (the K-major B operand) are kept in global memory already in
//     that layout (tc_pack_kernel: [K / 8 chunks][c_out][8], chunk blocks c_out x 16 + 16
//     bytes apart), so one thread moves a whole tap with one cp.async.bulk into a stage of a
//     ring of up to four, as soon as the MMAs that read the stage's previous tap have
//     completed; the copy completes the stage's mbarrier by its byte count.
//   - accumulators: R x c_out FP32 columns of TMEM (lane = pixel), D += A_t B_t^T over the
//     9 taps and K / 16 K-steps of 16.
//   - epilogue: warps w and w + 4 share TMEM lane quarter w (one pixel per thread) and read
//     half of its c_out columns each with tcgen05.ld, add bias and conditioning, scale, and
//     stage the row in shared memory (two buffers, alternating by row), from where all 256
//     threads write it out coalesced (conv_epilogue's outputs).
// Staging the input rows through TMA was measured first: tensor-map boxes whose innermost
// extent is one 8-channel chunk (16 bytes) move each pixel's chunk as a separate request, and
// operand staging then took most of a CTA's time. Coalesced 16-byte copies land the same
// layout at full rate; the weights, whose layout is chosen here, go as whole taps.
// Every wait on an mbarrier is bounded; on timeout the kernel sets an error flag, waits
// (bounded) for its copies in flight, frees its TMEM and stops.
#pragma once

namespace nop {

constexpr int TC_SLOTS = 130;                  // pixel slots per chunk block: x0 - 1 .. x0 + 128
constexpr int TC_CHUNK_A = (TC_SLOTS + 1) * 16;  // bytes between chunk blocks of an input row
constexpr int TC_THREADS = 256;                // eight warps: warps w, w + 4 share TMEM lane quarter w
constexpr int TC_PRODUCER = 128;               // thread that copies the weight taps (warp 4, lane 0)
constexpr int TC_MAX_BSTAGES = 4;
constexpr unsigned TC_SPIN_LIMIT = 1u << 20;   // bounded mbarrier waits (about a second at most)

// Set by a CTA whose wait gave up; every later CTA of the path then returns at once.
__device__ int tc_fault_flag;

// KC = K / 8: 8-channel chunks per pixel of the contraction (c_in / 8, doubled with X2).
template <int KC>
__host__ __device__ constexpr int tc_row_bytes() { return KC * TC_CHUNK_A; }
template <int CO>
__host__ __device__ constexpr int tc_chunk_b() { return CO * 16 + 16; }  // bytes between chunk blocks of a tap
template <int KC, int CO>
__host__ __device__ constexpr int tc_tap_bytes() { return KC * tc_chunk_b<CO>(); }
template <int CO>
__host__ __device__ constexpr int tc_stage_pitch() { return CO + 4; }
// Weight-ring stages: four where they fit beside the input rows in one CTA's shared memory
// (more taps in flight hide the copy latency behind the MMAs), else three.
template <int KC, int CO, int R>
__host__ __device__ constexpr int tc_bstages() {
  return (R + 2) * tc_row_bytes<KC>() + 4 * tc_tap_bytes<KC, CO>() + 512 <= 227 * 1024 ? 4 : 3;
}
template <int KC, int CO, int R>
__host__ __device__ constexpr int tc_operand_bytes() {
  return (R + 2) * tc_row_bytes<KC>() + tc_bstages<KC, CO, R>() * tc_tap_bytes<KC, CO>();
}
// Two staged output rows (FP32, rows tc_stage_pitch apart), then bias and conditioning.
template <int CO>
__host__ __device__ constexpr int tc_staged_bytes() { return 2 * 128 * tc_stage_pitch<CO>() * 4 + 2 * CO * 4; }
// The operand buffers, reused for the staged output rows, then 9 mbarriers and the TMEM address.
template <int KC, int CO, int R>
__host__ __device__ constexpr int tc_main_bytes() {
  return tc_operand_bytes<KC, CO, R>() > tc_staged_bytes<CO>() ? tc_operand_bytes<KC, CO, R>() : tc_staged_bytes<CO>();
}
template <int KC, int CO, int R>
__host__ __device__ constexpr int tc_smem_bytes() { return tc_main_bytes<KC, CO, R>() + 128 + 128 /* alignment */; }
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
// This thread's arrival on the mbarrier, raising the phase's expected transaction count by
// `bytes`: the phase completes once the arrivals are in and that many bytes have landed.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// One bulk copy of `bytes` from global to this CTA's shared memory (both addresses 16-byte
// aligned, bytes a multiple of 16) that counts its bytes against the mbarrier's phase.
__device__ __forceinline__ void tc_bulk_copy(uint32_t smem, const void* gmem, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem),
               "l"(gmem), "r"(bytes), "r"(bar)
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

// 32 or 16 consecutive accumulator columns of this thread's TMEM lane, as raw bits; the
// caller waits (tcgen05.wait::ld) before using them.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// Bias, conditioning and scale for n consecutive accumulator columns from column n0 (raw bits
// in r), into this pixel's staged row.
template <int N>
__device__ __forceinline__ void tc_stage_cols(const uint32_t* r, int n0, const float* sbias, const float* sfilm,
                                              float sc, float* stage_px) {
#pragma unroll
  for (int j = 0; j < N; j += 4) {
    const int n = n0 + j;
    float4 o;
    o.x = (__uint_as_float(r[j]) + sbias[n] + sfilm[n]) * sc;
    o.y = (__uint_as_float(r[j + 1]) + sbias[n + 1] + sfilm[n + 1]) * sc;
    o.z = (__uint_as_float(r[j + 2]) + sbias[n + 2] + sfilm[n + 2]) * sc;
    o.w = (__uint_as_float(r[j + 3]) + sbias[n + 3] + sfilm[n + 3]) * sc;
    *reinterpret_cast<float4*>(stage_px + n) = o;
  }
}

// The accumulator columns of one output row that the warps of pair half g (0 or 1) read from
// their TMEM lane quarter and stage: for c_out = 96, 32 columns at 32 g and 16 at 64 + 16 g;
// for 64, 32 at 32 g; for 16, all 16 in half 0. Loads of 32 columns start at multiples of 32
// and loads of 16 at multiples of 16 (row offsets r c_out are multiples of 16 too).
template <int CO>
__device__ __forceinline__ void tc_epilogue_row(uint32_t taddr_row, int g, const float* sbias, const float* sfilm,
                                                float sc, float* stage_px) {
  static_assert(CO == 16 || CO == 64 || CO == 96, "output widths of the network");
  if constexpr (CO == 16) {
    if (g != 0) return;  // warp-uniform
    uint32_t r[16];
    tmem_ld16(taddr_row, r);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    tc_stage_cols<16>(r, 0, sbias, sfilm, sc, stage_px);
  } else {
    uint32_t r[CO == 96 ? 48 : 32];
    tmem_ld32(taddr_row + 32 * g, r);
    if constexpr (CO == 96) tmem_ld16(taddr_row + 64 + 16 * g, r + 32);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    tc_stage_cols<32>(r, 32 * g, sbias, sfilm, sc, stage_px);
    if constexpr (CO == 96) tc_stage_cols<16>(r + 32, 64 + 16 * g, sbias, sfilm, sc, stage_px);
  }
}

// The epilogue stages one output row (128 pixels x CO channels, FP32) in shared memory with
// rows tc_stage_pitch(CO) floats apart: 16-byte aligned, and 8 consecutive pixels (one phase
// of a 16-byte store) fall in distinct bank groups. It is then written out in 16-byte pieces
// that consecutive threads take from consecutive addresses (coalesced): the FP32 result
// (added to what is there with accumulate), its BF16 rounding and its SiLU in BF16, as
// conv_epilogue does.
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

// Grid: (W / 128) x (B H / R) CTAs of TC_THREADS; R output rows per CTA. p.wpk holds the
// weights packed by tc_pack_kernel for (CI, CO, X2).
template <int CI, int CO, int R, bool X2>
__global__ void __launch_bounds__(TC_THREADS, 1) conv_tc_kernel(const __grid_constant__ ConvArgs p, int* err) {
  constexpr int KC = (X2 ? 2 : 1) * CI / 8;    // 8-channel chunks of the contraction
  constexpr int K = 8 * KC;
  static_assert(K % 16 == 0 && CO % 16 == 0 && CO <= 256, "UMMA shape: K steps of 16, N a multiple of 16");
  static_assert(R * CO <= 512, "accumulators fit in TMEM");
  static_assert(!X2 || CI == 16, "the second input only on 16-channel layers");
  constexpr int ROW = tc_row_bytes<KC>();       // bytes per staged input row
  constexpr int TAP = tc_tap_bytes<KC, CO>();   // bytes per staged weight tap
  constexpr uint32_t LBO_A = TC_CHUNK_A, LBO_B = tc_chunk_b<CO>(), SBO = 128;
  constexpr int COLS = tc_tmem_cols<CO, R>();
  constexpr uint32_t IDESC = umma_idesc_bf16<128, CO>();
  constexpr int S = tc_bstages<KC, CO, R>();
  constexpr int PITCH = tc_stage_pitch<CO>();
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 127) & ~(uintptr_t)127);
  unsigned char* sA = base;
  unsigned char* sB = base + (R + 2) * ROW;
  // b_full[S], b_empty[S], done (9 at most), then the TMEM address and the abort word
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + tc_main_bytes<KC, CO, R>());
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_MAX_BSTAGES + 1);
  volatile int* abort_word = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t done_bar = smem_u32(&bars[2 * S]);
  auto b_full = [&](int s) { return smem_u32(&bars[s]); };
  auto b_empty = [&](int s) { return smem_u32(&bars[S + s]); };

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * 128;
  const int row0 = blockIdx.y * R;  // first output row in the flattened (b, h) order
  const int b = row0 / p.H, h0 = row0 - b * p.H;

  if (tid == 0) {
    *abort_word = *(volatile int*)&tc_fault_flag;  // an earlier CTA's wait gave up: do nothing
    for (int s = 0; s < S; ++s) {
      mbar_init(b_full(s), 1);   // the producer's arrival plus the tap's bytes
      mbar_init(b_empty(s), 1);  // the commit of the MMAs that read the stage
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (*abort_word) return;  // uniform over the CTA: nothing allocated or in flight yet
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // The producer starts the first taps (one per stage), so that they are in flight together
  // with the input rows; the stage of tap t is t % S.
  int last_tap[TC_MAX_BSTAGES] = {-1, -1, -1, -1};  // the producer's last tap per stage
  auto copy_tap = [&](int t) {
    const int s = t % S;
    mbar_arrive_expect_tx(b_full(s), (uint32_t)TAP);
    tc_bulk_copy(smem_u32(sB + s * TAP), p.wpk + (size_t)t * TAP, (uint32_t)TAP, b_full(s));
    last_tap[s] = t;
  };
  if (tid == TC_PRODUCER)
    for (int t = 0; t < S; ++t) copy_tap(t);
  // The R + 2 input rows, by every thread: periodic in h and in x; with X2, chunks KC / 2 ..
  // KC - 1 from the second tensor.
  for (int idx = tid; idx < (R + 2) * TC_SLOTS * KC; idx += TC_THREADS) {
    const int i = idx / (TC_SLOTS * KC), rem = idx - i * (TC_SLOTS * KC);
    const int s = rem / KC, c = rem - s * KC;
    const int h = wrap1(h0 - 1 + i, p.H), x = wrap1(x0 - 1 + s, p.W);
    const size_t px = (size_t)(b * p.H + h) * p.W + x;
    const bf16* src = (X2 && c >= CI / 8) ? p.x2 + px * CI + 8 * (c - CI / 8) : p.x + px * CI + 8 * c;
    tc_cp16(smem_u32(sA + i * ROW + c * TC_CHUNK_A + s * 16), src);
  }
  tc_cp_done();  // this thread's input rows have landed
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();  // after it: every input row is in place and the TMEM address is known
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  if (tid == 0) {  // the MMA issuer
    for (int t = 0; t < 9 && ok; ++t) {
      const int s = t % S;
      if (!mbar_wait(b_full(s), (t / S) & 1)) {
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
        for (int kk = 0; kk < K / 16; ++kk) {
          const uint64_t ad = umma_desc(abase + kk * 2 * LBO_A, LBO_A, SBO);
          const uint64_t bd = umma_desc(bbase + kk * 2 * LBO_B, LBO_B, SBO);
          umma_bf16(tmem + (uint32_t)(r * CO), ad, bd, IDESC, (t > 0 || kk > 0) ? 1u : 0u);
        }
      }
      umma_commit(b_empty(s));  // the stage is free once these MMAs have read it
    }
    umma_commit(done_bar);  // arrives once every MMA issued above has completed
  } else if (tid == TC_PRODUCER) {  // the remaining taps, each into the stage its tap - S left
    for (int t = S; t < 9; ++t) {
      const int s = t % S;
      if (!mbar_wait(b_empty(s), ((t - S) / S) & 1)) {
        ok = false;
        break;
      }
      copy_tap(t);
    }
  }
  __syncwarp();
  const bool issued = __syncthreads_and(ok ? 1 : 0) != 0;
  // Wait for the accumulators (on the failure path, for whatever was issued).
  const bool fin = mbar_wait(done_bar, 0);
  const bool good = __syncthreads_and((issued && fin) ? 1 : 0) != 0;  // uniform over the CTA
  if (!good) {
    if (tid == 0) {
      atomicExch(&tc_fault_flag, 1);
      if (err) atomicExch(err, 1);
    }
    if (tid == TC_PRODUCER)  // the last copy into each stage has landed before the CTA ends
      for (int s = 0; s < S; ++s)
        if (last_tap[s] >= 0) mbar_wait(b_full(s), (last_tap[s] / S) & 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (good) {
    // The MMAs have completed: the operand buffers are free and hold the staged rows now.
    float* stage0 = reinterpret_cast<float*>(base);
    float* sbias = stage0 + 2 * 128 * PITCH;  // bias (0 if none), then the conditioning times alpha
    float* sfilm = sbias + CO;
    const float al = p.film ? p.alpha[b] : 0.0f;
    const float sc = p.scale_alpha ? p.alpha[b] : 1.0f;
    for (int n = tid; n < CO; n += TC_THREADS) {
      sbias[n] = p.bias ? p.bias[n] : 0.0f;
      sfilm[n] = p.film ? al * p.film[n] : 0.0f;
    }
    __syncthreads();
    const int quarter = warp & 3, half = warp >> 2;
    const int px = 32 * quarter + lane;  // this thread's TMEM lane: pixel x0 + px
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
      float* stage = stage0 + (r & 1) * 128 * PITCH;
      const uint32_t row_addr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(r * CO);
      tc_epilogue_row<CO>(row_addr, half, sbias, sfilm, sc, stage + px * PITCH);
      // every thread has staged row r and finished writing out row r - 1 (the other buffer)
      __syncthreads();
      tc_store_row<CO>(p, stage, (size_t)(row0 + r) * p.W + x0, tid);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
}

// The weights of a (CI, CO, X2) layer in the layout of the kernel's weight ring:
// out[t][c][n][8] (chunk blocks CO x 16 + 16 bytes apart, the last 16 bytes zero) =
// w[t][n][8 c' .. 8 c' + 7], c' = c mod (CI / 8) (with X2 the chunks repeat: both inputs
// meet the same weights). w is [9][CO][CI] BF16; out holds 9 tc_tap_bytes.
__global__ void tc_pack_kernel(const bf16* __restrict__ w, int CI, int CO, int KC, unsigned char* __restrict__ out) {
  const int per_chunk = CO + 1, n_items = 9 * KC * per_chunk;  // 16-byte items, one pad per chunk block
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n_items; idx += gridDim.x * blockDim.x) {
    const int t = idx / (KC * per_chunk), rem = idx - t * (KC * per_chunk);
    const int c = rem / per_chunk, n = rem - c * per_chunk;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (n < CO) v = *reinterpret_cast<const uint4*>(w + ((size_t)t * CO + n) * CI + 8 * (c % (CI / 8)));
    *reinterpret_cast<uint4*>(out + (size_t)idx * 16) = v;
  }
}

// ---------------------------------------------------------------- host side

// Whether the tensor-core path takes this convolution: rows of a multiple of 128 pixels, H a
// multiple of 4 (no CTA's rows straddle two samples), one input tensor or, on a 16-channel
// layer, the input and its BF16 remainder x2, no second weight half, and weights packed for
// the path (16-byte aligned operands).
inline bool tc_applies(const ConvArgs& a, int ci, int co) {
  const bool chans = (ci == 16 || ci == 64 || ci == 96) && (co == 16 || co == 64 || co == 96);
  const bool x2ok = a.x2 == nullptr || (ci == 16 && ((uintptr_t)a.x2 % 16) == 0);
  return chans && x2ok && a.w2 == nullptr && a.wpk != nullptr && a.W % 128 == 0 && a.H % 4 == 0 &&
         ((uintptr_t)a.x % 16) == 0 && ((uintptr_t)a.wpk % 16) == 0;
}

// Bytes of a layer's packed weights (tc_pack_kernel) and its 8-channel chunks per pixel.
inline int tc_kc(int ci, bool x2) { return (x2 ? 2 : 1) * ci / 8; }
inline size_t tc_pack_bytes(int ci, int co, bool x2) { return 9 * (size_t)tc_kc(ci, x2) * (co * 16 + 16); }

inline std::atomic<long long>& tc_counter() {
  static std::atomic<long long> n{0};
  return n;
}

template <int CI, int CO, int R, bool X2>
void launch_tc_rows(const ConvArgs& a, int* err, cudaStream_t s) {
  constexpr int KC = (X2 ? 2 : 1) * CI / 8;
  constexpr int bytes = tc_smem_bytes<KC, CO, R>();
  static_assert(bytes <= 227 * 1024, "fits in one CTA's shared memory");
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done.load(std::memory_order_relaxed) & bit)) {
    cudaFuncSetAttribute(conv_tc_kernel<CI, CO, R, X2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done.fetch_or(bit, std::memory_order_relaxed);
  }
  conv_tc_kernel<CI, CO, R, X2><<<dim3(a.W / 128, a.B * a.H / R), TC_THREADS, bytes, s>>>(a, err);
}

// Rows per CTA: 4 when that still gives two waves of CTAs over the SMs (operands reused by
// four rows), else fewer (more CTAs).
template <int CI, int CO, bool X2>
void launch_tc_x(const ConvArgs& a, int* err, int sms, cudaStream_t s) {
  const long long ctas4 = (long long)(a.W / 128) * ((long long)a.B * a.H) / 4;
  if (ctas4 >= 2LL * sms)
    launch_tc_rows<CI, CO, 4, X2>(a, err, s);
  else if (ctas4 * 2 >= sms)
    launch_tc_rows<CI, CO, 2, X2>(a, err, s);
  else
    launch_tc_rows<CI, CO, 1, X2>(a, err, s);
}

// Launches conv_tc_kernel for this convolution (tc_applies holds).
template <int CI, int CO>
bool launch_tc(const ConvArgs& a, int* err, int sms, cudaStream_t s) {
  if constexpr (CI == 16) {
    if (a.x2) {
      launch_tc_x<CI, CO, true>(a, err, sms, s);
      tc_counter().fetch_add(1, std::memory_order_relaxed);
      return true;
    }
  }
  launch_tc_x<CI, CO, false>(a, err, sms, s);
  tc_counter().fetch_add(1, std::memory_order_relaxed);
  return true;
}

}  // namespace nop
