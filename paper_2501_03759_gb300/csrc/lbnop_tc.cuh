// The periodic 3 x 3 convolution of lbnop.cu on the 5th-generation tensor cores (tcgen05):
// operands in shared memory in the MMA's canonical K-major layout, FP32 accumulators in
// tensor memory (TMEM), and warps specialised by role, so that loading, the MMAs and the
// epilogue of consecutive tiles overlap.
//
// Scope: rows of a multiple of 128 pixels (W % 128 == 0), H a multiple of 4, c_in and c_out
// in {16, 64, 96}; with X2, c_in = 16 and a second input tensor x2 (the BF16 remainder of
// the first), multiplied by the same weights: the contraction then runs over K = 32, the
// chunks of x followed by those of x2. That covers the finest level of the learned leap on
// 512 x 512 and larger fields, where most of its convolution work is; every other layer keeps
// the mma.sync kernels.
//
// The kernel is persistent: the grid holds as many CTAs per 128-pixel column block as fit on
// the GPU at once, and CTA g takes the g-th of that many equal runs of consecutive output rows
// (flattened over (b, h)), in tiles of up to 2 rows within one sample. Tile k:
//   - loader warps 8-11 copy its input rows (h - 1 .. h + rows, periodic in h) by 16-byte
//     cp.async, consecutive threads reading consecutive bytes, into slots of a ring of six:
//     input row i of tile k in slot (2 k + i) mod 6, as [K / 8 chunks][130 pixel slots]
//     [8 channels], pixel x0 - 1 + s (periodic in x) in pixel slot s. That is the K-major,
//     no-swizzle canonical layout of the MMA's A operand: 16-byte rows (one pixel's 8
//     channels) 16 bytes apart within a chunk block, chunk blocks 131 x 16 bytes apart. The
//     operand of tap (dy, dx) for output row r is input row r + 1 + dy from pixel slot 1 + dx
//     on: a shift of the descriptor's start address, no copy. A 2-row tile that follows a
//     2-row tile of the same sample finds its first two input rows in place (the previous
//     tile's last two) and copies two.
//   - warp 12 (lane 0) issues the 9 taps x K / 16 K-steps of MMAs per row into TMEM
//     accumulator buffer k mod 2 (2 x c_out FP32 columns, lane = pixel), D += A_t B_t^T,
//     while the epilogue still reads buffer (k + 1) mod 2.
//   - warp 13 (lane 0) streams the weight taps of all tiles in order: the weights are kept in
//     global memory already in the B operand's layout (tc_pack_kernel: [K / 8 chunks][c_out]
//     [8], chunk blocks c_out x 16 + 16 bytes apart), so one bulk copy moves a whole tap into
//     a stage of a ring of up to four, once the MMAs that read the stage's previous tap have
//     completed; the copy completes the stage's mbarrier by its byte count.
//   - epilogue warps 0-7: warps w and w + 4 share TMEM lane quarter w (one pixel per thread)
//     and read half of its c_out columns each with tcgen05.ld, add bias and conditioning,
//     scale, and stage the row in shared memory (in the tile's first two input slots, dead
//     once its MMAs are done, where they hold it), from where all 256 threads write it out
//     coalesced (conv_epilogue's outputs).
// mbarriers order the roles: a_full (rows loaded), mma_done (accumulators complete; slot pair
// free for a reloading tile), epi_done (accumulator buffer and staged slots free), and per
// weight stage b_full / b_empty. Tile k's input slots were last written for tile k - 2 and
// held its staged rows, so tile k's copies wait for tile k - 2's epilogue.
// Staging the input rows through TMA was measured first: tensor-map boxes whose innermost
// extent is one 8-channel chunk (16 bytes) move each pixel's chunk as a separate request, and
// operand staging then took most of a CTA's time. Coalesced 16-byte copies land the same
// layout at full rate; the weights, whose layout is chosen here, go as whole taps.
// Every wait on an mbarrier is bounded; on timeout the kernel sets an error flag, waits
// (bounded) for its copies and MMAs in flight, frees its TMEM and stops.
#pragma once

namespace nop {

constexpr int TC_SLOTS = 130;                  // pixel slots per chunk block: x0 - 1 .. x0 + 128
constexpr int TC_CHUNK_A = (TC_SLOTS + 1) * 16;  // bytes between chunk blocks of an input row
constexpr int TC_ROWS = 2;                     // output rows per tile at most
constexpr int TC_RING = 6;                     // input-row slots: two tiles in flight
constexpr int TC_EPI = 256;                    // warps 0-7: epilogue
constexpr int TC_LOAD = 128;                   // warps 8-11: input-row loaders
constexpr int TC_MMA_WARP = 12;                // lane 0 issues the MMAs; the warp owns the TMEM
constexpr int TC_PROD_WARP = 13;               // lane 0 streams the weight taps
constexpr int TC_THREADS = 14 * 32;
constexpr int TC_MAX_BSTAGES = 4;
constexpr int TC_BARS = 2 * TC_MAX_BSTAGES + 7;  // b_full, b_empty, a_full[2], mma_done[2], epi_done[2], final
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
// One staged output row: 128 pixels x CO FP32, pixel rows CO floats apart with their float4s
// permuted (tc_swz), then bias and conditioning.
template <int CO>
__host__ __device__ constexpr int tc_staged_bytes() { return 128 * CO * 4 + 2 * CO * 4; }
// The staged row goes over a tile's first two input slots where they hold it, else after the
// weight ring.
template <int KC, int CO>
__host__ __device__ constexpr bool tc_stage_in_a() { return 2 * tc_row_bytes<KC>() >= tc_staged_bytes<CO>(); }
template <int KC, int CO, int S>
__host__ __device__ constexpr int tc_main_bytes_s() {
  return TC_RING * tc_row_bytes<KC>() + S * tc_tap_bytes<KC, CO>() +
         (tc_stage_in_a<KC, CO>() ? 0 : tc_staged_bytes<CO>());
}
// Weight-ring stages: four where they fit in one CTA's shared memory (more taps in flight
// hide the copy latency behind the MMAs), else three, else two.
template <int KC, int CO>
__host__ __device__ constexpr int tc_bstages() {
  return tc_main_bytes_s<KC, CO, 4>() + 512 <= 227 * 1024 ? 4 : (tc_main_bytes_s<KC, CO, 3>() + 512 <= 227 * 1024 ? 3 : 2);
}
// The input slots, the weight ring, the staged row if separate; then the mbarriers, the TMEM
// address and an abort word (256 bytes), and alignment slack.
template <int KC, int CO>
__host__ __device__ constexpr int tc_main_bytes() { return tc_main_bytes_s<KC, CO, tc_bstages<KC, CO>()>(); }
template <int KC, int CO>
__host__ __device__ constexpr int tc_smem_bytes() { return tc_main_bytes<KC, CO>() + 256 + 128; }
// TMEM columns: a power of two >= 32 that holds two buffers of TC_ROWS accumulators of CO columns.
template <int CO>
__host__ __device__ constexpr int tc_tmem_cols() {
  constexpr int n = 2 * TC_ROWS * CO;
  return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : (n <= 256 ? 256 : 512)));
}
// Position of float4 j of pixel px in its staged row: consecutive pixels writing the same j
// (the TMEM read: one pixel per thread) and consecutive threads reading one pixel's float4s
// (the coalesced write-out) both fall in distinct bank groups.
template <int CO>
__device__ __forceinline__ int tc_swz(int px, int j) {
  return CO >= 32 ? (j ^ (px & 7)) : (j ^ ((px >> 1) & 3));
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
// Bias, conditioning and scale for N consecutive accumulator columns from column n0 (raw bits
// in r), into pixel px's staged row.
template <int CO, int N>
__device__ __forceinline__ void tc_stage_cols(const uint32_t* r, int n0, const float* sbias, const float* sfilm,
                                              float sc, float* stage, int px) {
#pragma unroll
  for (int j = 0; j < N; j += 4) {
    const int n = n0 + j;
    const float4 bb = *reinterpret_cast<const float4*>(sbias + n);
    const float4 ff = *reinterpret_cast<const float4*>(sfilm + n);
    float4 o;
    o.x = (__uint_as_float(r[j]) + bb.x + ff.x) * sc;
    o.y = (__uint_as_float(r[j + 1]) + bb.y + ff.y) * sc;
    o.z = (__uint_as_float(r[j + 2]) + bb.z + ff.z) * sc;
    o.w = (__uint_as_float(r[j + 3]) + bb.w + ff.w) * sc;
    *reinterpret_cast<float4*>(stage + px * CO + 4 * tc_swz<CO>(px, n / 4)) = o;
  }
}

// The accumulator columns of one output row that the warps of pair half g (0 or 1) read from
// their TMEM lane quarter and stage: for c_out = 96, 32 columns at 32 g and 16 at 64 + 16 g;
// for 64, 32 at 32 g; for 16, all 16 in half 0. Loads of 32 columns start at multiples of 32
// and loads of 16 at multiples of 16 (row and buffer offsets are multiples of 16 too).
template <int CO>
__device__ __forceinline__ void tc_epilogue_row(uint32_t taddr_row, int g, const float* sbias, const float* sfilm,
                                                float sc, float* stage, int px) {
  static_assert(CO == 16 || CO == 64 || CO == 96, "output widths of the network");
  if constexpr (CO == 16) {
    if (g != 0) return;  // warp-uniform
    uint32_t r[16];
    tmem_ld16(taddr_row, r);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    tc_stage_cols<CO, 16>(r, 0, sbias, sfilm, sc, stage, px);
  } else {
    uint32_t r[CO == 96 ? 48 : 32];
    tmem_ld32(taddr_row + 32 * g, r);
    if constexpr (CO == 96) tmem_ld16(taddr_row + 64 + 16 * g, r + 32);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    tc_stage_cols<CO, 32>(r, 32 * g, sbias, sfilm, sc, stage, px);
    if constexpr (CO == 96) tc_stage_cols<CO, 16>(r + 32, 64 + 16 * g, sbias, sfilm, sc, stage, px);
  }
}

// Writes out one staged output row (128 pixels from pix0) in 16-byte pieces that consecutive
// threads take from consecutive addresses (coalesced): the FP32 result (added to what is
// there with accumulate), its BF16 rounding and its SiLU in BF16, as conv_epilogue does.
template <int CO>
__device__ __forceinline__ void tc_store_row(const ConvArgs& p, const float* stage, size_t pix0, int tid) {
  constexpr int Q = CO / 4;
  const size_t o0 = pix0 * CO;  // item idx = 4 channels: global offset 4 idx
  for (int idx = tid; idx < 128 * Q; idx += TC_EPI) {
    const int px = idx / Q, c4 = idx - px * Q;
    const float4 v = *reinterpret_cast<const float4*>(stage + px * CO + 4 * tc_swz<CO>(px, c4));
    const size_t o = o0 + 4 * (size_t)idx;
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

// Named barrier 1 over the 256 epilogue threads, and the same barrier reducing a flag: true if
// it holds on every epilogue thread.
__device__ __forceinline__ void tc_epi_sync() { asm volatile("barrier.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ bool tc_epi_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbarrier.red.and.pred q, 1, 256, p;\n\tselp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

// Output rows of the tile starting at flattened row r: at most TC_ROWS, within the CTA's run
// (which ends before `last`) and within the sample.
__device__ __forceinline__ int tc_tile_rows(int r, int last, int H) {
  const int h = r % H;
  int n = last - r;
  n = n < TC_ROWS ? n : TC_ROWS;
  return n < H - h ? n : H - h;
}

// The tiles of one CTA, in order: rows [r0, r0 + rk), input slot base sk = 2 k mod 6, and
// whether the first two input rows are the previous tile's last two (a full tile of the same
// sample before it). Every role walks the same sequence.
struct TcTiles {
  int first, last, H;
  int k, r0, rk, sk;
  bool reuse;
  __device__ __forceinline__ void start(int f, int l, int h) {
    first = f;
    last = l;
    H = h;
    k = 0;
    r0 = f;
    sk = 0;
    reuse = false;
    rk = r0 < last ? tc_tile_rows(r0, last, H) : 0;
  }
  __device__ __forceinline__ bool more() const { return r0 < last; }
  __device__ __forceinline__ void next() {
    const bool full = rk == TC_ROWS;
    r0 += rk;
    ++k;
    sk = sk + 2 == TC_RING ? 0 : sk + 2;
    reuse = full && r0 < last && r0 % H != 0;
    rk = r0 < last ? tc_tile_rows(r0, last, H) : 0;
  }
};

// Grid: (W / 128) x G CTAs of TC_THREADS; CTA (x, g) takes flattened output rows
// [g N / G, (g + 1) N / G), N = B H, of column block x. p.wpk holds the weights packed by
// tc_pack_kernel for (CI, CO, X2).
template <int CI, int CO, bool X2>
__global__ void __launch_bounds__(TC_THREADS, 1) conv_tc_kernel(const __grid_constant__ ConvArgs p, int* err) {
  constexpr int KC = (X2 ? 2 : 1) * CI / 8;    // 8-channel chunks of the contraction
  constexpr int K = 8 * KC;
  static_assert(K % 16 == 0 && CO % 16 == 0 && CO <= 256, "UMMA shape: K steps of 16, N a multiple of 16");
  static_assert(2 * TC_ROWS * CO <= 512, "two accumulator buffers fit in TMEM");
  static_assert(!X2 || CI == 16, "the second input only on 16-channel layers");
  constexpr int ROW = tc_row_bytes<KC>();       // bytes per staged input row
  constexpr int TAP = tc_tap_bytes<KC, CO>();   // bytes per staged weight tap
  constexpr uint32_t LBO_A = TC_CHUNK_A, LBO_B = tc_chunk_b<CO>(), SBO = 128;
  constexpr int COLS = tc_tmem_cols<CO>();
  constexpr uint32_t IDESC = umma_idesc_bf16<128, CO>();
  constexpr int S = tc_bstages<KC, CO>();
  constexpr bool SIA = tc_stage_in_a<KC, CO>();
  constexpr int PER_ROW = TC_SLOTS * KC;        // 16-byte copies per input row
  static_assert(PER_ROW >= TC_LOAD, "a loader's copies advance by one row at most");
  extern __shared__ __align__(128) unsigned char tc_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 127) & ~(uintptr_t)127);
  unsigned char* sA = base;
  unsigned char* sB = base + TC_RING * ROW;
  float* stage_sep = reinterpret_cast<float*>(sB + S * TAP);  // the staged row when not in the input slots
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + tc_main_bytes<KC, CO>());
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + TC_BARS);
  volatile int* abort_word = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto b_full = [&](int s) { return smem_u32(&bars[s]); };
  auto b_empty = [&](int s) { return smem_u32(&bars[S + s]); };
  auto a_full = [&](int j) { return smem_u32(&bars[2 * S + j]); };
  auto mma_done = [&](int j) { return smem_u32(&bars[2 * S + 2 + j]); };
  auto epi_done = [&](int j) { return smem_u32(&bars[2 * S + 4 + j]); };
  const uint32_t final_bar = smem_u32(&bars[2 * S + 6]);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * 128;
  const int N = p.B * p.H;
  const int first = (int)((long long)blockIdx.y * N / gridDim.y);
  const int last = (int)((long long)(blockIdx.y + 1) * N / gridDim.y);

  if (tid == 0) {
    *abort_word = *(volatile int*)&tc_fault_flag;  // an earlier CTA's wait gave up: do nothing
    for (int s = 0; s < S; ++s) {
      mbar_init(b_full(s), 1);   // the producer's arrival plus the tap's bytes
      mbar_init(b_empty(s), 1);  // the commit of the MMAs that read the stage
    }
    for (int j = 0; j < 2; ++j) {
      mbar_init(a_full(j), TC_LOAD);   // every loader thread, once its copies have landed
      mbar_init(mma_done(j), 1);       // the commit after the tile's MMAs
      mbar_init(epi_done(j), TC_EPI);  // every epilogue thread, once done with the buffer
    }
    mbar_init(final_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (*abort_word || first >= last) return;  // uniform over the CTA: nothing allocated or in flight yet
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  TcTiles tl;
  tl.start(first, last, p.H);
  if (warp < TC_EPI / 32) {
    // ------------------------------------------------------------ epilogue warps 0-7
    const int quarter = warp & 3, half = warp >> 2;
    const int px = 32 * quarter + lane;  // this thread's TMEM lane: pixel x0 + px
    for (; tl.more(); tl.next()) {
      const int j = tl.k & 1;
      const bool fin = mbar_wait(mma_done(j), (uint32_t)((tl.k >> 1) & 1));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!tc_epi_and(fin)) {  // uniform over the epilogue warps
        ok = false;
        break;
      }
      float* stage = SIA ? reinterpret_cast<float*>(sA + tl.sk * ROW) : stage_sep;
      float* sbias = stage + 128 * CO;  // bias (0 if none), then the conditioning times alpha
      float* sfilm = sbias + CO;
      const int b = tl.r0 / p.H;
      const float al = p.film ? p.alpha[b] : 0.0f;
      const float sc = p.scale_alpha ? p.alpha[b] : 1.0f;
      for (int n = tid; n < CO; n += TC_EPI) {
        sbias[n] = p.bias ? p.bias[n] : 0.0f;
        sfilm[n] = p.film ? al * p.film[n] : 0.0f;
      }
      tc_epi_sync();
#pragma unroll 1
      for (int r = 0; r < tl.rk; ++r) {
        const uint32_t row_addr =
            tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)((j * TC_ROWS + r) * CO);
        tc_epilogue_row<CO>(row_addr, half, sbias, sfilm, sc, stage, px);
        tc_epi_sync();
        tc_store_row<CO>(p, stage, (size_t)(tl.r0 + r) * p.W + x0, tid);
        tc_epi_sync();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(epi_done(j));  // this thread's accumulator reads and staged-row reads are done
    }
  } else if (warp < (TC_EPI + TC_LOAD) / 32) {
    // ------------------------------------------------------------ loader warps 8-11
    const int ltid = tid - TC_EPI;
    const uint32_t sA32 = smem_u32(sA);
    for (; tl.more(); tl.next()) {
      const int j = tl.k & 1;
      // slots of input rows 2, 3: tile k - 2's first two, which held its staged rows
      if (tl.k >= 2 && !mbar_wait(epi_done(j), (uint32_t)(((tl.k >> 1) + 1) & 1))) {
        ok = false;
        break;
      }
      // slots of input rows 0, 1 when not reused: tile k - 1's last two, read by its MMAs
      if (!tl.reuse && tl.k >= 1 && !mbar_wait(mma_done(j ^ 1), (uint32_t)(((tl.k - 1) >> 1) & 1))) {
        ok = false;
        break;
      }
      const int b = tl.r0 / p.H, h0 = tl.r0 - b * p.H;
      // item (i, pixel slot, chunk), chunk fastest; each loader steps TC_LOAD items at a time
      const int i0 = tl.reuse ? 2 : 0;
      const int n_items = (tl.rk + 2 - i0) * PER_ROW;
      int i = i0, rem = ltid;
      size_t row_px = (size_t)(b * p.H + wrap1(h0 - 1 + i, p.H)) * p.W;  // first pixel of input row i
      int q = tl.sk + i >= TC_RING ? tl.sk + i - TC_RING : tl.sk + i;    // its slot
      for (int idx = ltid; idx < n_items; idx += TC_LOAD) {
        const int sl = rem / KC, c = rem - sl * KC;
        const size_t px = row_px + wrap1(x0 - 1 + sl, p.W);
        const bf16* src = (X2 && c >= CI / 8) ? p.x2 + px * CI + 8 * (c - CI / 8) : p.x + px * CI + 8 * c;
        tc_cp16(sA32 + (uint32_t)(q * ROW + c * TC_CHUNK_A + sl * 16), src);
        rem += TC_LOAD;
        if (rem >= PER_ROW) {
          rem -= PER_ROW;
          ++i;
          row_px = (size_t)(b * p.H + wrap1(h0 - 1 + i, p.H)) * p.W;
          q = q + 1 == TC_RING ? 0 : q + 1;
        }
      }
      tc_cp_done();  // this thread's copies have landed and are visible to the tensor cores
      mbar_arrive(a_full(j));
    }
  } else if (warp == TC_MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer (lane 0)
    if (lane == 0) {
      // Descriptors of input slot 0 and weight stage 0 at their first chunk: every operand
      // start is a 16-byte multiple from them, added to the start-address field (address / 16,
      // 14 bits, which holds every shared-memory address).
      const uint64_t a0 = umma_desc(smem_u32(sA), LBO_A, SBO);
      const uint64_t b0 = umma_desc(smem_u32(sB), LBO_B, SBO);
      for (; tl.more() && ok; tl.next()) {
        const int j = tl.k & 1;
        if (!mbar_wait(a_full(j), (uint32_t)((tl.k >> 1) & 1)) ||
            (tl.k >= 2 && !mbar_wait(epi_done(j), (uint32_t)(((tl.k >> 1) + 1) & 1)))) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dcol = tmem + (uint32_t)(j * TC_ROWS * CO);
        for (int t = 0; t < 9; ++t) {
          const int T = 9 * tl.k + t, s = T % S;
          if (!mbar_wait(b_full(s), (uint32_t)((T / S) & 1))) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const int dy = t / 3 - 1, dx = t % 3 - 1;
          const uint64_t bt = b0 + (uint64_t)((s * TAP) >> 4);
#pragma unroll
          for (int r = 0; r < TC_ROWS; ++r) {
            if (r < tl.rk) {
              int q = tl.sk + r + 1 + dy;  // the slot of input row r + 1 + dy
              q = q >= TC_RING ? q - TC_RING : q;
              const uint64_t at = a0 + (uint64_t)((q * ROW + (1 + dx) * 16) >> 4);
#pragma unroll
              for (int kk = 0; kk < K / 16; ++kk)
                umma_bf16(dcol + (uint32_t)(r * CO), at + (uint64_t)((kk * 2 * LBO_A) >> 4),
                          bt + (uint64_t)((kk * 2 * LBO_B) >> 4), IDESC, (t > 0 || kk > 0) ? 1u : 0u);
            }
          }
          umma_commit(b_empty(s));  // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        umma_commit(mma_done(j));  // the tile's accumulators are complete once this arrives
      }
      umma_commit(final_bar);  // every MMA issued above has completed once this arrives
      if (!mbar_wait(final_bar, 0)) ok = false;
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ weight producer (lane 0)
    if (lane == 0) {  // tap T of the run (tile T / 9, tap T % 9) into stage T % S
      int ntiles = 0;
      for (; tl.more(); tl.next()) ++ntiles;
      int last_tap[TC_MAX_BSTAGES] = {-1, -1, -1, -1};
      for (int T = 0; T < 9 * ntiles; ++T) {
        const int s = T % S;
        if (T >= S && !mbar_wait(b_empty(s), (uint32_t)(((T - S) / S) & 1))) {
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(b_full(s), (uint32_t)TAP);
        tc_bulk_copy(smem_u32(sB + s * TAP), p.wpk + (size_t)(T % 9) * TAP, (uint32_t)TAP, b_full(s));
        last_tap[s] = T;
      }
      // the last copy into each stage has landed before the CTA ends
      for (int s = 0; s < S; ++s)
        if (last_tap[s] >= 0 && !mbar_wait(b_full(s), (uint32_t)((last_tap[s] / S) & 1))) ok = false;
    }
    __syncwarp();
  }
  const bool all_ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (!all_ok && tid == 0) {
    atomicExch(&tc_fault_flag, 1);
    if (err) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == TC_MMA_WARP)
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

// ---------------------------------------------------------------- weight gradient

// The weight gradient dw[t][o][i] += sum_p dz(p)[o] x(p + d_t)[i] (t = 3 (dy + 1) + dx + 1, the
// data-parallel half of the backward pass of a convolution) on the tensor cores: the pixels are
// the contraction. The staging layout of the convolution above, [chunk][pixel slot][8
// channels], is then the canonical MN-major layout (8 pixels x 8 channels per 128-byte core
// matrix, channel chunks TC_CHUNK_A apart along M or N, 8-pixel groups 128 bytes apart along
// K), so both operands are staged exactly as the convolution stages its input rows and the
// descriptors keep their strides; the instruction descriptor marks A and B MN-major.
// A = dz of one row (M = c_out padded to 128 with zero chunks), B = x of the row dy away (N =
// c_in), shifted by dx through the start address; K = 16 pixels per MMA, 8 per row of 128.
//
// Grid: (W / 128) x 3 (dy) x G CTAs of WG_THREADS. CTA (x, dy, g) takes the g-th of G equal
// runs of the B H rows of column block x, accumulates its three dx taps in TMEM (3 c_in
// columns, lane = output channel) and adds them into dw with FP32 atomics at the end. Warps
// 0-7 stage (dz row, x row) pairs into a ring of stages (16-byte copies: eight warps keep
// enough of them in flight), and warps 0-3 read TMEM at the end; warp 8 allocates TMEM and
// its lane 0 issues the MMAs.
constexpr int WG_LOAD = 256;
constexpr int WG_MMA_WARP = WG_LOAD / 32;
constexpr int WG_THREADS = WG_LOAD + 32;
constexpr int WG_MCH = 16;  // chunks of the A operand: M = 128 channels

template <int CI>
__host__ __device__ constexpr int wg_stage_bytes() { return (WG_MCH + CI / 8) * TC_CHUNK_A; }
template <int CI>
__host__ __device__ constexpr int wg_stages() {
  return 4 * wg_stage_bytes<CI>() + 256 <= 227 * 1024 ? 4 : (3 * wg_stage_bytes<CI>() + 256 <= 227 * 1024 ? 3 : 2);
}
template <int CI>
__host__ __device__ constexpr int wg_smem_bytes() { return wg_stages<CI>() * wg_stage_bytes<CI>() + 256 + 128; }
template <int CI>
__host__ __device__ constexpr int wg_tmem_cols() {
  return 3 * CI <= 32 ? 32 : (3 * CI <= 64 ? 64 : (3 * CI <= 128 ? 128 : (3 * CI <= 256 ? 256 : 512)));
}
// kind::f16, FP32 accumulator, BF16 A and B, both MN-major (bits 15, 16), N >> 3, M >> 4.
template <int M, int N>
__host__ __device__ constexpr uint32_t umma_idesc_bf16_mn() {
  return umma_idesc_bf16<M, N>() | (1u << 15) | (1u << 16);
}

template <int CI, int CO>
__global__ void __launch_bounds__(WG_THREADS, 1) wgrad_tc_kernel(const __grid_constant__ WgradArgs p, int* err) {
  static_assert(CO <= 128 && CO % 16 == 0 && CI % 16 == 0 && 3 * CI <= 512, "M = 128 channels, 3 taps in TMEM");
  constexpr int ST = wg_stages<CI>(), STG = wg_stage_bytes<CI>();
  constexpr int COLS = wg_tmem_cols<CI>();
  constexpr uint32_t IDESC = umma_idesc_bf16_mn<128, CI>();
  // MN-major: the leading offset steps along K (8-pixel groups), the stride offset along M / N
  // (channel chunks)
  constexpr uint32_t LBO = 128, SBO = TC_CHUNK_A;
  constexpr int ZC = CO / 8, XC = CI / 8;  // chunks of dz and of x per pixel
  extern __shared__ __align__(128) unsigned char wg_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(wg_smem_raw) + 127) & ~(uintptr_t)127);
  // stage s: dz chunk blocks 0..15 (ZC.. zero), then the x chunk blocks
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + ST * STG);  // full[ST], empty[ST], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * 4 + 1);
  volatile int* abort_word = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto empty = [&](int s) { return smem_u32(&bars[ST + s]); };
  const uint32_t done_bar = smem_u32(&bars[2 * ST]);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * 128, dy = (int)blockIdx.y - 1;
  const int N = p.B * p.H;
  const int first = (int)((long long)blockIdx.z * N / gridDim.z);
  const int last = (int)((long long)(blockIdx.z + 1) * N / gridDim.z);
  const int nrows = last - first;

  if (tid == 0) {
    *abort_word = *(volatile int*)&tc_fault_flag;
    for (int s = 0; s < ST; ++s) {
      mbar_init(full(s), WG_LOAD);
      mbar_init(empty(s), 1);
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the zero chunks of every stage's A operand (M rows CO .. 127), written once
  for (int s = 0; s < ST; ++s)
    for (int k = tid; k < (WG_MCH - ZC) * TC_CHUNK_A / 16; k += WG_THREADS)
      reinterpret_cast<uint4*>(base + s * STG + ZC * TC_CHUNK_A)[k] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (*abort_word || nrows <= 0) return;  // uniform: nothing allocated or in flight
  if (warp == WG_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  if (warp < WG_MMA_WARP) {
    // ------------------------------------------------ loaders: row j of the run into stage j % ST
    const uint32_t base32 = smem_u32(base);
    for (int j = 0; j < nrows && ok; ++j) {
      const int s = j % ST;
      if (j >= ST && !mbar_wait(empty(s), (uint32_t)(((j - ST) / ST) & 1))) {
        ok = false;
        break;
      }
      const int row = first + j, b = row / p.H, h = row - b * p.H;
      const size_t zrow = ((size_t)row * p.W + x0) * CO;                                   // dz pixels x0 ..
      const size_t xrow = (size_t)(b * p.H + wrap1(h + dy, p.H)) * p.W;                    // x row h + dy
      // dz: pixel x0 + q - 1 in slot q (q = 1 .. 128), chunks 0 .. ZC - 1
      for (int idx = tid; idx < 128 * ZC; idx += WG_LOAD) {
        const int q = idx / ZC, c = idx - q * ZC;
        tc_cp16(base32 + (uint32_t)(s * STG + c * TC_CHUNK_A + (q + 1) * 16), p.dz + zrow + (size_t)q * CO + 8 * c);
      }
      // x: pixel x0 - 1 + q (periodic) in slot q (q = 0 .. 129)
      for (int idx = tid; idx < TC_SLOTS * XC; idx += WG_LOAD) {
        const int q = idx / XC, c = idx - q * XC;
        const size_t px = xrow + wrap1(x0 - 1 + q, p.W);
        tc_cp16(base32 + (uint32_t)(s * STG + (WG_MCH + c) * TC_CHUNK_A + q * 16), p.x + px * CI + 8 * c);
      }
      tc_cp_done();
      mbar_arrive(full(s));
    }
  } else if (lane == 0) {
    // ------------------------------------------------ MMA issuer: 3 dx taps x 8 K-steps per row
    const uint64_t d0 = umma_desc(smem_u32(base), LBO, SBO);
    for (int j = 0; j < nrows; ++j) {
      const int s = j % ST;
      if (!mbar_wait(full(s), (uint32_t)((j / ST) & 1))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t as = d0 + (uint64_t)((s * STG + 16) >> 4);                          // dz slot 1
      const uint64_t bs = d0 + (uint64_t)((s * STG + WG_MCH * TC_CHUNK_A) >> 4);         // x slot 0
#pragma unroll
      for (int dxi = 0; dxi < 3; ++dxi)
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
          umma_bf16(tmem + (uint32_t)(dxi * CI), as + (uint64_t)(kk * 16), bs + (uint64_t)(dxi + kk * 16), IDESC,
                    (j > 0 || kk > 0) ? 1u : 0u);
      umma_commit(empty(s));
    }
    umma_commit(done_bar);
  }
  __syncwarp();
  // every thread: the accumulators are complete (or the run gave up)
  const bool fin = mbar_wait(done_bar, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool good = __syncthreads_and((ok && fin) ? 1 : 0) != 0;
  if (!good && tid == 0) {
    atomicExch(&tc_fault_flag, 1);
    if (err) atomicExch(err, 1);
  }
  if (good && warp < 4) {
    // ------------------------------------------------ epilogue: TMEM lane 32 warp + lane = channel o
    const int o = 32 * warp + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < 3 * CI; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(lane_addr + (uint32_t)c0, r);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (o < CO) {
        const int dxi = c0 / CI, i0 = c0 - dxi * CI, t = 3 * (dy + 1) + dxi;
        float* d = p.dw + ((size_t)t * CO + o) * CI + i0;
#pragma unroll
        for (int e = 0; e < 16; ++e) atomicAdd(d + e, __uint_as_float(r[e]));
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == WG_MMA_WARP)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
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

// One persistent launch: as many CTAs per column block as fit on the GPU at once (never
// more than there are rows), each taking an equal run of rows.
template <int CI, int CO, bool X2>
void launch_tc_x(const ConvArgs& a, int* err, int sms, cudaStream_t s) {
  constexpr int KC = (X2 ? 2 : 1) * CI / 8;
  constexpr int bytes = tc_smem_bytes<KC, CO>();
  static_assert(bytes <= 227 * 1024, "fits in one CTA's shared memory");
  static std::atomic<int> per_sm[64];  // resident CTAs per SM, by device (0: not queried yet)
  int dev = 0;
  cudaGetDevice(&dev);
  int occ = per_sm[dev & 63].load(std::memory_order_relaxed);
  if (occ == 0) {
    cudaFuncSetAttribute(conv_tc_kernel<CI, CO, X2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv_tc_kernel<CI, CO, X2>, TC_THREADS, bytes) !=
            cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    if (occ > 512 / tc_tmem_cols<CO>()) occ = 512 / tc_tmem_cols<CO>();  // co-resident CTAs share TMEM
    per_sm[dev & 63].store(occ, std::memory_order_relaxed);
  }
  const int cols = a.W / 128, rows = a.B * a.H;
  const long long want = ((long long)sms * occ + cols - 1) / cols;
  const int G = (int)(want < rows ? want : rows);
  conv_tc_kernel<CI, CO, X2><<<dim3(cols, G), TC_THREADS, bytes, s>>>(a, err);
}

// The tensor-core weight gradient applies to rows of a multiple of 128 pixels (16-byte aligned
// tensors); every dz row pairs with its own sample's rows, so H is free.
inline bool wgrad_tc_applies(const WgradArgs& a) {
  return a.W % 128 == 0 && a.B * a.H >= 1 && ((uintptr_t)a.x % 16) == 0 && ((uintptr_t)a.dz % 16) == 0;
}

// One launch: (W / 128) x 3 (dy) x G CTAs, G equal runs of rows per column block and dy, as
// many CTAs as fit on the GPU at once (never more runs than rows).
template <int CI, int CO>
void launch_wgrad_tc(const WgradArgs& a, int* err, int sms, cudaStream_t s) {
  constexpr int bytes = wg_smem_bytes<CI>();
  static_assert(bytes <= 227 * 1024, "fits in one CTA's shared memory");
  static std::atomic<int> per_sm[64];
  int dev = 0;
  cudaGetDevice(&dev);
  int occ = per_sm[dev & 63].load(std::memory_order_relaxed);
  if (occ == 0) {
    cudaFuncSetAttribute(wgrad_tc_kernel<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wgrad_tc_kernel<CI, CO>, WG_THREADS, bytes) !=
            cudaSuccess ||
        occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    if (occ > 512 / wg_tmem_cols<CI>()) occ = 512 / wg_tmem_cols<CI>();  // co-resident CTAs share TMEM
    per_sm[dev & 63].store(occ, std::memory_order_relaxed);
  }
  const int cols = a.W / 128, rows = a.B * a.H;
  const long long want = ((long long)sms * occ) / (3LL * cols);
  const int G = (int)(want < 1 ? 1 : (want < rows ? want : rows));
  wgrad_tc_kernel<CI, CO><<<dim3(cols, 3, G), WG_THREADS, bytes, s>>>(a, err);
  tc_counter().fetch_add(1, std::memory_order_relaxed);
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
