// D2Q9 lattice constants and storage codecs shared by the lbch CUDA kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbch {

// Eq. 20a (c = 1) and Eq. 20b.
__host__ __device__ constexpr int cx(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
__host__ __device__ constexpr double wgt(int i) {
  return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
}

constexpr unsigned FULL = 0xffffffffu;

// Storage kinds (values of lbch_storage).
enum : int { ST_F32 = 0, ST_BF16 = 1, ST_F16 = 2 };

// FP16 deviations are stored scaled by 2^12 so that typical non-equilibrium parts
// (1e-6 .. 1e-1) sit in FP16's normal range; the scale is a power of two (exact).
constexpr float F16_SCALE = 4096.0f;
constexpr float F16_UNSCALE = 1.0f / 4096.0f;

// 16-bit deviation codecs on raw bits (bit patterns travel as uint16_t).
template <int ST>
struct Dev;

// Besides one value at a time (load, store), pairs packed in 32 bits with the first value
// in the low half: pack2 rounds both in one conversion; raw2 widens both without the
// storage scale, which the caller applies once to a sum (UNSCALE is a power of two, so
// scaling a sum is exact).
template <>
struct Dev<ST_BF16> {
  static constexpr float UNSCALE = 1.0f;
  __device__ __forceinline__ static float load(uint16_t b) {
    return __uint_as_float(static_cast<uint32_t>(b) << 16);  // exact widening
  }
  __device__ __forceinline__ static uint16_t store(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
  __device__ __forceinline__ static uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ __forceinline__ static void raw2(uint32_t u, float& lo, float& hi) {
    lo = __uint_as_float(u << 16);
    hi = __uint_as_float(u & 0xffff0000u);
  }
};

template <>
struct Dev<ST_F16> {
  static constexpr float UNSCALE = F16_UNSCALE;
  __device__ __forceinline__ static float load(uint16_t b) {
    return __half2float(__ushort_as_half(b)) * F16_UNSCALE;
  }
  __device__ __forceinline__ static uint16_t store(float v) {
    return __half_as_ushort(__float2half_rn(v * F16_SCALE));
  }
  __device__ __forceinline__ static uint32_t pack2(float lo, float hi) { return pack2_scaled(lo * F16_SCALE, hi * F16_SCALE); }
  // pack2 of values already multiplied by F16_SCALE (exact: a power of two), so that callers
  // can scale a pair in one packed multiply.
  __device__ __forceinline__ static uint32_t pack2_scaled(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ __forceinline__ static void raw2(uint32_t u, float& lo, float& hi) {
    const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u));
    lo = f.x;
    hi = f.y;
  }
};

// Device view of one population buffer.
//   F32:  plane i (0..8) at f32 + i*ps.
//   DEV:  f32 + 0*ps holds the post-collision rest population f*_0, f32 + 1*ps holds the
//         anchor mu_alpha of each node; plane i (1..8) of 16-bit deviations
//         d_i(x) = f*_i(x) - w_i mu_alpha(x + c_i), relative to the anchor of the node the
//         population streams to, sits at dev + (i-1)*ps. A reader at y rebuilds
//         f*_i(y - c_i) = w_i anchor(y) + d_i(y - c_i) from its own anchor.
struct Buf {
  float* f32;
  uint16_t* dev;
};

}  // namespace lbch
