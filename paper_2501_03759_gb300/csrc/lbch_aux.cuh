// Initial state, checkpoint transfer and FP64 reductions for lbch (not per step).
//
// The step kernel keeps post-collision populations f* (Eq. 17 right-hand side,
// before streaming); the canonical state of the paper is the post-streaming
// f_i(x, t) = f*_i(x - c_i). These kernels translate between the two and reduce
// phi = sum_i f_i (Eq. 22) and the free energy (Eq. 7 with Eq. 9 or Eq. 8).
#pragma once

#include "lbch_lattice.cuh"

namespace lbch {

constexpr int AUX_THREADS = 256;
constexpr int MAX_RED_BLOCKS = 2048;

struct Grid {
  int nx, ny;
  long long ps;  // plane stride of the population buffers (elements)
};

__device__ __forceinline__ long long wrapped(const Grid& g, int x, int y) {
  x = x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
  y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
  return (long long)y * g.nx + x;
}

// Canonical f_i at node (x, y): f*_i of the node the population came from (an FP32 value).
template <int ST>
__device__ __forceinline__ float pulled_f(const Buf& b, const Grid& g, int i, int x, int y) {
  const long long s = wrapped(g, x - cx(i), y - cy(i));
  if constexpr (ST == ST_F32) {
    return b.f32[(long long)i * g.ps + s];
  } else {
    if (i == 0) return b.f32[s];
    // w_i times this node's anchor plus the deviation stored at the source node.
    const long long own = (long long)y * g.nx + x;
    return fmaf((float)wgt(i), b.f32[g.ps + own], Dev<ST>::load(b.dev[(long long)(i - 1) * g.ps + s]));
  }
}
template <int ST>
__device__ __forceinline__ double pulled(const Buf& b, const Grid& g, int i, int x, int y) {
  return (double)pulled_f<ST>(b, g, i, x, y);
}

// Compensated (Kahan) FP32 sum: the error stays at FP32 rounding of the total.
struct KahanF32 {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// mu_alpha = f(phi) - k lap phi (Eq. 16, Eq. 26b) in FP64 from an FP64 phi plane;
// flags non-finite phi.
// FP32 -> FP64 copy of a device field (the staging plane of lbch_init_field_device).
__global__ void widen_kernel(const float* __restrict__ in, long long n, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

// Rows are spread over blocks and columns over threads (no 64-bit division per node).
__global__ void mu_alpha_kernel(const double* __restrict__ phi, double* __restrict__ mua, Grid g,
                                double k, double beta4, int* bad) {
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const long long id = (long long)y * g.nx + x;
      const double c = phi[id];
      double lap = 0.0;
#pragma unroll
      for (int i = 1; i < 9; ++i) lap += 2.0 * wgt(i) * (phi[wrapped(g, x + cx(i), y + cy(i))] - c);
      lap *= 3.0;
      mua[id] = beta4 * c * (c * c - 1.0) - k * lap;
      if (!isfinite(c)) atomicOr(bad, 1);
    }
}

// f = f^eq(phi0, mu_alpha) (Eq. 18) written in the step kernel's pre-streaming form, each
// value the FP32 rounding of its FP64 definition. The node-local part: the rest population,
// and for FP32 storage the two products every moving population takes, w mu_alpha(x) for the
// axis (w = 1/9) and diagonal (w = 1/36) velocities, into the scratch planes eq_ax and eq_dg
// (rounded once per node instead of once per population; init_gather_kernel places them).
template <int ST>
__global__ void init_state_kernel(const double* __restrict__ phi0, const double* __restrict__ mua,
                                  Buf b, Grid g, float* __restrict__ eq_ax, float* __restrict__ eq_dg) {
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const long long id = (long long)y * g.nx + x;
      const double m = mua[id];
      const double rest = phi0[id] + (wgt(0) - 1.0) * m;
      b.f32[id] = (float)rest;
      if constexpr (ST == ST_F32) {
        eq_ax[id] = (float)(wgt(1) * m);
        eq_dg[id] = (float)(wgt(5) * m);
      } else {
        // A reader at y + c_i rebuilds w_i anchor(y + c_i) + d_i(y) = w_i mu_alpha(y + c_i),
        // exactly f^eq_i there, with every deviation zero.
        b.f32[g.ps + id] = (float)m;
#pragma unroll
        for (int i = 1; i < 9; ++i) b.dev[(long long)(i - 1) * g.ps + id] = Dev<ST>::store(0.0f);
      }
    }
}

// FP32 storage: f*_i(y) must stream to f_i(y + c_i) = w_i mu_alpha(y + c_i), the product
// init_state_kernel rounded at y + c_i.
__global__ void init_gather_kernel(const float* __restrict__ eq_ax, const float* __restrict__ eq_dg, Buf b, Grid g) {
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const long long id = (long long)y * g.nx + x;
#pragma unroll
      for (int i = 1; i < 9; ++i)
        b.f32[(long long)i * g.ps + id] = (i <= 4 ? eq_ax : eq_dg)[wrapped(g, x + cx(i), y + cy(i))];
    }
}

// One canonical plane f_i(x, t) in FP64.
template <int ST>
__global__ void get_plane_kernel(Buf b, Grid g, int i, double* __restrict__ out) {
  const long long n = (long long)g.nx * g.ny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % g.nx), y = (int)(id / g.nx);
    out[id] = pulled<ST>(b, g, i, x, y);
  }
}

// FP32 state from one canonical FP64 plane: f*_i(y) = f_i(y + c_i); flags non-finite input.
__global__ void set_plane_f32_kernel(const double* __restrict__ in, Buf b, Grid g, int i, int* bad) {
  const long long n = (long long)g.nx * g.ny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % g.nx), y = (int)(id / g.nx);
    const double v = in[wrapped(g, x + cx(i), y + cy(i))];
    if (!isfinite(in[id])) atomicOr(bad, 1);
    b.f32[(long long)i * g.ps + id] = (float)v;
  }
}

// acc (+)= in, FP64 (phi of a canonical state, plane by plane); flags non-finite input.
__global__ void accumulate_kernel(const double* __restrict__ in, double* __restrict__ acc, long long n,
                                  int first, int* bad) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const double v = in[id];
    if (!isfinite(v)) atomicOr(bad, 1);
    acc[id] = first ? v : acc[id] + v;
  }
}

// Deviation storage from one canonical plane: rest population as is; a moving
// population as its deviation from w_i times the anchor (plane 1, already set) of
// the node it streams to.
template <int ST>
__global__ void set_plane_dev_kernel(const double* __restrict__ in, Buf b, Grid g, int i) {
  const long long n = (long long)g.nx * g.ny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % g.nx), y = (int)(id / g.nx);
    if (i == 0) {
      b.f32[id] = (float)in[id];
    } else {
      const long long dst = wrapped(g, x + cx(i), y + cy(i));
      const float want = (float)in[dst];
      b.dev[(long long)(i - 1) * g.ps + id] = Dev<ST>::store(want - (float)wgt(i) * b.f32[g.ps + dst]);
    }
  }
}

// Deviation storage, last pass of a state transfer: the rest population takes phi
// minus the moving populations as a reader rebuilds them, so the 16-bit rounding of
// the deviations does not change the mass (sum_i f_i(y) = phi(y) to FP32 rounding).
template <int ST>
__global__ void close_rest_kernel(const double* __restrict__ phi, Buf b, Grid g) {
  const long long n = (long long)g.nx * g.ny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % g.nx), y = (int)(id / g.nx);
    float moving = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) moving += (float)pulled<ST>(b, g, i, x, y);
    b.f32[id] = (float)(phi[id] - (double)moving);
  }
}

// Anchor plane (FP32) = mu_alpha of an FP64 mu plane.
__global__ void anchor_kernel(const double* __restrict__ mua, Buf b, Grid g) {
  const long long n = (long long)g.nx * g.ny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x)
    b.f32[g.ps + id] = (float)mua[id];
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = 0.0;
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  }
  return v;  // valid in thread 0
}

// phi = sum_i f_i (Eq. 22) per node into phi (FP64, for host transfer) or phi_f (FP32,
// for the energy). Rows are spread over blocks and columns over threads.
template <int ST>
__global__ void phi_kernel(Buf b, Grid g, double* __restrict__ phi_d, float* __restrict__ phi_f) {
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x)
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const long long id = (long long)y * g.nx + x;
      if (phi_d) {  // compensated FP32 sum (FP64 adds run at a small fraction of the FP32 rate)
        KahanF32 p;
#pragma unroll
        for (int i = 0; i < 9; ++i) p.add(pulled_f<ST>(b, g, i, x, y));
        phi_d[id] = p.value();
      } else {
        float p = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) p += pulled_f<ST>(b, g, i, x, y);
        phi_f[id] = p;
      }
    }
}

// Total mass sum_x phi(x). Streaming only permutes populations, so this is the sum of
// every stored population, no pull needed: 9 FP32 planes, or for 16-bit deviations
// sum_x [f*_0 + (1 - w_0) anchor + sum_i d_i] (w_i anchor(x) summed over i >= 1).
// Per-thread compensated FP32 sums, FP64 block sums to partial[blockIdx.x].
template <int ST>
__global__ void mass_kernel(Buf b, Grid g, double* __restrict__ partial) {
  __shared__ double sh[AUX_THREADS / 32];
  const long long n = (long long)g.nx * g.ny;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n4 = n / 4;  // float4 / 4-value chunks per plane (planes are 256-byte aligned)
  KahanF32 main, anchor;
  auto add_f32_plane = [&](const float* p, KahanF32& k) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
    for (long long q = t0; q < n4; q += stride) {
      const float4 v = __ldg(p4 + q);
      k.add(v.x); k.add(v.y); k.add(v.z); k.add(v.w);
    }
    for (long long q = 4 * n4 + t0; q < n; q += stride) k.add(__ldg(p + q));
  };
  if constexpr (ST == ST_F32) {
    for (int i = 0; i < 9; ++i) add_f32_plane(b.f32 + (long long)i * g.ps, main);
  } else {
    add_f32_plane(b.f32, main);
    add_f32_plane(b.f32 + g.ps, anchor);
    for (int i = 0; i < 8; ++i) {
      const uint16_t* d = b.dev + (long long)i * g.ps;
      const uint2* d4 = reinterpret_cast<const uint2*>(d);
      for (long long q = t0; q < n4; q += stride) {
        const uint2 v = __ldg(d4 + q);
        main.add(Dev<ST>::load(static_cast<uint16_t>(v.x & 0xffffu)));
        main.add(Dev<ST>::load(static_cast<uint16_t>(v.x >> 16)));
        main.add(Dev<ST>::load(static_cast<uint16_t>(v.y & 0xffffu)));
        main.add(Dev<ST>::load(static_cast<uint16_t>(v.y >> 16)));
      }
      for (long long q = 4 * n4 + t0; q < n; q += stride) main.add(Dev<ST>::load(__ldg(d + q)));
    }
  }
  double acc = main.value() + (1.0 - wgt(0)) * anchor.value();
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

struct EnergyConsts {
  float k, beta, beta4, alpha, half_eps, cw;
};

// Free-energy density (Eq. 7 with Eq. 9 or Eq. 8; stencils of Eq. 26; the n = 0,
// gamma = 1 guard where |grad phi|^2 < 1e-12) in FP32, block sums in FP64.
__global__ void energy_kernel(const float* __restrict__ phi, Grid g, EnergyConsts c,
                              double* __restrict__ partial) {
  __shared__ double sh[AUX_THREADS / 32];
  double acc = 0.0;
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x) {
    const long long rm = (long long)(y == 0 ? g.ny - 1 : y - 1) * g.nx;
    const long long r0 = (long long)y * g.nx;
    const long long rp = (long long)(y + 1 == g.ny ? 0 : y + 1) * g.nx;
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x + 1 == g.nx ? 0 : x + 1;
      const float p0 = phi[r0 + x];
      const float E = phi[r0 + xp], Wv = phi[r0 + xm], N = phi[rp + x], S = phi[rm + x];
      const float NE = phi[rp + xp], NW = phi[rp + xm], SW = phi[rm + xm], SE = phi[rm + xp];
      // Eq. 26a, 26b with the D2Q9 weights.
      const float gx = (E - Wv) * (1.0f / 3.0f) + ((NE - NW) + (SE - SW)) * (1.0f / 12.0f);
      const float gy = (N - S) * (1.0f / 3.0f) + ((NE - SE) + (NW - SW)) * (1.0f / 12.0f);
      const float lap = ((E + Wv) + (N + S)) * (2.0f / 3.0f) + ((NE + NW) + (SE + SW)) * (1.0f / 6.0f) -
                        p0 * (10.0f / 3.0f);
      const float g2 = fmaf(gx, gx, gy * gy);
      float gamma = 1.0f;
      if (g2 >= 1e-12f) {
        const float rs = rsqrtf(g2);
        const float n1 = gx * rs, n2 = gy * rs;
        const float n1s = n1 * n1, n2s = n2 * n2;
        gamma = fmaf(c.alpha, fmaf(4.0f, fmaf(n1s, n1s, n2s * n2s), -3.0f), 1.0f);
      }
      const float q = p0 * p0 - 1.0f;
      const float F = c.beta * q * q;                        // Eq. 4
      const float wv = fmaf(-c.cw, c.beta4 * p0 * q, lap);   // lap phi - f (Willmore) or lap phi
      const float e = fmaf(gamma, fmaf(0.5f * c.k, g2, F), c.half_eps * wv * wv);
      acc += (double)e;
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// The energy densities of energy_kernel and, beside them, the FP64 sum of phi itself (mass,
// Eq. 22), for a field given in FP32: partial_e[block] and partial_m[block].
__global__ void field_diag_kernel(const float* __restrict__ phi, Grid g, EnergyConsts c,
                                  double* __restrict__ partial_e, double* __restrict__ partial_m) {
  __shared__ double sh[AUX_THREADS / 32];
  double acc = 0.0, mass = 0.0;
  for (int y = blockIdx.x; y < g.ny; y += gridDim.x) {
    const long long rm = (long long)(y == 0 ? g.ny - 1 : y - 1) * g.nx;
    const long long r0 = (long long)y * g.nx;
    const long long rp = (long long)(y + 1 == g.ny ? 0 : y + 1) * g.nx;
    for (int x = threadIdx.x; x < g.nx; x += blockDim.x) {
      const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x + 1 == g.nx ? 0 : x + 1;
      const float p0 = phi[r0 + x];
      const float E = phi[r0 + xp], Wv = phi[r0 + xm], N = phi[rp + x], S = phi[rm + x];
      const float NE = phi[rp + xp], NW = phi[rp + xm], SW = phi[rm + xm], SE = phi[rm + xp];
      const float gx = (E - Wv) * (1.0f / 3.0f) + ((NE - NW) + (SE - SW)) * (1.0f / 12.0f);
      const float gy = (N - S) * (1.0f / 3.0f) + ((NE - SE) + (NW - SW)) * (1.0f / 12.0f);
      const float lap = ((E + Wv) + (N + S)) * (2.0f / 3.0f) + ((NE + NW) + (SE + SW)) * (1.0f / 6.0f) -
                        p0 * (10.0f / 3.0f);
      const float g2 = fmaf(gx, gx, gy * gy);
      float gamma = 1.0f;
      if (g2 >= 1e-12f) {
        const float rs = rsqrtf(g2);
        const float n1 = gx * rs, n2 = gy * rs;
        const float n1s = n1 * n1, n2s = n2 * n2;
        gamma = fmaf(c.alpha, fmaf(4.0f, fmaf(n1s, n1s, n2s * n2s), -3.0f), 1.0f);
      }
      const float q = p0 * p0 - 1.0f;
      const float F = c.beta * q * q;
      const float wv = fmaf(-c.cw, c.beta4 * p0 * q, lap);
      const float e = fmaf(gamma, fmaf(0.5f * c.k, g2, F), c.half_eps * wv * wv);
      acc += (double)e;
      mass += (double)p0;
    }
  }
  acc = block_sum(acc, sh);
  __syncthreads();  // warp 0 has read sh before the second sum reuses it
  mass = block_sum(mass, sh);
  if (threadIdx.x == 0) {
    partial_e[blockIdx.x] = acc;
    partial_m[blockIdx.x] = mass;
  }
}

// out[0] = sum of partial[0..n) in a fixed order (deterministic for a fixed n).
__global__ void final_sum_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double sh[1024 / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) out[0] = v;
}

// out[0] = sum of a[0..n), out[1] = sum of b[0..n): block 0 and block 1 of one launch, each in
// the order of final_sum_kernel.
__global__ void final_sum_pair_kernel(const double* __restrict__ a, const double* __restrict__ b, int n,
                                      double* __restrict__ out) {
  __shared__ double sh[1024 / 32];
  const double* p = blockIdx.x == 0 ? a : b;
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

}  // namespace lbch
