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

// Canonical f_i at node (x, y): f*_i of the node the population came from.
template <int ST>
__device__ __forceinline__ double pulled(const Buf& b, const Grid& g, int i, int x, int y) {
  const long long s = wrapped(g, x - cx(i), y - cy(i));
  if constexpr (ST == ST_F32) {
    return (double)b.f32[(long long)i * g.ps + s];
  } else {
    if (i == 0) return (double)b.f32[s];
    return (double)fmaf((float)wgt(i), b.f32[g.ps + s], Dev<ST>::load(b.dev[(long long)(i - 1) * g.ps + s]));
  }
}

// mu_alpha = f(phi) - k lap phi (Eq. 16, Eq. 26b) in FP64 from an FP64 phi plane;
// flags non-finite phi.
__global__ void mu_alpha_kernel(const double* __restrict__ phi, double* __restrict__ mua, Grid g,
                                double k, double beta4, int* bad) {
  const long long n = (long long)g.nx * g.ny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % g.nx), y = (int)(id / g.nx);
    const double c = phi[id];
    double lap = 0.0;
#pragma unroll
    for (int i = 1; i < 9; ++i) lap += 2.0 * wgt(i) * (phi[wrapped(g, x + cx(i), y + cy(i))] - c);
    lap *= 3.0;
    mua[id] = beta4 * c * (c * c - 1.0) - k * lap;
    if (!isfinite(c)) atomicOr(bad, 1);
  }
}

// f = f^eq(phi0, mu_alpha) (Eq. 18) written in the step kernel's pre-streaming form.
template <int ST>
__global__ void init_state_kernel(const double* __restrict__ phi0, const double* __restrict__ mua,
                                  Buf b, Grid g) {
  const long long n = (long long)g.nx * g.ny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % g.nx), y = (int)(id / g.nx);
    const double m = mua[id];
    const double rest = phi0[id] + (wgt(0) - 1.0) * m;
    if constexpr (ST == ST_F32) {
      b.f32[id] = (float)rest;
#pragma unroll
      for (int i = 1; i < 9; ++i)  // f*_i(y) must stream to f_i(y + c_i) = w_i mu_alpha(y + c_i)
        b.f32[(long long)i * g.ps + id] = (float)(wgt(i) * mua[wrapped(g, x + cx(i), y + cy(i))]);
    } else {
      b.f32[id] = (float)rest;
      b.f32[g.ps + id] = (float)m;
      const float mf = (float)m;
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        // Reader rebuilds w_i anchor(y) + d_i(y); it must give w_i mu_alpha(y + c_i).
        const float want = (float)(wgt(i) * mua[wrapped(g, x + cx(i), y + cy(i))]);
        b.dev[(long long)(i - 1) * g.ps + id] = Dev<ST>::store(want - (float)wgt(i) * mf);
      }
    }
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

// Deviation storage from one canonical plane: rest population as is; moving
// populations as deviations from w_i times the anchor already in plane 1.
template <int ST>
__global__ void set_plane_dev_kernel(const double* __restrict__ in, Buf b, Grid g, int i) {
  const long long n = (long long)g.nx * g.ny;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % g.nx), y = (int)(id / g.nx);
    if (i == 0) {
      b.f32[id] = (float)in[id];
    } else {
      const float want = (float)in[wrapped(g, x + cx(i), y + cy(i))];
      b.dev[(long long)(i - 1) * g.ps + id] = Dev<ST>::store(want - (float)wgt(i) * b.f32[g.ps + id]);
    }
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

// phi = sum_i f_i (Eq. 22) per node, summed in FP64; optionally written out as FP64
// (phi_d) or FP32 (phi_f); block partial sums of phi go to partial[blockIdx.x].
template <int ST>
__global__ void phi_kernel(Buf b, Grid g, double* __restrict__ phi_d, float* __restrict__ phi_f,
                           double* __restrict__ partial) {
  __shared__ double sh[AUX_THREADS / 32];
  const long long n = (long long)g.nx * g.ny;
  double acc = 0.0;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % g.nx), y = (int)(id / g.nx);
    double p = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) p += pulled<ST>(b, g, i, x, y);
    if (phi_d) phi_d[id] = p;
    if (phi_f) phi_f[id] = (float)p;
    acc += p;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0 && partial) partial[blockIdx.x] = acc;
}

struct EnergyConsts {
  float k, beta, beta4, alpha, half_eps, cw;
};

// Free-energy density (Eq. 7 with Eq. 9 or Eq. 8; stencils of Eq. 26; the n = 0,
// gamma = 1 guard where |grad phi|^2 < 1e-24) in FP32, block sums in FP64.
__global__ void energy_kernel(const float* __restrict__ phi, Grid g, EnergyConsts c,
                              double* __restrict__ partial) {
  __shared__ double sh[AUX_THREADS / 32];
  const long long n = (long long)g.nx * g.ny;
  double acc = 0.0;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(id % g.nx), y = (int)(id / g.nx);
    const float p0 = phi[id];
    float gx = 0.0f, gy = 0.0f, lap = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const float v = phi[wrapped(g, x + cx(i), y + cy(i))];
      const float w3 = 3.0f * (float)wgt(i);
      gx = fmaf(w3 * cx(i), v, gx);
      gy = fmaf(w3 * cy(i), v, gy);
      lap = fmaf(2.0f * w3, v - p0, lap);
    }
    const float g2 = fmaf(gx, gx, gy * gy);
    float gamma = 1.0f;
    if (g2 >= 1e-24f) {
      const float rs = rsqrtf(g2);
      const float n1 = gx * rs, n2 = gy * rs;
      const float n1s = n1 * n1, n2s = n2 * n2;
      gamma = fmaf(c.alpha, fmaf(4.0f, fmaf(n1s, n1s, n2s * n2s), -3.0f), 1.0f);
    }
    const float q = p0 * p0 - 1.0f;
    const float F = c.beta * q * q;              // Eq. 4
    const float wv = fmaf(-c.cw, c.beta4 * p0 * q, lap);  // lap phi - f (Willmore) or lap phi
    const float e = fmaf(gamma, fmaf(0.5f * c.k, g2, F), c.half_eps * wv * wv);
    acc += (double)e;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// out[0] = sum of partial[0..n) in a fixed order (deterministic for a fixed n).
__global__ void final_sum_kernel(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double sh[1024 / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += partial[i];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) out[0] = v;
}

}  // namespace lbch
