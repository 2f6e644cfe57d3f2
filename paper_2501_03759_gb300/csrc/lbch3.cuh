// 3D time step on the D3Q15 lattice (the C-ABI of include/lbch3.h), included at the
// end of lbch_api.cu.
//
// One step is four kernels over the periodic grid, each one thread per node with
// rows (y, z) across blocks and x across threads:
//   phi3_kernel      f_in,i(x) = f*_i(x - c_i); phi = sum_i f_in,i            (Eqs. 17, 22)
//   point3_kernel    grad phi, lap phi (Eq. 26, D3Q15 weights), n, gamma(n) (Eqs. 3, 6),
//                    Q (Eq. 15 reading), w, mu_alpha (Eq. 16), local part of mu_beta
//   mub3_kernel      mu_beta = local - div Q + eps lap w                         (Eqs. 13, 16)
//   collide3_kernel  g = grad mu_beta; MRT collision in the Eq. 24 moment basis;
//                    store f* (Eqs. 17-19, 25)
// Intermediate fields live in the workspace, so the step moves more than the 120
// bytes per node the populations need; the 2D path is the fused one.
#pragma once

namespace lbch3 {

// Eq. 21a (c = 1) and Eq. 21b.
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 14) ? 1 : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 13) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 3 || i == 7 || i == 9 || i == 12 || i == 13) ? 1 : ((i == 4 || i == 8 || i == 10 || i == 11 || i == 14) ? -1 : 0);
}
__host__ __device__ constexpr int cz(int i) {
  return (i == 5 || i == 7 || i == 10 || i == 11 || i == 13) ? 1 : ((i == 6 || i == 8 || i == 9 || i == 12 || i == 14) ? -1 : 0);
}
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0); }

// Row k of the Eq. 24 moment basis at velocity i, as the function of c it names.
__host__ __device__ constexpr int mrow(int k, int i) {
  const int x = cx(i), y = cy(i), z = cz(i), c2 = x * x + y * y + z * z;
  return k == 0 ? 1
       : k == 1 ? c2 - 2
       : k == 2 ? (15 * c2 * c2 - 55 * c2 + 32) / 2
       : k == 3 ? x
       : k == 4 ? (5 * c2 - 13) * x / 2
       : k == 5 ? y
       : k == 6 ? (5 * c2 - 13) * y / 2
       : k == 7 ? z
       : k == 8 ? (5 * c2 - 13) * z / 2
       : k == 9 ? 3 * x * x - c2
       : k == 10 ? y * y - z * z
       : k == 11 ? x * y
       : k == 12 ? y * z
       : k == 13 ? x * z
       : x * y * z;
}
__host__ __device__ constexpr int mnorm(int k) {
  int s = 0;
  for (int i = 0; i < 15; ++i) s += mrow(k, i) * mrow(k, i);
  return s;
}

struct Grid3 {
  int nx, ny, nz;
  long long ps;  // plane stride (elements)
};

struct Consts3 {
  float k, kq, kiso, beta4, beta12, alpha, a16, eps, cw, cfp, cnk;
  float s[15];
};

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ long long node(const Grid3& g, int x, int y, int z) {
  return ((long long)wrapi(z, g.nz) * g.ny + wrapi(y, g.ny)) * g.nx + wrapi(x, g.nx);
}

// Gradient (Eq. 26a) and Laplacian (Eq. 26b) of an FP32 field at (x, y, z). The
// gradient pairs opposite neighbours (c_{2j+1} = -c_{2j+2} in Eq. 21a), so each term is
// an exact difference and a locally uniform field gives exactly zero; the Laplacian
// sums differences from the centre.
__device__ __forceinline__ void stencil(const float* __restrict__ v, const Grid3& g, int x, int y, int z,
                                        float& gx, float& gy, float& gz, float& lap) {
  const float c = v[node(g, x, y, z)];
  float t[15];
#pragma unroll
  for (int i = 1; i < 15; ++i) t[i] = v[node(g, x + cx(i), y + cy(i), z + cz(i))];
  float sx = 0.0f, sy = 0.0f, sz = 0.0f, sl = 0.0f;
#pragma unroll
  for (int i = 1; i < 15; i += 2) {  // pairs (i, i+1) with c_{i+1} = -c_i
    const float d = t[i] - t[i + 1];
    const float w = (float)(3.0 * wgt(i));
    if (cx(i) != 0) sx = fmaf(w * cx(i), d, sx);
    if (cy(i) != 0) sy = fmaf(w * cy(i), d, sy);
    if (cz(i) != 0) sz = fmaf(w * cz(i), d, sz);
    sl = fmaf(2.0f * w, (t[i] - c) + (t[i + 1] - c), sl);
  }
  gx = sx;
  gy = sy;
  gz = sz;
  lap = sl;
}

#define LBCH3_FOR_NODES(g)                                                         \
  for (long long row = blockIdx.x; row < (long long)(g).ny * (g).nz; row += gridDim.x) \
    for (int x = threadIdx.x; x < (g).nx; x += blockDim.x)

__global__ void phi3_kernel(const float* __restrict__ f, Grid3 g, float* __restrict__ phi) {
  LBCH3_FOR_NODES(g) {
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    float p = 0.0f;
#pragma unroll
    for (int i = 0; i < 15; ++i) p += f[(long long)i * g.ps + node(g, x - cx(i), y - cy(i), z - cz(i))];
    phi[row * g.nx + x] = p;
  }
}

__global__ void point3_kernel(const float* __restrict__ phi, Grid3 g, Consts3 c, float* __restrict__ Qx,
                              float* __restrict__ Qy, float* __restrict__ Qz, float* __restrict__ W,
                              float* __restrict__ A, float* __restrict__ mua) {
  LBCH3_FOR_NODES(g) {
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    const long long id = row * g.nx + x;
    float dx, dy, dz, lap;
    stencil(phi, g, x, y, z, dx, dy, dz, lap);
    const float g2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool ok = g2 >= 1e-12f;  // n = 0, gamma = 1 below this
    const float rs = rsqrtf(ok ? g2 : 1.0f);
    const float n1 = dx * rs, n2 = dy * rs, n3 = dz * rs;  // Eq. 3
    const float n1s = n1 * n1, n2s = n2 * n2, n3s = n3 * n3;
    const float S4 = fmaf(n1s, n1s, fmaf(n2s, n2s, n3s * n3s));
    const float gm1 = ok ? c.alpha * fmaf(4.0f, S4, -3.0f) : 0.0f;  // gamma - 1, Eq. 6
    const float t = ok ? c.kq * c.a16 * (g2 * rs) : 0.0f;         // k_q |grad phi| 16 alpha
    const float kg = fmaf(c.k, gm1, c.kiso);
    Qx[id] = fmaf(kg, dx, t * (n1 * (n1s - S4)));  // P grad_n gamma = 16 alpha n (n^2 - sum n^4)
    Qy[id] = fmaf(kg, dy, t * (n2 * (n2s - S4)));
    Qz[id] = fmaf(kg, dz, t * (n3 * (n3s - S4)));
    const float p = phi[id], p2 = p * p;
    const float fb = c.beta4 * p * (p2 - 1.0f);
    const float fp = fmaf(c.beta12, p2, -c.beta4);
    const float w = fmaf(-c.cw, fb, lap);
    W[id] = w;
    mua[id] = fmaf(-c.k, lap, fb);
    A[id] = fmaf(gm1, fb, fmaf(-c.cfp * fp, w, c.cnk * lap));
  }
}

__global__ void mub3_kernel(const float* __restrict__ Qx, const float* __restrict__ Qy,
                            const float* __restrict__ Qz, const float* __restrict__ W,
                            const float* __restrict__ A, Grid3 g, float eps, float* __restrict__ mub) {
  LBCH3_FOR_NODES(g) {
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    float ax, ay, az, al, bx, by, bz, bl, qx, qy, qz, ql, wx, wy, wz, wl;
    stencil(Qx, g, x, y, z, ax, ay, az, al);
    stencil(Qy, g, x, y, z, bx, by, bz, bl);
    stencil(Qz, g, x, y, z, qx, qy, qz, ql);
    stencil(W, g, x, y, z, wx, wy, wz, wl);
    const long long id = row * g.nx + x;
    mub[id] = A[id] - (ax + by + qz) + eps * wl;
  }
}

__global__ void collide3_kernel(const float* __restrict__ src, const float* __restrict__ mub,
                                const float* __restrict__ mua, Grid3 g, Consts3 c, float* __restrict__ dst) {
  LBCH3_FOR_NODES(g) {
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    const long long id = row * g.nx + x;
    float gx, gy, gz, unused;
    stencil(mub, g, x, y, z, gx, gy, gz, unused);
    float f[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) f[i] = src[(long long)i * g.ps + node(g, x - cx(i), y - cy(i), z - cz(i))];
    float phi = 0.0f;
#pragma unroll
    for (int i = 0; i < 15; ++i) phi += f[i];
    const float m_a = mua[id];
    // Moments, their equilibria (Eq. 18) and the source moments (Eq. 19) in closed form:
    // m^eq = (phi, -2 phi + mu_a, 16 phi - 15 mu_a, 0, ...); F_m nonzero on j and q.
    float nk[15];
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      float m = 0.0f;
#pragma unroll
      for (int i = 0; i < 15; ++i)
        if (mrow(k, i) != 0) m = fmaf((float)mrow(k, i), f[i], m);
      const float meq = k == 0 ? phi : (k == 1 ? fmaf(-2.0f, phi, m_a) : (k == 2 ? fmaf(16.0f, phi, -15.0f * m_a) : 0.0f));
      const float gk = (k == 3 || k == 4) ? gx : ((k == 5 || k == 6) ? gy : gz);
      const float Fm = (k == 3 || k == 5 || k == 7) ? -gk * (1.0f / 3.0f)
                     : (k == 4 || k == 6 || k == 8) ? gk * (7.0f / 9.0f) : 0.0f;
      const float ms = fmaf(-c.s[k], m - meq, m) + (1.0f - 0.5f * c.s[k]) * Fm;  // Eq. 17 in moments
      nk[k] = ms * (1.0f / (float)mnorm(k));
    }
    float o[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) {
      float v = 0.0f;
#pragma unroll
      for (int k = 0; k < 15; ++k)
        if (mrow(k, i) != 0) v = fmaf((float)mrow(k, i), nk[k], v);
      o[i] = v;
    }
    // Rest population closes the mass exactly (sum_i f* = sum_i f, Eq. 34).
    float d = 0.0f;
#pragma unroll
    for (int i = 1; i < 15; ++i) d += f[i] - o[i];
    o[0] = f[0] + d;
#pragma unroll
    for (int i = 0; i < 15; ++i) dst[(long long)i * g.ps + id] = o[i];
  }
}

__global__ void mu_alpha3_kernel(const double* __restrict__ phi, double* __restrict__ mua, Grid3 g, double k,
                                 double beta4, int* bad) {
  LBCH3_FOR_NODES(g) {
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    const long long id = row * g.nx + x;
    const double c = phi[id];
    double lap = 0.0;
#pragma unroll
    for (int i = 1; i < 15; ++i) lap += 2.0 * wgt(i) * (phi[node(g, x + cx(i), y + cy(i), z + cz(i))] - c);
    lap *= 3.0;
    mua[id] = beta4 * c * (c * c - 1.0) - k * lap;
    if (!isfinite(c)) atomicOr(bad, 1);
  }
}

// f = f^eq(phi0, mu_alpha) in the pre-streaming form (f*_i(x) streams to f_i(x + c_i)).
__global__ void init3_kernel(const double* __restrict__ phi0, const double* __restrict__ mua, Grid3 g,
                             float* __restrict__ f) {
  LBCH3_FOR_NODES(g) {
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    const long long id = row * g.nx + x;
    f[id] = (float)(phi0[id] + (wgt(0) - 1.0) * mua[id]);
#pragma unroll
    for (int i = 1; i < 15; ++i)
      f[(long long)i * g.ps + id] = (float)(wgt(i) * mua[node(g, x + cx(i), y + cy(i), z + cz(i))]);
  }
}

__global__ void phi3_f64_kernel(const float* __restrict__ f, Grid3 g, double* __restrict__ phi) {
  LBCH3_FOR_NODES(g) {
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    double p = 0.0;
#pragma unroll
    for (int i = 0; i < 15; ++i) p += (double)f[(long long)i * g.ps + node(g, x - cx(i), y - cy(i), z - cz(i))];
    phi[row * g.nx + x] = p;
  }
}

__global__ void mass3_kernel(const float* __restrict__ f, Grid3 g, double* __restrict__ partial) {
  __shared__ double sh[lbch::AUX_THREADS / 32];
  const long long n = (long long)g.nx * g.ny * g.nz;
  lbch::KahanF32 k;
  for (int i = 0; i < 15; ++i)
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
      k.add(f[(long long)i * g.ps + q]);
  const double acc = lbch::block_sum(k.value(), sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void energy3_kernel(const float* __restrict__ phi, Grid3 g, lbch::EnergyConsts c,
                               double* __restrict__ partial) {
  __shared__ double sh[lbch::AUX_THREADS / 32];
  double acc = 0.0;
  LBCH3_FOR_NODES(g) {
    const int y = (int)(row % g.ny), z = (int)(row / g.ny);
    float dx, dy, dz, lap;
    stencil(phi, g, x, y, z, dx, dy, dz, lap);
    const float p0 = phi[row * g.nx + x];
    const float g2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float gamma = 1.0f;
    if (g2 >= 1e-12f) {
      const float rs = rsqrtf(g2);
      const float a = dx * rs, b = dy * rs, e = dz * rs;
      gamma = fmaf(c.alpha, fmaf(4.0f, fmaf(a * a, a * a, fmaf(b * b, b * b, e * e * e * e)), -3.0f), 1.0f);
    }
    const float q = p0 * p0 - 1.0f;
    const float F = c.beta * q * q;
    const float wv = fmaf(-c.cw, c.beta4 * p0 * q, lap);
    acc += (double)fmaf(gamma, fmaf(0.5f * c.k, g2, F), c.half_eps * wv * wv);
  }
  acc = lbch::block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

}  // namespace lbch3

struct lbch3_ctx {
  lbch3_params p;
  double k, beta, s[15];
  cudaStream_t stream;
  lbch3::Grid3 g;
  lbch3::Consts3 cs;
  float* buf[2];
  int cur;
  float *phi, *Qx, *Qy, *Qz, *W, *A, *mua, *mub;
  double* stage;
  double* partial;
  double* result;
  int* flags;
  int blocks;      // row-blocks for the node kernels
  int red_blocks;  // blocks for the reductions
  bool has_state, failed;
  char err[512];
};

namespace {

const char* check3(const lbch3_params* p) {
  if (!p) return "params is NULL";
  if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nx > 4096 || p->ny > 4096 || p->nz > 4096)
    return "nx, ny, nz must be in [1, 4096]";
  if ((long long)p->nx * p->ny * p->nz >= (1LL << 31)) return "nx*ny*nz must be < 2^31";
  if (!(p->M > 0.0) || !std::isfinite(p->M) || !(p->sigma > 0.0) || !(p->D > 0.0) || !(p->eps >= 0.0))
    return "M, sigma, D must be > 0 and eps >= 0";
  if (!(p->alpha >= 0.0 && p->alpha < 1.0)) return "alpha must be in [0, 1)";
  if (p->regularization < LBCH_REG_NONE || p->regularization > LBCH_REG_LINEAR) return "unknown regularization";
  if (p->flags & ~(unsigned)(LBCH_Q_LITERAL | LBCH_MU_NESTED | LBCH_S35_EXPLICIT)) return "unknown flag bits";
  for (int i = 1; i < 15; ++i) {
    if ((i == 3 || i == 5 || i == 7) && !(p->flags & LBCH_S35_EXPLICIT)) continue;
    if (!(p->s[i] > 0.0 && p->s[i] < 2.0)) return "relaxation rates s_1..s_14 must lie in (0, 2)";
  }
  return nullptr;
}

long long ps3(const lbch3_params* p) { return ((long long)p->nx * p->ny * p->nz + 63) / 64 * 64; }

bool cuda3_failed(lbch3_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return false;
  c->failed = true;
  snprintf(c->err, sizeof(c->err), "%s: %s", what, cudaGetErrorString(e));
  return true;
}

lbch_status pre3(lbch3_ctx* c, bool need_state) {
  if (!c) return LBCH_EINVAL;
  if (c->failed) return LBCH_ESTATE;
  if (need_state && !c->has_state) {
    snprintf(c->err, sizeof(c->err), "no state: call lbch3_init_field first");
    return LBCH_EINVAL;
  }
  return LBCH_OK;
}

lbch_status sync3(lbch3_ctx* c, const char* what) {
  if (cuda3_failed(c, cudaGetLastError(), what)) return LBCH_ECUDA;
  if (cuda3_failed(c, cudaStreamSynchronize(c->stream), what)) return LBCH_ECUDA;
  return LBCH_OK;
}

}  // namespace

extern "C" {

size_t lbch3_workspace_bytes(const lbch3_params* p) {
  if (check3(p)) return 0;
  const size_t ps = (size_t)ps3(p);
  return 2 * align_up(ps * 15 * sizeof(float)) + 8 * align_up(ps * sizeof(float)) + align_up(ps * sizeof(double)) +
         align_up(MAX_RED_BLOCKS * sizeof(double)) + align_up(8 * sizeof(double)) + align_up(16 * sizeof(int));
}

lbch_status lbch3_create(const lbch3_params* p, void* d_workspace, size_t bytes, void* cuda_stream, lbch3_ctx** out) {
  if (!out || check3(p)) return LBCH_EINVAL;
  const size_t need = lbch3_workspace_bytes(p);
  if (!d_workspace || bytes < need || ((uintptr_t)d_workspace % ALIGN) != 0) return LBCH_ENOMEM;
  lbch3_ctx* c = new (std::nothrow) lbch3_ctx();
  if (!c) return LBCH_ENOMEM;
  c->p = *p;
  c->beta = 3.0 * p->sigma / (4.0 * p->D);  // Eq. 5
  c->k = 3.0 * p->sigma * p->D / 8.0;
  for (int i = 0; i < 15; ++i) c->s[i] = p->s[i];
  if (!(p->flags & LBCH_S35_EXPLICIT)) c->s[3] = c->s[5] = c->s[7] = 1.0 / (3.0 * p->M + 0.5);
  c->stream = (cudaStream_t)cuda_stream;
  const long long ps = ps3(p);
  c->g = lbch3::Grid3{p->nx, p->ny, p->nz, ps};
  char* q = (char*)d_workspace;
  for (int b = 0; b < 2; ++b) {
    c->buf[b] = (float*)q;
    q += align_up((size_t)ps * 15 * sizeof(float));
  }
  float** planes[8] = {&c->phi, &c->Qx, &c->Qy, &c->Qz, &c->W, &c->A, &c->mua, &c->mub};
  for (float** pl : planes) {
    *pl = (float*)q;
    q += align_up((size_t)ps * sizeof(float));
  }
  c->stage = (double*)q;
  q += align_up((size_t)ps * sizeof(double));
  c->partial = (double*)q;
  q += align_up(MAX_RED_BLOCKS * sizeof(double));
  c->result = (double*)q;
  q += align_up(8 * sizeof(double));
  c->flags = (int*)q;
  const bool nested = p->flags & LBCH_MU_NESTED;
  const double eps = p->regularization == LBCH_REG_NONE ? 0.0 : p->eps;
  lbch3::Consts3& k = c->cs;
  k.k = (float)c->k;
  k.kq = (float)((p->flags & LBCH_Q_LITERAL) ? 1.0 : c->k);
  k.kiso = (float)(nested ? c->k : 0.0);
  k.beta4 = (float)(4.0 * c->beta);
  k.beta12 = (float)(12.0 * c->beta);
  k.alpha = (float)p->alpha;
  k.a16 = (float)(16.0 * p->alpha);
  k.eps = (float)eps;
  k.cw = p->regularization == LBCH_REG_LINEAR ? 0.0f : 1.0f;
  k.cfp = p->regularization == LBCH_REG_WILLMORE ? (float)eps : 0.0f;
  k.cnk = (float)(nested ? c->k : 0.0);
  for (int i = 0; i < 15; ++i) k.s[i] = (float)c->s[i];
  const long long rows = (long long)p->ny * p->nz;
  c->blocks = (int)(rows < (1LL << 30) ? rows : (1LL << 30));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long nn = (long long)p->nx * p->ny * p->nz;
  long long rb = (nn + AUX_THREADS - 1) / AUX_THREADS;
  const long long cap = (long long)(sms > 0 ? sms : 152) * 8 < MAX_RED_BLOCKS ? (long long)(sms > 0 ? sms : 152) * 8
                                                                              : MAX_RED_BLOCKS;
  c->red_blocks = (int)(rb < cap ? rb : cap);
  c->cur = 0;
  c->has_state = false;
  c->failed = false;
  c->err[0] = 0;
  *out = c;
  return LBCH_OK;
}

lbch_status lbch3_init_field(lbch3_ctx* c, const double* h_phi0) {
  lbch_status st = pre3(c, false);
  if (st != LBCH_OK) return st;
  if (!h_phi0) return LBCH_EINVAL;
  const size_t n = (size_t)c->p.nx * c->p.ny * c->p.nz;
  c->has_state = false;
  double* mua = reinterpret_cast<double*>(c->Qx);  // Qx and Qy together hold one FP64 plane
  if (cuda3_failed(c, cudaMemcpyAsync(c->stage, h_phi0, n * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                   "init_field: copy") ||
      cuda3_failed(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "init_field: clear"))
    return LBCH_ECUDA;
  lbch3::mu_alpha3_kernel<<<c->blocks, 128, 0, c->stream>>>(c->stage, mua, c->g, c->k, 4.0 * c->beta, c->flags);
  lbch3::init3_kernel<<<c->blocks, 128, 0, c->stream>>>(c->stage, mua, c->g, c->buf[0]);
  int bad = 0;
  if (cuda3_failed(c, cudaMemcpyAsync(&bad, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "init_field"))
    return LBCH_ECUDA;
  if ((st = sync3(c, "init_field")) != LBCH_OK) return st;
  if (bad) {
    snprintf(c->err, sizeof(c->err), "init_field: phi0 holds NaN or Inf");
    return LBCH_ENONFINITE;
  }
  c->cur = 0;
  c->has_state = true;
  return LBCH_OK;
}

lbch_status lbch3_step(lbch3_ctx* c, int64_t n) {
  lbch_status st = pre3(c, true);
  if (st != LBCH_OK) return st;
  if (n < 0) return LBCH_EINVAL;
  const dim3 grid(c->blocks), block(128);
  for (int64_t t = 0; t < n; ++t) {
    const float* src = c->buf[c->cur];
    float* dst = c->buf[c->cur ^ 1];
    lbch3::phi3_kernel<<<grid, block, 0, c->stream>>>(src, c->g, c->phi);
    lbch3::point3_kernel<<<grid, block, 0, c->stream>>>(c->phi, c->g, c->cs, c->Qx, c->Qy, c->Qz, c->W, c->A, c->mua);
    lbch3::mub3_kernel<<<grid, block, 0, c->stream>>>(c->Qx, c->Qy, c->Qz, c->W, c->A, c->g, c->cs.eps, c->mub);
    lbch3::collide3_kernel<<<grid, block, 0, c->stream>>>(src, c->mub, c->mua, c->g, c->cs, dst);
    c->cur ^= 1;
  }
  if (cuda3_failed(c, cudaGetLastError(), "step: launch")) return LBCH_ECUDA;
  return LBCH_OK;
}

lbch_status lbch3_get_field(lbch3_ctx* c, double* h_phi) {
  lbch_status st = pre3(c, true);
  if (st != LBCH_OK) return st;
  if (!h_phi) return LBCH_EINVAL;
  const size_t n = (size_t)c->p.nx * c->p.ny * c->p.nz;
  lbch3::phi3_f64_kernel<<<c->blocks, 128, 0, c->stream>>>(c->buf[c->cur], c->g, c->stage);
  if (cuda3_failed(c, cudaMemcpyAsync(h_phi, c->stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                   "get_field: copy"))
    return LBCH_ECUDA;
  return sync3(c, "get_field");
}

lbch_status lbch3_mass(lbch3_ctx* c, double* out) {
  lbch_status st = pre3(c, true);
  if (st != LBCH_OK) return st;
  if (!out) return LBCH_EINVAL;
  lbch3::mass3_kernel<<<c->red_blocks, AUX_THREADS, 0, c->stream>>>(c->buf[c->cur], c->g, c->partial);
  final_sum_kernel<<<1, 1024, 0, c->stream>>>(c->partial, c->red_blocks, c->result);
  if (cuda3_failed(c, cudaMemcpyAsync(out, c->result, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "mass"))
    return LBCH_ECUDA;
  if ((st = sync3(c, "mass")) != LBCH_OK) return st;
  return std::isfinite(*out) ? LBCH_OK : LBCH_ENONFINITE;
}

lbch_status lbch3_free_energy(lbch3_ctx* c, double* out) {
  lbch_status st = pre3(c, true);
  if (st != LBCH_OK) return st;
  if (!out) return LBCH_EINVAL;
  lbch3::phi3_kernel<<<c->blocks, 128, 0, c->stream>>>(c->buf[c->cur], c->g, c->phi);
  EnergyConsts ec;
  const double eps = c->p.regularization == LBCH_REG_NONE ? 0.0 : c->p.eps;
  ec.k = (float)c->k;
  ec.beta = (float)c->beta;
  ec.beta4 = (float)(4.0 * c->beta);
  ec.alpha = (float)c->p.alpha;
  ec.half_eps = (float)(0.5 * eps);
  ec.cw = c->p.regularization == LBCH_REG_LINEAR ? 0.0f : 1.0f;
  lbch3::energy3_kernel<<<c->red_blocks, AUX_THREADS, 0, c->stream>>>(c->phi, c->g, ec, c->partial);
  final_sum_kernel<<<1, 1024, 0, c->stream>>>(c->partial, c->red_blocks, c->result + 1);
  if (cuda3_failed(c, cudaMemcpyAsync(out, c->result + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                   "free_energy"))
    return LBCH_ECUDA;
  if ((st = sync3(c, "free_energy")) != LBCH_OK) return st;
  return std::isfinite(*out) ? LBCH_OK : LBCH_ENONFINITE;
}

const char* lbch3_last_error(const lbch3_ctx* c) { return c ? c->err : "context is NULL"; }

void lbch3_destroy(lbch3_ctx* c) { delete c; }

}  // extern "C"
