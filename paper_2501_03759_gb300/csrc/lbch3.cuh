// 3D time step on the D3Q15 lattice (the C-ABI of include/lbch3.h), included at the
// end of lbch_api.cu.
//
// One step is three kernels over the periodic grid:
//   phi3_kernel      f_in,i(x) = f*_i(x - c_i); phi = sum_i f_in,i            (Eqs. 17, 22)
//   mu3_kernel       grad phi, lap phi (Eq. 26, D3Q15 weights), n, gamma(n) (Eqs. 3, 6),
//                    Q (Eq. 15 reading), w, mu_alpha (Eq. 16), then
//                    mu_beta = (gamma - 1) f - div Q + eps (lap w - f' w)     (Eqs. 13, 16)
//   collide3_kernel  g = grad mu_beta; MRT collision in the Eq. 24 moment basis;
//                    store f* (Eqs. 17-19, 25)
// phi3 and collide3 run one thread per node, x across threads. mu3 sweeps z through an
// x-y tile: each plane of phi and of (Q, w) passes once through shared memory and every
// thread keeps its column's partial stencil sums in registers. The intermediate fields
// that reach HBM are phi, mu_alpha and mu_beta (12 bytes written, about 14 read per
// node) besides the 120 bytes of populations.
#pragma once

namespace lbch3 {

// Eq. 21a (c = 1) and Eq. 21b.
__host__ __device__ __forceinline__ constexpr int cx(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 14) ? 1 : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 13) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int cy(int i) {
  return (i == 3 || i == 7 || i == 9 || i == 12 || i == 13) ? 1 : ((i == 4 || i == 8 || i == 10 || i == 11 || i == 14) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int cz(int i) {
  return (i == 5 || i == 7 || i == 10 || i == 11 || i == 13) ? 1 : ((i == 6 || i == 8 || i == 9 || i == 12 || i == 14) ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr double wgt(int i) {
  return i == 0 ? 2.0 / 9.0 : (i <= 6 ? 1.0 / 9.0 : 1.0 / 72.0);
}

// Row k of the Eq. 24 moment basis at velocity i, as the function of c it names.
__host__ __device__ __forceinline__ constexpr int mrow(int k, int i) {
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

// The basis as a compile-time table, so that every entry the collision uses is a
// literal after unrolling (rows, and their squared norms for M^-1 = M^T diag(1/|M_k|^2)).
struct Basis3 {
  int m[15][15];
  int norm[15];
};
__host__ __device__ constexpr Basis3 make_basis3() {
  Basis3 b{};
  for (int k = 0; k < 15; ++k) {
    b.norm[k] = 0;
    for (int i = 0; i < 15; ++i) {
      b.m[k][i] = mrow(k, i);
      b.norm[k] += b.m[k][i] * b.m[k][i];
    }
  }
  return b;
}
constexpr Basis3 kBasis3 = make_basis3();
template <int K, int I>
struct MR {
  static constexpr int v = kBasis3.m[K][I];
};
template <int K>
struct MN {
  static constexpr int v = kBasis3.norm[K];
};

struct Grid3 {
  int nx, ny, nz;
  int segs;      // x segments of NX3 nodes per row (node kernels)
  long long ps;  // plane stride (elements)
};

constexpr int NX3 = 128;  // threads per block of the node kernels, along x

struct Consts3 {
  float k, kq, kiso, beta4, beta12, alpha, a16, eps, cw, cfp, cnk;
  float s[15];
};

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
__device__ __forceinline__ int modn(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// A node and the offsets of its neighbours (x fastest; 32-bit, since n < 2^31).
struct Site {
  int x, y, z, id;
  int xo[3];     // x - 1, x, x + 1 (periodic)
  int ro[3][3];  // (z + dz) ny nx + (y + dy) nx for dy, dz in {-1, 0, 1} (periodic)
  __device__ __forceinline__ int at(int dx, int dy, int dz) const { return ro[dy + 1][dz + 1] + xo[dx + 1]; }
};

// The node of this thread in node-kernel block b (x segment fastest, then y, then z);
// false past the end of the row.
__device__ __forceinline__ bool site_of(const Grid3& g, int b, Site& s) {
  const int seg = b % g.segs, row = b / g.segs;
  s.x = seg * NX3 + (int)threadIdx.x;
  if (s.x >= g.nx) return false;
  s.y = row % g.ny;
  s.z = row / g.ny;
  s.xo[0] = s.x == 0 ? g.nx - 1 : s.x - 1;
  s.xo[1] = s.x;
  s.xo[2] = s.x + 1 == g.nx ? 0 : s.x + 1;
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) s.ro[dy + 1][dz + 1] = (wrapi(s.z + dz, g.nz) * g.ny + wrapi(s.y + dy, g.ny)) * g.nx;
  s.id = s.ro[1][1] + s.x;
  return true;
}

// Gradient (Eq. 26a) and Laplacian (Eq. 26b) from the centre value c and the
// neighbour values t[i] = v(x + c_i), i = 1..14. The gradient pairs opposite
// velocities (c_{2j} = -c_{2j-1} in Eq. 21a), so each term is an exact difference and a
// locally uniform field gives exactly zero; the Laplacian sums differences from c.
__device__ __forceinline__ void grad_lap(float c, const float (&t)[15], float& gx, float& gy, float& gz, float& lap) {
  float sx = 0.0f, sy = 0.0f, sz = 0.0f, sl = 0.0f;
#pragma unroll
  for (int i = 1; i < 15; i += 2) {
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

__device__ __forceinline__ void stencil(const float* __restrict__ v, const Site& s, float& gx, float& gy, float& gz,
                                        float& lap) {
  float t[15];
#pragma unroll
  for (int i = 1; i < 15; ++i) t[i] = v[s.at(cx(i), cy(i), cz(i))];
  grad_lap(v[s.id], t, gx, gy, gz, lap);
}

// Population load with a 256-byte L2 fetch (.L2::256B): a block's 128 threads read 512
// contiguous bytes of each plane row (0.7636 -> 0.7602 ms per 256^3 step on GB300).
__device__ __forceinline__ float ld_pop(const float* p) {
  float v;
  asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

__global__ void __launch_bounds__(NX3) phi3_kernel(const float* __restrict__ f, Grid3 g, float* __restrict__ phi) {
  Site s;
  if (!site_of(g, blockIdx.x, s)) return;
  float p = 0.0f;
#pragma unroll
  for (int i = 0; i < 15; ++i) p += ld_pop(f + (long long)i * g.ps + s.at(-cx(i), -cy(i), -cz(i)));
  phi[s.id] = p;
}

// ---------------------------------------------------------------- mu3_kernel

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}

constexpr int MU_TX = 30, MU_TY = 14;                // mu_beta outputs per plane and tile
constexpr int MU_QX = MU_TX + 2, MU_QY = MU_TY + 2;  // (Q, w) region: one thread per column
constexpr int MU_PX = MU_TX + 4, MU_PY = MU_TY + 4;  // phi region
constexpr int MU_THREADS = 32 * MU_QY;
constexpr int MU_PHI_PER_THREAD = (MU_PX * MU_PY + MU_THREADS - 1) / MU_THREADS;
constexpr int MU_RING = 5;  // phi planes in shared memory: MU_RING - 1 in flight ahead of the sweep
static_assert(MU_QX == 32, "one lane per (Q, w) column");

// mu3_kernel's work list: tiles_x * tiles_y tiles, each a column of nz planes, in the
// order (tile, z); block b sweeps planes [b per_block, (b + 1) per_block) of that list.
struct MuTiles {
  int tiles_x, tiles_y;
  long long per_block;
};

// Anisotropic quantities at one node from its phi, grad phi and lap phi: Q (reading of
// Eq. 15 under LBCH_Q_LITERAL / LBCH_MU_NESTED), w = lap phi - f (Eq. 9; 0 for the
// linear regularisation), mu_alpha (Eq. 16) and the local part of mu_beta.
struct Aniso {
  float qx, qy, qz, w, mua, a;
};
__device__ __forceinline__ Aniso aniso(const Consts3& c, float p, float dx, float dy, float dz, float lap) {
  Aniso r;
  const float g2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const bool ok = g2 >= 1e-12f;  // n = 0, gamma = 1 below this
  const float rs = rsqrtf(ok ? g2 : 1.0f);
  const float n1 = dx * rs, n2 = dy * rs, n3 = dz * rs;  // Eq. 3
  const float n1s = n1 * n1, n2s = n2 * n2, n3s = n3 * n3;
  const float S4 = fmaf(n1s, n1s, fmaf(n2s, n2s, n3s * n3s));
  const float gm1 = ok ? c.alpha * fmaf(4.0f, S4, -3.0f) : 0.0f;  // gamma - 1, Eq. 6
  const float t = ok ? c.kq * c.a16 * (g2 * rs) : 0.0f;         // k_q |grad phi| 16 alpha
  const float kg = fmaf(c.k, gm1, c.kiso);
  r.qx = fmaf(kg, dx, t * (n1 * (n1s - S4)));  // P grad_n gamma = 16 alpha n (n^2 - sum n^4)
  r.qy = fmaf(kg, dy, t * (n2 * (n2s - S4)));
  r.qz = fmaf(kg, dz, t * (n3 * (n3s - S4)));
  const float p2 = p * p;
  const float fb = c.beta4 * p * (p2 - 1.0f);
  const float fp = fmaf(c.beta12, p2, -c.beta4);
  r.w = fmaf(-c.cw, fb, lap);
  r.mua = fmaf(-c.k, lap, fb);
  r.a = fmaf(gm1, fb, fmaf(-c.cfp * fp, r.w, c.cnk * lap));
  return r;
}

// Stencil weights of Eq. 26 on D3Q15: 3 w_i for the gradient, 6 w_i for the Laplacian.
constexpr float G1 = 3.0f / 9.0f, G7 = 3.0f / 72.0f, L1 = 6.0f / 9.0f, L7 = 6.0f / 72.0f;

// What one plane p of phi gives the stencils at (x, y): the centre c, the in-plane axis
// terms of the gradient and Laplacian at (x, y, p), and the sums over the four in-plane
// diagonal neighbours (x +- 1, y +- 1, p) that the corner velocities of planes p -+ 1
// use: X = sum s_x v, Y = sum s_y v, S = sum v. Differences and pair sums are formed
// first, so a locally uniform field gives exact zeros.
struct PhiPlane {
  float c, gx, gy, lap, X, Y, S;
};
__device__ __forceinline__ PhiPlane phi_plane(const float (*v)[MU_PX], int rx, int ry) {
  PhiPlane r;
  const float c = v[ry][rx], e = v[ry][rx + 1], w = v[ry][rx - 1], n = v[ry + 1][rx], s = v[ry - 1][rx];
  const float ne = v[ry + 1][rx + 1], nw = v[ry + 1][rx - 1], se = v[ry - 1][rx + 1], sw = v[ry - 1][rx - 1];
  r.c = c;
  r.gx = G1 * (e - w);
  r.gy = G1 * (n - s);
  r.lap = L1 * (((e - c) + (w - c)) + ((n - c) + (s - c)));
  r.X = (ne - nw) + (se - sw);
  r.Y = (ne - se) + (nw - sw);
  r.S = (ne + nw) + (se + sw);
  return r;
}

// The same for one plane of (Q_x, Q_y, Q_z, w): in-plane parts of div Q and lap w, the
// diagonal sums X = sum s_x Q_x, Y = sum s_y Q_y, Z = sum Q_z, W = sum w, and the centre
// Q_z and w.
struct QPlane {
  float div, lapw, X, Y, Z, W, qz, w;
};
__device__ __forceinline__ QPlane q_plane(const float (*q)[MU_QY][MU_QX], int rx, int ry) {
  QPlane r;
  const float (*Qx)[MU_QX] = q[0];
  const float (*Qy)[MU_QX] = q[1];
  const float (*Qz)[MU_QX] = q[2];
  const float (*W)[MU_QX] = q[3];
  const float wc = W[ry][rx];
  r.div = G1 * ((Qx[ry][rx + 1] - Qx[ry][rx - 1]) + (Qy[ry + 1][rx] - Qy[ry - 1][rx]));
  r.lapw = L1 * (((W[ry][rx + 1] - wc) + (W[ry][rx - 1] - wc)) + ((W[ry + 1][rx] - wc) + (W[ry - 1][rx] - wc)));
  r.X = (Qx[ry + 1][rx + 1] - Qx[ry + 1][rx - 1]) + (Qx[ry - 1][rx + 1] - Qx[ry - 1][rx - 1]);
  r.Y = (Qy[ry + 1][rx + 1] - Qy[ry - 1][rx + 1]) + (Qy[ry + 1][rx - 1] - Qy[ry - 1][rx - 1]);
  r.Z = (Qz[ry + 1][rx + 1] + Qz[ry + 1][rx - 1]) + (Qz[ry - 1][rx + 1] + Qz[ry - 1][rx - 1]);
  r.W = (W[ry + 1][rx + 1] + W[ry + 1][rx - 1]) + (W[ry - 1][rx + 1] + W[ry - 1][rx - 1]);
  r.qz = Qz[ry][rx];
  r.w = wc;
  return r;
}

// Each block sweeps its runs of (x-y tile, z range) in turn; thread (lane, warp) owns the column
// (x0 - 1 + lane, y0 - 1 + warp) of the (Q, w) region and sweeps z. Each plane of phi
// and of (Q, w) passes through shared memory once; the thread keeps what the planes
// below contributed to its column's stencils in registers:
//   phi plane p arrives  ->  grad phi, lap phi, Q, w, mu_alpha on plane p - 1
//   (Q, w) plane p - 1   ->  mu_beta on plane p - 2 (interior columns)
// Two barriers per plane; phi planes arrive by cp.async MU_RING - 1 planes ahead.
__global__ void __launch_bounds__(MU_THREADS, 2) mu3_kernel(const float* __restrict__ phi, Grid3 g, Consts3 c,
                                                            MuTiles mt, float* __restrict__ mua,
                                                            float* __restrict__ mub) {
  __shared__ float sphi[MU_RING][MU_PY][MU_PX];
  __shared__ float sq[4][MU_QY][MU_QX];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long total = (long long)mt.tiles_x * mt.tiles_y * g.nz;
  const long long end = min(total, ((long long)blockIdx.x + 1) * mt.per_block);
  for (long long idx = (long long)blockIdx.x * mt.per_block; idx < end;) {
    const int tile = (int)(idx / g.nz);
    const int z0 = (int)(idx % g.nz);
    const int z1 = (int)min((long long)g.nz, z0 + (end - idx));
    idx += z1 - z0;
    const int x0 = (tile % mt.tiles_x) * MU_TX;
    const int y0 = (tile / mt.tiles_x) * MU_TY;
    __syncthreads();  // the previous run's reads of the rings are done
    const int gx = x0 - 1 + lane, gy = y0 - 1 + warp;  // this column
    const bool out = lane >= 1 && lane <= MU_TX && warp >= 1 && warp <= MU_TY && gx < g.nx && gy < g.ny;

    // phi plane p (z0 - 2 <= p <= z1 + 1) lands by cp.async in ring slot (p - z0 + 2) % MU_RING;
    // every thread commits one group per plane (empty past the last one).
    int src_off[MU_PHI_PER_THREAD];  // in-plane offset of each element this thread copies
#pragma unroll
    for (int j = 0; j < MU_PHI_PER_THREAD; ++j) {
      const int r = threadIdx.x + j * MU_THREADS;
      const int rx = r % MU_PX, ry = r / MU_PX;
      src_off[j] = r < MU_PX * MU_PY ? modn(y0 - 2 + ry, g.ny) * g.nx + modn(x0 - 2 + rx, g.nx) : 0;
    }
    auto issue = [&](int p) {
      if (p <= z1 + 1) {
        const float* src = phi + (long long)modn(p, g.nz) * g.ny * g.nx;
        float* dst = &sphi[(p - z0 + 2) % MU_RING][0][0];
#pragma unroll
        for (int j = 0; j < MU_PHI_PER_THREAD; ++j) {
          const int r = threadIdx.x + j * MU_THREADS;
          if (r < MU_PX * MU_PY) cp_async4(dst + r, src + src_off[j]);
        }
      }
      lbch::cp_async_commit();
    };

    PhiPlane p1{}, p2{};  // phi planes p - 1 and p - 2 of this column
    QPlane q1{}, q2{};    // (Q, w) planes t - 1 and t - 2 (t = p - 1)
    float a1 = 0.0f;      // local part of mu_beta on plane t - 1
#pragma unroll
    for (int k = 0; k < MU_RING - 1; ++k) issue(z0 - 2 + k);
    for (int p = z0 - 2; p <= z1 + 1; ++p) {
      lbch::cp_async_wait<MU_RING - 2>();  // this thread's copies of plane p have landed
      __syncthreads();                     // and everyone's; slot of plane p - 1 is free
      issue(p + MU_RING - 1);
      const PhiPlane p0 = phi_plane(sphi[(p - z0 + 2) % MU_RING], lane + 1, warp + 1);
      const int t = p - 1;  // plane whose phi stencils p0 completes
      const bool have_q = t >= z0 - 1;
      float a0 = 0.0f;
      if (have_q) {
        const float dx = p1.gx + G7 * (p0.X + p2.X);
        const float dy = p1.gy + G7 * (p0.Y + p2.Y);
        const float dz = G1 * (p0.c - p2.c) + G7 * (p0.S - p2.S);
        const float lap = p1.lap + L1 * ((p0.c - p1.c) + (p2.c - p1.c)) +
                          L7 * ((p0.S - 4.0f * p1.c) + (p2.S - 4.0f * p1.c));
        const Aniso r = aniso(c, p1.c, dx, dy, dz, lap);
        sq[0][warp][lane] = r.qx;
        sq[1][warp][lane] = r.qy;
        sq[2][warp][lane] = r.qz;
        sq[3][warp][lane] = r.w;
        if (out && t >= z0 && t < z1) mua[(t * g.ny + gy) * g.nx + gx] = r.mua;
        a0 = r.a;
      }
      p2 = p1;
      p1 = p0;
      __syncthreads();
      if (have_q && out) {
        const QPlane q0 = q_plane(sq, lane, warp);
        const int s = t - 1;  // mu_beta plane that (Q, w) of plane t completes
        if (s >= z0 && s < z1) {
          const float div = q1.div + G7 * (((q0.X + q2.X) + (q0.Y + q2.Y)) + (q0.Z - q2.Z)) + G1 * (q0.qz - q2.qz);
          const float lapw = q1.lapw + L1 * ((q0.w - q1.w) + (q2.w - q1.w)) +
                             L7 * ((q0.W - 4.0f * q1.w) + (q2.W - 4.0f * q1.w));
          mub[(s * g.ny + gy) * g.nx + gx] = fmaf(c.eps, lapw, a1 - div);  // Eq. 13 minus mu_alpha
        }
        q2 = q1;
        q1 = q0;
      }
      a1 = a0;
    }
  }
}

// ---------------------------------------------------------------- collide3_kernel

// Moment k of f (row k of Eq. 24 applied to f[0..14]); entries are literals.
template <int K, int I = 0>
__device__ __forceinline__ float moment(const float (&f)[15]) {
  if constexpr (I == 15) {
    return 0.0f;
  } else {
    constexpr int m = MR<K, I>::v;
    const float rest = moment<K, I + 1>(f);
    if constexpr (m == 0) return rest;
    else if constexpr (m == 1) return f[I] + rest;
    else if constexpr (m == -1) return rest - f[I];
    else return fmaf((float)m, f[I], rest);
  }
}

// Population i of M^T n (column i of Eq. 24 against the scaled post-collision moments).
template <int I, int K = 0>
__device__ __forceinline__ float back(const float (&n)[15]) {
  if constexpr (K == 15) {
    return 0.0f;
  } else {
    constexpr int m = MR<K, I>::v;
    const float rest = back<I, K + 1>(n);
    if constexpr (m == 0) return rest;
    else if constexpr (m == 1) return n[K] + rest;
    else if constexpr (m == -1) return rest - n[K];
    else return fmaf((float)m, n[K], rest);
  }
}

// FAST: s_k = 1 for every moment but phi (k = 0) and j (k = 3, 5, 7), so those others take
// m* = m^eq + F_m / 2 and need not be formed from f.
template <int K, bool FAST>
__device__ __forceinline__ void relax(const float (&f)[15], float phi, float m_a, float gx, float gy, float gz,
                                      const Consts3& c, float (&nk)[15]) {
  // m^eq = (phi, -2 phi + mu_a, 16 phi - 15 mu_a, 0, ...) (Eq. 18 in the Eq. 24 basis);
  // F_m = M F is nonzero on j (-g/3) and q (7 g/9) only (Eq. 19).
  const float meq = K == 0 ? phi : (K == 1 ? fmaf(-2.0f, phi, m_a) : (K == 2 ? fmaf(16.0f, phi, -15.0f * m_a) : 0.0f));
  const float gk = (K == 3 || K == 4) ? gx : ((K == 5 || K == 6) ? gy : gz);
  const float Fm = (K == 3 || K == 5 || K == 7) ? -gk * (1.0f / 3.0f) : ((K == 4 || K == 6 || K == 8) ? gk * (7.0f / 9.0f) : 0.0f);
  float ms;
  if constexpr (FAST && K != 0 && K != 3 && K != 5 && K != 7) {
    ms = fmaf(0.5f, Fm, meq);
  } else {
    const float m = moment<K>(f);
    ms = fmaf(-c.s[K], m - meq, m) + (1.0f - 0.5f * c.s[K]) * Fm;  // Eq. 17 in moments
  }
  nk[K] = ms * (1.0f / (float)MN<K>::v);
  if constexpr (K + 1 < 15) relax<K + 1, FAST>(f, phi, m_a, gx, gy, gz, c, nk);
}

template <int I>
__device__ __forceinline__ void unproject(const float (&nk)[15], float (&o)[15]) {
  o[I] = back<I>(nk);
  if constexpr (I + 1 < 15) unproject<I + 1>(nk, o);
}

template <bool FAST>
__global__ void __launch_bounds__(NX3) collide3_kernel(const float* __restrict__ src, const float* __restrict__ mub,
                                                       const float* __restrict__ mua, Grid3 g, Consts3 c,
                                                       float* __restrict__ dst) {
  Site s;
  if (!site_of(g, blockIdx.x, s)) return;
  float f[15];
#pragma unroll
  for (int i = 0; i < 15; ++i) f[i] = ld_pop(src + (long long)i * g.ps + s.at(-cx(i), -cy(i), -cz(i)));
  float gx, gy, gz, unused;
  stencil(mub, s, gx, gy, gz, unused);
  float phi = 0.0f;
#pragma unroll
  for (int i = 0; i < 15; ++i) phi += f[i];
  float nk[15], o[15];
  relax<0, FAST>(f, phi, mua[s.id], gx, gy, gz, c, nk);
  unproject<0>(nk, o);
  // Rest population closes the mass exactly (sum_i f* = sum_i f, Eq. 34).
  float d = 0.0f;
#pragma unroll
  for (int i = 1; i < 15; ++i) d += f[i] - o[i];
  o[0] = f[0] + d;
#pragma unroll
  for (int i = 0; i < 15; ++i) dst[(long long)i * g.ps + s.id] = o[i];
}

// ---------------------------------------------------------------- init and diagnostics

__global__ void __launch_bounds__(NX3) mu_alpha3_kernel(const double* __restrict__ phi, double* __restrict__ mua,
                                                        Grid3 g, double k, double beta4, int* bad) {
  Site s;
  if (!site_of(g, blockIdx.x, s)) return;
  const double c = phi[s.id];
  double lap = 0.0;
#pragma unroll
  for (int i = 1; i < 15; ++i) lap += 2.0 * wgt(i) * (phi[s.at(cx(i), cy(i), cz(i))] - c);
  lap *= 3.0;
  mua[s.id] = beta4 * c * (c * c - 1.0) - k * lap;
  if (!isfinite(c)) atomicOr(bad, 1);
}

// f = f^eq(phi0, mu_alpha) in the pre-streaming form (f*_i(x) streams to f_i(x + c_i)).
__global__ void __launch_bounds__(NX3) init3_kernel(const double* __restrict__ phi0, const double* __restrict__ mua,
                                                    Grid3 g, float* __restrict__ f) {
  Site s;
  if (!site_of(g, blockIdx.x, s)) return;
  f[s.id] = (float)(phi0[s.id] + (wgt(0) - 1.0) * mua[s.id]);
#pragma unroll
  for (int i = 1; i < 15; ++i) f[(long long)i * g.ps + s.id] = (float)(wgt(i) * mua[s.at(cx(i), cy(i), cz(i))]);
}

__global__ void __launch_bounds__(NX3) phi3_f64_kernel(const float* __restrict__ f, Grid3 g, double* __restrict__ phi) {
  Site s;
  if (!site_of(g, blockIdx.x, s)) return;
  double p = 0.0;
#pragma unroll
  for (int i = 0; i < 15; ++i) p += (double)f[(long long)i * g.ps + s.at(-cx(i), -cy(i), -cz(i))];
  phi[s.id] = p;
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

// Energy density (reading C11 in 3D) per node; blocks stride over the node-kernel
// blocks with NX3 threads each.
__global__ void __launch_bounds__(NX3) energy3_kernel(const float* __restrict__ phi, Grid3 g, lbch::EnergyConsts c,
                                                      int node_blocks, double* __restrict__ partial) {
  __shared__ double sh[NX3 / 32];
  double acc = 0.0;
  for (int b = blockIdx.x; b < node_blocks; b += gridDim.x) {
    Site s;
    if (!site_of(g, b, s)) continue;
    float dx, dy, dz, lap;
    stencil(phi, s, dx, dy, dz, lap);
    const float p0 = phi[s.id];
    const float g2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float gamma = 1.0f;
    if (g2 >= 1e-12f) {
      const float rs = rsqrtf(g2);
      const float a = dx * rs, b2 = dy * rs, e = dz * rs;
      gamma = fmaf(c.alpha, fmaf(4.0f, fmaf(a * a, a * a, fmaf(b2 * b2, b2 * b2, e * e * e * e)), -3.0f), 1.0f);
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
  float *phi, *mua, *mub;
  double* stage;
  double* partial;
  double* result;
  int* flags;
  int blocks;      // blocks of the node kernels (NX3 x-nodes each)
  int red_blocks;  // blocks for the reductions
  lbch3::MuTiles mt;
  int mu_blocks;   // blocks of mu3_kernel
  bool fast;       // s_k = 1 except for phi and j: the reduced collision
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
  return 2 * align_up(ps * 15 * sizeof(float)) + 3 * align_up(ps * sizeof(float)) + align_up(ps * sizeof(double)) +
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
  const int segs = (p->nx + lbch3::NX3 - 1) / lbch3::NX3;
  c->g = lbch3::Grid3{p->nx, p->ny, p->nz, segs, ps};
  char* q = (char*)d_workspace;
  for (int b = 0; b < 2; ++b) {
    c->buf[b] = (float*)q;
    q += align_up((size_t)ps * 15 * sizeof(float));
  }
  float** planes[3] = {&c->phi, &c->mua, &c->mub};
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
  c->fast = true;
  for (int i = 1; i < 15; ++i)
    if (i != 3 && i != 5 && i != 7 && c->s[i] != 1.0) c->fast = false;
  c->blocks = segs * p->ny * p->nz;  // < 2^31: segs * nx-rows <= (nx + 127) / 128 * ny * nz
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  {  // mu3: one resident wave of persistent blocks, each with an equal run of planes
    lbch3::MuTiles& mt = c->mt;
    mt.tiles_x = (p->nx + lbch3::MU_TX - 1) / lbch3::MU_TX;
    mt.tiles_y = (p->ny + lbch3::MU_TY - 1) / lbch3::MU_TY;
    const long long total = (long long)mt.tiles_x * mt.tiles_y * p->nz;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lbch3::mu3_kernel, lbch3::MU_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    const long long wave = (long long)(sms > 0 ? sms : 152) * per_sm;
    long long per_block = (total + wave - 1) / wave;
    if (per_block < 4) per_block = 4;  // a run re-reads 3 planes at its start
    mt.per_block = per_block;
    c->mu_blocks = (int)((total + per_block - 1) / per_block);
  }
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
  double* mua = reinterpret_cast<double*>(c->buf[1]);  // the second population buffer is free during init
  if (cuda3_failed(c, cudaMemcpyAsync(c->stage, h_phi0, n * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                   "init_field: copy") ||
      cuda3_failed(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "init_field: clear"))
    return LBCH_ECUDA;
  lbch3::mu_alpha3_kernel<<<c->blocks, lbch3::NX3, 0, c->stream>>>(c->stage, mua, c->g, c->k, 4.0 * c->beta, c->flags);
  lbch3::init3_kernel<<<c->blocks, lbch3::NX3, 0, c->stream>>>(c->stage, mua, c->g, c->buf[0]);
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
  for (int64_t t = 0; t < n; ++t) {
    const float* src = c->buf[c->cur];
    float* dst = c->buf[c->cur ^ 1];
    lbch3::phi3_kernel<<<c->blocks, lbch3::NX3, 0, c->stream>>>(src, c->g, c->phi);
    lbch3::mu3_kernel<<<c->mu_blocks, lbch3::MU_THREADS, 0, c->stream>>>(c->phi, c->g, c->cs, c->mt, c->mua, c->mub);
    if (c->fast)
      lbch3::collide3_kernel<true><<<c->blocks, lbch3::NX3, 0, c->stream>>>(src, c->mub, c->mua, c->g, c->cs, dst);
    else
      lbch3::collide3_kernel<false><<<c->blocks, lbch3::NX3, 0, c->stream>>>(src, c->mub, c->mua, c->g, c->cs, dst);
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
  lbch3::phi3_f64_kernel<<<c->blocks, lbch3::NX3, 0, c->stream>>>(c->buf[c->cur], c->g, c->stage);
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
  lbch3::phi3_kernel<<<c->blocks, lbch3::NX3, 0, c->stream>>>(c->buf[c->cur], c->g, c->phi);
  EnergyConsts ec;
  const double eps = c->p.regularization == LBCH_REG_NONE ? 0.0 : c->p.eps;
  ec.k = (float)c->k;
  ec.beta = (float)c->beta;
  ec.beta4 = (float)(4.0 * c->beta);
  ec.alpha = (float)c->p.alpha;
  ec.half_eps = (float)(0.5 * eps);
  ec.cw = c->p.regularization == LBCH_REG_LINEAR ? 0.0f : 1.0f;
  lbch3::energy3_kernel<<<c->red_blocks, lbch3::NX3, 0, c->stream>>>(c->phi, c->g, ec, c->blocks, c->partial);
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
