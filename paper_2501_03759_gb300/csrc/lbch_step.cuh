// Fused time step of the MRT lattice Boltzmann scheme for the anisotropic
// Cahn-Hilliard equation (arXiv 2501.03759, Section 3), one kernel per step.
//
// What one launch computes, for every node x of the periodic grid:
//   f_in,i(x)  = f*_i(x - c_i)                      pull streaming of the previous step
//   phi        = sum_i f_in,i                       Eq. 22
//   grad phi, lap phi                               Eq. 26a, 26b
//   n, gamma(n), P grad_n gamma, Q, f, f', w, mu_a  Eqs. 2, 6, 15, 9, 13, 16
//   mu_beta = (gamma-1) f - div Q + eps(lap w - f' w)   Eqs. 13, 16 (split reading)
//   g = grad mu_beta, F_m = M F                     Eqs. 26a, 19, 25
//   m* = m - S(m - m^eq) + (I - S/2) F_m, f* = M^-1 m*   Eqs. 17, 23, 25
// and stores f* (the state before streaming) in the other buffer.
//
// Work decomposition (GB300): one warp owns a strip of 128 consecutive columns
// (4 per lane, so rows move as 16-byte vectors) and sweeps a segment of rows top to
// bottom. phi is needed up to 3 nodes away from an output node, so each warp keeps
// a rolling three-row window of every stencil in registers: when the phi row r
// arrives it completes grad/lap phi of row r-1, mu_beta of row r-2 and
// grad mu_beta of row r-3, and collides row r-3. Left/right neighbours come from
// warp shuffles; the 4 strip columns at each edge are halo, so a strip yields 120
// output columns. Rows arrive by cp.async into a per-warp shared-memory ring of
// landing slots, fetched PF_DIST rows ahead of use; a row stays in the ring until
// its collision three rows later (each lane reads back only what it copied, so no
// barrier is needed). No tensor cores: the 9x9 moment transform is a handful of
// adds with constant +-1/+-2 entries.
#pragma once

#include "lbch_f2.cuh"
#include "lbch_lattice.cuh"

namespace lbch {

constexpr int STRIP_W = 128;                 // columns per warp strip
constexpr int HALO_W = 4;                    // halo columns on each side
constexpr int OUT_W = STRIP_W - 2 * HALO_W;  // output columns per strip
// A field exactly STRIP_W wide is one strip that covers the whole periodic row: the lane
// neighbour exchanges below rotate (lane 0's left neighbour is lane 31), so every column is
// computed from its true periodic neighbours and all STRIP_W columns are output. In a strip
// of a wider (or narrower) field the rotated-in values reach only halo columns: an output
// column depends on columns at most HALO_W (the stencil depth) away, inside the strip.
__host__ __device__ constexpr int n_strips_for(int nx) { return nx == STRIP_W ? 1 : (nx + OUT_W - 1) / OUT_W; }
constexpr int STEP_WARPS = 4;                // warps per CTA
// Pipeline depth per storage (measured on GB300 at 8192^2): fetch one row ahead and collide
// row r-3 right after its grad mu_beta. The 16-bit storages keep 12 warps per SM (their
// landing slots are smaller); colliding row r-4 first in the iteration with no prefetch
// instead ran 10% slower once their per-row instruction count had come down, and one row
// of prefetch with r-4 needs a sixth slot, which costs a CTA per SM; so does two rows of
// prefetch with r-3 (0.547 -> 0.710 ms per 8192^2 BF16 launch).
template <int ST, bool VEC>
struct Pipe {
  static constexpr bool DEV16 = ST != ST_F32;
  static constexpr int PF_DIST = 1;                     // rows fetched ahead of the phi row
  static constexpr int LAG = 3;                         // phi row r collides row r - LAG
  static constexpr int SLOTS = PF_DIST + 1 + LAG;       // rows held per warp: r-LAG .. r+PF_DIST
  // 16-byte units per slot: 9 per lane for FP32 planes (or pulled values on the scalar
  // path); rest + anchor + 8 half-width deviation planes = 6 per lane for vector DEV.
  static constexpr int SLOT_F4 = (DEV16 && VEC ? 6 : 9) * 32;
  static constexpr int MIN_CTAS = DEV16 && VEC ? 3 : 2;  // CTAs per SM the launch bounds plan for
};
template <int ST, bool VEC>
constexpr int step_smem() { return STEP_WARPS * Pipe<ST, VEC>::SLOTS * Pipe<ST, VEC>::SLOT_F4 * 16; }

// Constants shared by every field a launch steps.
struct StepArgs {
  // Chemical potential constants.
  float k;     // gradient energy coefficient (Eq. 5)
  float kq;    // factor on |grad phi| P grad_n gamma in Q (k, or 1 for the literal Eq. 15)
  float kiso;  // k times the isotropic part kept in Q (0 split, k nested)
  float beta4, beta12;  // 4 beta and 12 beta (f and f')
  float eps;   // eps on lap w (0 without regularisation)
  float cw;    // w = lap phi - cw f  (1 Willmore, 0 linear)
  float cfp;   // eps on f' w (Willmore only)
  float cnk;   // k lap phi added to mu_beta in nested form
  // Collision: n_k = (m*_k)/|row k of M|^2 in terms of m_k, m^eq_k and g.
  float c1a, c1b, c2a, c2b, c3a, c3g, c4a, c4g, c5a, c5g, c6a, c6g, c7, c8;
};

// One periodic field: its buffers, its size and work split, and its anisotropy.
struct Field {
  Buf src, dst;
  long long ps;  // plane stride in elements
  int nx, ny;
  int n_strips, seg_len;
  float alpha, a16;  // alpha and 16 alpha (Eq. 6)
};

__device__ __forceinline__ int imod(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// The value of the lane to the left (lane 31 for lane 0) and to the right (lane 0 for 31).
__device__ __forceinline__ float from_lane_left(float v) {
  return __shfl_sync(FULL, v, (threadIdx.x + 31) & 31);
}
__device__ __forceinline__ float from_lane_right(float v) {
  return __shfl_sync(FULL, v, (threadIdx.x + 1) & 31);
}

// Left/right neighbour sums and differences of a per-column quantity over the strip:
// s_j = q_{j-1} + q_{j+1}, d_j = q_{j+1} - q_{j-1} for this lane's columns j = 0..3 (pairs
// (0, 1) and (2, 3)), with the outer neighbours from the adjacent lanes.
__device__ __forceinline__ void neighbours(const F2 (&q)[2], F2 (&s)[2], F2 (&d)[2]) {
  const float left = from_lane_left(q[1].y);
  const float right = from_lane_right(q[0].x);
  const F2 A = f2(left, q[0].x), B = f2(q[0].y, q[1].x), C = f2(q[1].y, right);
  s[0] = A + B;
  s[1] = B + C;
  d[0] = B - A;
  d[1] = C - B;
}

// Per-lane addressing of the strip.
struct Cols {
  long long c0;  // aligned first column (vector path)
  int cs[6];     // columns xs + 4 lane + k - 1, k = 0..5 (scalar path), mod nx
};

// Row copies ask L2 to fetch 256-byte blocks (.L2::256B): a warp's row of one plane is 512
// (FP32) or 256 (16-bit) contiguous bytes, so each miss brings in the neighbouring sectors the
// warp reads next. Measured on GB300 at 8192^2: 0.844 -> 0.821 ms per FP32 launch and
// 0.548 -> 0.542 ms per BF16 launch (a 128-byte hint gave no FP32 gain).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global.L2::256B [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global.L2::256B [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One warp's landing slot for one phi row r, as 16-byte units [q][lane]:
//   vector F32:  q = i holds plane i of row r - c_iy at the strip's aligned columns (raw f*);
//   vector DEV:  q = 0 the rest plane of row r, q = 1 the anchor plane of row r, then (as
//                8-byte units [k][lane]) the deviation plane k+1 of row r - c_(k+1)y;
//   scalar path: q = i holds f_in,i itself (pulled and rebuilt when it was fetched).
// Fetches phi row r (rows ro_m = r-1, ro_0 = r, ro_p = r+1) into a slot; the vector path
// copies asynchronously (cp.async), the scalar path loads and stores synchronously.
template <int ST, bool VEC>
__device__ __forceinline__ void issue_row(const Field& fd, float4* slot, int lane, long long ro_m,
                                          long long ro_0, long long ro_p, const Cols& cl) {
#define LBCH_RO(I) (cy(I) == 1 ? ro_m : (cy(I) == -1 ? ro_p : ro_0))
  if constexpr (VEC) {
    if constexpr (ST == ST_F32) {
#pragma unroll
      for (int i = 0; i < 9; ++i)
        cp_async16(slot + i * 32 + lane, fd.src.f32 + (long long)i * fd.ps + LBCH_RO(i) + cl.c0);
    } else {
      cp_async16(slot + lane, fd.src.f32 + ro_0 + cl.c0);
      cp_async16(slot + 32 + lane, fd.src.f32 + fd.ps + ro_0 + cl.c0);
      uint2* ds = reinterpret_cast<uint2*>(slot + 64);
#pragma unroll
      for (int i = 1; i < 9; ++i)
        cp_async8(ds + (i - 1) * 32 + lane, fd.src.dev + (long long)(i - 1) * fd.ps + LBCH_RO(i) + cl.c0);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      float v[4];
      const long long ro = LBCH_RO(i);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = cl.cs[j - cx(i) + 1];  // pull: f_in,i(x) = f*_i(x - c_i)
        if constexpr (ST == ST_F32) {
          v[j] = __ldg(fd.src.f32 + (long long)i * fd.ps + ro + c);
        } else if (i == 0) {
          v[j] = __ldg(fd.src.f32 + ro + c);
        } else {  // w_i times the anchor of this node, plus the deviation from the source node
          v[j] = fmaf((float)wgt(i), __ldg(fd.src.f32 + fd.ps + ro_0 + cl.cs[j + 1]),
                      Dev<ST>::load(__ldg(fd.src.dev + (long long)(i - 1) * fd.ps + ro + c)));
        }
      }
      slot[i * 32 + lane] = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
#undef LBCH_RO
}

// Pull shift along x of a per-column quantity of the strip: column j takes column j - 1
// (c_x = 1) or column j + 1 (c_x = -1).
__device__ __forceinline__ void from_left(F2 (&v)[2]) {
  const float prev = from_lane_left(v[1].y);
  v[1] = f2(v[0].y, v[1].x);
  v[0] = f2(prev, v[0].x);
}
__device__ __forceinline__ void from_right(F2 (&v)[2]) {
  const float next = from_lane_right(v[0].x);
  v[0] = f2(v[0].y, v[1].x);
  v[1] = f2(v[1].y, next);
}

__device__ __forceinline__ void to_pairs(const float4 t, F2 (&v)[2]) {
  v[0] = f2(t.x, t.y);
  v[1] = f2(t.z, t.w);
}

// f_in,I at this lane's 4 columns from a landed slot.
template <int ST, bool VEC, int I>
__device__ __forceinline__ void read_row(const float4* slot, int lane, F2 (&v)[2]) {
  constexpr bool REBUILD = VEC && ST != ST_F32 && I != 0;
  if constexpr (!REBUILD) {
    to_pairs(slot[I * 32 + lane], v);
  } else {  // deviations of the source nodes (row r - c_Iy), shifted below
    const uint2 raw = reinterpret_cast<const uint2*>(slot + 64)[(I - 1) * 32 + lane];
    Dev<ST>::raw2(raw.x, v[0].x, v[0].y);
    Dev<ST>::raw2(raw.y, v[1].x, v[1].y);
    if constexpr (Dev<ST>::UNSCALE != 1.0f) {
      v[0] = splat(Dev<ST>::UNSCALE) * v[0];
      v[1] = splat(Dev<ST>::UNSCALE) * v[1];
    }
  }
  if constexpr (VEC) {  // the pull shift along x happens here, one shuffle per plane
    if constexpr (cx(I) == 1) {
      from_left(v);
    } else if constexpr (cx(I) == -1) {
      from_right(v);
    }
  }
  if constexpr (REBUILD) {  // f*_I(y - c_I) = w_I anchor(y) + d_I(y - c_I)
    const F2 w = splat((float)wgt(I));
    F2 m[2];
    to_pairs(slot[32 + lane], m);
    v[0] = fma2(w, m[0], v[0]);
    v[1] = fma2(w, m[1], v[1]);
  }
}

// Grouped deviation sums of a landed DEV row at this lane's 4 columns, pulled along x, in
// storage units (FP16 values still carry their scale). The eight moving planes fall into
// three groups by c_x: gp = d1 + d5 + d8 (c_x = 1), gm = d3 + d6 + d7 (c_x = -1) and
// g0 = d2 + d4; with H also their c_y-signed parts hp = d5 - d8, hm = d6 - d7 and
// h0 = d2 - d4. A group shares one pull shift, so it takes one shuffle instead of one per
// plane. Every population arriving at a node is rebuilt on that node's anchor, the weights
// w_1..w_8 sum to 5/9, and the anchor terms cancel in j_x and j_y, so
//   phi = f*_0 + (5/9) anchor + (gp + gm + g0),  j_x = gp - gm,  j_y = hp + hm + h0.
struct DevSums {
  F2 gp[2], gm[2], g0[2], hp[2], hm[2], h0[2];
};
template <int ST, bool H>
__device__ __forceinline__ void dev_sums(const float4* slot, int lane, DevSums& s) {
  const uint2* ds = reinterpret_cast<const uint2*>(slot + 64);
  F2 d[9][2];
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const uint2 raw = ds[(i - 1) * 32 + lane];
    Dev<ST>::raw2(raw.x, d[i][0].x, d[i][0].y);
    Dev<ST>::raw2(raw.y, d[i][1].x, d[i][1].y);
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    s.gp[k] = (d[1][k] + d[5][k]) + d[8][k];
    s.gm[k] = (d[3][k] + d[6][k]) + d[7][k];
    s.g0[k] = d[2][k] + d[4][k];
    if constexpr (H) {
      s.hp[k] = d[5][k] - d[8][k];
      s.hm[k] = d[6][k] - d[7][k];
      s.h0[k] = d[2][k] - d[4][k];
    }
  }
  from_left(s.gp);
  from_right(s.gm);
  if constexpr (H) {
    from_left(s.hp);
    from_right(s.hm);
  }
}

// phi at this lane's columns of a landed DEV row from its rest population, anchor and
// group sums.
template <int ST>
__device__ __forceinline__ void dev_phi(const float4* slot, int lane, const DevSums& s, F2 (&ph)[2]) {
  F2 rest[2], anc[2];
  to_pairs(slot[lane], rest);
  to_pairs(slot[32 + lane], anc);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    F2 g = (s.gp[k] + s.gm[k]) + s.g0[k];
    if constexpr (Dev<ST>::UNSCALE != 1.0f) g = splat(Dev<ST>::UNSCALE) * g;
    ph[k] = fma2(splat(5.0f / 9.0f), anc[k], rest[k]) + g;
  }
}

// Pointwise part at two nodes: Q (Eq. 15 reading), w, mu_alpha (Eq. 16) and the local part A
// of mu_beta (Eq. 13 minus Eq. 16's mu_alpha).
__device__ __forceinline__ void pointwise(const StepArgs& a, const Field& fd, F2 phi, F2 dx, F2 dy, F2 lap,
                                          F2& Qx, F2& Qy, F2& w, F2& A, F2& mua) {
  const F2 g2 = fma2(dx, dx, dy * dy);
  const bool okx = g2.x >= 1e-12f, oky = g2.y >= 1e-12f;  // n = 0, gamma = 1 below this
  const F2 rs = f2(rsqrtf(okx ? g2.x : 1.0f), rsqrtf(oky ? g2.y : 1.0f));
  const F2 n1 = dx * rs, n2 = dy * rs;  // Eq. 2
  const F2 n1s = n1 * n1, n2s = n2 * n2;
  const F2 S4 = fma2(n1s, n1s, n2s * n2s);
  F2 gm1 = splat(fd.alpha) * fma2(splat(4.0f), S4, splat(-3.0f));  // gamma - 1, Eq. 6
  // k_q |grad phi| P grad_n gamma with grad_n gamma = 16 alpha n^3, P = I - n n^T.
  F2 t = splat(a.kq * fd.a16) * (g2 * rs);
  if (!okx) gm1.x = t.x = 0.0f;
  if (!oky) gm1.y = t.y = 0.0f;
  const F2 kg = fma2(splat(a.k), gm1, splat(a.kiso));
  Qx = fma2(kg, dx, t * (n1 * (n1s - S4)));
  Qy = fma2(kg, dy, t * (n2 * (n2s - S4)));
  const F2 phi2 = phi * phi;
  const F2 fb = (splat(a.beta4) * phi) * (phi2 - splat(1.0f));  // f = F'(phi), Eq. 9
  const F2 fp = fma2(splat(a.beta12), phi2, splat(-a.beta4));   // f'(phi), Eq. 13
  w = fma2(splat(-a.cw), fb, lap);
  mua = fma2(splat(-a.k), lap, fb);
  A = fma2(gm1, fb, fma2(splat(-a.cfp) * fp, w, splat(a.cnk) * lap));
}

// Eq. 17 at two nodes in moment space (Eqs. 23, 25) with the closed forms
// m^eq = (phi, -4 phi + 2 mu_a, 4 phi - 3 mu_a, 0, ...) and
// M F = (0, 0, 0, -g_x/3, g_x/3, -g_y/3, g_y/3, 0, 0), and M^-1 = M^T diag(1/|row|^2).
// FAST: s_1 = s_2 = s_4 = s_6 = s_7 = s_8 = 1, so those moments take their (forced)
// equilibrium and need not be formed; the result equals the general path's, whose
// (1 - s_k) m_k terms are then exactly zero.
// FAST collision from the three moments it needs, phi = m_0, j_x = m_3 and j_y = m_5 (the
// others take their equilibrium): o[1..8] of f*; o[0] is left to the caller.
__device__ __forceinline__ void collide_fast(const StepArgs& a, F2 phi, F2 m3, F2 m5, F2 mua, F2 gx, F2 gy,
                                             F2 (&o)[9]) {
  const F2 n0 = phi * splat(1.0f / 9.0f);
  const F2 n1 = splat(a.c1b) * fma2(splat(2.0f), mua, splat(-4.0f) * phi);
  const F2 n2 = splat(a.c2b) * fma2(splat(-3.0f), mua, splat(4.0f) * phi);
  const F2 n4 = splat(a.c4g) * gx, n6 = splat(a.c6g) * gy;
  const F2 n3 = fma2(splat(a.c3a), m3, splat(a.c3g) * gx);
  const F2 n5 = fma2(splat(a.c5a), m5, splat(a.c5g) * gy);
  const F2 A0 = fma2(splat(-2.0f), n2, n0 - n1);
  const F2 X = fma2(splat(-2.0f), n4, n3), Y = fma2(splat(-2.0f), n6, n5);
  o[1] = A0 + X;
  o[3] = A0 - X;
  o[2] = A0 + Y;
  o[4] = A0 - Y;
  const F2 D0 = fma2(splat(2.0f), n1, n0 + n2);
  const F2 U = n3 + n4, V = n5 + n6;
  const F2 P = U + V, Mv = U - V;
  o[5] = D0 + P;
  o[7] = D0 - P;
  o[6] = D0 - Mv;
  o[8] = D0 + Mv;
}

template <bool FAST>
__device__ __forceinline__ void collide(const StepArgs& a, const F2 (&f)[9], F2 mua, F2 gx, F2 gy, F2 (&o)[9],
                                        F2& phi_out) {
  const F2 ab = f[1] + f[3], bb = f[2] + f[4];
  const F2 Sa = ab + bb;
  const F2 e = f[5] + f[7], h = f[6] + f[8];
  const F2 Sd = e + h;
  const F2 phi = (f[0] + Sa) + Sd;
  const F2 x1 = f[1] - f[3], y1 = f[2] - f[4];
  const F2 p = f[5] - f[7], q = f[6] - f[8];
  const F2 pm = p - q, pp = p + q;
  const F2 m3 = x1 + pm, m5 = y1 + pp;
  if constexpr (FAST) {
    collide_fast(a, phi, m3, m5, mua, gx, gy, o);
  } else {
    const F2 n0 = phi * splat(1.0f / 9.0f);
    const F2 m1 = fma2(splat(-4.0f), f[0], fma2(splat(2.0f), Sd, splat(0.0f) - Sa));
    const F2 m2 = fma2(splat(4.0f), f[0], fma2(splat(-2.0f), Sa, Sd));
    const F2 m4 = fma2(splat(-2.0f), x1, pm), m6 = fma2(splat(-2.0f), y1, pp);
    const F2 m7 = ab - bb, m8 = e - h;
    const F2 n1 = fma2(splat(a.c1a), m1, splat(a.c1b) * fma2(splat(2.0f), mua, splat(-4.0f) * phi));
    const F2 n2 = fma2(splat(a.c2a), m2, splat(a.c2b) * fma2(splat(-3.0f), mua, splat(4.0f) * phi));
    const F2 n4 = fma2(splat(a.c4a), m4, splat(a.c4g) * gx);
    const F2 n6 = fma2(splat(a.c6a), m6, splat(a.c6g) * gy);
    const F2 n7 = splat(a.c7) * m7;
    const F2 n8 = splat(a.c8) * m8;
    const F2 n3 = fma2(splat(a.c3a), m3, splat(a.c3g) * gx);
    const F2 n5 = fma2(splat(a.c5a), m5, splat(a.c5g) * gy);
    const F2 A0 = fma2(splat(-2.0f), n2, n0 - n1);
    const F2 B = A0 + n7, C = A0 - n7;
    const F2 X = fma2(splat(-2.0f), n4, n3), Y = fma2(splat(-2.0f), n6, n5);
    o[1] = B + X;
    o[3] = B - X;
    o[2] = C + Y;
    o[4] = C - Y;
    const F2 D0 = fma2(splat(2.0f), n1, n0 + n2);
    const F2 E = D0 + n8, G = D0 - n8;
    const F2 U = n3 + n4, V = n5 + n6;
    const F2 P = U + V, Mv = U - V;
    o[5] = E + P;
    o[7] = E - P;
    o[6] = G - Mv;
    o[8] = G + Mv;
  }
  // Row 0 of M^-1 m* would be n0 - 4 n1 + 4 n2, but FP32 n0 = phi/9 carries a fixed
  // relative bias. Since sum_i f*_i = sum_i f_i (m_0 is conserved, Eq. 34), the rest
  // population takes what the moving ones gave up: f*_0 = f_0 + sum_{i>=1} (f_i - f*_i).
  // The differences of nearby values are exact and small, so the only rounding at the
  // scale of phi is the final add.
  o[0] = f[0] + ((((f[1] - o[1]) + (f[2] - o[2])) + ((f[3] - o[3]) + (f[4] - o[4]))) +
                 (((f[5] - o[5]) + (f[6] - o[6])) + ((f[7] - o[7]) + (f[8] - o[8]))));
  phi_out = phi;
}

__device__ __forceinline__ void unpair(const F2 (&v)[2], float (&s)[4]) {
  s[0] = v[0].x;
  s[1] = v[0].y;
  s[2] = v[1].x;
  s[3] = v[1].y;
}

// Stores one collided row. DEV storage keeps the rest population and this node's
// anchor in FP32 and d_i = f*_i - w_i anchor(x + c_i) in 16 bits; the rest population
// is closed on the values a reader will rebuild, so sum_i f*_i = phi holds (mass is
// conserved to FP32 rounding, not 16-bit rounding). dmu[i-1] is the anchor of the node
// population i streams to, at this lane's columns.
template <int ST>
__device__ __forceinline__ void store_row_vec(const Field& fd, long long ro, long long col, const F2 (&o)[9][2],
                                              const F2 (&mua)[2], const F2 (&dmu)[8][2], const F2 (&phi)[2]) {
  if constexpr (ST == ST_F32) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
      *reinterpret_cast<float4*>(fd.dst.f32 + (long long)i * fd.ps + ro + col) =
          make_float4(o[i][0].x, o[i][0].y, o[i][1].x, o[i][1].y);
  } else {
    using D = Dev<ST>;
    // Columns (0, 1) and (2, 3) of each plane round in one conversion; f*_i as its reader
    // rebuilds it (anchor term plus the stored deviation) closes the rest population.
    F2 sum[2];
    uint32_t pk[8][2];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const F2 w = splat((float)wgt(i)), nw = splat(-(float)wgt(i));
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const F2 dv = fma2(nw, dmu[i - 1][k], o[i][k]);
        if constexpr (ST == ST_F16) {  // the storage scale for both columns in one packed multiply
          const F2 sv = splat(F16_SCALE) * dv;
          pk[i - 1][k] = D::pack2_scaled(sv.x, sv.y);
        } else {
          pk[i - 1][k] = D::pack2(dv.x, dv.y);
        }
        F2 back;
        D::raw2(pk[i - 1][k], back.x, back.y);
        if constexpr (D::UNSCALE != 1.0f) back = splat(D::UNSCALE) * back;
        const F2 rb = fma2(w, dmu[i - 1][k], back);
        sum[k] = i == 1 ? rb : sum[k] + rb;
      }
    }
    const F2 rest0 = phi[0] - sum[0], rest1 = phi[1] - sum[1];
    // Streaming stores (st.global.cs, evict first in L2): 0.542 -> 0.538 ms per 8192^2 BF16
    // launch on GB300. The FP32 planes keep plain stores: streaming ones ran 0.821 -> 0.834 ms.
    __stcs(reinterpret_cast<float4*>(fd.dst.f32 + ro + col), make_float4(rest0.x, rest0.y, rest1.x, rest1.y));
    __stcs(reinterpret_cast<float4*>(fd.dst.f32 + fd.ps + ro + col), make_float4(mua[0].x, mua[0].y, mua[1].x, mua[1].y));
#pragma unroll
    for (int i = 0; i < 8; ++i)
      __stcs(reinterpret_cast<uint2*>(fd.dst.dev + (long long)i * fd.ps + ro + col), make_uint2(pk[i][0], pk[i][1]));
  }
}

// Scalar-path store for columns that may be partly out of range (grids whose width is not a
// multiple of 4): the first nvalid of the 4 columns at col0.
template <int ST>
__device__ __forceinline__ void store_row_masked(const Field& fd, long long ro, int col0, int nvalid,
                                                 const F2 (&o2)[9][2], const F2 (&mua2)[2],
                                                 const F2 (&dmu2)[8][2], const F2 (&phi2)[2]) {
  float o[9][4], mua[4], dmu[8][4], phi[4];
#pragma unroll
  for (int i = 0; i < 9; ++i) unpair(o2[i], o[i]);
#pragma unroll
  for (int i = 0; i < 8; ++i) unpair(dmu2[i], dmu[i]);
  unpair(mua2, mua);
  unpair(phi2, phi);
  if constexpr (ST == ST_F32) {
    for (int j = 0; j < 4; ++j)
      if (j < nvalid)
#pragma unroll
        for (int i = 0; i < 9; ++i) fd.dst.f32[(long long)i * fd.ps + ro + col0 + j] = o[i][j];
  } else {
    using D = Dev<ST>;
    for (int j = 0; j < 4; ++j) {
      if (j >= nvalid) break;
      float sum = 0.0f;
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const float w = (float)wgt(i);
        const uint16_t d = D::store(fmaf(-w, dmu[i - 1][j], o[i][j]));
        sum += fmaf(w, dmu[i - 1][j], D::load(d));
        fd.dst.dev[(long long)(i - 1) * fd.ps + ro + col0 + j] = d;
      }
      fd.dst.f32[ro + col0 + j] = phi[j] - sum;
      fd.dst.f32[fd.ps + ro + col0 + j] = mua[j];
    }
  }
}

// 16-bit storages with the default rates cache phi, j_x and j_y of a landed row in its slot
// (over the deviations, which nothing reads after that) when the row's phi is formed; the
// collision three rows later reads them back instead of summing the deviations again.
template <int ST, bool VEC, bool FAST>
struct DevCache {
  static constexpr bool ON = VEC && FAST && ST != ST_F32;
};
__device__ __forceinline__ F2* cache_of(float4* slot) { return reinterpret_cast<F2*>(slot + 64); }
__device__ __forceinline__ const F2* cache_of(const float4* slot) { return reinterpret_cast<const F2*>(slot + 64); }

// Collides row `row` of this warp's strip from its landing slot and stores it.
// mu_m, mu_c, mu_p: mu_alpha of rows row-1, row, row+1 at this lane's columns.
template <int ST, bool VEC, bool FAST>
__device__ __forceinline__ void collide_row(const StepArgs& a, const Field& fd, const float4* slot, int lane,
                                            int row, bool store, int ocol0, int nvalid, const F2 (&mu_m)[2],
                                            const F2 (&mu_c)[2], const F2 (&mu_p)[2], const F2 (&gx)[2],
                                            const F2 (&gy)[2]) {
  F2 o[9][2], phic[2];
  if constexpr (DevCache<ST, VEC, FAST>::ON) {  // phi, j_x and j_y cached when the row landed
    const F2* cache = cache_of(slot);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      F2 oj[9];
      phic[k] = cache[k * 32 + lane];
      collide_fast(a, phic[k], cache[(2 + k) * 32 + lane], cache[(4 + k) * 32 + lane], mu_c[k], gx[k], gy[k],
                   oj);
      o[0][k] = splat(0.0f);  // the DEV store closes the rest population from phi
#pragma unroll
      for (int i = 1; i < 9; ++i) o[i][k] = oj[i];
    }
  } else {
    F2 fr[9][2];
    read_row<ST, VEC, 0>(slot, lane, fr[0]);
    read_row<ST, VEC, 1>(slot, lane, fr[1]);
    read_row<ST, VEC, 2>(slot, lane, fr[2]);
    read_row<ST, VEC, 3>(slot, lane, fr[3]);
    read_row<ST, VEC, 4>(slot, lane, fr[4]);
    read_row<ST, VEC, 5>(slot, lane, fr[5]);
    read_row<ST, VEC, 6>(slot, lane, fr[6]);
    read_row<ST, VEC, 7>(slot, lane, fr[7]);
    read_row<ST, VEC, 8>(slot, lane, fr[8]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      F2 f[9], oj[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = fr[i][k];
      collide<FAST>(a, f, mu_c[k], gx[k], gy[k], oj, phic[k]);
#pragma unroll
      for (int i = 0; i < 9; ++i) o[i][k] = oj[i];
    }
  }
  F2 dmu[8][2];
  if constexpr (ST != ST_F32) {  // anchors of the destination nodes x + c_i
    float ext[3][6];             // rows row-1, row, row+1; columns -1 .. 4 of this lane
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const F2(&m)[2] = r == 0 ? mu_m : (r == 1 ? mu_c : mu_p);
      ext[r][0] = from_lane_left(m[1].y);
      ext[r][1] = m[0].x;
      ext[r][2] = m[0].y;
      ext[r][3] = m[1].x;
      ext[r][4] = m[1].y;
      ext[r][5] = from_lane_right(m[0].x);
    }
#pragma unroll
    for (int i = 1; i < 9; ++i)
#pragma unroll
      for (int k = 0; k < 2; ++k)
        dmu[i - 1][k] = f2(ext[1 + cy(i)][2 * k + cx(i) + 1], ext[1 + cy(i)][2 * k + cx(i) + 2]);
  }
  if (store) {
    const long long ro = (long long)row * fd.nx;
    if constexpr (VEC) {
      store_row_vec<ST>(fd, ro, ocol0, o, mu_c, dmu, phic);
    } else {
      store_row_masked<ST>(fd, ro, ocol0, nvalid, o, mu_c, dmu, phic);
    }
  }
}

// One warp's work: the rows [seg * seg_len, ...) of strip `strip` of field fd.
template <int ST, bool VEC, bool FAST>
__device__ __forceinline__ void step_warp(const StepArgs& a, const Field& fd, int strip, int seg, float4* slots,
                                          int lane) {
  using PP = Pipe<ST, VEC>;
  constexpr int PF_DIST = PP::PF_DIST, COLLIDE_LAG = PP::LAG, SLOTS = PP::SLOTS, SLOT_F4 = PP::SLOT_F4;
  const int y0 = seg * fd.seg_len;
  const int y1 = min(y0 + fd.seg_len, fd.ny);
  const bool full_row = fd.nx == STRIP_W;  // one strip over the whole periodic row
  const int xs = full_row ? 0 : strip * OUT_W - HALO_W;  // strip start column (before wrap)

  Cols cl;
  cl.c0 = imod(xs + 4 * lane, fd.nx);
#pragma unroll
  for (int k = 0; k < 6; ++k) cl.cs[k] = imod(xs + 4 * lane + k - 1, fd.nx);

  // Output columns of this lane: strip columns 4 lane + j in [HALO_W, STRIP_W - HALO_W), or
  // all of them for a full row.
  const int ocol0 = xs + 4 * lane;  // global column of element 0
  const bool lane_out = full_row || (lane >= 1 && lane <= 30 && ocol0 < fd.nx);
  const int nvalid = min(4, fd.nx - ocol0);

  // Rolling accumulators (see the header comment): index 1 = row completing next, 0 = row
  // after; U and V hold the y-difference terms of the last two rows (phi and mu_beta).
  F2 Ax1[2], Al1[2], Ax0[2], Al0[2], U1[2], U0[2], php[2];
  F2 T1[2], T0[2];
  F2 Gx1[2], Gx0[2], V1[2], V0[2];
  F2 mu1[2], mu2[2], mu3[2];  // mu_alpha of rows r-2, r-3, r-4
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    Ax1[k] = Al1[k] = Ax0[k] = Al0[k] = U1[k] = U0[k] = php[k] = splat(0.0f);
    T1[k] = T0[k] = Gx1[k] = Gx0[k] = V1[k] = V0[k] = splat(0.0f);
    mu1[k] = mu2[k] = mu3[k] = splat(0.0f);
  }

  // phi rows y0-3 .. ; row y collides at phi row y + COLLIDE_LAG.
  const int n_it = (y1 - y0) + 3 + COLLIDE_LAG;
  // Rows r-1, r, r+1 (mod ny) of the next phi row to fetch.
  int fm = imod(y0 - 4, fd.ny), f0 = imod(y0 - 3, fd.ny), fp = imod(y0 - 2, fd.ny);
  auto fetch_next = [&](float4* slot) {
    issue_row<ST, VEC>(fd, slot, lane, (long long)fm * fd.nx, (long long)f0 * fd.nx, (long long)fp * fd.nx, cl);
    fm = f0;
    f0 = fp;
    fp = fp + 1 == fd.ny ? 0 : fp + 1;
  };
#pragma unroll
  for (int d = 0; d < PF_DIST; ++d) {
    if (d < n_it) fetch_next(slots + d * SLOT_F4);
    cp_async_commit();
  }
  const F2 K12 = splat(1.0f / 12.0f), K6 = splat(1.0f / 6.0f), K3 = splat(1.0f / 3.0f);
  const F2 K23 = splat(2.0f / 3.0f), KM103 = splat(-10.0f / 3.0f), K4 = splat(4.0f);
  const F2 EPS = splat(a.eps);
  int s_cur = 0, s_pf = PF_DIST, s_col = SLOTS - COLLIDE_LAG;  // slots of rows r, r+PF_DIST, r-LAG
  for (int it = 0; it < n_it; ++it) {
    // 1. Fetch row r + PF_DIST.
    if (it + PF_DIST < n_it) fetch_next(slots + s_pf * SLOT_F4);
    cp_async_commit();
    // 2. Wait for row r; pull it and sum phi (Eq. 22).
    cp_async_wait<PF_DIST>();
    F2 ph[2];
    if constexpr (VEC && ST != ST_F32) {  // grouped: one shuffle per c_x group
      float4* slot = slots + s_cur * SLOT_F4;
      DevSums ds;
      dev_sums<ST, DevCache<ST, VEC, FAST>::ON>(slot, lane, ds);
      dev_phi<ST>(slot, lane, ds, ph);
      if constexpr (DevCache<ST, VEC, FAST>::ON) {
        F2* cache = cache_of(slot);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          F2 jx = ds.gp[k] - ds.gm[k], jy = (ds.hp[k] + ds.hm[k]) + ds.h0[k];
          if constexpr (Dev<ST>::UNSCALE != 1.0f) {
            jx = splat(Dev<ST>::UNSCALE) * jx;
            jy = splat(Dev<ST>::UNSCALE) * jy;
          }
          cache[k * 32 + lane] = ph[k];
          cache[(2 + k) * 32 + lane] = jx;
          cache[(4 + k) * 32 + lane] = jy;
        }
      }
    } else {
      const float4* slot = slots + s_cur * SLOT_F4;
      F2 v[2];
      read_row<ST, VEC, 0>(slot, lane, ph);
#define LBCH_PULL(I)                    \
  read_row<ST, VEC, I>(slot, lane, v); \
  ph[0] = ph[0] + v[0];                \
  ph[1] = ph[1] + v[1];
      LBCH_PULL(1) LBCH_PULL(2) LBCH_PULL(3) LBCH_PULL(4)
      LBCH_PULL(5) LBCH_PULL(6) LBCH_PULL(7) LBCH_PULL(8)
#undef LBCH_PULL
    }
    // 3. grad phi and lap phi of row r-1 (Eq. 26a, 26b), rolling over rows.
    F2 dx[2], dy[2], lp[2];
    {
      F2 s[2], d[2];
      neighbours(ph, s, d);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const F2 e = d[k] * K12;
        const F2 u = fma2(s[k], K12, ph[k] * K3);
        const F2 t = fma2(s[k], K6, ph[k] * K23);
        dx[k] = Ax1[k] + e;
        dy[k] = u - U1[k];
        lp[k] = Al1[k] + t;
        Ax1[k] = fma2(K4, e, Ax0[k]);
        U1[k] = U0[k];
        Al1[k] = Al0[k] + fma2(s[k], K23, ph[k] * KM103);
        Ax0[k] = e;
        U0[k] = u;
        Al0[k] = t;
      }
    }
    // 4. Pointwise at row r-1.
    F2 Qx[2], Qy[2], w[2], Aq[2], mun[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) pointwise(a, fd, php[k], dx[k], dy[k], lp[k], Qx[k], Qy[k], w[k], Aq[k], mun[k]);
#pragma unroll
    for (int k = 0; k < 2; ++k) php[k] = ph[k];
    // 5. mu_beta of row r-2: A - div Q + eps lap w (Eq. 26 on Q and w).
    F2 mub[2];
    {
      F2 sx[2], dqx[2], sqy[2], dqy[2], sw[2], dw[2];
      neighbours(Qx, sx, dqx);
      neighbours(Qy, sqy, dqy);
      neighbours(w, sw, dw);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const F2 aa = dqx[k] * K12;
        const F2 bb = fma2(sqy[k], K12, Qy[k] * K3);
        const F2 cc = EPS * fma2(sw[k], K6, w[k] * K23);
        mub[k] = T1[k] + ((cc - aa) - bb);
        T1[k] = T0[k] + fma2(EPS, fma2(sw[k], K23, w[k] * KM103), fma2(splat(-4.0f), aa, Aq[k]));
        T0[k] = (bb - aa) + cc;
      }
    }
    // 6. grad mu_beta of row r-3 (Eq. 26a).
    F2 gx[2], gy[2];
    {
      F2 s[2], d[2];
      neighbours(mub, s, d);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const F2 e = d[k] * K12;
        const F2 u = fma2(s[k], K12, mub[k] * K3);
        gx[k] = Gx1[k] + e;
        gy[k] = u - V1[k];
        Gx1[k] = fma2(K4, e, Gx0[k]);
        V1[k] = V0[k];
        Gx0[k] = e;
        V0[k] = u;
      }
    }
    // 7. Collide row r-3.
    static_assert(COLLIDE_LAG == 3, "row r-3 collides right after its grad mu_beta");
    if (it >= 6)
      collide_row<ST, VEC, FAST>(a, fd, slots + s_col * SLOT_F4, lane, y0 + it - 6, lane_out, ocol0, nvalid, mu3,
                                 mu2, mu1, gx, gy);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      mu3[k] = mu2[k];
      mu2[k] = mu1[k];
      mu1[k] = mun[k];
    }
    s_cur = s_cur + 1 == SLOTS ? 0 : s_cur + 1;
    s_pf = s_pf + 1 == SLOTS ? 0 : s_pf + 1;
    s_col = s_col + 1 == SLOTS ? 0 : s_col + 1;
  }
  cp_async_wait<0>();
}

// Single field: warp w takes strip w % n_strips of segment w / n_strips.
template <int ST, bool VEC, bool FAST>
__global__ void __launch_bounds__(STEP_WARPS * 32, (Pipe<ST, VEC>::MIN_CTAS))
    step_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ Field fd, long long n_warps) {
  extern __shared__ float4 smem_slots[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const long long warp = (long long)blockIdx.x * STEP_WARPS + wib;
  if (warp >= n_warps) return;  // whole warps only: shuffles see all 32 lanes
  float4* slots = smem_slots + wib * (Pipe<ST, VEC>::SLOTS * Pipe<ST, VEC>::SLOT_F4);
  step_warp<ST, VEC, FAST>(a, fd, (int)(warp % fd.n_strips), (int)(warp / fd.n_strips), slots, lane);
}

}  // namespace lbch
