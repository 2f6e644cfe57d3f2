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

#include "lbch_lattice.cuh"

namespace lbch {

constexpr int STRIP_W = 128;                 // columns per warp strip
constexpr int HALO_W = 4;                    // halo columns on each side
constexpr int OUT_W = STRIP_W - 2 * HALO_W;  // output columns per strip
constexpr int STEP_WARPS = 4;                // warps per CTA
// Pipeline depth per storage (measured on GB300 at 8192^2): fetch one row ahead and collide
// row r-3 right after its grad mu_beta. The 16-bit storages keep 12 warps per SM (their
// landing slots are smaller); colliding row r-4 first in the iteration with no prefetch
// instead ran 10% slower once their per-row instruction count had come down, and one row
// of prefetch with r-4 needs a sixth slot, which costs a CTA per SM.
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

// Left/right neighbour sums and differences of a per-column quantity over the strip.
__device__ __forceinline__ void neighbours(const float (&q)[4], float (&s)[4], float (&d)[4]) {
  const float left = __shfl_up_sync(FULL, q[3], 1);
  const float right = __shfl_down_sync(FULL, q[0], 1);
  s[0] = left + q[1];
  d[0] = q[1] - left;
  s[1] = q[0] + q[2];
  d[1] = q[2] - q[0];
  s[2] = q[1] + q[3];
  d[2] = q[3] - q[1];
  s[3] = q[2] + right;
  d[3] = right - q[2];
}

// Per-lane addressing of the strip.
struct Cols {
  long long c0;  // aligned first column (vector path)
  int cs[6];     // columns xs + 4 lane + k - 1, k = 0..5 (scalar path), mod nx
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
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

// f_in,I at this lane's 4 columns from a landed slot.
template <int ST, bool VEC, int I>
__device__ __forceinline__ void read_row(const float4* slot, int lane, float (&v)[4]) {
  constexpr bool REBUILD = VEC && ST != ST_F32 && I != 0;
  if constexpr (!REBUILD) {
    const float4 t = slot[I * 32 + lane];
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {  // deviations of the source nodes (row r - c_Iy), shifted below
    const uint2 raw = reinterpret_cast<const uint2*>(slot + 64)[(I - 1) * 32 + lane];
    v[0] = Dev<ST>::load(static_cast<uint16_t>(raw.x & 0xffffu));
    v[1] = Dev<ST>::load(static_cast<uint16_t>(raw.x >> 16));
    v[2] = Dev<ST>::load(static_cast<uint16_t>(raw.y & 0xffffu));
    v[3] = Dev<ST>::load(static_cast<uint16_t>(raw.y >> 16));
  }
  if constexpr (VEC) {  // the pull shift along x happens here, one shuffle per plane
    if constexpr (cx(I) == 1) {  // take the column to the left
      const float prev = __shfl_up_sync(FULL, v[3], 1);
      v[3] = v[2]; v[2] = v[1]; v[1] = v[0]; v[0] = prev;
    } else if constexpr (cx(I) == -1) {  // take the column to the right
      const float next = __shfl_down_sync(FULL, v[0], 1);
      v[0] = v[1]; v[1] = v[2]; v[2] = v[3]; v[3] = next;
    }
  }
  if constexpr (REBUILD) {  // f*_I(y - c_I) = w_I anchor(y) + d_I(y - c_I)
    const float w = (float)wgt(I);
    const float4 m = slot[32 + lane];
    v[0] = fmaf(w, m.x, v[0]);
    v[1] = fmaf(w, m.y, v[1]);
    v[2] = fmaf(w, m.z, v[2]);
    v[3] = fmaf(w, m.w, v[3]);
  }
}

// Pull shift along x of a per-column quantity of the strip: column j takes column j - 1
// (c_x = 1) or column j + 1 (c_x = -1).
__device__ __forceinline__ void from_left(float (&v)[4]) {
  const float prev = __shfl_up_sync(FULL, v[3], 1);
  v[3] = v[2]; v[2] = v[1]; v[1] = v[0]; v[0] = prev;
}
__device__ __forceinline__ void from_right(float (&v)[4]) {
  const float next = __shfl_down_sync(FULL, v[0], 1);
  v[0] = v[1]; v[1] = v[2]; v[2] = v[3]; v[3] = next;
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
  float gp[4], gm[4], g0[4], hp[4], hm[4], h0[4];
};
template <int ST, bool H>
__device__ __forceinline__ void dev_sums(const float4* slot, int lane, DevSums& s) {
  const uint2* ds = reinterpret_cast<const uint2*>(slot + 64);
  float d[9][4];
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const uint2 raw = ds[(i - 1) * 32 + lane];
    Dev<ST>::raw2(raw.x, d[i][0], d[i][1]);
    Dev<ST>::raw2(raw.y, d[i][2], d[i][3]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    s.gp[j] = (d[1][j] + d[5][j]) + d[8][j];
    s.gm[j] = (d[3][j] + d[6][j]) + d[7][j];
    s.g0[j] = d[2][j] + d[4][j];
    if constexpr (H) {
      s.hp[j] = d[5][j] - d[8][j];
      s.hm[j] = d[6][j] - d[7][j];
      s.h0[j] = d[2][j] - d[4][j];
    }
  }
  from_left(s.gp);
  from_right(s.gm);
  if constexpr (H) {
    from_left(s.hp);
    from_right(s.hm);
  }
}

// phi at column j of a landed DEV row from its rest population, anchor and group sums.
template <int ST>
__device__ __forceinline__ float dev_phi(const float4* slot, int lane, const DevSums& s, int j) {
  const float4 r = slot[lane], m = slot[32 + lane];
  const float rest = j == 0 ? r.x : (j == 1 ? r.y : (j == 2 ? r.z : r.w));
  const float anc = j == 0 ? m.x : (j == 1 ? m.y : (j == 2 ? m.z : m.w));
  return fmaf(5.0f / 9.0f, anc, rest) + Dev<ST>::UNSCALE * ((s.gp[j] + s.gm[j]) + s.g0[j]);
}

// Pointwise part at one node: Q (Eq. 15 reading), w, mu_alpha (Eq. 16) and the
// local part A of mu_beta (Eq. 13 minus Eq. 16's mu_alpha).
__device__ __forceinline__ void pointwise(const StepArgs& a, const Field& fd, float phi, float dx, float dy,
                                          float lap, float& Qx, float& Qy, float& w, float& A,
                                          float& mua) {
  const float g2 = fmaf(dx, dx, dy * dy);
  const bool ok = g2 >= 1e-12f;  // n = 0, gamma = 1 below this
  const float rs = rsqrtf(ok ? g2 : 1.0f);
  const float n1 = dx * rs, n2 = dy * rs;  // Eq. 2
  const float n1s = n1 * n1, n2s = n2 * n2;
  const float S4 = fmaf(n1s, n1s, n2s * n2s);
  const float gm1 = ok ? fd.alpha * fmaf(4.0f, S4, -3.0f) : 0.0f;  // gamma - 1, Eq. 6
  // k_q |grad phi| P grad_n gamma with grad_n gamma = 16 alpha n^3, P = I - n n^T.
  const float t = ok ? a.kq * fd.a16 * (g2 * rs) : 0.0f;
  const float kg = fmaf(a.k, gm1, a.kiso);
  Qx = fmaf(kg, dx, t * (n1 * (n1s - S4)));
  Qy = fmaf(kg, dy, t * (n2 * (n2s - S4)));
  const float phi2 = phi * phi;
  const float fb = a.beta4 * phi * (phi2 - 1.0f);  // f = F'(phi), Eq. 9
  const float fp = fmaf(a.beta12, phi2, -a.beta4); // f'(phi), Eq. 13
  w = fmaf(-a.cw, fb, lap);
  mua = fmaf(-a.k, lap, fb);
  A = fmaf(gm1, fb, fmaf(-a.cfp * fp, w, a.cnk * lap));
}

// Eq. 17 at one node in moment space (Eqs. 23, 25) with the closed forms
// m^eq = (phi, -4 phi + 2 mu_a, 4 phi - 3 mu_a, 0, ...) and
// M F = (0, 0, 0, -g_x/3, g_x/3, -g_y/3, g_y/3, 0, 0), and M^-1 = M^T diag(1/|row|^2).
// FAST: s_1 = s_2 = s_4 = s_6 = s_7 = s_8 = 1, so those moments take their (forced)
// equilibrium and need not be formed; the result equals the general path's, whose
// (1 - s_k) m_k terms are then exactly zero.
// FAST collision from the three moments it needs, phi = m_0, j_x = m_3 and j_y = m_5 (the
// others take their equilibrium): o[1..8] of f*; o[0] is left to the caller.
__device__ __forceinline__ void collide_fast(const StepArgs& a, float phi, float m3, float m5, float mua, float gx,
                                             float gy, float (&o)[9]) {
  const float n0 = phi * (1.0f / 9.0f);
  const float n1 = a.c1b * fmaf(2.0f, mua, -4.0f * phi);
  const float n2 = a.c2b * fmaf(-3.0f, mua, 4.0f * phi);
  const float n4 = a.c4g * gx, n6 = a.c6g * gy;
  const float n3 = fmaf(a.c3a, m3, a.c3g * gx);
  const float n5 = fmaf(a.c5a, m5, a.c5g * gy);
  const float A0 = fmaf(-2.0f, n2, n0 - n1);
  const float X = fmaf(-2.0f, n4, n3), Y = fmaf(-2.0f, n6, n5);
  o[1] = A0 + X;
  o[3] = A0 - X;
  o[2] = A0 + Y;
  o[4] = A0 - Y;
  const float D0 = fmaf(2.0f, n1, n0 + n2);
  const float U = n3 + n4, V = n5 + n6;
  const float P = U + V, Mv = U - V;
  o[5] = D0 + P;
  o[7] = D0 - P;
  o[6] = D0 - Mv;
  o[8] = D0 + Mv;
}

template <bool FAST>
__device__ __forceinline__ void collide(const StepArgs& a, const float (&f)[9], float mua,
                                        float gx, float gy, float (&o)[9], float& phi_out) {
  const float ab = f[1] + f[3], bb = f[2] + f[4];
  const float Sa = ab + bb;
  const float e = f[5] + f[7], h = f[6] + f[8];
  const float Sd = e + h;
  const float phi = f[0] + Sa + Sd;
  const float x1 = f[1] - f[3], y1 = f[2] - f[4];
  const float p = f[5] - f[7], q = f[6] - f[8];
  const float pm = p - q, pp = p + q;
  const float m3 = x1 + pm, m5 = y1 + pp;
  if constexpr (FAST) {
    collide_fast(a, phi, m3, m5, mua, gx, gy, o);
  } else {
    const float n0 = phi * (1.0f / 9.0f);
    const float m1 = fmaf(-4.0f, f[0], fmaf(2.0f, Sd, -Sa));
    const float m2 = fmaf(4.0f, f[0], fmaf(-2.0f, Sa, Sd));
    const float m4 = fmaf(-2.0f, x1, pm), m6 = fmaf(-2.0f, y1, pp);
    const float m7 = ab - bb, m8 = e - h;
    const float n1 = fmaf(a.c1a, m1, a.c1b * fmaf(2.0f, mua, -4.0f * phi));
    const float n2 = fmaf(a.c2a, m2, a.c2b * fmaf(-3.0f, mua, 4.0f * phi));
    const float n4 = fmaf(a.c4a, m4, a.c4g * gx);
    const float n6 = fmaf(a.c6a, m6, a.c6g * gy);
    const float n7 = a.c7 * m7;
    const float n8 = a.c8 * m8;
    const float n3 = fmaf(a.c3a, m3, a.c3g * gx);
    const float n5 = fmaf(a.c5a, m5, a.c5g * gy);
    const float A0 = fmaf(-2.0f, n2, n0 - n1);
    const float B = A0 + n7, C = A0 - n7;
    const float X = fmaf(-2.0f, n4, n3), Y = fmaf(-2.0f, n6, n5);
    o[1] = B + X;
    o[3] = B - X;
    o[2] = C + Y;
    o[4] = C - Y;
    const float D0 = fmaf(2.0f, n1, n0 + n2);
    const float E = D0 + n8, G = D0 - n8;
    const float U = n3 + n4, V = n5 + n6;
    const float P = U + V, Mv = U - V;
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

// Stores one collided row. DEV storage keeps the rest population and this node's
// anchor in FP32 and d_i = f*_i - w_i anchor(x + c_i) in 16 bits; the rest population
// is closed on the values a reader will rebuild, so sum_i f*_i = phi holds (mass is
// conserved to FP32 rounding, not 16-bit rounding). dmu[i-1][j] is the anchor of the
// node population i of column j streams to.
template <int ST, bool VEC>
__device__ __forceinline__ void store_row(const Field& fd, long long ro, long long col,
                                          const float (&o)[9][4], const float (&mua)[4],
                                          const float (&dmu)[8][4], const float (&phi)[4]) {
  if constexpr (ST == ST_F32) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      float* p = fd.dst.f32 + (long long)i * fd.ps + ro + col;
      if constexpr (VEC) {
        *reinterpret_cast<float4*>(p) = make_float4(o[i][0], o[i][1], o[i][2], o[i][3]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = o[i][j];
      }
    }
  } else {
    using D = Dev<ST>;
    // Columns (0, 1) and (2, 3) of each plane round in one conversion; f*_i as its reader
    // rebuilds it (anchor term plus the stored deviation) closes the rest population.
    float rest[4], sum[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    uint32_t pk[8][2];
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      const float w = (float)wgt(i);
      float dv[4], back[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) dv[j] = o[i][j] - w * dmu[i - 1][j];
      pk[i - 1][0] = D::pack2(dv[0], dv[1]);
      pk[i - 1][1] = D::pack2(dv[2], dv[3]);
      D::raw2(pk[i - 1][0], back[0], back[1]);
      D::raw2(pk[i - 1][1], back[2], back[3]);
#pragma unroll
      for (int j = 0; j < 4; ++j) sum[j] += fmaf(w, dmu[i - 1][j], back[j] * D::UNSCALE);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) rest[j] = phi[j] - sum[j];
    float* p0 = fd.dst.f32 + ro + col;
    float* pm = fd.dst.f32 + fd.ps + ro + col;
    if constexpr (VEC) {
      *reinterpret_cast<float4*>(p0) = make_float4(rest[0], rest[1], rest[2], rest[3]);
      *reinterpret_cast<float4*>(pm) = make_float4(mua[0], mua[1], mua[2], mua[3]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        p0[j] = rest[j];
        pm[j] = mua[j];
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      uint16_t* pd = fd.dst.dev + (long long)i * fd.ps + ro + col;
      if constexpr (VEC) {
        *reinterpret_cast<uint2*>(pd) = make_uint2(pk[i][0], pk[i][1]);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) pd[j] = static_cast<uint16_t>(pk[i][j >> 1] >> (16 * (j & 1)));
      }
    }
  }
}

// Scalar-path store for columns that may be partly out of range (not 4-aligned grids).
template <int ST>
__device__ __forceinline__ void store_row_masked(const Field& fd, long long ro, int col0, int nvalid,
                                                 const float (&o)[9][4], const float (&mua)[4],
                                                 const float (&dmu)[8][4], const float (&phi)[4]) {
  if (nvalid >= 4) {
    store_row<ST, false>(fd, ro, col0, o, mua, dmu, phi);
    return;
  }
  // Fewer than 4 valid columns: write them one at a time.
  if constexpr (ST == ST_F32) {
    for (int j = 0; j < nvalid; ++j)
#pragma unroll
      for (int i = 0; i < 9; ++i) fd.dst.f32[(long long)i * fd.ps + ro + col0 + j] = o[i][j];
  } else {
    using D = Dev<ST>;
    for (int j = 0; j < nvalid; ++j) {
      float sum = 0.0f;
#pragma unroll
      for (int i = 1; i < 9; ++i) {
        const float w = (float)wgt(i);
        const uint16_t d = D::store(o[i][j] - w * dmu[i - 1][j]);
        sum += fmaf(w, dmu[i - 1][j], D::load(d));
        fd.dst.dev[(long long)(i - 1) * fd.ps + ro + col0 + j] = d;
      }
      fd.dst.f32[ro + col0 + j] = phi[j] - sum;
      fd.dst.f32[fd.ps + ro + col0 + j] = mua[j];
    }
  }
}

// Collides row `row` of this warp's strip from its landing slot and stores it.
// mu_m, mu_c, mu_p: mu_alpha of rows row-1, row, row+1 at this lane's columns.
template <int ST, bool VEC, bool FAST>
__device__ __forceinline__ void collide_row(const StepArgs& a, const Field& fd, const float4* slot, int lane,
                                            int row,
                                            bool store, int ocol0, int nvalid, const float (&mu_m)[4],
                                            const float (&mu_c)[4], const float (&mu_p)[4],
                                            const float (&gx)[4], const float (&gy)[4]) {
  float o[9][4], phic[4];
  if constexpr (VEC && FAST && ST != ST_F32) {  // phi, j_x and j_y straight from the deviations
    DevSums ds;
    dev_sums<ST, true>(slot, lane, ds);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float oj[9];
      phic[j] = dev_phi<ST>(slot, lane, ds, j);
      const float m3 = Dev<ST>::UNSCALE * (ds.gp[j] - ds.gm[j]);
      const float m5 = Dev<ST>::UNSCALE * ((ds.hp[j] + ds.hm[j]) + ds.h0[j]);
      collide_fast(a, phic[j], m3, m5, mu_c[j], gx[j], gy[j], oj);
      o[0][j] = 0.0f;  // the DEV store closes the rest population from phi
#pragma unroll
      for (int i = 1; i < 9; ++i) o[i][j] = oj[i];
    }
  } else {
    float fr[9][4];
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
    for (int j = 0; j < 4; ++j) {
      float f[9], oj[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = fr[i][j];
      collide<FAST>(a, f, mu_c[j], gx[j], gy[j], oj, phic[j]);
#pragma unroll
      for (int i = 0; i < 9; ++i) o[i][j] = oj[i];
    }
  }
  float dmu[8][4];
  if constexpr (ST != ST_F32) {  // anchors of the destination nodes x + c_i
    float ext[3][6];             // rows row-1, row, row+1; columns -1 .. 4 of this lane
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float(&m)[4] = k == 0 ? mu_m : (k == 1 ? mu_c : mu_p);
      ext[k][0] = __shfl_up_sync(FULL, m[3], 1);
      ext[k][1] = m[0];
      ext[k][2] = m[1];
      ext[k][3] = m[2];
      ext[k][4] = m[3];
      ext[k][5] = __shfl_down_sync(FULL, m[0], 1);
    }
#pragma unroll
    for (int i = 1; i < 9; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) dmu[i - 1][j] = ext[1 + cy(i)][j + cx(i) + 1];
  }
  if (store) {
    const long long ro = (long long)row * fd.nx;
    if constexpr (VEC) {
      store_row<ST, true>(fd, ro, ocol0, o, mu_c, dmu, phic);
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
  const int xs = strip * OUT_W - HALO_W;  // strip start column (before wrap)

  Cols cl;
  cl.c0 = imod(xs + 4 * lane, fd.nx);
#pragma unroll
  for (int k = 0; k < 6; ++k) cl.cs[k] = imod(xs + 4 * lane + k - 1, fd.nx);

  // Output columns of this lane: strip columns 4 lane + j in [HALO_W, STRIP_W - HALO_W).
  const int ocol0 = strip * OUT_W + 4 * lane - HALO_W;  // global column of element 0
  const bool lane_out = lane >= 1 && lane <= 30 && ocol0 < fd.nx;
  const int nvalid = min(4, fd.nx - ocol0);

  // Rolling accumulators (see the header comment): index 1 = row completing next, 0 = row after.
  float Ax1[4], Ay1[4], Al1[4], Ax0[4], Ay0[4], Al0[4], php[4];
  float T1[4], T0[4];
  float Gx1[4], Gy1[4], Gx0[4], Gy0[4];
  float mu1[4], mu2[4], mu3[4];  // mu_alpha of rows r-2, r-3, r-4
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    Ax1[j] = Ay1[j] = Al1[j] = Ax0[j] = Ay0[j] = Al0[j] = php[j] = 0.0f;
    T1[j] = T0[j] = Gx1[j] = Gy1[j] = Gx0[j] = Gy0[j] = 0.0f;
    mu1[j] = mu2[j] = mu3[j] = 0.0f;
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
  int s_cur = 0, s_pf = PF_DIST, s_col = SLOTS - COLLIDE_LAG;  // slots of rows r, r+PF_DIST, r-LAG
  for (int it = 0; it < n_it; ++it) {
    // 1. Fetch row r + PF_DIST.
    if (it + PF_DIST < n_it) fetch_next(slots + s_pf * SLOT_F4);
    cp_async_commit();
    // 2. Wait for row r; pull it and sum phi (Eq. 22).
    cp_async_wait<PF_DIST>();
    float ph[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if constexpr (VEC && ST != ST_F32) {  // grouped: one shuffle per c_x group
      const float4* slot = slots + s_cur * SLOT_F4;
      DevSums ds;
      dev_sums<ST, false>(slot, lane, ds);
#pragma unroll
      for (int j = 0; j < 4; ++j) ph[j] = dev_phi<ST>(slot, lane, ds, j);
    } else {
      const float4* slot = slots + s_cur * SLOT_F4;
      float v[4];
#define LBCH_PULL(I)                    \
  read_row<ST, VEC, I>(slot, lane, v); \
  ph[0] += v[0]; ph[1] += v[1]; ph[2] += v[2]; ph[3] += v[3];
      LBCH_PULL(0) LBCH_PULL(1) LBCH_PULL(2) LBCH_PULL(3) LBCH_PULL(4)
      LBCH_PULL(5) LBCH_PULL(6) LBCH_PULL(7) LBCH_PULL(8)
#undef LBCH_PULL
    }
    // 3. grad phi and lap phi of row r-1 (Eq. 26a, 26b), rolling over rows.
    float dx[4], dy[4], lp[4];
    {
      float s[4], d[4];
      neighbours(ph, s, d);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float e = d[j] * (1.0f / 12.0f);
        const float u = fmaf(s[j], 1.0f / 12.0f, ph[j] * (1.0f / 3.0f));
        const float t = fmaf(s[j], 1.0f / 6.0f, ph[j] * (2.0f / 3.0f));
        dx[j] = Ax1[j] + e;
        dy[j] = Ay1[j] + u;
        lp[j] = Al1[j] + t;
        Ax1[j] = fmaf(4.0f, e, Ax0[j]);
        Ay1[j] = Ay0[j];
        Al1[j] = Al0[j] + fmaf(s[j], 2.0f / 3.0f, ph[j] * (-10.0f / 3.0f));
        Ax0[j] = e;
        Ay0[j] = -u;
        Al0[j] = t;
      }
    }
    // 4. Pointwise at row r-1.
    float Qx[4], Qy[4], w[4], Aq[4], mun[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) pointwise(a, fd, php[j], dx[j], dy[j], lp[j], Qx[j], Qy[j], w[j], Aq[j], mun[j]);
#pragma unroll
    for (int j = 0; j < 4; ++j) php[j] = ph[j];
    // 5. mu_beta of row r-2: A - div Q + eps lap w (Eq. 26 on Q and w).
    float mub[4];
    {
      float sx[4], dqx[4], sqy[4], dqy[4], sw[4], dw[4];
      neighbours(Qx, sx, dqx);
      neighbours(Qy, sqy, dqy);
      neighbours(w, sw, dw);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float aa = dqx[j] * (1.0f / 12.0f);
        const float bb = fmaf(sqy[j], 1.0f / 12.0f, Qy[j] * (1.0f / 3.0f));
        const float cc = a.eps * fmaf(sw[j], 1.0f / 6.0f, w[j] * (2.0f / 3.0f));
        mub[j] = T1[j] + (cc - aa - bb);
        T1[j] = T0[j] + (fmaf(-4.0f, aa, Aq[j]) +
                         a.eps * fmaf(sw[j], 2.0f / 3.0f, w[j] * (-10.0f / 3.0f)));
        T0[j] = (bb - aa) + cc;
      }
    }
    // 6. grad mu_beta of row r-3 (Eq. 26a).
    float gx[4], gy[4];
    {
      float s[4], d[4];
      neighbours(mub, s, d);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float e = d[j] * (1.0f / 12.0f);
        const float u = fmaf(s[j], 1.0f / 12.0f, mub[j] * (1.0f / 3.0f));
        gx[j] = Gx1[j] + e;
        gy[j] = Gy1[j] + u;
        Gx1[j] = fmaf(4.0f, e, Gx0[j]);
        Gy1[j] = Gy0[j];
        Gx0[j] = e;
        Gy0[j] = -u;
      }
    }
    // 7. Collide row r-3.
    static_assert(COLLIDE_LAG == 3, "row r-3 collides right after its grad mu_beta");
    if (it >= 6)
      collide_row<ST, VEC, FAST>(a, fd, slots + s_col * SLOT_F4, lane, y0 + it - 6, lane_out, ocol0, nvalid, mu3,
                                 mu2, mu1, gx, gy);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      mu3[j] = mu2[j];
      mu2[j] = mu1[j];
      mu1[j] = mun[j];
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
