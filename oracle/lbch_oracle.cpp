// FP64 CPU oracle for the MRT lattice Boltzmann scheme for the anisotropic
// Cahn-Hilliard equation (arXiv 2501.03759). TEST INFRASTRUCTURE ONLY: see
// lbch_oracle.h for the contract, the pins, and what is unpinned.
//
// One time step follows Section 3 of the paper as whole-field passes over plain
// arrays, with periodic (modulo) neighbour indexing and no tiling or fusion:
//   1. phi = sum_i f_i                                     (Eq. 22)
//   2. grad phi, lap phi                                   (Eq. 26a, 26b)
//   3. n, gamma(n), grad_n gamma, P, Q, f(phi), f'(phi),
//      w = lap phi - f, mu_alpha = f - k lap phi           (Eqs. 2, 6, 15, 9, 13, 16)
//   4. div Q, lap w, mu_beta = mu - mu_alpha               (Eqs. 13, 16, 26)
//   5. grad mu_beta and F_i = -w_i c_i . grad mu_beta      (Eqs. 26a, 19)
//   6. collision f* = f - M^-1 S M (f - f^eq) + M^-1 (I - S/2) M F   (Eq. 17)
//   7. streaming f_i(x + c_i, t + 1) = f*_i(x)             (Eq. 17, periodic)
//
// Readings where the paper is silent or garbled (each is a named choice):
//   - Eq. 15 drops the k that Eq. 14 carries once F ~ k|grad phi|^2/2 is used; the
//     default keeps it: Q = gamma k grad phi + k |grad phi| P grad_n gamma.
//     ORC_Q_LITERAL drops it as printed.
//   - mu_beta = mu - mu_alpha (Eq. 16). By default the isotropic part of -div Q
//     cancels against the -k lap phi inside mu_alpha analytically, so
//     mu_beta = (gamma - 1) f - div Qt + eps (lap w - f' w) with
//     Qt = (gamma - 1) k grad phi + k |grad phi| P grad_n gamma; then gamma = 1
//     gives mu_beta = eps(...) only, and mu_beta = 0 when also eps = 0 (the
//     isotropic reduction stated after Eq. 16). ORC_MU_NESTED takes mu - mu_alpha
//     with the full Q and nested Eq. 26a stencils instead.
//   - n = grad phi/|grad phi| is undefined where grad phi = 0: where
//     |grad phi|^2 < 1e-12 the node takes n = 0, gamma = 1, P grad_n gamma = 0
//     (a threshold an FP32 gradient can resolve: its rounding noise stays below 1e-14).
//   - grad_n gamma is the R^2 gradient of Eq. 6 in n: 16 alpha (n_1^3, n_2^3).
//   - Only s_3 = s_5 is fixed (by M = c_s^2 (1/s_3 - 1/2) dt after Eq. 38);
//     the other rates are inputs.
//   - Initial state: f = f^eq(phi0, mu_alpha(phi0)).
//   - Discrete energy: sum over nodes of gamma (k/2 |grad phi|^2 + F) + eps/2 G,
//     with the Eq. 26 stencils and unit cell area.

#include "lbch_oracle.h"

#include <cmath>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// Eq. 20a (c = 1) and Eq. 20b.
const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
const double WGT[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                       1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
// c_s = c / sqrt(3), c = dx/dt = 1 (text after Eq. 21); dt = dx = 1.
const double CS2 = 1.0 / 3.0;
const double GUARD = 1e-12;

// Eq. 23.
const double MROWS[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}};

// Gauss-Jordan inversion with partial pivoting of a 9x9 matrix.
void invert9(const double a_in[9][9], double inv[9][9]) {
  double a[9][18];
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 18; ++c) a[r][c] = c < 9 ? a_in[r][c] : (c - 9 == r ? 1.0 : 0.0);
  for (int col = 0; col < 9; ++col) {
    int piv = col;
    for (int r = col + 1; r < 9; ++r)
      if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
    if (piv != col)
      for (int c = 0; c < 18; ++c) std::swap(a[col][c], a[piv][c]);
    const double d = a[col][col];
    for (int c = 0; c < 18; ++c) a[col][c] /= d;
    for (int r = 0; r < 9; ++r) {
      if (r == col) continue;
      const double m = a[r][col];
      if (m == 0.0) continue;
      for (int c = 0; c < 18; ++c) a[r][c] -= m * a[col][c];
    }
  }
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) inv[r][c] = a[r][c + 9];
}

struct Scheme {
  int nx, ny;
  double k, beta, eps, alpha;
  int reg;
  unsigned flags;
  double s[9];
  double Minv[9][9];
  double A[9][9];  // M^-1 S M
  double B[9][9];  // M^-1 (I - S/2) M
};

int derive(const orc_params* p, orc_derived* d) {
  if (!p || !d) return -1;
  if (!(p->sigma > 0) || !(p->D > 0) || !(p->M > 0)) return -1;
  // Eq. 5: sigma = 4 sqrt(2 k beta)/3, D = sqrt(2k/beta).
  // From the second, k = beta D^2/2; then sqrt(2 k beta) = beta D, so
  // sigma = 4 beta D/3, beta = 3 sigma/(4D), k = 3 sigma D/8.
  d->beta = 3.0 * p->sigma / (4.0 * p->D);
  d->k = d->beta * p->D * p->D / 2.0;
  for (int i = 0; i < 9; ++i) d->s[i] = p->s[i];
  if (!(p->flags & ORC_S35_EXPLICIT)) {
    // After Eq. 38: M = c_s^2 (1/s_{3,5} - 1/2) dt with dt = 1.
    const double s35 = 1.0 / (p->M / CS2 + 0.5);
    d->s[3] = s35;
    d->s[5] = s35;
  }
  for (int i = 1; i < 9; ++i)
    if (!(d->s[i] > 0.0 && d->s[i] < 2.0)) return -1;
  return 0;
}

int make_scheme(const orc_params* p, Scheme* sc) {
  orc_derived d;
  if (derive(p, &d) != 0) return -1;
  if (p->nx < 1 || p->ny < 1) return -1;
  sc->nx = p->nx;
  sc->ny = p->ny;
  sc->k = d.k;
  sc->beta = d.beta;
  sc->eps = p->eps;
  sc->alpha = p->alpha;
  sc->reg = p->regularization;
  sc->flags = p->flags;
  for (int i = 0; i < 9; ++i) sc->s[i] = d.s[i];
  invert9(MROWS, sc->Minv);
  // A = M^-1 S M, B = M^-1 (I - S/2) M, exactly the bracketed matrices of Eq. 17.
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) {
      double a = 0.0, b = 0.0;
      for (int m = 0; m < 9; ++m) {
        a += sc->Minv[i][m] * sc->s[m] * MROWS[m][j];
        b += sc->Minv[i][m] * (1.0 - sc->s[m] / 2.0) * MROWS[m][j];
      }
      sc->A[i][j] = a;
      sc->B[i][j] = b;
    }
  return 0;
}

inline int wrap(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

// Eq. 26a at node (x, y) of field chi.
inline void grad26(const Scheme& sc, const double* chi, int x, int y, double* gx, double* gy) {
  double sx = 0.0, sy = 0.0;
  for (int i = 0; i < 9; ++i) {
    const double v = chi[wrap(y + CY[i], sc.ny) * sc.nx + wrap(x + CX[i], sc.nx)];
    sx += WGT[i] * CX[i] * v;
    sy += WGT[i] * CY[i] * v;
  }
  *gx = sx / CS2;
  *gy = sy / CS2;
}

// Eq. 26b at node (x, y) of field chi.
inline double lap26(const Scheme& sc, const double* chi, int x, int y) {
  const double c = chi[y * sc.nx + x];
  double s = 0.0;
  for (int i = 0; i < 9; ++i) {
    const double v = chi[wrap(y + CY[i], sc.ny) * sc.nx + wrap(x + CX[i], sc.nx)];
    s += 2.0 * WGT[i] * (v - c);
  }
  return s / CS2;
}

// Eq. 4 and the derivatives given after Eq. 9 and Eq. 13.
inline double bulkF(const Scheme& sc, double phi) {
  return sc.beta * (phi - 1.0) * (phi - 1.0) * (phi + 1.0) * (phi + 1.0);
}
inline double bulk_f(const Scheme& sc, double phi) {
  return 4.0 * sc.beta * phi * (phi + 1.0) * (phi - 1.0);
}
inline double bulk_fp(const Scheme& sc, double phi) {
  return 4.0 * sc.beta * (3.0 * phi * phi - 1.0);
}

// Anisotropy at one node from grad phi (Eqs. 2, 6 and the projection after Eq. 14).
struct Aniso {
  double gamma;   // gamma(n), Eq. 6
  double Pgx, Pgy;  // P grad_n gamma
  double gnorm;   // |grad phi|
};

inline Aniso anisotropy(const Scheme& sc, double dx, double dy) {
  Aniso a;
  const double g2 = dx * dx + dy * dy;
  a.gnorm = std::sqrt(g2);
  if (g2 < GUARD) {
    a.gamma = 1.0;
    a.Pgx = 0.0;
    a.Pgy = 0.0;
    return a;
  }
  const double n1 = dx / a.gnorm, n2 = dy / a.gnorm;   // Eq. 2
  const double n1_4 = n1 * n1 * n1 * n1, n2_4 = n2 * n2 * n2 * n2;
  a.gamma = 1.0 + sc.alpha * (4.0 * (n1_4 + n2_4) - 3.0);  // Eq. 6, d = 2
  const double gn1 = 16.0 * sc.alpha * n1 * n1 * n1;       // grad_n gamma
  const double gn2 = 16.0 * sc.alpha * n2 * n2 * n2;
  // P = I - n n^T applied to grad_n gamma.
  const double P11 = 1.0 - n1 * n1, P12 = -n1 * n2, P22 = 1.0 - n2 * n2;
  a.Pgx = P11 * gn1 + P12 * gn2;
  a.Pgy = P12 * gn1 + P22 * gn2;
  return a;
}

struct Fields {
  std::vector<double> phi, dx, dy, lap, gamma, Qx, Qy, w, mua, mub, gx, gy, lap2;
  explicit Fields(size_t n)
      : phi(n), dx(n), dy(n), lap(n), gamma(n), Qx(n), Qy(n), w(n), mua(n), mub(n), gx(n), gy(n),
        lap2(n) {}
};

// Steps 1-5 of the header: all fields the collision needs.
void compute_fields(const Scheme& sc, const double* f, Fields& F) {
  const int nx = sc.nx, ny = sc.ny;
  const size_t N = size_t(nx) * ny;
  // 1. Eq. 22.
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t id = size_t(y) * nx + x;
      double s = 0.0;
      for (int i = 0; i < 9; ++i) s += f[i * N + id];
      F.phi[id] = s;
    }
  // 2. Eq. 26a, 26b on phi.
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t id = size_t(y) * nx + x;
      grad26(sc, F.phi.data(), x, y, &F.dx[id], &F.dy[id]);
      F.lap[id] = lap26(sc, F.phi.data(), x, y);
    }
  // 3. Pointwise anisotropy, Q, w, mu_alpha.
  const bool literal_q = sc.flags & ORC_Q_LITERAL;
  const bool nested = sc.flags & ORC_MU_NESTED;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t id = size_t(y) * nx + x;
      const Aniso a = anisotropy(sc, F.dx[id], F.dy[id]);
      F.gamma[id] = a.gamma;
      const double kq = literal_q ? 1.0 : sc.k;  // factor on |grad phi| P grad_n gamma
      // Eq. 15; in split form the isotropic part k grad phi is left to mu_alpha.
      const double iso = nested ? a.gamma : (a.gamma - 1.0);
      F.Qx[id] = iso * sc.k * F.dx[id] + kq * a.gnorm * a.Pgx;
      F.Qy[id] = iso * sc.k * F.dy[id] + kq * a.gnorm * a.Pgy;
      const double fb = bulk_f(sc, F.phi[id]);
      F.w[id] = F.lap[id] - fb;                  // Delta phi - f(phi), Eq. 9
      F.mua[id] = fb - sc.k * F.lap[id];         // Eq. 16
    }
  // Linear regularisation needs lap(lap phi) (Eq. 12).
  if (sc.reg == 2) {
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) F.lap2[size_t(y) * nx + x] = lap26(sc, F.lap.data(), x, y);
  }
  // 4. mu_beta = mu - mu_alpha (Eqs. 13/12, 16).
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t id = size_t(y) * nx + x;
      double qxx, qxy, qyx, qyy;
      grad26(sc, F.Qx.data(), x, y, &qxx, &qxy);
      grad26(sc, F.Qy.data(), x, y, &qyx, &qyy);
      const double divQ = qxx + qyy;
      const double phi = F.phi[id];
      const double fb = bulk_f(sc, phi);
      double reg = 0.0;
      if (sc.reg == 1) {
        reg = sc.eps * (lap26(sc, F.w.data(), x, y) - bulk_fp(sc, phi) * F.w[id]);  // Eq. 13
      } else if (sc.reg == 2) {
        reg = sc.eps * F.lap2[id];  // Eq. 12
      }
      if (nested) {
        const double mu = F.gamma[id] * fb - divQ + reg;  // Eq. 11 with Eq. 13 or 12
        F.mub[id] = mu - F.mua[id];
      } else {
        F.mub[id] = (F.gamma[id] - 1.0) * fb - divQ + reg;
      }
    }
  // 5. Eq. 26a on mu_beta.
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t id = size_t(y) * nx + x;
      grad26(sc, F.mub.data(), x, y, &F.gx[id], &F.gy[id]);
    }
}

void equilibrium(double phi, double mua, double feq[9]) {
  // Eq. 18.
  for (int i = 0; i < 9; ++i) feq[i] = WGT[i] * mua;
  feq[0] = phi + (WGT[0] - 1.0) * mua;
}

void source(double gx, double gy, double F[9]) {
  // Eq. 19.
  for (int i = 0; i < 9; ++i) F[i] = -WGT[i] * (CX[i] * gx + CY[i] * gy);
}

void collide(const Scheme& sc, const double f[9], double phi, double mua, double gx, double gy,
             double out[9]) {
  double feq[9], F[9], neq[9];
  equilibrium(phi, mua, feq);
  source(gx, gy, F);
  for (int j = 0; j < 9; ++j) neq[j] = f[j] - feq[j];
  // Eq. 17 with dt = 1.
  for (int i = 0; i < 9; ++i) {
    double relax = 0.0, force = 0.0;
    for (int j = 0; j < 9; ++j) {
      relax += sc.A[i][j] * neq[j];
      force += sc.B[i][j] * F[j];
    }
    out[i] = f[i] - relax + force;
  }
}

void step_once(const Scheme& sc, double* f, Fields& F, std::vector<double>& fstar) {
  const int nx = sc.nx, ny = sc.ny;
  const size_t N = size_t(nx) * ny;
  compute_fields(sc, f, F);
  // 6. Collision at every node.
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t id = size_t(y) * nx + x;
      double fi[9], fo[9];
      for (int i = 0; i < 9; ++i) fi[i] = f[i * N + id];
      collide(sc, fi, F.phi[id], F.mua[id], F.gx[id], F.gy[id], fo);
      for (int i = 0; i < 9; ++i) fstar[i * N + id] = fo[i];
    }
  // 7. Streaming, periodic: f_i(x + c_i) = f*_i(x).
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x)
      for (int i = 0; i < 9; ++i) {
        const size_t dst = size_t(wrap(y + CY[i], ny)) * nx + wrap(x + CX[i], nx);
        f[i * N + dst] = fstar[i * N + size_t(y) * nx + x];
      }
}

}  // namespace

extern "C" {

int orc_derive(const orc_params* p, orc_derived* out) { return derive(p, out); }

void orc_matrices(double* M81, double* Minv81) {
  double inv[9][9];
  invert9(MROWS, inv);
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) {
      if (M81) M81[r * 9 + c] = MROWS[r][c];
      if (Minv81) Minv81[r * 9 + c] = inv[r][c];
    }
}

void orc_equilibrium(double phi, double mu_alpha, double feq[9]) { equilibrium(phi, mu_alpha, feq); }

void orc_source(double gx, double gy, double F[9]) { source(gx, gy, F); }

void orc_collide_site(const orc_params* p, const double f[9], double phi, double mu_alpha,
                      double gx, double gy, double out[9]) {
  Scheme sc;
  if (make_scheme(p, &sc) != 0) {
    for (int i = 0; i < 9; ++i) out[i] = NAN;
    return;
  }
  collide(sc, f, phi, mu_alpha, gx, gy, out);
}

int orc_init(const orc_params* p, const double* phi0, double* f) {
  Scheme sc;
  if (make_scheme(p, &sc) != 0) return -1;
  const int nx = sc.nx, ny = sc.ny;
  const size_t N = size_t(nx) * ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t id = size_t(y) * nx + x;
      const double mua = bulk_f(sc, phi0[id]) - sc.k * lap26(sc, phi0, x, y);  // Eq. 16
      double feq[9];
      equilibrium(phi0[id], mua, feq);
      for (int i = 0; i < 9; ++i) f[i * N + id] = feq[i];
    }
  return 0;
}

int orc_step(const orc_params* p, double* f, int64_t nsteps) {
  Scheme sc;
  if (make_scheme(p, &sc) != 0) return -1;
  const size_t N = size_t(sc.nx) * sc.ny;
  Fields F(N);
  std::vector<double> fstar(9 * N);
  for (int64_t t = 0; t < nsteps; ++t) step_once(sc, f, F, fstar);
  return 0;
}

int orc_phi(const orc_params* p, const double* f, double* phi) {
  Scheme sc;
  if (make_scheme(p, &sc) != 0) return -1;
  const size_t N = size_t(sc.nx) * sc.ny;
  for (size_t id = 0; id < N; ++id) {
    double s = 0.0;
    for (int i = 0; i < 9; ++i) s += f[i * N + id];
    phi[id] = s;
  }
  return 0;
}

int orc_fields(const orc_params* p, const double* f, double* out12) {
  Scheme sc;
  if (make_scheme(p, &sc) != 0) return -1;
  const size_t N = size_t(sc.nx) * sc.ny;
  Fields F(N);
  compute_fields(sc, f, F);
  const std::vector<double>* src[12] = {&F.phi, &F.dx, &F.dy, &F.lap, &F.gamma, &F.Qx,
                                        &F.Qy,  &F.w,  &F.mua, &F.mub, &F.gx, &F.gy};
  for (int q = 0; q < 12; ++q) std::memcpy(out12 + q * N, src[q]->data(), N * sizeof(double));
  return 0;
}

double orc_mass(const orc_params* p, const double* f) {
  Scheme sc;
  if (make_scheme(p, &sc) != 0) return NAN;
  const size_t N = size_t(sc.nx) * sc.ny;
  double m = 0.0;
  for (size_t id = 0; id < N; ++id)
    for (int i = 0; i < 9; ++i) m += f[i * N + id];
  return m;
}

double orc_energy(const orc_params* p, const double* f) {
  Scheme sc;
  if (make_scheme(p, &sc) != 0) return NAN;
  const int nx = sc.nx, ny = sc.ny;
  const size_t N = size_t(nx) * ny;
  std::vector<double> phi(N), row(ny);
  orc_phi(p, f, phi.data());
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y) {
    double acc = 0.0;
    for (int x = 0; x < nx; ++x) {
      const size_t id = size_t(y) * nx + x;
      double dx, dy;
      grad26(sc, phi.data(), x, y, &dx, &dy);
      const double lap = lap26(sc, phi.data(), x, y);
      const Aniso a = anisotropy(sc, dx, dy);
      // Eq. 7: gamma(n) (k/2 |grad phi|^2 + F(phi)) + eps/2 G(phi).
      double e = a.gamma * (0.5 * sc.k * (dx * dx + dy * dy) + bulkF(sc, phi[id]));
      if (sc.reg == 1) {
        const double w = lap - bulk_f(sc, phi[id]);  // Eq. 9
        e += 0.5 * sc.eps * w * w;
      } else if (sc.reg == 2) {
        e += 0.5 * sc.eps * lap * lap;  // Eq. 8
      }
      acc += e;
    }
    row[y] = acc;
  }
  double E = 0.0;
  for (int y = 0; y < ny; ++y) E += row[y];
  return E;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

}  // extern "C"

// ===================================================================================
// 3D: D3Q15, the same scheme with d = 3 (Eqs. 3, 6, 17-19, 21, 22, 24, 26).
// ===================================================================================

namespace {

// Eq. 21a (c = 1) and Eq. 21b.
const int CX3[15] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
const int CY3[15] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1};
const int CZ3[15] = {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1};
const double W3[15] = {2.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                       1.0 / 9.0,  1.0 / 9.0,  1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0,
                       1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0};

// Row k of Eq. 24 as the function of c it names, at velocity i.
double m3_row(int k, int i) {
  const double x = CX3[i], y = CY3[i], z = CZ3[i], c2 = x * x + y * y + z * z;
  switch (k) {
    case 0: return 1.0;                                      // rho
    case 1: return c2 - 2.0;                                 // e
    case 2: return (15.0 * c2 * c2 - 55.0 * c2 + 32.0) / 2;  // epsilon
    case 3: return x;                                        // j_x
    case 4: return (5.0 * c2 - 13.0) / 2.0 * x;              // q_x
    case 5: return y;                                        // j_y
    case 6: return (5.0 * c2 - 13.0) / 2.0 * y;              // q_y
    case 7: return z;                                        // j_z
    case 8: return (5.0 * c2 - 13.0) / 2.0 * z;              // q_z
    case 9: return 3.0 * x * x - c2;                         // 3 p_xx
    case 10: return y * y - z * z;                           // p_ww
    case 11: return x * y;                                   // p_xy
    case 12: return y * z;                                   // p_yz
    case 13: return x * z;                                   // p_xz
    default: return x * y * z;                               // m_xyz
  }
}

// Gauss-Jordan inversion of an n x n row-major matrix (n <= 15).
void invert_n(int n, const double* a_in, double* inv) {
  double a[15][30];
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < 2 * n; ++c) a[r][c] = c < n ? a_in[r * n + c] : (c - n == r ? 1.0 : 0.0);
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
    if (piv != col)
      for (int c = 0; c < 2 * n; ++c) std::swap(a[col][c], a[piv][c]);
    const double d = a[col][col];
    for (int c = 0; c < 2 * n; ++c) a[col][c] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double m = a[r][col];
      if (m == 0.0) continue;
      for (int c = 0; c < 2 * n; ++c) a[r][c] -= m * a[col][c];
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) inv[r * n + c] = a[r][c + n];
}

struct Scheme3 {
  int nx, ny, nz;
  double k, beta, eps, alpha;
  int reg;
  unsigned flags;
  double s[15];
  double M[15][15], Minv[15][15], A[15][15], B[15][15];
};

int make_scheme3(const orc3_params* p, Scheme3* sc) {
  if (!p || p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
  if (!(p->sigma > 0) || !(p->D > 0) || !(p->M > 0)) return -1;
  sc->nx = p->nx;
  sc->ny = p->ny;
  sc->nz = p->nz;
  sc->beta = 3.0 * p->sigma / (4.0 * p->D);  // Eq. 5, as in 2D
  sc->k = sc->beta * p->D * p->D / 2.0;
  sc->eps = p->eps;
  sc->alpha = p->alpha;
  sc->reg = p->regularization;
  sc->flags = p->flags;
  for (int i = 0; i < 15; ++i) sc->s[i] = p->s[i];
  if (!(p->flags & ORC_S35_EXPLICIT)) {
    const double sj = 1.0 / (p->M / CS2 + 0.5);  // the j moments carry the flux (after Eq. 38)
    sc->s[3] = sc->s[5] = sc->s[7] = sj;
  }
  for (int i = 1; i < 15; ++i)
    if (!(sc->s[i] > 0.0 && sc->s[i] < 2.0)) return -1;
  double m[225], mi[225];
  for (int r = 0; r < 15; ++r)
    for (int c = 0; c < 15; ++c) m[r * 15 + c] = m3_row(r, c);
  invert_n(15, m, mi);
  for (int r = 0; r < 15; ++r)
    for (int c = 0; c < 15; ++c) {
      sc->M[r][c] = m[r * 15 + c];
      sc->Minv[r][c] = mi[r * 15 + c];
    }
  for (int i = 0; i < 15; ++i)
    for (int j = 0; j < 15; ++j) {
      double a = 0.0, b = 0.0;
      for (int q = 0; q < 15; ++q) {
        a += sc->Minv[i][q] * sc->s[q] * sc->M[q][j];
        b += sc->Minv[i][q] * (1.0 - sc->s[q] / 2.0) * sc->M[q][j];
      }
      sc->A[i][j] = a;
      sc->B[i][j] = b;
    }
  return 0;
}

inline size_t idx3(const Scheme3& sc, int x, int y, int z) {
  return (size_t(wrap(z, sc.nz)) * sc.ny + wrap(y, sc.ny)) * sc.nx + wrap(x, sc.nx);
}

// Eq. 26a in 3D.
inline void grad3(const Scheme3& sc, const double* chi, int x, int y, int z, double g[3]) {
  double s[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 15; ++i) {
    const double v = chi[idx3(sc, x + CX3[i], y + CY3[i], z + CZ3[i])];
    s[0] += W3[i] * CX3[i] * v;
    s[1] += W3[i] * CY3[i] * v;
    s[2] += W3[i] * CZ3[i] * v;
  }
  for (int d = 0; d < 3; ++d) g[d] = s[d] / CS2;
}

// Eq. 26b in 3D.
inline double lap3(const Scheme3& sc, const double* chi, int x, int y, int z) {
  const double c = chi[idx3(sc, x, y, z)];
  double s = 0.0;
  for (int i = 0; i < 15; ++i) s += 2.0 * W3[i] * (chi[idx3(sc, x + CX3[i], y + CY3[i], z + CZ3[i])] - c);
  return s / CS2;
}

struct Aniso3 {
  double gamma, Pg[3], gnorm;
};

// Eqs. 3, 6 and the projection after Eq. 14, with the n = 0 guard.
inline Aniso3 anisotropy3(double alpha, const double g[3]) {
  Aniso3 a;
  const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
  a.gnorm = std::sqrt(g2);
  if (g2 < GUARD) {
    a.gamma = 1.0;
    a.Pg[0] = a.Pg[1] = a.Pg[2] = 0.0;
    return a;
  }
  double n[3], gn[3], s4 = 0.0;
  for (int d = 0; d < 3; ++d) {
    n[d] = g[d] / a.gnorm;
    s4 += n[d] * n[d] * n[d] * n[d];
    gn[d] = 16.0 * alpha * n[d] * n[d] * n[d];
  }
  a.gamma = 1.0 + alpha * (4.0 * s4 - 3.0);  // Eq. 6, d = 3
  for (int d = 0; d < 3; ++d) {
    double v = 0.0;
    for (int e = 0; e < 3; ++e) v += ((d == e ? 1.0 : 0.0) - n[d] * n[e]) * gn[e];  // P = I - n n^T
    a.Pg[d] = v;
  }
  return a;
}

struct Fields3 {
  std::vector<double> phi, dx, dy, dz, lap, gamma, Qx, Qy, Qz, w, mua, mub, gx, gy, gz, lap2;
  explicit Fields3(size_t n)
      : phi(n), dx(n), dy(n), dz(n), lap(n), gamma(n), Qx(n), Qy(n), Qz(n), w(n), mua(n), mub(n), gx(n),
        gy(n), gz(n), lap2(n) {}
};

void compute_fields3(const Scheme3& sc, const double* f, Fields3& F) {
  const int nx = sc.nx, ny = sc.ny, nz = sc.nz;
  const size_t N = size_t(nx) * ny * nz;
  const bool literal_q = sc.flags & ORC_Q_LITERAL, nested = sc.flags & ORC_MU_NESTED;
#pragma omp parallel for schedule(static)
  for (long long id = 0; id < (long long)N; ++id) {
    double s = 0.0;
    for (int i = 0; i < 15; ++i) s += f[i * N + id];  // Eq. 22
    F.phi[id] = s;
  }
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const size_t id = idx3(sc, x, y, z);
        double g[3];
        grad3(sc, F.phi.data(), x, y, z, g);
        F.dx[id] = g[0];
        F.dy[id] = g[1];
        F.dz[id] = g[2];
        F.lap[id] = lap3(sc, F.phi.data(), x, y, z);
        const Aniso3 a = anisotropy3(sc.alpha, g);
        F.gamma[id] = a.gamma;
        const double kq = literal_q ? 1.0 : sc.k;
        const double iso = nested ? a.gamma : (a.gamma - 1.0);
        F.Qx[id] = iso * sc.k * g[0] + kq * a.gnorm * a.Pg[0];  // Eq. 15
        F.Qy[id] = iso * sc.k * g[1] + kq * a.gnorm * a.Pg[1];
        F.Qz[id] = iso * sc.k * g[2] + kq * a.gnorm * a.Pg[2];
        const double phi = F.phi[id];
        const double fb = 4.0 * sc.beta * phi * (phi + 1.0) * (phi - 1.0);
        F.w[id] = F.lap[id] - fb;
        F.mua[id] = fb - sc.k * F.lap[id];  // Eq. 16
      }
  if (sc.reg == 2) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) F.lap2[idx3(sc, x, y, z)] = lap3(sc, F.lap.data(), x, y, z);
  }
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const size_t id = idx3(sc, x, y, z);
        double gxq[3], gyq[3], gzq[3];
        grad3(sc, F.Qx.data(), x, y, z, gxq);
        grad3(sc, F.Qy.data(), x, y, z, gyq);
        grad3(sc, F.Qz.data(), x, y, z, gzq);
        const double divQ = gxq[0] + gyq[1] + gzq[2];
        const double phi = F.phi[id];
        const double fb = 4.0 * sc.beta * phi * (phi + 1.0) * (phi - 1.0);
        const double fp = 4.0 * sc.beta * (3.0 * phi * phi - 1.0);
        double reg = 0.0;
        if (sc.reg == 1) reg = sc.eps * (lap3(sc, F.w.data(), x, y, z) - fp * F.w[id]);  // Eq. 13
        else if (sc.reg == 2) reg = sc.eps * F.lap2[id];                                  // Eq. 12
        F.mub[id] = nested ? F.gamma[id] * fb - divQ + reg - F.mua[id] : (F.gamma[id] - 1.0) * fb - divQ + reg;
      }
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const size_t id = idx3(sc, x, y, z);
        double g[3];
        grad3(sc, F.mub.data(), x, y, z, g);
        F.gx[id] = g[0];
        F.gy[id] = g[1];
        F.gz[id] = g[2];
      }
}

void equilibrium3(double phi, double mua, double feq[15]) {
  for (int i = 0; i < 15; ++i) feq[i] = W3[i] * mua;  // Eq. 18
  feq[0] = phi + (W3[0] - 1.0) * mua;
}

void source3(double gx, double gy, double gz, double F[15]) {
  for (int i = 0; i < 15; ++i) F[i] = -W3[i] * (CX3[i] * gx + CY3[i] * gy + CZ3[i] * gz);  // Eq. 19
}

void collide3(const Scheme3& sc, const double f[15], double phi, double mua, double gx, double gy, double gz,
              double out[15]) {
  double feq[15], F[15], neq[15];
  equilibrium3(phi, mua, feq);
  source3(gx, gy, gz, F);
  for (int j = 0; j < 15; ++j) neq[j] = f[j] - feq[j];
  for (int i = 0; i < 15; ++i) {  // Eq. 17, dt = 1
    double relax = 0.0, force = 0.0;
    for (int j = 0; j < 15; ++j) {
      relax += sc.A[i][j] * neq[j];
      force += sc.B[i][j] * F[j];
    }
    out[i] = f[i] - relax + force;
  }
}

}  // namespace

extern "C" {

void orc3_matrices(double* M225, double* Minv225) {
  orc3_params p = {};
  p.nx = p.ny = p.nz = 1;
  p.M = 0.1;
  p.sigma = 0.01;
  p.D = 5.0;
  for (int i = 0; i < 15; ++i) p.s[i] = 1.0;
  Scheme3 sc;
  make_scheme3(&p, &sc);
  for (int r = 0; r < 15; ++r)
    for (int c = 0; c < 15; ++c) {
      if (M225) M225[r * 15 + c] = sc.M[r][c];
      if (Minv225) Minv225[r * 15 + c] = sc.Minv[r][c];
    }
}

void orc3_equilibrium(double phi, double mu_alpha, double feq[15]) { equilibrium3(phi, mu_alpha, feq); }

void orc3_source(double gx, double gy, double gz, double F[15]) { source3(gx, gy, gz, F); }

void orc3_collide_site(const orc3_params* p, const double f[15], double phi, double mu_alpha, double gx,
                       double gy, double gz, double out[15]) {
  Scheme3 sc;
  if (make_scheme3(p, &sc) != 0) {
    for (int i = 0; i < 15; ++i) out[i] = NAN;
    return;
  }
  collide3(sc, f, phi, mu_alpha, gx, gy, gz, out);
}

int orc3_init(const orc3_params* p, const double* phi0, double* f) {
  Scheme3 sc;
  if (make_scheme3(p, &sc) != 0) return -1;
  const size_t N = size_t(sc.nx) * sc.ny * sc.nz;
#pragma omp parallel for collapse(2) schedule(static)
  for (int z = 0; z < sc.nz; ++z)
    for (int y = 0; y < sc.ny; ++y)
      for (int x = 0; x < sc.nx; ++x) {
        const size_t id = idx3(sc, x, y, z);
        const double ph = phi0[id];
        const double mua = 4.0 * sc.beta * ph * (ph + 1.0) * (ph - 1.0) - sc.k * lap3(sc, phi0, x, y, z);
        double feq[15];
        equilibrium3(ph, mua, feq);
        for (int i = 0; i < 15; ++i) f[i * N + id] = feq[i];
      }
  return 0;
}

int orc3_step(const orc3_params* p, double* f, int64_t nsteps) {
  Scheme3 sc;
  if (make_scheme3(p, &sc) != 0) return -1;
  const int nx = sc.nx, ny = sc.ny, nz = sc.nz;
  const size_t N = size_t(nx) * ny * nz;
  Fields3 F(N);
  std::vector<double> fstar(15 * N);
  for (int64_t t = 0; t < nsteps; ++t) {
    compute_fields3(sc, f, F);
#pragma omp parallel for schedule(static)
    for (long long id = 0; id < (long long)N; ++id) {
      double fi[15], fo[15];
      for (int i = 0; i < 15; ++i) fi[i] = f[i * N + id];
      collide3(sc, fi, F.phi[id], F.mua[id], F.gx[id], F.gy[id], F.gz[id], fo);
      for (int i = 0; i < 15; ++i) fstar[i * N + id] = fo[i];
    }
    // Streaming, periodic: f_i(x + c_i) = f*_i(x).
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
          for (int i = 0; i < 15; ++i)
            f[i * N + idx3(sc, x + CX3[i], y + CY3[i], z + CZ3[i])] = fstar[i * N + idx3(sc, x, y, z)];
  }
  return 0;
}

int orc3_fields(const orc3_params* p, const double* f, double* out4) {
  Scheme3 sc;
  if (make_scheme3(p, &sc) != 0) return -1;
  const size_t N = size_t(sc.nx) * sc.ny * sc.nz;
  Fields3 F(N);
  compute_fields3(sc, f, F);
  const std::vector<double>* src[4] = {&F.phi, &F.gamma, &F.mua, &F.mub};
  for (int q = 0; q < 4; ++q)
    for (size_t id = 0; id < N; ++id) out4[q * N + id] = (*src[q])[id];
  return 0;
}

int orc3_phi(const orc3_params* p, const double* f, double* phi) {
  Scheme3 sc;
  if (make_scheme3(p, &sc) != 0) return -1;
  const size_t N = size_t(sc.nx) * sc.ny * sc.nz;
  for (size_t id = 0; id < N; ++id) {
    double s = 0.0;
    for (int i = 0; i < 15; ++i) s += f[i * N + id];
    phi[id] = s;
  }
  return 0;
}

double orc3_mass(const orc3_params* p, const double* f) {
  Scheme3 sc;
  if (make_scheme3(p, &sc) != 0) return NAN;
  const size_t N = size_t(sc.nx) * sc.ny * sc.nz;
  double m = 0.0;
  for (size_t id = 0; id < N; ++id)
    for (int i = 0; i < 15; ++i) m += f[i * N + id];
  return m;
}

double orc3_energy(const orc3_params* p, const double* f) {
  Scheme3 sc;
  if (make_scheme3(p, &sc) != 0) return NAN;
  const int nx = sc.nx, ny = sc.ny, nz = sc.nz;
  const size_t N = size_t(nx) * ny * nz;
  std::vector<double> phi(N), plane(nz);
  orc3_phi(p, f, phi.data());
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z) {
    double acc = 0.0;
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const double ph = phi[idx3(sc, x, y, z)];
        double g[3];
        grad3(sc, phi.data(), x, y, z, g);
        const double lap = lap3(sc, phi.data(), x, y, z);
        const Aniso3 a = anisotropy3(sc.alpha, g);
        const double F = sc.beta * (ph - 1.0) * (ph - 1.0) * (ph + 1.0) * (ph + 1.0);  // Eq. 4
        double e = a.gamma * (0.5 * sc.k * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) + F);  // Eq. 7
        if (sc.reg == 1) {
          const double w = lap - 4.0 * sc.beta * ph * (ph + 1.0) * (ph - 1.0);  // Eq. 9
          e += 0.5 * sc.eps * w * w;
        } else if (sc.reg == 2) {
          e += 0.5 * sc.eps * lap * lap;  // Eq. 8
        }
        acc += e;
      }
    plane[z] = acc;
  }
  double E = 0.0;
  for (int z = 0; z < nz; ++z) E += plane[z];
  return E;
}

}  // extern "C"
