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
//     |grad phi|^2 < 1e-24 the node takes n = 0, gamma = 1, P grad_n gamma = 0.
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
const double GUARD = 1e-24;

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
