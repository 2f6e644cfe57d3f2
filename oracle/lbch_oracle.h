/*
 * FP64 CPU oracle for the multiple-relaxation-time lattice Boltzmann scheme for
 * the anisotropic Cahn-Hilliard equation (Liu, Wang, Liu, arXiv 2501.03759).
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA path. Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg load it. It
 * shares no code, header, table or constant with the CUDA library, and the CUDA
 * library never calls it.
 *
 * Layout: a state is 9 planes of nx*ny doubles, plane i first, then row y, then
 * column x (x fastest): f[i*nx*ny + y*nx + x]. Planes follow the D2Q9 order of
 * Eq. 20a. The state is the post-streaming distribution f_i(x, t) of Eq. 17.
 *
 * Pins (tests check each against something other than this code):
 *   orc_matrices       Eq. 23 printed values; M M^T diagonal; M^-1 M = I.
 *   orc_equilibrium    moment constraints Eq. 27b.
 *   orc_source         moment constraints Eq. 27c.
 *   orc_collide_site   single-relaxation reduction (all s_i equal).
 *   orc_step           mass conservation (Eq. 34), energy decay, isotropic tanh
 *                      profile (Eq. 40 with Eq. 5), continuum linear dispersion
 *                      (Eqs. 10, 13, 15, 16, 38) on the axes, the diagonals and a
 *                      generic angle (gamma of Eq. 6 between its extremes), with
 *                      Willmore (Eq. 13) and linear (Eq. 12) regularisation, lattice
 *                      rotation/mirror equivariance, constant-field fixed point.
 *   orc_fields         mu_beta on a circular interface converges at second order to
 *                      the continuum value of Eqs. 2, 6, 15, 16 (the tangential term
 *                      with and without k: readings C1 and ORC_Q_LITERAL); the
 *                      ORC_MU_NESTED difference equals k (lap - div grad) phi from
 *                      Fourier symbols of Eq. 26; the n = 0 guard fires only in bulk.
 *   orc_energy         Eq. 7 with Eq. 9 or Eq. 8 on fields with closed-form sums.
 * Each of these pins fails under planted mistakes in its branch (a mutation test
 * builds altered copies of this oracle and runs the pins against them).
 * Parity unpinned: the absolute shapes and energy curves of the paper's figures
 * (their values are not printed).
 */
#ifndef LBCH_ORACLE_H
#define LBCH_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_Q_LITERAL = 1u,    /* Eq. 15 as printed: no k on the |grad phi| P grad_n gamma term */
  ORC_MU_NESTED = 2u,    /* mu_beta = mu - mu_alpha with the full Q of Eq. 15 (nested stencils) */
  ORC_S35_EXPLICIT = 4u  /* take s[3], s[5] as given instead of deriving them from M */
};

typedef struct {
  int32_t nx, ny;                 /* periodic grid, x fastest */
  double M, sigma, D, eps, alpha; /* Eq. 39 parameters and the anisotropy strength of Eq. 6 */
  double s[9];                    /* relaxation rates of S = diag(s_0..s_8), Eq. 25 */
  int32_t regularization;         /* 0 none, 1 Willmore (Eq. 9, Eq. 13), 2 linear (Eq. 8, Eq. 12) */
  uint32_t flags;                 /* ORC_* bits */
} orc_params;

typedef struct {
  double k, beta;   /* from sigma and D by inverting Eq. 5 */
  double s[9];      /* rates actually used (s_3 = s_5 from M unless ORC_S35_EXPLICIT) */
} orc_derived;

/* Fills *out. Returns 0, or -1 if a parameter is outside its domain. */
int orc_derive(const orc_params* p, orc_derived* out);

/* M of Eq. 23 (row-major 9x9) and its inverse obtained by Gauss-Jordan elimination. */
void orc_matrices(double* M81, double* Minv81);

/* f^eq of Eq. 18 at one node. */
void orc_equilibrium(double phi, double mu_alpha, double feq[9]);

/* F_i of Eq. 19 at one node, given grad mu_beta = (gx, gy). */
void orc_source(double gx, double gy, double F[9]);

/* One node of Eq. 17 in matrix form (post-collision value, before streaming). */
void orc_collide_site(const orc_params* p, const double f[9], double phi, double mu_alpha,
                      double gx, double gy, double out[9]);

/* f(x, 0) = f^eq(phi0, mu_alpha(phi0)), mu_alpha from Eq. 16 with the Laplacian of Eq. 26b. */
int orc_init(const orc_params* p, const double* phi0, double* f);

/* Advances the state nsteps time steps of Eq. 17 in place. */
int orc_step(const orc_params* p, double* f, int64_t nsteps);

/* phi = sum_i f_i (Eq. 22). */
int orc_phi(const orc_params* p, const double* f, double* phi);

/* Intermediate fields of one step from the state f (each nx*ny, in this order):
 * phi, dphi_x, dphi_y, lap_phi, gamma, Qx, Qy, w, mu_alpha, mu_beta, gx, gy.
 * Qx, Qy are the components of the vector field whose divergence enters mu_beta. */
int orc_fields(const orc_params* p, const double* f, double* out12);

/* Sum over nodes of phi (Eq. 22). */
double orc_mass(const orc_params* p, const double* f);

/* Discrete free energy: Eq. 7 with G of Eq. 9 (or Eq. 8), stencils of Eq. 26. */
double orc_energy(const orc_params* p, const double* f);

/* Number of OpenMP threads for the whole-field passes (rows split across threads;
 * results do not depend on it). Returns the number now in use. */
int orc_set_threads(int n);

/* ---- 3D: D3Q15 (Eq. 21, Eq. 24), Section 3 with d = 3 ------------------------------
 * State: 15 planes of nx*ny*nz doubles, plane i first, then z, then y, then x (x
 * fastest), in the velocity order of Eq. 21a. Readings specific to 3D:
 *   - Eq. 24 names the moments (rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, p_ww,
 *     p_xy, p_yz, p_xz, m_xyz) but orders the eight diagonal velocities differently from
 *     Eq. 21a, and its last row is not orthogonal to j_x; the oracle builds each row as
 *     the function of c it names, evaluated at the velocities of Eq. 21a (last row
 *     c_x c_y c_z).
 *   - s_3 = s_5 = s_7 (the j moments) = 1/(M/c_s^2 + 1/2) unless ORC_S35_EXPLICIT.
 * Pins: Eq. 21 and Eq. 24 printed values (with the two discrepancies named exactly),
 * Eq. 27 moment constraints, orthogonality, single-relaxation reduction, mass
 * conservation, energy decay, continuum linear dispersion along axis, face and body
 * diagonals, cube rotation equivariance, a separate NumPy route, and (orc3_fields) mu_beta
 * on a spherical interface against the continuum value of Eqs. 3, 6, 15, 16. */
typedef struct {
  int32_t nx, ny, nz;
  double M, sigma, D, eps, alpha;
  double s[15];
  int32_t regularization;
  uint32_t flags;
} orc3_params;

void orc3_matrices(double* M225, double* Minv225);
void orc3_equilibrium(double phi, double mu_alpha, double feq[15]);
void orc3_source(double gx, double gy, double gz, double F[15]);
void orc3_collide_site(const orc3_params* p, const double f[15], double phi, double mu_alpha,
                       double gx, double gy, double gz, double out[15]);
int orc3_init(const orc3_params* p, const double* phi0, double* f);
/* phi, gamma, mu_alpha and mu_beta of the state f (4 planes of nx*ny*nz, in that order):
 * the pointwise fields one step computes before the collision (Eqs. 3, 6, 13, 15, 16, 22). */
int orc3_fields(const orc3_params* p, const double* f, double* out4);
int orc3_step(const orc3_params* p, double* f, int64_t nsteps);
int orc3_phi(const orc3_params* p, const double* f, double* phi);
double orc3_mass(const orc3_params* p, const double* f);
double orc3_energy(const orc3_params* p, const double* f);

#ifdef __cplusplus
}
#endif
#endif
