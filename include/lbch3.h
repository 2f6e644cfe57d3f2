/*
 * lbch3: the same time step in 3D, on the D3Q15 lattice (arXiv 2501.03759, Section 3
 * with d = 3; Eqs. 3, 6, 17-19, 21, 22, 24, 26), on a periodic nx x ny x nz grid.
 *
 * The model and the readings are those of lbch.h, with these 3D specifics:
 *   - Velocities and weights of Eq. 21a, 21b (in that order).
 *   - Moment basis of Eq. 24 (rho, e, eps, j_x, q_x, j_y, q_y, j_z, q_z, 3p_xx, p_ww,
 *     p_xy, p_yz, p_xz, m_xyz), each row built as the function of c it names at the
 *     velocities of Eq. 21a. The print orders the diagonal velocities differently and
 *     its last row is not orthogonal to j_x; the last row here is c_x c_y c_z.
 *   - s_3 = s_5 = s_7 (the j moments) = 1/(M/c_s^2 + 1/2) unless LBCH_S35_EXPLICIT.
 *   - gamma(n) = 1 + alpha (4 (n_1^4 + n_2^4 + n_3^4) - 3) (Eq. 6, d = 3).
 * Populations are stored in FP32 (120 bytes read and written per node update).
 *
 * Errors, streams and the caller-owned workspace follow lbch.h; lbch3 never allocates.
 */
#ifndef LBCH3_H
#define LBCH3_H

#include "lbch.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbch3_ctx lbch3_ctx; /* opaque; lbch3_create / lbch3_destroy */

typedef struct {
  int32_t nx, ny, nz;   /* periodic grid, x fastest; each in [1, 4096], nx*ny*nz < 2^31 */
  double M, sigma, D, eps, alpha; /* as in lbch_params */
  double s[15];         /* relaxation rates s_0..s_14 of the D3Q15 moments; s_1..s_14 in (0, 2) */
  int32_t regularization; /* LBCH_REG_* */
  uint32_t flags;         /* LBCH_Q_LITERAL | LBCH_MU_NESTED | LBCH_S35_EXPLICIT (s_3, s_5, s_7) */
} lbch3_params;

/* Device workspace (two population buffers; FP32 planes of phi, mu_alpha and mu_beta;
 * one FP64 staging plane; a reduction area); 0 for invalid parameters. */
size_t lbch3_workspace_bytes(const lbch3_params* p);

/* Creates a 3D context on the current device; same rules as lbch_create. */
lbch_status lbch3_create(const lbch3_params* p, void* d_workspace, size_t bytes, void* cuda_stream,
                         lbch3_ctx** out);

/* f = f^eq(phi0, mu_alpha(phi0)); h_phi0: nx*ny*nz doubles, x fastest, then y, then z.
 * Synchronises. LBCH_ENONFINITE if phi0 holds NaN/Inf. */
lbch_status lbch3_init_field(lbch3_ctx* c, const double* h_phi0);

/* Advances n >= 0 time steps (three kernel launches per step); asynchronous. */
lbch_status lbch3_step(lbch3_ctx* c, int64_t n);

/* phi = sum_i f_i to h_phi (nx*ny*nz doubles). Synchronises. */
lbch_status lbch3_get_field(lbch3_ctx* c, double* h_phi);

/* Total mass and free energy (Eq. 7 with Eq. 9 or 8, D3Q15 stencils), FP64 sums. */
lbch_status lbch3_mass(lbch3_ctx* c, double* out);
lbch_status lbch3_free_energy(lbch3_ctx* c, double* out);

const char* lbch3_last_error(const lbch3_ctx* c);
void lbch3_destroy(lbch3_ctx* c);

#ifdef __cplusplus
}
#endif
#endif
