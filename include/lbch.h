/*
 * lbch: one time step of the multiple-relaxation-time lattice Boltzmann scheme for
 * the anisotropic Cahn-Hilliard equation (Liu, Wang, Liu, arXiv 2501.03759,
 * Sections 2-3), on a periodic 2D grid, on one NVIDIA GB300 GPU (sm_103a).
 *
 * The problem (Section 2): an order parameter phi(x, t) on a periodic N_x x N_y
 * lattice evolves by the Cahn-Hilliard equation d phi/dt = div(M grad mu) (Eq. 10)
 * with the chemical potential of Eq. 13 (Willmore regularisation, Eq. 9), the
 * fourfold anisotropy gamma(n) = 1 + alpha cos 4 theta (Eq. 6) and the vector field
 * Q of Eq. 15. The scheme (Section 3) splits mu = mu_alpha + mu_beta (Eq. 16) and
 * evolves D2Q9 populations f_i (Eq. 20) by the MRT update of Eq. 17 with the
 * equilibrium of Eq. 18, the source of Eq. 19, the moment matrix of Eq. 23 and the
 * isotropic stencils of Eq. 26; phi = sum_i f_i (Eq. 22). Lattice units: dx = dt =
 * c = 1, c_s^2 = 1/3.
 *
 * Readings the library takes where the paper is silent or garbled (flags select
 * the alternatives):
 *   - Eq. 15 is used with the factor k that Eq. 14 carries on its second term:
 *     Q = gamma k grad phi + k |grad phi| P grad_n gamma.  LBCH_Q_LITERAL drops it.
 *   - mu_beta = mu - mu_alpha with the isotropic k lap phi cancelled analytically:
 *     mu_beta = (gamma-1) f - div((gamma-1) k grad phi + k|grad phi| P grad_n gamma)
 *               + eps (lap w - f'(phi) w),  w = lap phi - f(phi).
 *     LBCH_MU_NESTED takes mu - mu_alpha with the full Q instead.
 *   - Where |grad phi|^2 < 1e-12 a node takes n = 0, gamma = 1, P grad_n gamma = 0
 *     (FP32 rounding of a zero gradient stays below this, so it never picks a direction).
 *   - grad_n gamma = 16 alpha (n_1^3, n_2^3), the gradient of Eq. 6 in R^2.
 *   - s_3 = s_5 = 1/(M/c_s^2 + 1/2) (from M = c_s^2 (1/s_{3,5} - 1/2) dt, after
 *     Eq. 38) unless LBCH_S35_EXPLICIT; the other rates are inputs (default 1).
 *   - Initial populations: f = f^eq(phi0, mu_alpha(phi0)), Eq. 18 with Eq. 16.
 *   - Free energy: sum over nodes of gamma(n)(k/2 |grad phi|^2 + F(phi))
 *     + eps/2 G(phi), with the stencils of Eq. 26 (Eqs. 1, 4, 7, 8, 9).
 *
 * Threading and streams: a context is used by one host thread at a time. All GPU
 * work of a context goes to the CUDA stream given at creation, in call order.
 *
 * Errors: every call returns an lbch_status and never aborts or throws. After a
 * CUDA error the context is failed: every later call except lbch_destroy and
 * lbch_last_error returns LBCH_ESTATE.
 */
#ifndef LBCH_H
#define LBCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbch_ctx lbch_ctx; /* opaque; created by lbch_create, freed by lbch_destroy */

typedef enum {
  LBCH_OK = 0,
  LBCH_EINVAL = -1,      /* bad argument, parameter, size or call order */
  LBCH_ECUDA = -2,       /* a CUDA call failed; the context is now failed */
  LBCH_ENOMEM = -3,      /* the caller's workspace is too small or misaligned */
  LBCH_ENONFINITE = -4,  /* NaN or Inf in an input field or in a reduced result */
  LBCH_ESTATE = -5       /* the context failed earlier */
} lbch_status;

/* How the populations are stored between steps; arithmetic is FP32 in all cases. */
typedef enum {
  LBCH_STORE_F32 = 0,       /* 9 FP32 planes: 72 bytes read+written per node update */
  LBCH_STORE_BF16_DEV = 1,  /* FP32 rest population and mu_alpha anchor per node, plus the 8
                               moving populations as BF16 deviations from omega_i times the
                               anchor of the node they stream to: 48 bytes */
  LBCH_STORE_F16_DEV = 2    /* as above with FP16 deviations scaled by 2^12: 48 bytes */
} lbch_storage;

enum {
  LBCH_Q_LITERAL = 1u,    /* Eq. 15 exactly as printed (no k on its second term) */
  LBCH_MU_NESTED = 2u,    /* mu_beta = mu - mu_alpha with the full Q of Eq. 15 */
  LBCH_S35_EXPLICIT = 4u  /* use s[3], s[5] as given instead of deriving them from M */
};

enum { LBCH_REG_NONE = 0, LBCH_REG_WILLMORE = 1, LBCH_REG_LINEAR = 2 };

typedef struct {
  int32_t nx, ny;      /* periodic grid, x fastest; 1 <= nx, ny <= 65536 */
  double M;            /* mobility (Eq. 10), > 0; sets s_3 = s_5 */
  double sigma, D;     /* surface tension and interface thickness (Eq. 5), > 0 */
  double eps;          /* regularisation strength epsilon (Eq. 7), >= 0 */
  double alpha;        /* anisotropy strength (Eq. 6), 0 <= alpha < 1 */
  double s[9];         /* relaxation rates s_0..s_8 of S (Eq. 25); each of s_1..s_8 in (0, 2) */
  int32_t storage;       /* lbch_storage */
  int32_t regularization;/* LBCH_REG_*: none, Willmore (Eq. 9, Eq. 13, the paper's choice),
                            linear (Eq. 8, Eq. 12) */
  uint32_t flags;        /* LBCH_Q_LITERAL | LBCH_MU_NESTED | LBCH_S35_EXPLICIT */
} lbch_params;

/* Device workspace a context needs for these parameters (population buffers,
 * one FP64 staging plane of nx*ny, a small reduction area); 0 if the parameters
 * are invalid. */
size_t lbch_workspace_bytes(const lbch_params* p);

/* Creates a context on the current CUDA device.
 *   d_workspace: device memory of at least lbch_workspace_bytes(p) bytes, 256-byte
 *                aligned, owned by the caller; it must outlive the context. The
 *                library never allocates or frees device memory.
 *   cuda_stream: a cudaStream_t (NULL for the legacy default stream).
 * Returns LBCH_EINVAL for bad parameters, LBCH_ENOMEM if the workspace is too small
 * or misaligned, LBCH_ECUDA if the device cannot run the kernels. *out is set only
 * on LBCH_OK. */
lbch_status lbch_create(const lbch_params* p, void* d_workspace, size_t bytes,
                        void* cuda_stream, lbch_ctx** out);

/* Sets the state to f = f^eq(phi0, mu_alpha(phi0)) (Eq. 18, Eq. 16, Eq. 26b) at t = 0.
 *   h_phi0: host array of nx*ny doubles, row-major (x fastest), read before return.
 * Synchronises the stream. LBCH_ENONFINITE (state left unset) if phi0 holds NaN/Inf. */
lbch_status lbch_init_field(lbch_ctx* ctx, const double* h_phi0);

/* lbch_init_field from a device field: h_phi0 replaced by d_phi0, nx*ny FP32 values in
 * device memory (x fastest). Asynchronous; it does not check for NaN/Inf. */
lbch_status lbch_init_field_device(lbch_ctx* ctx, const float* d_phi0);

/* Writes phi(x, t) = sum_i f_i(x, t) as FP32 to d_phi (nx*ny values, device memory).
 * Asynchronous. */
lbch_status lbch_get_phi_device(lbch_ctx* ctx, float* d_phi);

/* Advances the state n >= 0 time steps of Eq. 17. Asynchronous: enqueues the n step
 * kernels on the stream and returns. From the first call with n >= 16 on, runs of 16 steps
 * are replayed from a CUDA graph that the context captures once on a private stream and
 * keeps (with its driver resources) until lbch_destroy; the results are those of
 * single launches, bit for bit. While the caller is capturing the stream itself, the
 * kernels are launched one by one. LBCH_EINVAL before any init/set_state. */
lbch_status lbch_step(lbch_ctx* ctx, int64_t n);

/* Total mass sum_x phi(x) (Eq. 22), accumulated in FP64 on the GPU. Synchronises. */
lbch_status lbch_mass(lbch_ctx* ctx, double* out);

/* Discrete free energy (Eq. 7 with G of Eq. 9 or Eq. 8), densities in FP32, sum in
 * FP64 on the GPU. Synchronises. LBCH_ENONFINITE if the result is NaN/Inf. */
lbch_status lbch_free_energy(lbch_ctx* ctx, double* out);

/* Copies phi(x, t) = sum_i f_i(x, t) (Eq. 22) to h_phi (nx*ny doubles). Synchronises. */
lbch_status lbch_get_field(lbch_ctx* ctx, double* h_phi);

/* Copies the post-streaming populations f_i(x, t) of Eq. 17 to h_f9: 9 planes of
 * nx*ny doubles, plane i in the D2Q9 order of Eq. 20a. Synchronises. */
lbch_status lbch_get_state(lbch_ctx* ctx, double* h_f9);

/* Replaces the state with h_f9 (same layout as lbch_get_state); checkpoint/resume.
 * Synchronises. LBCH_ENONFINITE (state left unset) if h_f9 holds NaN/Inf. */
lbch_status lbch_set_state(lbch_ctx* ctx, const double* h_f9);

/* Asynchronous forms of lbch_mass and lbch_free_energy (same kernels, same FP64 sums):
 * the result goes to one double in device memory, d_out, and the call returns without
 * synchronising, so that diagnostics can be chained with steps on the stream and read
 * back once. They do not check the result for NaN/Inf. */
lbch_status lbch_mass_device(lbch_ctx* ctx, double* d_out);
lbch_status lbch_free_energy_device(lbch_ctx* ctx, double* d_out);

/* Mass and free energy of a field phi given in device memory (nx*ny FP32 values, x fastest),
 * with this context's parameters, asynchronously: d_out2[0] = sum_x phi (FP64 sum of the
 * FP32 values, Eq. 22), d_out2[1] = the discrete free energy of lbch_free_energy (Eq. 7 with
 * G of Eq. 9 or Eq. 8; for the field lbch_get_phi_device writes, the same value bit for bit).
 * One pass over the field; the state is not read and need not be set. */
lbch_status lbch_field_diagnostics_device(lbch_ctx* ctx, const float* d_phi, double* d_out2);

/* Bytes of one state (the population buffer a step reads) for these parameters; 0 if
 * they are invalid. */
size_t lbch_state_bytes(const lbch_params* p);

/* Device-side checkpoint: copies the current state into d_dst (device memory of at least
 * lbch_state_bytes(p) bytes, owned by the caller), asynchronously. The copy is an
 * opaque image of the library's storage, valid only for a context with the same
 * parameters. LBCH_EINVAL if bytes is too small or there is no state. */
lbch_status lbch_save_state_device(lbch_ctx* ctx, void* d_dst, size_t bytes);

/* Makes an image saved by lbch_save_state_device the current state, asynchronously. The
 * continuation is bit for bit the one the saved context would have taken. The step
 * counter is left as it is. */
lbch_status lbch_restore_state_device(lbch_ctx* ctx, const void* d_src, size_t bytes);

/* Number of time steps taken since the last lbch_init_field / lbch_set_state /
 * lbch_init_field_device, or the value last given to lbch_set_steps_taken. */
int64_t lbch_steps_taken(const lbch_ctx* ctx);

/* Sets the step counter that lbch_steps_taken reports (bookkeeping only, no GPU work):
 * a caller that re-initialises the state from a field standing for a later time (the
 * learned leap of lbnop.h) keeps the simulated time this way. LBCH_EINVAL if steps < 0. */
lbch_status lbch_set_steps_taken(lbch_ctx* ctx, int64_t steps);

/* Human-readable description of the last error on this context ("" if none). */
const char* lbch_last_error(const lbch_ctx* ctx);

/* Frees the host-side context. Never touches the workspace. NULL is ignored. */
void lbch_destroy(lbch_ctx* ctx);

/* ---- Batches: many independent periodic fields stepped together --------------------
 *
 * A batch holds `count` fields that share the scheme parameters of `common` (M, sigma, D,
 * eps, s, storage, regularization, flags) and differ in size nx[i] x ny[i] and anisotropy
 * strength alpha[i] (Eq. 6). One kernel launch advances every field by one time step
 * (Eq. 17), so many small problems (parameter sweeps) fill the GPU together.
 * Initial conditions, fields and diagnostics are per field and mean exactly what they
 * mean for a single context; each field evolves exactly as it would alone. */
typedef struct lbch_batch lbch_batch; /* opaque; lbch_batch_create / lbch_batch_destroy */

/* Device workspace for a batch (every field's population buffers, one shared scratch
 * area, the work tables); 0 for invalid arguments. nx, ny: arrays of count sizes. */
size_t lbch_batch_workspace_bytes(const lbch_params* common, int32_t count, const int32_t* nx,
                                  const int32_t* ny);

/* Creates a batch on the current device. alpha: count strengths (NULL: common->alpha for
 * all). The workspace rules are those of lbch_create. Creation also tunes the work split:
 * it times a few row-segment lengths on the zeroed buffers (about a hundred launches) and
 * captures a CUDA graph of 64 steps, which holds driver resources until lbch_batch_destroy.
 * Returns LBCH_EINVAL, LBCH_ENOMEM or LBCH_ECUDA as lbch_create does. */
lbch_status lbch_batch_create(const lbch_params* common, int32_t count, const int32_t* nx,
                              const int32_t* ny, const double* alpha, void* d_workspace,
                              size_t bytes, void* cuda_stream, lbch_batch** out);

/* lbch_init_field for field i (0 <= i < count). Fields may only be (re)initialised while
 * the batch has taken an even number of steps; LBCH_EINVAL otherwise. */
lbch_status lbch_batch_init_field(lbch_batch* b, int32_t i, const double* h_phi0);

/* Advances every field n >= 0 time steps; asynchronous like lbch_step. LBCH_EINVAL until
 * every field has been initialised. */
lbch_status lbch_batch_step(lbch_batch* b, int64_t n);

/* lbch_get_field, lbch_mass and lbch_free_energy for field i; each synchronises. The
 * fields share one scratch area, so calls on one batch must not overlap. */
lbch_status lbch_batch_get_field(lbch_batch* b, int32_t i, double* h_phi);
/* lbch_get_phi_device for field i (asynchronous, on the batch's stream). */
lbch_status lbch_batch_get_phi_device(lbch_batch* b, int32_t i, float* d_phi);
lbch_status lbch_batch_mass(lbch_batch* b, int32_t i, double* out);
lbch_status lbch_batch_free_energy(lbch_batch* b, int32_t i, double* out);

/* Rows per warp the creation-time tuner chose (-1 for NULL). */
int32_t lbch_batch_rows_target(const lbch_batch* b);

/* Time steps taken since creation (-1 for NULL). */
int64_t lbch_batch_steps_taken(const lbch_batch* b);

/* Description of the last error on this batch ("" if none). */
const char* lbch_batch_last_error(const lbch_batch* b);

/* Frees the batch's host objects and its CUDA graph; never touches the workspace. */
void lbch_batch_destroy(lbch_batch* b);

/* Free energy of a state the caller holds in device memory, computed without any
 * device allocation. This is a library convenience with no counterpart in the paper.
 * It serves callers that cannot call cudaMalloc, or cannot hand this library an
 * allocator: code whose device memory all comes from a pool fixed at start-up, or a
 * host application that is only allowed to launch work on memory it already owns.
 * It computes the same quantity as lbch_free_energy, without a context or workspace.
 *   p:            scheme parameters (nx, ny, sigma, D, eps, alpha, regularization; the
 *                 storage field is ignored and not validated: the state is FP32).
 *   d_f9:         device array of the post-streaming populations f_i(x, t) in FP32, 9
 *                 planes, plane i starting at d_f9 + i * plane_stride, each row-major with
 *                 x fastest (the layout of lbch_get_state, in FP32 on the device).
 *   plane_stride: elements between planes, >= nx * ny.
 *   d_out:        device pointer to one double that receives the energy.
 *   cuda_stream:  stream for the work (NULL for the legacy default stream); the call
 *                 returns without synchronising it.
 * The scratch (phi in FP32 and the FP64 partial sums) lives in one file-scope
 * __device__ array of 16,793,600 bytes that every GPU loading the library holds until
 * the process exits. So nx * ny may be at most 4,194,304 (2048 x 2048); larger grids
 * return LBCH_EINVAL. The first call on each device resolves that array's device
 * address (cudaGetSymbolAddress) and the SM count; make that first call before any
 * stream capture. All calls share the array and every call overwrites the parts it
 * reads (nothing carries over between calls), so calls that overlap on the GPU race.
 * Returns LBCH_EINVAL for bad arguments, LBCH_ECUDA if set-up or a launch fails. A CUDA
 * error left pending by earlier work of the calling thread is reported as LBCH_ECUDA
 * before anything is launched, and stays pending for the caller to read. */
lbch_status lbch_free_energy_static(const lbch_params* p, const float* d_f9, int64_t plane_stride,
                                    double* d_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
