/*
 * lbnop: a learned leap for the anisotropic Cahn-Hilliard LBM of lbch.h.
 *
 * A periodic convolutional U-Net maps phi(t) on an H x W field to phi(t + K), K lattice
 * steps later (the surrogate is not part of arXiv 2501.03759; the scheme of its Section 3
 * generates its training data and is the reference it is checked against). The library
 * holds the network, runs it forward, trains it (mean squared error, Adam), and alternates
 * leaps with steps of an lbch context.
 *
 * Network (the flat parameter layout below follows this table, in this order):
 *   sig = root mean square of phi (1 for a zero field)
 *   phi / sig (H x W, FP32) -> 4 x 4 space-to-depth -> 16 channels at level 0 (H/4 x W/4)
 *   layer  c_in c_out level activation
 *   e0a      16   96   0   SiLU  (its pre-activation also gets alpha v, alpha of Eq. 6;
 *                               its input is stored as two BF16 halves, hi = bf16(x) and
 *                               lo = bf16(x - hi), both multiplied by its weights; so is
 *                               the input of lin and lina)
 *   e0b      96   96   0   SiLU  -> h0
 *   e1a      96   64   1   SiLU  (input: 2 x 2 average pool of h0)
 *   e1b      64   64   1   SiLU  -> h1
 *   e2a      64   96   2   SiLU  (input: pool of h1)
 *   e2b      96   96   2   SiLU  -> h2
 *   m3a      96   96   3   SiLU  (input: pool of h2)
 *   m3b      96   96   3   SiLU  -> h3
 *   d2a      96   96   2   SiLU  (input: nearest 2x upsampling of h3, plus h2)
 *   d2b      96   64   2   none
 *   d1a      64   64   1   SiLU  (input: upsampled d2b output, plus h1)
 *   d1b      64   96   1   none
 *   d0a      96   96   0   SiLU  (input: upsampled d1b output, plus h0)
 *   out      96   16   0   none
 *   lin      16   16   0   none  (input: the e0a input; a linear path whose weights are
 *                               also kept as two BF16 halves, hi and lo = bf16(w - hi))
 *   lina     16   16   0   none  (input: the e0a input; output multiplied by alpha)
 *   out + lin + lina -> 4 x 4 depth-to-space -> D (H x W)
 *   phi_out = phi + scale sig (D - mean D)  (mean over the field, so mass is conserved)
 * Every layer is a 3 x 3 cross-correlation with periodic wrap plus a bias:
 *   z(p) = sum_{(dy, dx) in {-1,0,1}^2} W[3 (dy + 1) + (dx + 1)] x(p + (dy, dx)) + b.
 * Flat parameters (FP32, 826,096 values): for each layer in table order, W as
 * [9][c_out][c_in], then b [c_out]; after e0a's bias, its conditioning vector v [c_out].
 *
 * Arithmetic: the convolutions are implicit GEMMs on BF16 tensor-core operands with FP32
 * accumulation. Weights are kept in FP32 (master copy, Adam state) and rounded to BF16
 * for the GEMMs; activations and gradients between layers are stored in BF16; the head
 * (D, its mean, phi_out) and the loss are FP32 with FP64 sums.
 *
 * Ownership and errors follow lbch.h: the caller owns the device workspace (the library
 * never allocates), all work goes to the caller's stream, and calls return lbch_status.
 */
#ifndef LBNOP_H
#define LBNOP_H

#include "lbch.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbnop_ctx lbnop_ctx;

#define LBNOP_MAX_BATCH 64

typedef struct {
  int32_t H, W;          /* field size, multiples of 32, each in [32, 8192] */
  int32_t max_batch;     /* fields per forward or training step, in [1, LBNOP_MAX_BATCH] */
  double scale;          /* phi_out = phi + scale sig (D - mean D); > 0 */
} lbnop_params;

/* Number of FP32 parameters (826,096). */
int64_t lbnop_param_count(void);

/* Device workspace for these parameters (weights, Adam state, activations and gradients
 * for max_batch fields); 0 if the parameters are invalid. */
size_t lbnop_workspace_bytes(const lbnop_params* p);

lbch_status lbnop_create(const lbnop_params* p, void* d_workspace, size_t bytes, void* cuda_stream,
                         lbnop_ctx** out);

/* Loads parameters from host FP32 (lbnop_param_count values, layout above) and resets the
 * Adam state. Synchronises. LBCH_ENONFINITE if any value is NaN or Inf. */
lbch_status lbnop_set_params(lbnop_ctx* c, const float* h_theta);
lbch_status lbnop_get_params(lbnop_ctx* c, float* h_theta);   /* synchronises */

/* phi_out = network(phi, alpha) for `batch` fields. d_phi, d_phi_out: device FP32,
 * [batch][H][W] (they may be the same buffer); h_alpha: host, batch values (anisotropy
 * strength per field). Asynchronous. */
lbch_status lbnop_forward(lbnop_ctx* c, const float* d_phi, const double* h_alpha, int32_t batch,
                          float* d_phi_out);

/* Forward, loss = sum_b w_b sum_x (phi_out - target)^2 / (batch H W), and its gradient in
 * the parameters (kept in the context; read with lbnop_get_grads). d_target: device FP32
 * [batch][H][W]; h_weight: host, batch weights w_b >= 0, or NULL for all ones. Writes the
 * loss to *h_loss if h_loss is not NULL (synchronises then). */
lbch_status lbnop_backward(lbnop_ctx* c, const float* d_phi, const double* h_alpha, const float* d_target,
                           const double* h_weight, int32_t batch, double* h_loss);
lbch_status lbnop_get_grads(lbnop_ctx* c, float* h_grad);     /* synchronises */

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with learning rate lr
 * on the gradient g of the last lbnop_backward, scaled first by min(1, max_norm / |g|)
 * (|g| the L2 norm over all parameters) when a clip is set. Asynchronous. */
lbch_status lbnop_adam(lbnop_ctx* c, double lr);

/* Global-norm gradient clipping for the following Adam steps: max_norm > 0 clips, 0 (the
 * default) turns it off; LBCH_EINVAL for a negative or non-finite value. */
lbch_status lbnop_set_clip(lbnop_ctx* c, double max_norm);

/* The L2 norm over all parameters of the last lbnop_backward's gradient, before any
 * clipping. Synchronises. LBCH_EINVAL before the first backward. */
lbch_status lbnop_grad_norm(lbnop_ctx* c, double* h_norm);

/* lbnop_backward followed by lbnop_adam. */
lbch_status lbnop_train_step(lbnop_ctx* c, const float* d_phi, const double* h_alpha, const float* d_target,
                             const double* h_weight, int32_t batch, double lr, double* h_loss);

/* Runs `cycles` times: one leap of the network on the field of `lbm` (phi = sum f),
 * f = f^eq(phi_out) as in lbch_init_field, then lbm_steps steps of the scheme. The lbch
 * context must have nx = W, ny = H, FP32 storage, and work on the same CUDA stream as
 * this context. Asynchronous. Every leap is applied unchecked, and each re-initialisation
 * restarts the step counter of `lbm`, so afterwards lbch_steps_taken counts only the last
 * lbm_steps; lbnop_leap_run_judged checks every leap and keeps the simulated time. */
lbch_status lbnop_leap_run(lbnop_ctx* c, lbch_ctx* lbm, double alpha, int64_t cycles, int64_t lbm_steps);

/* The leaps of lbnop_leap_run and lbnop_leap_run_judged average the network over `turns`
 * quarter turns of the field: 1 (the default) runs the network alone; 4 runs it on the field
 * turned by 0, 90, 180 and 270 degrees (one forward of four fields), turns each prediction
 * back and takes the mean. The scheme commutes with the square's quarter turns (its
 * velocities, weights, relaxation rates and gamma of Eq. 6 are invariant under them) and the
 * network only approximately, so the mean is an estimate of the same step that is exactly
 * equivariant; it costs one batch-4 forward per leap. Mass stays conserved (each prediction
 * conserves it). 4 needs H = W and max_batch >= 4; LBCH_EINVAL otherwise. */
lbch_status lbnop_set_leap_turns(lbnop_ctx* c, int32_t turns);

/* The plain scheme as the judge of each leap in lbnop_leap_run_judged. */
typedef struct {
  int64_t leap_steps;      /* K > 0: the lattice steps one leap stands for. A rejected leap is
                              replaced by K steps of the scheme from the saved pre-leap state. */
  double energy_rtol;      /* >= 0: the free energy (Eq. 7) must not rise by more than
                              energy_rtol |E| across a leap, nor across the lbm_steps
                              correction steps after it (the energy law of Section 4) */
  double mass_atol;        /* >= 0: |sum phi after the leap - sum phi before| <= mass_atol H W */
  int64_t audit_every;     /* >= 0; 0 = no audits. Every audit_every-th cycle runs the K plain
                              steps as well, compares phi (relative L2) with the leap's, and
                              continues from the plain state */
  double phi_rtol;         /* >= 0: an audited leap whose phi is further than this from the
                              plain result counts as rejected */
} lbnop_judge;

/* What the judge saw during one lbnop_leap_run_judged call. */
typedef struct {
  int64_t accepted;            /* leaps kept (audited leaps within phi_rtol included) */
  int64_t rejected;            /* leaps replaced by plain steps (sum of the four below) */
  int64_t rejected_nonfinite;  /* NaN/Inf in the mass or energy after the leap or correction */
  int64_t rejected_mass;       /* mass moved by more than mass_atol H W */
  int64_t rejected_energy;     /* energy rose across the leap or across its correction steps */
  int64_t rejected_audit;      /* audited leaps further than phi_rtol from the plain result */
  int64_t audits;              /* audited cycles */
  int64_t lbm_steps;           /* lattice steps of the scheme run in total */
  double max_audit_err;        /* largest relative L2 phi error an audit measured */
  double max_leap_rise;        /* largest (E_after - E_before)/|E_before| across a judged leap */
  double max_corr_rise;        /* the same across the correction steps after a judged leap */
} lbnop_judge_stats;

/* lbnop_leap_run with the plain scheme as judge and fallback. Each of the `cycles` cycles
 * saves the state of `lbm` in this context's workspace, leaps, re-initialises f =
 * f^eq(phi_out), runs lbm_steps steps, and reads back the mass and free energy (FP64 sums on
 * the device) before the leap, after it and after the correction. The readings of cycle k
 * are copied to the host on a side stream while cycle k + 1 already runs (two saved states
 * in the workspace); the host judges cycle k from them.
 * If any is NaN/Inf, the mass moved by more than mass_atol H W, or the energy rose by
 * more than energy_rtol |E| across the leap or the correction, the saved state is
 * restored and K + lbm_steps plain steps are run instead (cycle k + 1, started on the
 * rejected state, is discarded and run again), so that a run in which every leap is
 * rejected equals the plain scheme bit for bit. Audited cycles (audit_every)
 * run the plain K steps next to the leap instead of re-initialising, and continue from
 * the plain state. After each cycle the step counter of `lbm` (lbch_steps_taken) has
 * advanced by K + lbm_steps: simulated time, whether the cycle leapt or not.
 * The lbch context must satisfy what lbnop_leap_run requires. `stats` (may be NULL)
 * receives the counts. LBCH_EINVAL for an invalid judge. */
lbch_status lbnop_leap_run_judged(lbnop_ctx* c, lbch_ctx* lbm, double alpha, int64_t cycles,
                                  int64_t lbm_steps, const lbnop_judge* judge, lbnop_judge_stats* stats);

/* Operator entry points (device pointers, the given stream, asynchronous), as used by
 * the network. BF16 tensors are uint16_t bit patterns, channels last:
 *   x [B][H][W][c_in], w [9][c_out][c_in], y [B][H][W][c_out].
 * c_in and c_out must be 16, 64 or 96 (the widths of the network); any H, W >= 1.
 *   conv3x3:             y = conv(x, w) + bias (bias may be NULL), FP32 out.
 *   conv3x3_bwd_data:    dx = sum_d w_d^T dy(p - d), FP32 out ([B][H][W][c_in]).
 *   conv3x3_bwd_weight:  dw[d] = sum_p dy(p) x(p + d)^T, FP32 out ([9][c_out][c_in]),
 *                        dy being BF16 [B][H][W][c_out].
 * Errors: LBCH_EINVAL for NULL pointers or unsupported shapes; LBCH_ECUDA if a launch fails.
 * A CUDA error left pending by earlier work of the calling thread is reported as LBCH_ECUDA
 * before anything is launched, and stays pending for the caller to read. */
lbch_status lbnop_conv3x3(const uint16_t* d_x, const uint16_t* d_w, const float* d_bias, int32_t B, int32_t H,
                          int32_t W, int32_t c_in, int32_t c_out, float* d_y, void* cuda_stream);
/* The same convolution with weights packed once for the tensor-core path: lbnop_conv3x3_pack
 * writes w ([9][c_out][c_in] BF16, 16-byte aligned) into d_packed (16-byte aligned, caller
 * owned, lbnop_conv3x3_packed_bytes(c_in, c_out) bytes; 0 for unsupported widths) in the
 * layout that path copies whole weight taps from, [9][c_in / 8][c_out][8] with 16 zero bytes
 * after each [c_out][8] block. lbnop_conv3x3_packed then runs conv3x3 with it: d_packed is
 * read where the tensor-core path takes the shape (W a multiple of 128, H a multiple of 4),
 * d_w elsewhere; d_packed may be NULL, which keeps every shape on the mma.sync kernels.
 * lbnop_conv3x3 is lbnop_conv3x3_packed with d_packed = NULL (the library allocates nothing). */
size_t lbnop_conv3x3_packed_bytes(int32_t c_in, int32_t c_out);
lbch_status lbnop_conv3x3_pack(const uint16_t* d_w, int32_t c_in, int32_t c_out, void* d_packed, void* cuda_stream);
lbch_status lbnop_conv3x3_packed(const uint16_t* d_x, const uint16_t* d_w, const void* d_packed, const float* d_bias,
                                 int32_t B, int32_t H, int32_t W, int32_t c_in, int32_t c_out, float* d_y,
                                 void* cuda_stream);
lbch_status lbnop_conv3x3_bwd_data(const uint16_t* d_dy, const uint16_t* d_w, int32_t B, int32_t H, int32_t W,
                                   int32_t c_in, int32_t c_out, float* d_dx, void* cuda_stream);
lbch_status lbnop_conv3x3_bwd_weight(const uint16_t* d_x, const uint16_t* d_dy, int32_t B, int32_t H, int32_t W,
                                     int32_t c_in, int32_t c_out, float* d_dw, void* cuda_stream);

/* Number of launches this process has run on the tcgen05 tensor-core path (operands staged
 * in shared memory, FP32 accumulators in tensor memory) since the library was loaded. That
 * path takes every forward convolution whose rows are a multiple of 128 pixels long (H a
 * multiple of 4) with packed weights: one input tensor, or on the network's first layer the
 * input and its BF16 remainder (K = 32); and every weight gradient (conv3x3_bwd_weight, and
 * the network's backward pass) whose rows are a multiple of 128 pixels. The others run on
 * mma.sync kernels. A diagnostic for tests and benchmarks. */
int64_t lbnop_tc_launches(void);

/* 1 if a tcgen05 convolution of this process (on the current device) gave up one of its
 * bounded waits (about a second each): its outputs are invalid, and every later launch of that
 * path returns without work. 0 if none did, -1 if the flag cannot be read. Read it after
 * synchronising the stream the convolutions ran on. The calls of an lbnop context that
 * synchronise (set_params, backward, train_step, grad_norm, get_grads, and
 * leap_run_judged at its end) check it themselves and fail with LBCH_ECUDA. */
int32_t lbnop_tc_fault(void);

const char* lbnop_last_error(const lbnop_ctx* c);
void lbnop_destroy(lbnop_ctx* c);

#ifdef __cplusplus
}
#endif
#endif
