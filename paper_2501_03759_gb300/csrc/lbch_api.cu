// C-ABI of the lbch library (declared in include/lbch.h): parameter checks,
// workspace layout, kernel launches on the caller's stream, error reporting.
// Every step of the method runs in the kernels of lbch_step.cuh / lbch_aux.cuh;
// host code here only validates, lays out memory and launches.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "lbch.h"
#include "lbch3.h"
#include "lbch_aux.cuh"
#include "lbch_step.cuh"

using namespace lbch;

struct lbch_ctx {
  lbch_params p;
  double k, beta;
  double s[9];
  cudaStream_t stream;
  int device;
  // Workspace layout.
  char* ws;
  size_t ws_bytes;
  long long ps;     // plane stride (elements)
  Buf buf[2];       // population buffers (ping-pong)
  int cur;          // buffer holding the current post-collision state
  bool has_state;
  int64_t steps;
  double* stage0;   // FP64 plane (host transfers)
  double* stage1;   // FP64 plane (mu_alpha, phi accumulation, FP32 phi for the energy)
  double* partial;  // MAX_RED_BLOCKS doubles
  double* result;   // 8 doubles
  int* flags;       // 16 ints
  // Launch shapes.
  StepArgs sa;      // constants of the scheme
  Field fld;        // geometry and work split of the field (buffers set per launch)
  long long n_warps;
  bool vec;
  bool fast;  // s_1 = s_2 = s_4 = s_6 = s_7 = s_8 = 1: reduced collision
  int step_blocks;
  int aux_blocks;
  cudaGraphExec_t graph;  // GRAPH_STEPS step launches from buffer 0, captured at first use
  bool graph_off;         // capture failed once, or the caller's stream is being captured
  bool failed;
  char err[512];
};

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

long long plane_stride(const lbch_params* p) {
  const long long n = (long long)p->nx * p->ny;
  return (n + 63) / 64 * 64;  // keeps every plane 256-byte aligned
}

size_t state_bytes(const lbch_params* p) {
  const long long ps = plane_stride(p);
  if (p->storage == LBCH_STORE_F32) return align_up((size_t)ps * 9 * sizeof(float));
  return align_up((size_t)ps * 2 * sizeof(float)) + align_up((size_t)ps * 8 * sizeof(uint16_t));
}

const char* check_params(const lbch_params* p) {
  if (!p) return "params is NULL";
  if (p->nx < 1 || p->ny < 1 || p->nx > 65536 || p->ny > 65536) return "nx, ny must be in [1, 65536]";
  if (!(p->M > 0.0) || !std::isfinite(p->M)) return "M must be finite and > 0";
  if (!(p->sigma > 0.0) || !std::isfinite(p->sigma)) return "sigma must be finite and > 0";
  if (!(p->D > 0.0) || !std::isfinite(p->D)) return "D must be finite and > 0";
  if (!(p->eps >= 0.0) || !std::isfinite(p->eps)) return "eps must be finite and >= 0";
  if (!(p->alpha >= 0.0 && p->alpha < 1.0)) return "alpha must be in [0, 1) so that gamma > 0";
  if (p->storage < LBCH_STORE_F32 || p->storage > LBCH_STORE_F16_DEV) return "unknown storage";
  if (p->regularization < LBCH_REG_NONE || p->regularization > LBCH_REG_LINEAR)
    return "unknown regularization";
  if (p->flags & ~(unsigned)(LBCH_Q_LITERAL | LBCH_MU_NESTED | LBCH_S35_EXPLICIT)) return "unknown flag bits";
  for (int i = 1; i < 9; ++i) {
    if ((i == 3 || i == 5) && !(p->flags & LBCH_S35_EXPLICIT)) continue;
    if (!(p->s[i] > 0.0 && p->s[i] < 2.0)) return "relaxation rates s_1..s_8 must lie in (0, 2)";
  }
  const double s35 = 1.0 / (p->M * 3.0 + 0.5);
  if (!(p->flags & LBCH_S35_EXPLICIT) && !(s35 > 0.0 && s35 < 2.0)) return "M gives s_3 outside (0, 2)";
  return nullptr;
}

void set_err(lbch_ctx* c, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof(c->err), fmt, ap);
  va_end(ap);
}

// Records a CUDA error (the context becomes failed). Returns true on error.
bool cuda_failed(lbch_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return false;
  c->failed = true;
  set_err(c, "%s: %s", what, cudaGetErrorString(e));
  return true;
}

lbch_status precheck(lbch_ctx* c, bool need_state) {
  if (!c) return LBCH_EINVAL;
  if (c->failed) return LBCH_ESTATE;
  if (need_state && !c->has_state) {
    set_err(c, "no state: call lbch_init_field or lbch_set_state first");
    return LBCH_EINVAL;
  }
  return LBCH_OK;
}

Grid grid_of(const lbch_ctx* c) { return Grid{c->p.nx, c->p.ny, c->ps}; }

// The step kernel instantiation for a context: storage, 16-byte rows (nx % 4 == 0), and
// whether the relaxation rates allow the reduced collision.
template <int ST>
const void* step_entry(bool vec, bool fast) {
  if (vec) return fast ? (const void*)step_kernel<ST, true, true> : (const void*)step_kernel<ST, true, false>;
  return fast ? (const void*)step_kernel<ST, false, true> : (const void*)step_kernel<ST, false, false>;
}

template <int ST>
void launch_step(lbch_ctx* c, const Field& f, cudaStream_t s) {
  const dim3 g(c->step_blocks), b(STEP_WARPS * 32);
  const StepArgs& a = c->sa;
  if (c->vec) {
    if (c->fast)
      step_kernel<ST, true, true><<<g, b, step_smem<ST, true>(), s>>>(a, f, c->n_warps);
    else
      step_kernel<ST, true, false><<<g, b, step_smem<ST, true>(), s>>>(a, f, c->n_warps);
  } else {
    if (c->fast)
      step_kernel<ST, false, true><<<g, b, step_smem<ST, false>(), s>>>(a, f, c->n_warps);
    else
      step_kernel<ST, false, false><<<g, b, step_smem<ST, false>(), s>>>(a, f, c->n_warps);
  }
}

template <int ST>
cudaError_t configure_step_kernel(bool vec, bool fast) {
  return cudaFuncSetAttribute(step_entry<ST>(vec, fast), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              vec ? step_smem<ST, true>() : step_smem<ST, false>());
}

template <int ST>
int step_occupancy(bool vec, bool fast) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step_entry<ST>(vec, fast), STEP_WARPS * 32,
                                                vec ? step_smem<ST, true>() : step_smem<ST, false>());
  return nb;
}

void fill_step_consts(lbch_ctx* c) {
  StepArgs& a = c->sa;
  const lbch_params& p = c->p;
  const bool nested = p.flags & LBCH_MU_NESTED;
  const double eps = p.regularization == LBCH_REG_NONE ? 0.0 : p.eps;
  a.k = (float)c->k;
  a.kq = (float)((p.flags & LBCH_Q_LITERAL) ? 1.0 : c->k);
  a.kiso = (float)(nested ? c->k : 0.0);
  a.beta4 = (float)(4.0 * c->beta);
  a.beta12 = (float)(12.0 * c->beta);
  c->fld.alpha = (float)p.alpha;
  c->fld.a16 = (float)(16.0 * p.alpha);
  a.eps = (float)eps;
  a.cw = p.regularization == LBCH_REG_LINEAR ? 0.0f : 1.0f;
  a.cfp = p.regularization == LBCH_REG_WILLMORE ? (float)eps : 0.0f;
  a.cnk = (float)(nested ? c->k : 0.0);
  const double* s = c->s;
  // n_k = m*_k / |row_k|^2 (|row|^2 = 9, 36, 36, 6, 12, 6, 12, 4, 4), with
  // m*_k = (1 - s_k) m_k + s_k m^eq_k + (1 - s_k/2) F_k, F_3 = -g_x/3, F_4 = g_x/3,
  // F_5 = -g_y/3, F_6 = g_y/3.
  a.c1a = (float)((1.0 - s[1]) / 36.0);
  a.c1b = (float)(s[1] / 36.0);
  a.c2a = (float)((1.0 - s[2]) / 36.0);
  a.c2b = (float)(s[2] / 36.0);
  a.c3a = (float)((1.0 - s[3]) / 6.0);
  a.c3g = (float)(-(1.0 - 0.5 * s[3]) / 18.0);
  a.c4a = (float)((1.0 - s[4]) / 12.0);
  a.c4g = (float)((1.0 - 0.5 * s[4]) / 36.0);
  a.c5a = (float)((1.0 - s[5]) / 6.0);
  a.c5g = (float)(-(1.0 - 0.5 * s[5]) / 18.0);
  a.c6a = (float)((1.0 - s[6]) / 12.0);
  a.c6g = (float)((1.0 - 0.5 * s[6]) / 36.0);
  a.c7 = (float)((1.0 - s[7]) / 4.0);
  a.c8 = (float)((1.0 - s[8]) / 4.0);
}

// f^eq of the FP64 phi0 in stage0 and its mu_alpha in stage1 into b; FP32 storage rounds
// the two products w mu_alpha per node into scratch planes of the other population buffer.
template <int ST>
void launch_init(lbch_ctx* c, Buf b) {
  float* eq_ax = c->buf[1].f32;
  float* eq_dg = c->buf[1].f32 + c->ps;
  init_state_kernel<ST><<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->stage0, c->stage1, b, grid_of(c), eq_ax,
                                                                      eq_dg);
  if constexpr (ST == ST_F32)
    init_gather_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(eq_ax, eq_dg, b, grid_of(c));
}

template <int ST>
void launch_phi(lbch_ctx* c, double* phi_d, float* phi_f) {
  phi_kernel<ST><<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->buf[c->cur], grid_of(c), phi_d, phi_f);
}

template <int ST>
void launch_mass(lbch_ctx* c, double* partial) {
  mass_kernel<ST><<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->buf[c->cur], grid_of(c), partial);
}

template <int ST>
void launch_get_plane(lbch_ctx* c, int i) {
  get_plane_kernel<ST><<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->buf[c->cur], grid_of(c), i, c->stage0);
}

template <int ST>
void launch_close_rest(lbch_ctx* c) {
  if constexpr (ST != ST_F32)
    close_rest_kernel<ST><<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->stage1, c->buf[c->cur], grid_of(c));
}

template <int ST>
void launch_set_dev(lbch_ctx* c, int i) {
  if constexpr (ST != ST_F32)
    set_plane_dev_kernel<ST><<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->stage0, c->buf[c->cur], grid_of(c), i);
}

// Calls FN<storage kind>(args...) for the context's storage.
#define DISPATCH(ST_VAL, FN, ...)                  \
  switch (ST_VAL) {                                \
    case ST_F32: FN<ST_F32>(__VA_ARGS__); break;   \
    case ST_BF16: FN<ST_BF16>(__VA_ARGS__); break; \
    default: FN<ST_F16>(__VA_ARGS__); break;       \
  }

// phi in FP32 (stage1), the energy densities, and their fixed-order FP64 sum into d_out.
void launch_energy(lbch_ctx* c, double* d_out) {
  float* phi_f = reinterpret_cast<float*>(c->stage1);
  DISPATCH(c->p.storage, launch_phi, c, nullptr, phi_f);
  EnergyConsts ec;
  const double eps = c->p.regularization == LBCH_REG_NONE ? 0.0 : c->p.eps;
  ec.k = (float)c->k;
  ec.beta = (float)c->beta;
  ec.beta4 = (float)(4.0 * c->beta);
  ec.alpha = (float)c->p.alpha;
  ec.half_eps = (float)(0.5 * eps);
  ec.cw = c->p.regularization == LBCH_REG_LINEAR ? 0.0f : 1.0f;
  energy_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(phi_f, grid_of(c), ec, c->partial);
  final_sum_kernel<<<1, 1024, 0, c->stream>>>(c->partial, c->aux_blocks, d_out);
}

lbch_status finish(lbch_ctx* c, const char* what) {
  if (cuda_failed(c, cudaGetLastError(), what)) return LBCH_ECUDA;
  return LBCH_OK;
}

// One time step from buffer `cur` on stream s.
void launch_one_step(lbch_ctx* c, int cur, cudaStream_t s) {
  Field f = c->fld;
  f.src = c->buf[cur];
  f.dst = c->buf[cur ^ 1];
  DISPATCH(c->p.storage, launch_step, c, f, s);
}

// Steps are replayed from a CUDA graph of GRAPH_STEPS launches (an even number, so the
// buffer parity returns): on small fields a step takes a few microseconds, comparable to
// the launch overhead the graph removes. The graph is captured on a private stream at the
// first call that can use it; a failed capture falls back to direct launches for good.
constexpr int GRAPH_STEPS = 16;

bool ensure_graph(lbch_ctx* c) {
  if (c->graph) return true;
  if (c->graph_off) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return false;  // the caller is capturing this stream: plain launches join its graph
  }
  cudaStream_t cap = nullptr;
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    for (int k = 0; k < GRAPH_STEPS; ++k) launch_one_step(c, k & 1, cap);
    ok = cudaStreamEndCapture(cap, &g) == cudaSuccess;
  }
  if (ok) ok = cudaGraphInstantiate(&c->graph, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (cap) cudaStreamDestroy(cap);
  if (!ok) {
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_off = true;
    cudaGetLastError();  // a failed capture is not an error of the context
  }
  return ok;
}

lbch_status sync_flag(lbch_ctx* c, int* host_flag, const char* what) {
  if (cuda_failed(c, cudaMemcpyAsync(host_flag, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream), what))
    return LBCH_ECUDA;
  if (cuda_failed(c, cudaStreamSynchronize(c->stream), what)) return LBCH_ECUDA;
  return LBCH_OK;
}

// Staging planes, reduction partials, results and flags of one field.
size_t scratch_bytes(const lbch_params* p) {
  const size_t n = (size_t)p->nx * p->ny;
  return 2 * align_up(n * sizeof(double)) + align_up(MAX_RED_BLOCKS * sizeof(double)) +
         align_up(8 * sizeof(double)) + align_up(16 * sizeof(int));
}

// Sets up a context whose two population buffers start at `state` and whose scratch
// (scratch_bytes(p)) starts at `scratch`; both 256-byte aligned device addresses.
lbch_status ctx_setup(const lbch_params* p, char* state, char* scratch, cudaStream_t stream, lbch_ctx** out) {
  lbch_ctx* c = new (std::nothrow) lbch_ctx();
  if (!c) return LBCH_ENOMEM;
  c->p = *p;
  c->beta = 3.0 * p->sigma / (4.0 * p->D);  // Eq. 5 solved for beta and k
  c->k = 3.0 * p->sigma * p->D / 8.0;
  for (int i = 0; i < 9; ++i) c->s[i] = p->s[i];
  if (!(p->flags & LBCH_S35_EXPLICIT)) c->s[3] = c->s[5] = 1.0 / (p->M * 3.0 + 0.5);  // after Eq. 38
  c->stream = stream;
  c->ws = state;
  c->ws_bytes = 0;
  c->ps = plane_stride(p);
  const size_t sb = state_bytes(p);
  const size_t n = (size_t)p->nx * p->ny;
  for (int b = 0; b < 2; ++b) {
    char* base = state + b * sb;
    c->buf[b].f32 = (float*)base;
    c->buf[b].dev = p->storage == LBCH_STORE_F32
                        ? nullptr
                        : (uint16_t*)(base + align_up((size_t)c->ps * 2 * sizeof(float)));
  }
  char* q = scratch;
  c->stage0 = (double*)q;
  q += align_up(n * sizeof(double));
  c->stage1 = (double*)q;
  q += align_up(n * sizeof(double));
  c->partial = (double*)q;
  q += align_up(MAX_RED_BLOCKS * sizeof(double));
  c->result = (double*)q;
  q += align_up(8 * sizeof(double));
  c->flags = (int*)q;
  c->cur = 0;
  c->has_state = false;
  c->steps = 0;
  c->failed = false;
  c->err[0] = 0;

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  c->vec = (p->nx % 4) == 0;
  c->fast = c->s[1] == 1.0 && c->s[2] == 1.0 && c->s[4] == 1.0 && c->s[6] == 1.0 && c->s[7] == 1.0 &&
            c->s[8] == 1.0;
  if (e == cudaSuccess) {
    switch (p->storage) {
      case LBCH_STORE_F32: e = configure_step_kernel<ST_F32>(c->vec, c->fast); break;
      case LBCH_STORE_BF16_DEV: e = configure_step_kernel<ST_BF16>(c->vec, c->fast); break;
      default: e = configure_step_kernel<ST_F16>(c->vec, c->fast); break;
    }
  }
  if (e != cudaSuccess) {
    delete c;
    return LBCH_ECUDA;
  }
  c->device = dev;
  int per_sm = 0;
  switch (p->storage) {
    case LBCH_STORE_F32: per_sm = step_occupancy<ST_F32>(c->vec, c->fast); break;
    case LBCH_STORE_BF16_DEV: per_sm = step_occupancy<ST_BF16>(c->vec, c->fast); break;
    default: per_sm = step_occupancy<ST_F16>(c->vec, c->fast); break;
  }
  if (per_sm < 1) {
    delete c;
    return LBCH_ECUDA;
  }
  // Strips of 120 output columns; segments of rows sized so that all warps fit in one
  // resident wave when the grid allows (each warp pays 6 warm-up rows).
  Field& f = c->fld;
  f.ps = c->ps;
  f.nx = p->nx;
  f.ny = p->ny;
  f.n_strips = n_strips_for(p->nx);
  const long long resident = (long long)sms * per_sm * STEP_WARPS;
  long long segs = resident / f.n_strips;
  if (segs < 1) segs = 1;
  // Small fields are latency-bound (one warp walks its segment row by row), so they take
  // segments down to 2 rows: measured 22 -> 8 us per step at 64^2-256^2, 22 -> 14 us at 512^2.
  const long long max_segs = (p->ny + 1) / 2;
  if (segs > max_segs) segs = max_segs;
  f.seg_len = (int)((p->ny + segs - 1) / segs);
  segs = (p->ny + f.seg_len - 1) / f.seg_len;
  c->n_warps = (long long)f.n_strips * segs;
  c->step_blocks = (int)((c->n_warps + STEP_WARPS - 1) / STEP_WARPS);
  fill_step_consts(c);
  long long ab = ((long long)n + AUX_THREADS - 1) / AUX_THREADS;
  const long long cap = (long long)sms * 8 < MAX_RED_BLOCKS ? (long long)sms * 8 : MAX_RED_BLOCKS;
  c->aux_blocks = (int)(ab < cap ? ab : cap);
  *out = c;
  return LBCH_OK;
}

}  // namespace

extern "C" {

size_t lbch_workspace_bytes(const lbch_params* p) {
  if (check_params(p)) return 0;
  return 2 * state_bytes(p) + scratch_bytes(p);
}

lbch_status lbch_create(const lbch_params* p, void* d_workspace, size_t bytes, void* cuda_stream,
                        lbch_ctx** out) {
  if (!out) return LBCH_EINVAL;
  if (check_params(p)) return LBCH_EINVAL;
  const size_t need = lbch_workspace_bytes(p);
  if (!d_workspace || bytes < need || ((uintptr_t)d_workspace % ALIGN) != 0) return LBCH_ENOMEM;
  char* ws = (char*)d_workspace;
  lbch_status st = ctx_setup(p, ws, ws + 2 * state_bytes(p), (cudaStream_t)cuda_stream, out);
  if (st == LBCH_OK) (*out)->ws_bytes = bytes;
  return st;
}

lbch_status lbch_init_field(lbch_ctx* c, const double* h_phi0) {
  lbch_status st = precheck(c, false);
  if (st != LBCH_OK) return st;
  if (!h_phi0) return LBCH_EINVAL;
  const size_t n = (size_t)c->p.nx * c->p.ny;
  c->has_state = false;
  if (cuda_failed(c, cudaMemcpyAsync(c->stage0, h_phi0, n * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                  "init_field: copy phi0"))
    return LBCH_ECUDA;
  if (cuda_failed(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "init_field: clear flag"))
    return LBCH_ECUDA;
  mu_alpha_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->stage0, c->stage1, grid_of(c), c->k,
                                                                4.0 * c->beta, c->flags);
  c->cur = 0;
  DISPATCH(c->p.storage, launch_init, c, c->buf[0]);
  if ((st = finish(c, "init_field: launch")) != LBCH_OK) return st;
  int bad = 0;
  if ((st = sync_flag(c, &bad, "init_field")) != LBCH_OK) return st;
  if (bad) {
    set_err(c, "init_field: phi0 holds NaN or Inf");
    return LBCH_ENONFINITE;
  }
  c->has_state = true;
  c->steps = 0;
  return LBCH_OK;
}

lbch_status lbch_init_field_device(lbch_ctx* c, const float* d_phi0) {
  lbch_status st = precheck(c, false);
  if (st != LBCH_OK) return st;
  if (!d_phi0) return LBCH_EINVAL;
  c->has_state = false;
  widen_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(d_phi0, (long long)c->p.nx * c->p.ny, c->stage0);
  mu_alpha_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->stage0, c->stage1, grid_of(c), c->k,
                                                                4.0 * c->beta, c->flags);
  c->cur = 0;
  DISPATCH(c->p.storage, launch_init, c, c->buf[0]);
  if ((st = finish(c, "init_field_device: launch")) != LBCH_OK) return st;
  c->has_state = true;
  c->steps = 0;
  return LBCH_OK;
}

lbch_status lbch_get_phi_device(lbch_ctx* c, float* d_phi) {
  lbch_status st = precheck(c, true);
  if (st != LBCH_OK) return st;
  if (!d_phi) return LBCH_EINVAL;
  DISPATCH(c->p.storage, launch_phi, c, nullptr, d_phi);
  return finish(c, "get_phi_device: launch");
}

lbch_status lbch_step(lbch_ctx* c, int64_t n) {
  lbch_status st = precheck(c, true);
  if (st != LBCH_OK) return st;
  if (n < 0) {
    set_err(c, "step: n must be >= 0");
    return LBCH_EINVAL;
  }
  int64_t left = n;
  if (left >= GRAPH_STEPS + (c->cur ? 1 : 0) && ensure_graph(c)) {
    if (c->cur == 1) {  // back to parity 0, where the graph starts
      launch_one_step(c, 1, c->stream);
      c->cur = 0;
      --left;
    }
    for (; left >= GRAPH_STEPS; left -= GRAPH_STEPS)
      if (cuda_failed(c, cudaGraphLaunch(c->graph, c->stream), "step: graph launch")) return LBCH_ECUDA;
  }
  for (; left > 0; --left) {
    launch_one_step(c, c->cur, c->stream);
    c->cur ^= 1;
  }
  c->steps += n;
  return finish(c, "step: launch");
}

lbch_status lbch_mass(lbch_ctx* c, double* out) {
  lbch_status st = precheck(c, true);
  if (st != LBCH_OK) return st;
  if (!out) return LBCH_EINVAL;
  DISPATCH(c->p.storage, launch_mass, c, c->partial);
  final_sum_kernel<<<1, 1024, 0, c->stream>>>(c->partial, c->aux_blocks, c->result);
  if ((st = finish(c, "mass: launch")) != LBCH_OK) return st;
  double v = 0.0;
  if (cuda_failed(c, cudaMemcpyAsync(&v, c->result, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "mass: copy"))
    return LBCH_ECUDA;
  if (cuda_failed(c, cudaStreamSynchronize(c->stream), "mass: sync")) return LBCH_ECUDA;
  *out = v;
  if (!std::isfinite(v)) {
    set_err(c, "mass is not finite");
    return LBCH_ENONFINITE;
  }
  return LBCH_OK;
}

lbch_status lbch_free_energy(lbch_ctx* c, double* out) {
  lbch_status st = precheck(c, true);
  if (st != LBCH_OK) return st;
  if (!out) return LBCH_EINVAL;
  launch_energy(c, c->result + 1);
  if ((st = finish(c, "free_energy: launch")) != LBCH_OK) return st;
  double v = 0.0;
  if (cuda_failed(c, cudaMemcpyAsync(&v, c->result + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                  "free_energy: copy"))
    return LBCH_ECUDA;
  if (cuda_failed(c, cudaStreamSynchronize(c->stream), "free_energy: sync")) return LBCH_ECUDA;
  *out = v;
  if (!std::isfinite(v)) {
    set_err(c, "free energy is not finite");
    return LBCH_ENONFINITE;
  }
  return LBCH_OK;
}

lbch_status lbch_get_field(lbch_ctx* c, double* h_phi) {
  lbch_status st = precheck(c, true);
  if (st != LBCH_OK) return st;
  if (!h_phi) return LBCH_EINVAL;
  const size_t n = (size_t)c->p.nx * c->p.ny;
  DISPATCH(c->p.storage, launch_phi, c, c->stage0, nullptr);
  if ((st = finish(c, "get_field: launch")) != LBCH_OK) return st;
  if (cuda_failed(c, cudaMemcpyAsync(h_phi, c->stage0, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                  "get_field: copy"))
    return LBCH_ECUDA;
  if (cuda_failed(c, cudaStreamSynchronize(c->stream), "get_field: sync")) return LBCH_ECUDA;
  return LBCH_OK;
}

lbch_status lbch_get_state(lbch_ctx* c, double* h_f9) {
  lbch_status st = precheck(c, true);
  if (st != LBCH_OK) return st;
  if (!h_f9) return LBCH_EINVAL;
  const size_t n = (size_t)c->p.nx * c->p.ny;
  for (int i = 0; i < 9; ++i) {
    DISPATCH(c->p.storage, launch_get_plane, c, i);
    if ((st = finish(c, "get_state: launch")) != LBCH_OK) return st;
    if (cuda_failed(c, cudaMemcpyAsync(h_f9 + i * n, c->stage0, n * sizeof(double), cudaMemcpyDeviceToHost,
                                       c->stream),
                    "get_state: copy"))
      return LBCH_ECUDA;
  }
  if (cuda_failed(c, cudaStreamSynchronize(c->stream), "get_state: sync")) return LBCH_ECUDA;
  return LBCH_OK;
}

lbch_status lbch_set_state(lbch_ctx* c, const double* h_f9) {
  lbch_status st = precheck(c, false);
  if (st != LBCH_OK) return st;
  if (!h_f9) return LBCH_EINVAL;
  const size_t n = (size_t)c->p.nx * c->p.ny;
  const Grid g = grid_of(c);
  c->has_state = false;
  c->cur = 0;
  if (cuda_failed(c, cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream), "set_state: clear flag"))
    return LBCH_ECUDA;
  if (c->p.storage == LBCH_STORE_F32) {
    for (int i = 0; i < 9; ++i) {
      if (cuda_failed(c, cudaMemcpyAsync(c->stage0, h_f9 + i * n, n * sizeof(double), cudaMemcpyHostToDevice,
                                         c->stream),
                      "set_state: copy"))
        return LBCH_ECUDA;
      set_plane_f32_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->stage0, c->buf[0], g, i, c->flags);
    }
  } else {
    // phi = sum_i f_i, then the anchor mu_alpha(phi), then each plane against it.
    for (int i = 0; i < 9; ++i) {
      if (cuda_failed(c, cudaMemcpyAsync(c->stage0, h_f9 + i * n, n * sizeof(double), cudaMemcpyHostToDevice,
                                         c->stream),
                      "set_state: copy"))
        return LBCH_ECUDA;
      accumulate_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->stage0, c->stage1, (long long)n, i == 0,
                                                                      c->flags);
    }
    mu_alpha_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->stage1, c->stage0, g, c->k, 4.0 * c->beta,
                                                                  c->flags);
    anchor_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(c->stage0, c->buf[0], g);
    for (int i = 1; i < 9; ++i) {
      if (cuda_failed(c, cudaMemcpyAsync(c->stage0, h_f9 + i * n, n * sizeof(double), cudaMemcpyHostToDevice,
                                         c->stream),
                      "set_state: copy"))
        return LBCH_ECUDA;
      DISPATCH(c->p.storage, launch_set_dev, c, i);
    }
    DISPATCH(c->p.storage, launch_close_rest, c);  // rest = phi - rebuilt moving populations
  }
  if ((st = finish(c, "set_state: launch")) != LBCH_OK) return st;
  int bad = 0;
  if ((st = sync_flag(c, &bad, "set_state")) != LBCH_OK) return st;
  if (bad) {
    set_err(c, "set_state: state holds NaN or Inf");
    return LBCH_ENONFINITE;
  }
  c->has_state = true;
  c->steps = 0;
  return LBCH_OK;
}

lbch_status lbch_mass_device(lbch_ctx* c, double* d_out) {
  lbch_status st = precheck(c, true);
  if (st != LBCH_OK) return st;
  if (!d_out) return LBCH_EINVAL;
  DISPATCH(c->p.storage, launch_mass, c, c->partial);
  final_sum_kernel<<<1, 1024, 0, c->stream>>>(c->partial, c->aux_blocks, d_out);
  return finish(c, "mass_device: launch");
}

lbch_status lbch_free_energy_device(lbch_ctx* c, double* d_out) {
  lbch_status st = precheck(c, true);
  if (st != LBCH_OK) return st;
  if (!d_out) return LBCH_EINVAL;
  launch_energy(c, d_out);
  return finish(c, "free_energy_device: launch");
}

lbch_status lbch_field_diagnostics_device(lbch_ctx* c, const float* d_phi, double* d_out2) {
  lbch_status st = precheck(c, false);
  if (st != LBCH_OK) return st;
  if (!d_phi || !d_out2) return LBCH_EINVAL;
  EnergyConsts ec;
  const double eps = c->p.regularization == LBCH_REG_NONE ? 0.0 : c->p.eps;
  ec.k = (float)c->k;
  ec.beta = (float)c->beta;
  ec.beta4 = (float)(4.0 * c->beta);
  ec.alpha = (float)c->p.alpha;
  ec.half_eps = (float)(0.5 * eps);
  ec.cw = c->p.regularization == LBCH_REG_LINEAR ? 0.0f : 1.0f;
  // mass partial sums in the second staging plane (nx ny doubles >= the block count)
  field_diag_kernel<<<c->aux_blocks, AUX_THREADS, 0, c->stream>>>(d_phi, grid_of(c), ec, c->partial, c->stage1);
  final_sum_pair_kernel<<<2, 1024, 0, c->stream>>>(c->stage1, c->partial, c->aux_blocks, d_out2);
  return finish(c, "field_diagnostics_device: launch");
}

size_t lbch_state_bytes(const lbch_params* p) { return check_params(p) ? 0 : state_bytes(p); }

lbch_status lbch_save_state_device(lbch_ctx* c, void* d_dst, size_t bytes) {
  lbch_status st = precheck(c, true);
  if (st != LBCH_OK) return st;
  const size_t sb = state_bytes(&c->p);
  if (!d_dst || bytes < sb) {
    set_err(c, "save_state_device: destination is NULL or smaller than %zu bytes", sb);
    return LBCH_EINVAL;
  }
  if (cuda_failed(c, cudaMemcpyAsync(d_dst, c->buf[c->cur].f32, sb, cudaMemcpyDeviceToDevice, c->stream),
                  "save_state_device: copy"))
    return LBCH_ECUDA;
  return LBCH_OK;
}

lbch_status lbch_restore_state_device(lbch_ctx* c, const void* d_src, size_t bytes) {
  lbch_status st = precheck(c, false);
  if (st != LBCH_OK) return st;
  const size_t sb = state_bytes(&c->p);
  if (!d_src || bytes < sb) {
    set_err(c, "restore_state_device: source is NULL or smaller than %zu bytes", sb);
    return LBCH_EINVAL;
  }
  if (cuda_failed(c, cudaMemcpyAsync(c->buf[0].f32, d_src, sb, cudaMemcpyDeviceToDevice, c->stream),
                  "restore_state_device: copy"))
    return LBCH_ECUDA;
  c->cur = 0;
  c->has_state = true;
  return LBCH_OK;
}

int64_t lbch_steps_taken(const lbch_ctx* c) { return c ? c->steps : -1; }

lbch_status lbch_set_steps_taken(lbch_ctx* c, int64_t steps) {
  if (!c || steps < 0) return LBCH_EINVAL;
  c->steps = steps;
  return LBCH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Allocation-free free energy (lbch_free_energy_static): the same phi -> energy ->
// fixed-order FP64 sum as lbch_free_energy, with its scratch in one static device array.

namespace {

constexpr long long STATIC_MAX_NODES = 1LL << 22;  // 2048 x 2048
constexpr size_t STATIC_PARTIAL_BYTES = (size_t)MAX_RED_BLOCKS * sizeof(double);
constexpr size_t STATIC_SCRATCH_BYTES = STATIC_PARTIAL_BYTES + (size_t)STATIC_MAX_NODES * sizeof(float);

// FP64 partial sums (first MAX_RED_BLOCKS doubles), then phi in FP32.
static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_static_mu;
void* g_static_addr[MAX_DEVICES];  // device address of g_static_scratch, per device
int g_static_sms[MAX_DEVICES];

// phi = sum_i f_i (Eq. 22) of canonical FP32 populations, summed in FP64, stored in FP32.
__global__ void phi_canonical_kernel(const float* __restrict__ f, long long ps, long long n,
                                     float* __restrict__ phi) {
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < n;
       id += (long long)gridDim.x * blockDim.x) {
    double p = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) p += (double)f[(long long)i * ps + id];
    phi[id] = (float)p;
  }
}

// Resolves the scratch address and SM count of the current device once.
cudaError_t static_setup(void** addr, int* sms) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_static_sms[dev] = n;
    g_static_addr[dev] = p;
  }
  *addr = g_static_addr[dev];
  *sms = g_static_sms[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" {

lbch_status lbch_free_energy_static(const lbch_params* p, const float* d_f9, int64_t plane_stride,
                                    double* d_out, void* cuda_stream) {
  if (!p || !d_f9 || !d_out) return LBCH_EINVAL;
  lbch_params q = *p;
  q.storage = LBCH_STORE_F32;  // the state is FP32 whatever the caller left in this field
  if (check_params(&q)) return LBCH_EINVAL;
  // An error pending from earlier work is the caller's: report it without launching,
  // and leave it pending (peek, not get).
  if (cudaPeekAtLastError() != cudaSuccess) return LBCH_ECUDA;
  const long long n = (long long)p->nx * p->ny;
  if (plane_stride < n) return LBCH_EINVAL;
  if (n > STATIC_MAX_NODES) return LBCH_EINVAL;  // beyond the static scratch
  void* base = nullptr;
  int sms = 0;
  if (static_setup(&base, &sms) != cudaSuccess) return LBCH_ECUDA;
  double* partial = reinterpret_cast<double*>(base);
  float* phi = reinterpret_cast<float*>(static_cast<char*>(base) + STATIC_PARTIAL_BYTES);
  long long blocks = (n + AUX_THREADS - 1) / AUX_THREADS;
  const long long cap = (long long)sms * 8 < MAX_RED_BLOCKS ? (long long)sms * 8 : MAX_RED_BLOCKS;
  if (blocks > cap) blocks = cap;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double k = 3.0 * p->sigma * p->D / 8.0, beta = 3.0 * p->sigma / (4.0 * p->D);  // Eq. 5
  const double eps = p->regularization == LBCH_REG_NONE ? 0.0 : p->eps;
  EnergyConsts ec;
  ec.k = (float)k;
  ec.beta = (float)beta;
  ec.beta4 = (float)(4.0 * beta);
  ec.alpha = (float)p->alpha;
  ec.half_eps = (float)(0.5 * eps);
  ec.cw = p->regularization == LBCH_REG_LINEAR ? 0.0f : 1.0f;
  // Every partial slot the final sum reads, and every phi value the energy kernel reads,
  // is written earlier in this same call: nothing needs clearing.
  phi_canonical_kernel<<<(int)blocks, AUX_THREADS, 0, st>>>(d_f9, plane_stride, n, phi);
  if (cudaGetLastError() != cudaSuccess) return LBCH_ECUDA;
  energy_kernel<<<(int)blocks, AUX_THREADS, 0, st>>>(phi, Grid{p->nx, p->ny, plane_stride}, ec, partial);
  if (cudaGetLastError() != cudaSuccess) return LBCH_ECUDA;
  final_sum_kernel<<<1, 1024, 0, st>>>(partial, (int)blocks, d_out);
  return cudaGetLastError() == cudaSuccess ? LBCH_OK : LBCH_ECUDA;
}

const char* lbch_last_error(const lbch_ctx* c) { return c ? c->err : "context is NULL"; }

void lbch_destroy(lbch_ctx* c) {
  if (c && c->graph) cudaGraphExecDestroy(c->graph);
  delete c;
}

}  // extern "C"

#include "lbch_batch.cuh"
#include "lbch3.cuh"
