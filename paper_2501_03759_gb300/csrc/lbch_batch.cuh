// Batched stepping of many independent periodic fields (the C-ABI lbch_batch_*),
// included at the end of lbch_api.cu so that it shares the context machinery.
//
// One kernel launch advances every field of the batch by one time step. Each warp
// reads its (field, strip, segment) from a task table and its field's geometry from
// a field table, then runs the same warp body as the single-field kernel, so every
// node is computed exactly as it would be alone. Kernel boundaries separate the time
// steps: there is no grid-wide barrier and no spin-wait. Steps are replayed from CUDA
// graphs of BATCH_GRAPH_STEPS launches to amortise launch cost. At creation a small
// autotuner times candidate row-segment lengths on the zeroed buffers and keeps the
// fastest.
#pragma once

#include <algorithm>
#include <vector>

namespace lbch {

constexpr int BATCH_GRAPH_STEPS = 64;                             // launches per CUDA graph (even)
constexpr int BATCH_ROW_TARGETS[] = {32, 64, 128, 256, 512, 1024};  // rows per warp tried by the tuner
constexpr int N_ROW_TARGETS = sizeof(BATCH_ROW_TARGETS) / sizeof(int);

template <int ST, bool VEC, bool FAST>
__global__ void __launch_bounds__(STEP_WARPS * 32, (Pipe<ST, VEC>::MIN_CTAS))
    step_batch_kernel(const __grid_constant__ StepArgs a, const Field* __restrict__ fields,
                      const int4* __restrict__ tasks, int n_tasks, int parity) {
  extern __shared__ float4 smem_slots[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int warp = blockIdx.x * STEP_WARPS + wib;
  if (warp >= n_tasks) return;  // whole warps only
  const int4 t = tasks[warp];   // field, strip, segment
  Field fd = fields[t.x];
  if (parity) {
    const Buf tmp = fd.src;
    fd.src = fd.dst;
    fd.dst = tmp;
  }
  float4* slots = smem_slots + wib * (Pipe<ST, VEC>::SLOTS * Pipe<ST, VEC>::SLOT_F4);
  step_warp<ST, VEC, FAST>(a, fd, t.y, t.z, slots, lane);
}

}  // namespace lbch

struct lbch_batch {
  int count;
  std::vector<lbch_ctx*> fields;  // one context per field, sharing the scratch area
  std::vector<long long> nodes;
  lbch_params common;
  cudaStream_t stream;
  cudaStream_t capture;          // private stream used only to capture the graph
  StepArgs sa;
  bool vec, fast;
  Field* d_fields;               // field table (parity 0 buffers), device
  int4* d_tasks;                 // task table, device
  size_t max_tasks;
  int n_tasks;
  int blocks;
  int rows_target;               // chosen by the tuner
  float tune_ms[N_ROW_TARGETS];
  int cur;
  int64_t steps;
  cudaGraphExec_t graph;
  bool failed;
  char err[512];
};

namespace {

void batch_err(lbch_batch* b, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->err, sizeof(b->err), fmt, ap);
  va_end(ap);
}

bool batch_cuda_failed(lbch_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return false;
  b->failed = true;
  batch_err(b, "%s: %s", what, cudaGetErrorString(e));
  return true;
}

// Parameters of field i: the common ones with this field's size and anisotropy.
lbch_params field_params(const lbch_params* common, int32_t nx, int32_t ny, double alpha) {
  lbch_params p = *common;
  p.nx = nx;
  p.ny = ny;
  p.alpha = alpha;
  return p;
}

int n_strips_of(int nx) { return n_strips_for(nx); }

// Task list for a rows-per-warp target: largest fields first (longest work first),
// and within a field the strips of a segment next to each other (they share halos).
void build_tasks(const int32_t* nx, const int32_t* ny, int count, int rows, std::vector<int4>& tasks,
                 std::vector<int>& seg_len) {
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (long long)nx[x] * ny[x] > (long long)nx[y] * ny[y];
  });
  tasks.clear();
  seg_len.assign(count, 1);
  for (int f : order) {
    const int segs = std::max(1, (ny[f] + rows - 1) / rows);
    const int len = (ny[f] + segs - 1) / segs;
    seg_len[f] = len;
    const int nseg = (ny[f] + len - 1) / len;
    for (int g = 0; g < nseg; ++g)
      for (int s = 0; s < n_strips_of(nx[f]); ++s) tasks.push_back(make_int4(f, s, g, 0));
  }
}

size_t max_task_count(const int32_t* nx, const int32_t* ny, int count) {
  size_t m = 0;
  std::vector<int4> t;
  std::vector<int> l;
  for (int r = 0; r < N_ROW_TARGETS; ++r) {
    build_tasks(nx, ny, count, BATCH_ROW_TARGETS[r], t, l);
    m = std::max(m, t.size());
  }
  return m;
}

const char* check_batch(const lbch_params* common, int32_t count, const int32_t* nx, const int32_t* ny,
                        const double* alpha) {
  if (!common || !nx || !ny || count < 1 || count > (1 << 20)) return "bad batch arguments";
  for (int i = 0; i < count; ++i) {
    const lbch_params p = field_params(common, nx[i], ny[i], alpha ? alpha[i] : common->alpha);
    if (const char* e = check_params(&p)) return e;
  }
  return nullptr;
}

template <int ST, bool VEC, bool FAST>
void launch_batch_kernel(lbch_batch* b, cudaStream_t s, int parity) {
  step_batch_kernel<ST, VEC, FAST><<<b->blocks, STEP_WARPS * 32, step_smem<ST, VEC>(), s>>>(
      b->sa, b->d_fields, b->d_tasks, b->n_tasks, parity);
}

template <int ST>
void launch_batch(lbch_batch* b, cudaStream_t s, int parity) {
  if (b->vec) {
    if (b->fast) launch_batch_kernel<ST, true, true>(b, s, parity);
    else launch_batch_kernel<ST, true, false>(b, s, parity);
  } else {
    if (b->fast) launch_batch_kernel<ST, false, true>(b, s, parity);
    else launch_batch_kernel<ST, false, false>(b, s, parity);
  }
}

template <int ST>
const void* batch_entry(bool vec, bool fast) {
  if (vec)
    return fast ? (const void*)step_batch_kernel<ST, true, true> : (const void*)step_batch_kernel<ST, true, false>;
  return fast ? (const void*)step_batch_kernel<ST, false, true> : (const void*)step_batch_kernel<ST, false, false>;
}

template <int ST>
cudaError_t configure_batch_kernel(bool vec, bool fast) {
  return cudaFuncSetAttribute(batch_entry<ST>(vec, fast), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              vec ? step_smem<ST, true>() : step_smem<ST, false>());
}

void batch_launch(lbch_batch* b, cudaStream_t s, int parity) {
  DISPATCH(b->common.storage, launch_batch, b, s, parity);
}

// Uploads a task list for `rows` and sets the per-field segment lengths in the field table.
lbch_status batch_use_rows(lbch_batch* b, const int32_t* nx, const int32_t* ny, int rows) {
  std::vector<int4> tasks;
  std::vector<int> seg_len;
  build_tasks(nx, ny, b->count, rows, tasks, seg_len);
  std::vector<Field> table(b->count);
  for (int i = 0; i < b->count; ++i) {
    Field f = b->fields[i]->fld;
    f.seg_len = seg_len[i];
    f.src = b->fields[i]->buf[0];
    f.dst = b->fields[i]->buf[1];
    table[i] = f;
  }
  if (batch_cuda_failed(b, cudaMemcpyAsync(b->d_tasks, tasks.data(), tasks.size() * sizeof(int4),
                                           cudaMemcpyHostToDevice, b->stream), "batch: upload tasks") ||
      batch_cuda_failed(b, cudaMemcpyAsync(b->d_fields, table.data(), table.size() * sizeof(Field),
                                           cudaMemcpyHostToDevice, b->stream), "batch: upload fields") ||
      batch_cuda_failed(b, cudaStreamSynchronize(b->stream), "batch: upload sync"))
    return LBCH_ECUDA;
  b->n_tasks = (int)tasks.size();
  b->blocks = (b->n_tasks + STEP_WARPS - 1) / STEP_WARPS;
  b->rows_target = rows;
  return LBCH_OK;
}

}  // namespace

extern "C" {

size_t lbch_batch_workspace_bytes(const lbch_params* common, int32_t count, const int32_t* nx, const int32_t* ny) {
  if (check_batch(common, count, nx, ny, nullptr)) return 0;
  size_t total = 0, scratch = 0;
  for (int i = 0; i < count; ++i) {
    const lbch_params p = field_params(common, nx[i], ny[i], common->alpha);
    total += 2 * state_bytes(&p);
    scratch = std::max(scratch, scratch_bytes(&p));
  }
  return total + scratch + align_up((size_t)count * sizeof(Field)) +
         align_up(max_task_count(nx, ny, count) * sizeof(int4));
}

lbch_status lbch_batch_create(const lbch_params* common, int32_t count, const int32_t* nx, const int32_t* ny,
                              const double* alpha, void* d_workspace, size_t bytes, void* cuda_stream,
                              lbch_batch** out) {
  if (!out || check_batch(common, count, nx, ny, alpha)) return LBCH_EINVAL;
  const size_t need = lbch_batch_workspace_bytes(common, count, nx, ny);
  if (!d_workspace || bytes < need || ((uintptr_t)d_workspace % ALIGN) != 0) return LBCH_ENOMEM;
  lbch_batch* b = new (std::nothrow) lbch_batch();
  if (!b) return LBCH_ENOMEM;
  b->count = count;
  b->common = *common;
  b->stream = (cudaStream_t)cuda_stream;
  b->capture = nullptr;
  b->graph = nullptr;
  b->cur = 0;
  b->steps = 0;
  b->failed = false;
  b->err[0] = 0;
  // Layout: field states, shared scratch, field table, task table.
  char* q = (char*)d_workspace;
  size_t scratch = 0;
  for (int i = 0; i < count; ++i) {
    const lbch_params p = field_params(common, nx[i], ny[i], alpha ? alpha[i] : common->alpha);
    scratch = std::max(scratch, scratch_bytes(&p));
  }
  char* states = q;
  size_t state_total = 0;
  for (int i = 0; i < count; ++i) {
    const lbch_params p = field_params(common, nx[i], ny[i], common->alpha);
    state_total += 2 * state_bytes(&p);
  }
  char* shared_scratch = states + state_total;
  b->d_fields = (Field*)(shared_scratch + scratch);
  b->d_tasks = (int4*)((char*)b->d_fields + align_up((size_t)count * sizeof(Field)));
  b->max_tasks = max_task_count(nx, ny, count);
  b->fields.assign(count, nullptr);
  b->nodes.assign(count, 0);
  char* st = states;
  bool all_vec = true;
  for (int i = 0; i < count; ++i) {
    const lbch_params p = field_params(common, nx[i], ny[i], alpha ? alpha[i] : common->alpha);
    lbch_status r = ctx_setup(&p, st, shared_scratch, b->stream, &b->fields[i]);
    if (r != LBCH_OK) {
      lbch_batch_destroy(b);
      return r;
    }
    st += 2 * state_bytes(&p);
    b->nodes[i] = (long long)nx[i] * ny[i];
    all_vec = all_vec && b->fields[i]->vec;
  }
  b->sa = b->fields[0]->sa;  // the same scheme constants for every field
  b->fast = b->fields[0]->fast;
  b->vec = all_vec;
  cudaError_t e;
  switch (common->storage) {
    case LBCH_STORE_F32: e = configure_batch_kernel<ST_F32>(b->vec, b->fast); break;
    case LBCH_STORE_BF16_DEV: e = configure_batch_kernel<ST_BF16>(b->vec, b->fast); break;
    default: e = configure_batch_kernel<ST_F16>(b->vec, b->fast); break;
  }
  if (batch_cuda_failed(b, e, "batch: configure") ||
      batch_cuda_failed(b, cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "batch: stream")) {
    lbch_batch_destroy(b);
    return LBCH_ECUDA;
  }
  // Autotune the row-segment length on zeroed buffers (the kernel's work does not depend
  // on the values), then capture the graph for the winner.
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  bool ok = !batch_cuda_failed(b, cudaMemsetAsync(states, 0, state_total, b->stream), "batch: clear") &&
            !batch_cuda_failed(b, cudaEventCreate(&t0), "batch: event") &&
            !batch_cuda_failed(b, cudaEventCreate(&t1), "batch: event");
  int best = 0;
  for (int r = 0; ok && r < N_ROW_TARGETS; ++r) {
    if (batch_use_rows(b, nx, ny, BATCH_ROW_TARGETS[r]) != LBCH_OK) {
      ok = false;
      break;
    }
    for (int w = 0; w < 2; ++w) batch_launch(b, b->stream, w & 1);
    cudaEventRecord(t0, b->stream);
    for (int k = 0; k < 6; ++k) batch_launch(b, b->stream, k & 1);
    cudaEventRecord(t1, b->stream);
    if (batch_cuda_failed(b, cudaEventSynchronize(t1), "batch: tune")) {
      ok = false;
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, t0, t1);
    b->tune_ms[r] = ms / 6.0f;
    if (b->tune_ms[r] < b->tune_ms[best]) best = r;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (ok) ok = batch_use_rows(b, nx, ny, BATCH_ROW_TARGETS[best]) == LBCH_OK;
  if (ok) {
    cudaGraph_t g = nullptr;
    ok = !batch_cuda_failed(b, cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal),
                            "batch: capture");
    if (ok) {
      for (int k = 0; k < BATCH_GRAPH_STEPS; ++k) batch_launch(b, b->capture, k & 1);
      ok = !batch_cuda_failed(b, cudaStreamEndCapture(b->capture, &g), "batch: capture end");
    }
    if (ok) ok = !batch_cuda_failed(b, cudaGraphInstantiate(&b->graph, g, 0), "batch: instantiate");
    if (g) cudaGraphDestroy(g);
  }
  if (!ok) {
    lbch_batch_destroy(b);
    return LBCH_ECUDA;
  }
  *out = b;
  return LBCH_OK;
}

lbch_status lbch_batch_init_field(lbch_batch* b, int32_t i, const double* h_phi0) {
  if (!b || i < 0 || i >= b->count) return LBCH_EINVAL;
  if (b->failed) return LBCH_ESTATE;
  lbch_ctx* c = b->fields[i];
  if (b->cur != 0) {  // keep every field on the batch's buffer parity
    batch_err(b, "init_field: initialise fields before the first step or after an even number of steps");
    return LBCH_EINVAL;
  }
  lbch_status st = lbch_init_field(c, h_phi0);
  if (st != LBCH_OK) batch_err(b, "field %d: %s", i, lbch_last_error(c));
  if (st == LBCH_ECUDA) b->failed = true;
  return st;
}

lbch_status lbch_batch_step(lbch_batch* b, int64_t n) {
  if (!b || n < 0) return LBCH_EINVAL;
  if (b->failed) return LBCH_ESTATE;
  for (lbch_ctx* c : b->fields)
    if (!c->has_state) {
      batch_err(b, "step: every field needs lbch_batch_init_field first");
      return LBCH_EINVAL;
    }
  int64_t left = n;
  if (b->cur == 1 && left > 0) {  // back to parity 0 so that graphs can be replayed
    batch_launch(b, b->stream, 1);
    b->cur = 0;
    --left;
  }
  while (left >= BATCH_GRAPH_STEPS) {
    if (batch_cuda_failed(b, cudaGraphLaunch(b->graph, b->stream), "step: graph launch")) return LBCH_ECUDA;
    left -= BATCH_GRAPH_STEPS;
  }
  for (; left > 0; --left) {
    batch_launch(b, b->stream, b->cur);
    b->cur ^= 1;
  }
  b->steps += n;
  for (lbch_ctx* c : b->fields) {
    c->cur = b->cur;
    c->steps = b->steps;
  }
  if (batch_cuda_failed(b, cudaGetLastError(), "step: launch")) return LBCH_ECUDA;
  return LBCH_OK;
}

#define LBCH_BATCH_FIELD_CALL(NAME, CALL)                              \
  lbch_status NAME {                                                   \
    if (!b || i < 0 || i >= b->count) return LBCH_EINVAL;             \
    if (b->failed) return LBCH_ESTATE;                                 \
    lbch_ctx* c = b->fields[i];                                        \
    lbch_status st = CALL;                                             \
    if (st != LBCH_OK) batch_err(b, "field %d: %s", i, lbch_last_error(c)); \
    if (st == LBCH_ECUDA) b->failed = true;                            \
    return st;                                                         \
  }

LBCH_BATCH_FIELD_CALL(lbch_batch_get_field(lbch_batch* b, int32_t i, double* h_phi), lbch_get_field(c, h_phi))
LBCH_BATCH_FIELD_CALL(lbch_batch_get_phi_device(lbch_batch* b, int32_t i, float* d_phi), lbch_get_phi_device(c, d_phi))
LBCH_BATCH_FIELD_CALL(lbch_batch_mass(lbch_batch* b, int32_t i, double* out), lbch_mass(c, out))
LBCH_BATCH_FIELD_CALL(lbch_batch_free_energy(lbch_batch* b, int32_t i, double* out), lbch_free_energy(c, out))
#undef LBCH_BATCH_FIELD_CALL

int32_t lbch_batch_rows_target(const lbch_batch* b) { return b ? b->rows_target : -1; }

int64_t lbch_batch_steps_taken(const lbch_batch* b) { return b ? b->steps : -1; }

const char* lbch_batch_last_error(const lbch_batch* b) { return b ? b->err : "batch is NULL"; }

void lbch_batch_destroy(lbch_batch* b) {
  if (!b) return;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (lbch_ctx* c : b->fields) delete c;
  delete b;
}

}  // extern "C"
