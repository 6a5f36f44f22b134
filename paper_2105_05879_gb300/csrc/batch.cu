// batch.cu -- batches of queries over any mix of plans in one persistent,
// graph-captured launch, and the autotuner of the query kernel's ring.
//
// A batch is a fixed list of queries (plan, x, J, K, S, eps, seed, outputs).
// At creation the host resolves every query into a device descriptor, deals
// the queries to the CTAs plan by plan (largest rows first), each plan's
// longest first onto the least-loaded CTA by estimated cost (bytes gathered
// plus refined), uploads descriptors and schedule to the caller's workspace,
// and (optionally) captures the launch into a CUDA graph that
// kerdock_batch_launch replays.  Inputs are read at replay time, so a caller
// refills the same x buffers and replays.
#include <algorithm>
#include <cstring>
#include <new>
#include <queue>
#include <unordered_map>
#include <vector>

#include "kerdock_internal.cuh"

namespace {

// Candidate ring geometries tried by the autotuners.
const int kTuneRingKb[] = {64, 96, 128, 160};
const int kTuneCrows[] = {1, 2, 4, 8};

struct Timer {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~Timer() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};

}  // namespace

struct kerdock_batch_s {
  int device = -1;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  std::vector<kd::QueryDesc> descs;
  std::vector<int32_t> order;
  std::vector<int64_t> cta_start;
  kd::Dims dims;
  kd::Tuning tuning;
  kd::LaunchCfg cfg{};
  bool means_in_smem = true;
  int grid = 0;
  kd::QueryDesc* d_descs = nullptr;
  int32_t* d_order = nullptr;
  int64_t* d_cta_start = nullptr;
  float* d_means = nullptr;
  uint32_t* status = nullptr;
  bool use_graph = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

struct WsLayout {
  size_t descs, order, cta, means, total;
};

WsLayout ws_layout(int64_t count, int grid, const kd::Dims& dm, bool means_in_smem) {
  WsLayout w{};
  size_t off = 0;
  w.descs = off;
  off = kd::align_up(off + size_t(count) * sizeof(kd::QueryDesc), 256);
  w.order = off;
  off = kd::align_up(off + size_t(count) * sizeof(int32_t), 256);
  w.cta = off;
  off = kd::align_up(off + size_t(grid + 1) * sizeof(int64_t), 256);
  w.means = off;
  if (!means_in_smem) off = kd::align_up(off + size_t(grid) * 2 * size_t(dm.KL) * 4, 256);
  w.total = off;
  return w;
}

int validate_query(const kerdock_query_t& q, int device) {
  if (q.plan == nullptr || q.x == nullptr || q.out_idx == nullptr || q.out_val == nullptr ||
      q.out_count == nullptr)
    return KERDOCK_ERR_INVALID_ARG;
  const kd::Plan& p = q.plan->p;
  if (!p.bound) return KERDOCK_ERR_NOT_BOUND;
  if (!p.preprocessed) return KERDOCK_ERR_NOT_PREPROCESSED;
  if (p.device != device) return KERDOCK_ERR_INVALID_ARG;
  if (q.J < 1 || q.K < 1 || q.K > kd::kMaxK || int64_t(q.J) * q.K > kd::kMaxN)
    return KERDOCK_ERR_UNSUPPORTED;
  if (q.S < 1 || q.S > p.m) return KERDOCK_ERR_INVALID_ARG;
  if (q.flags < 0 || q.flags > KERDOCK_FLAG_FULL_OUTPUT) return KERDOCK_ERR_INVALID_ARG;
  if (!(q.flags & KERDOCK_FLAG_FULL_OUTPUT) && !(q.eps > 0.0f)) return KERDOCK_ERR_INVALID_ARG;
  if (q.index < 0) return KERDOCK_ERR_INVALID_ARG;
  return KERDOCK_OK;
}

int device_sms(int* device, int* sms) {
  KD_CUDA_TRY(cudaGetDevice(device));
  KD_CUDA_TRY(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, *device));
  return KERDOCK_OK;
}

void destroy_graph(kerdock_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// The schedule of deal() as a pure function of the queries' plans (any
// pointer identifying each query's plan), row bytes and costs: order[] lists
// the queries CTA by CTA, CTA c's from cta_start[c] to cta_start[c + 1].
void plan_major_schedule(const void* const* plan_ids, const uint32_t* row_bytes,
                         const double* cost, int64_t count, int grid, std::vector<int32_t>& order,
                         std::vector<int64_t>& cta_start) {
  // plan groups in order of first appearance
  std::unordered_map<const void*, int> group_of;
  std::vector<uint32_t> group_row_bytes;
  std::vector<int> group(static_cast<size_t>(count));
  for (int64_t i = 0; i < count; ++i) {
    const auto ins = group_of.emplace(plan_ids[i], int(group_row_bytes.size()));
    if (ins.second) group_row_bytes.push_back(row_bytes[i]);
    group[size_t(i)] = ins.first->second;
  }
  const size_t ngroups = group_row_bytes.size();
  std::vector<int> gorder(ngroups);
  for (size_t g = 0; g < ngroups; ++g) gorder[g] = int(g);
  std::stable_sort(gorder.begin(), gorder.end(), [&](int x, int y) {
    return group_row_bytes[size_t(x)] > group_row_bytes[size_t(y)];
  });
  std::vector<int> grank(ngroups);
  for (size_t k = 0; k < ngroups; ++k) grank[size_t(gorder[k])] = int(k);
  std::vector<int32_t> by_cost(static_cast<size_t>(count));
  for (int64_t i = 0; i < count; ++i) by_cost[size_t(i)] = int32_t(i);
  std::stable_sort(by_cost.begin(), by_cost.end(), [&](int32_t x, int32_t y) {
    const int gx = grank[size_t(group[size_t(x)])], gy = grank[size_t(group[size_t(y)])];
    return gx != gy ? gx < gy : cost[x] > cost[y];
  });
  using Load = std::pair<double, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int c = 0; c < grid; ++c) heap.push({0.0, c});
  std::vector<std::vector<int32_t>> per_cta(static_cast<size_t>(grid));
  for (int32_t qi : by_cost) {
    Load top = heap.top();
    heap.pop();
    per_cta[size_t(top.second)].push_back(qi);
    top.first += cost[qi];
    heap.push(top);
  }
  order.clear();
  cta_start.assign(size_t(grid) + 1, 0);
  for (int c = 0; c < grid; ++c) {
    cta_start[size_t(c) + 1] = cta_start[size_t(c)] + int64_t(per_cta[size_t(c)].size());
    for (int32_t qi : per_cta[size_t(c)]) order.push_back(qi);
  }
}

// Deal the queries to the CTAs by cost (any unit), plan by plan: the plans in
// decreasing order of row size, each plan's queries longest first onto the
// least-loaded CTA (loads carried from plan to plan), every CTA running its
// share of one plan before the next.  So all CTAs sweep one representation at
// a time, and the rows in flight share its address translations: on GB300 the
// mixed batch of seven plans (n = 64 ... 4096, 2048 queries) took 5.20 ms this
// way against 6.59 ms with one longest-first order over all queries, 7.1 ms
// with each CTA's list rotated to a different starting point and 7.7 ms
// shuffled.  Fills the host order and per-CTA start arrays.
void deal(kerdock_batch_s* b, const std::vector<double>& cost) {
  const size_t count = cost.size();
  std::vector<const void*> plan_ids(count);
  std::vector<uint32_t> row_bytes(count);
  for (size_t i = 0; i < count; ++i) {
    plan_ids[i] = b->descs[i].R;
    row_bytes[i] = b->descs[i].row_bytes;
  }
  plan_major_schedule(plan_ids.data(), row_bytes.data(), cost.data(), int64_t(count), b->grid,
                      b->order, b->cta_start);
}

// Upload the schedule (order and per-CTA starts) on the batch's stream and
// wait for it: the host arrays are the copies' sources.
cudaError_t upload_schedule(kerdock_batch_s* b) {
  cudaError_t e = cudaMemcpyAsync(b->d_order, b->order.data(), b->order.size() * sizeof(int32_t),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_cta_start, b->cta_start.data(),
                        b->cta_start.size() * sizeof(int64_t), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e;
}

// Set the ring geometry and (re)capture the launch into a graph when asked.
int configure(kerdock_batch_s* b, const kd::Tuning& tu) {
  kd::LaunchCfg cfg{};
  if (!kd::make_cfg(b->dims, tu, b->means_in_smem, cfg, true)) return KERDOCK_ERR_UNSUPPORTED;
  cfg.means_gmem = b->means_in_smem ? nullptr : b->d_means;
  cfg.status = b->status;
  b->cfg = cfg;
  b->tuning = tu;
  destroy_graph(b);
  int rc = kd::prepare_batch_kernel(b->cfg);  // not a stream operation: before any capture
  if (rc != KERDOCK_OK) return rc;
  if (b->use_graph) {
    KD_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    rc = kd::launch_batch(b->cfg, b->d_descs, b->d_order, b->d_cta_start, b->grid, b->stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t end = cudaStreamEndCapture(b->stream, &graph);
    if (rc != KERDOCK_OK || end != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc != KERDOCK_OK ? rc : KERDOCK_ERR_CUDA;
    }
    b->graph = graph;
    KD_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  }
  return KERDOCK_OK;
}

int launch(kerdock_batch_s* b) {
  if (b->exec) {
    KD_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
    return KERDOCK_OK;
  }
  return kd::launch_batch(b->cfg, b->d_descs, b->d_order, b->d_cta_start, b->grid, b->stream);
}

// Time reps back-to-back runs of fn on stream (milliseconds per run).
template <class Fn>
int time_runs(cudaStream_t stream, int reps, Fn fn, float* ms) {
  Timer t;
  KD_CUDA_TRY(cudaEventCreate(&t.e0));
  KD_CUDA_TRY(cudaEventCreate(&t.e1));
  int rc = fn();  // warm-up
  if (rc != KERDOCK_OK) return rc;
  KD_CUDA_TRY(cudaEventRecord(t.e0, stream));
  for (int r = 0; r < reps; ++r) {
    rc = fn();
    if (rc != KERDOCK_OK) return rc;
  }
  KD_CUDA_TRY(cudaEventRecord(t.e1, stream));
  KD_CUDA_TRY(cudaEventSynchronize(t.e1));
  float total = 0.f;
  KD_CUDA_TRY(cudaEventElapsedTime(&total, t.e0, t.e1));
  *ms = total / float(reps);
  return KERDOCK_OK;
}

}  // namespace

extern "C" {

size_t kerdock_batch_workspace_bytes(const kerdock_query_t* queries, int64_t count) {
  if (queries == nullptr || count < 1) return 0;
  int device = 0, sms = 0;
  if (device_sms(&device, &sms) != KERDOCK_OK) return 0;
  kd::Dims dm;
  for (int64_t i = 0; i < count; ++i) {
    if (queries[i].plan == nullptr) return 0;
    kd::dims_add(dm, queries[i].plan->p, queries[i].K, queries[i].S);
  }
  const int grid = int(count < sms ? count : sms);
  return ws_layout(count, grid, dm, kd::means_fit_smem(dm)).total;
}

int kerdock_batch_create(kerdock_batch_t* batch, const kerdock_query_t* queries, int64_t count,
                         void* ws_dev, size_t ws_bytes, void* stream, int32_t options) {
  if (batch == nullptr) return KERDOCK_ERR_INVALID_ARG;
  *batch = nullptr;
  if (queries == nullptr || count < 1 || count > (int64_t(1) << 31) - 1 || ws_dev == nullptr)
    return KERDOCK_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws_dev) & 255) return KERDOCK_ERR_ALIGNMENT;
  if (options & ~KERDOCK_BATCH_GRAPH) return KERDOCK_ERR_INVALID_ARG;
  int device = 0, sms = 0;
  int rc = device_sms(&device, &sms);
  if (rc != KERDOCK_OK) return rc;
  auto* b = new (std::nothrow) kerdock_batch_s();
  if (b == nullptr) return KERDOCK_ERR_INVALID_ARG;
  b->device = device;
  b->num_sms = sms;
  b->stream = static_cast<cudaStream_t>(stream);
  b->descs.resize(size_t(count));
  std::vector<double> cost(static_cast<size_t>(count));
  for (int64_t i = 0; i < count; ++i) {
    const kerdock_query_t& q = queries[i];
    rc = validate_query(q, device);
    if (rc != KERDOCK_OK) {
      delete b;
      return rc;
    }
    const kd::Plan& p = q.plan->p;
    kd::QueryDesc d = kd::plan_desc(p);
    kd::set_query_params(d, q.J, q.K, q.S, q.eps, q.seed, q.flags);
    d.x = q.x;
    d.out_idx = q.out_idx;
    d.out_val = q.out_val;
    d.out_count = q.out_count;
    d.ctr_base = q.index * d.N;
    b->descs[size_t(i)] = d;
    kd::dims_add(b->dims, p, q.K, q.S);
    cost[size_t(i)] = double(d.N) * double(d.row_bytes) + double(q.S) * double(p.n) * 4.0 +
                      65536.0;
    if (i == 0) b->status = p.status();
  }
  b->means_in_smem = kd::means_fit_smem(b->dims);
  b->grid = int(count < sms ? count : sms);
  deal(b, cost);
  const WsLayout w = ws_layout(count, b->grid, b->dims, b->means_in_smem);
  if (ws_bytes < w.total) {
    delete b;
    return KERDOCK_ERR_CAPACITY;
  }
  char* base = static_cast<char*>(ws_dev);
  b->d_descs = reinterpret_cast<kd::QueryDesc*>(base + w.descs);
  b->d_order = reinterpret_cast<int32_t*>(base + w.order);
  b->d_cta_start = reinterpret_cast<int64_t*>(base + w.cta);
  b->d_means = b->means_in_smem ? nullptr : reinterpret_cast<float*>(base + w.means);
  cudaError_t e = cudaMemcpyAsync(b->d_descs, b->descs.data(), b->descs.size() * sizeof(kd::QueryDesc),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = upload_schedule(b);
  if (e != cudaSuccess) {
    delete b;
    return KERDOCK_ERR_CUDA;
  }
  b->use_graph = (options & KERDOCK_BATCH_GRAPH) && b->stream != nullptr;
  rc = configure(b, kd::Tuning{});
  if (rc != KERDOCK_OK) {
    destroy_graph(b);
    delete b;
    return rc;
  }
  *batch = b;
  return KERDOCK_OK;
}

int kerdock_batch_launch(kerdock_batch_t batch) {
  if (batch == nullptr) return KERDOCK_ERR_INVALID_ARG;
  return launch(batch);
}

int kerdock_batch_set_tuning(kerdock_batch_t batch, int32_t ring_kb, int32_t crows) {
  if (batch == nullptr || ring_kb < 0 || crows < 0) return KERDOCK_ERR_INVALID_ARG;
  kd::Tuning tu;
  tu.ring_kb = ring_kb;
  tu.crows = crows;
  return configure(batch, tu);
}

int kerdock_batch_set_costs(kerdock_batch_t batch, const double* cost, int64_t count) {
  if (batch == nullptr || cost == nullptr || count != int64_t(batch->descs.size()))
    return KERDOCK_ERR_INVALID_ARG;
  std::vector<double> c(static_cast<size_t>(count));
  for (int64_t i = 0; i < count; ++i) {
    if (!(cost[i] >= 0.0) || !(cost[i] <= 1e300)) return KERDOCK_ERR_INVALID_ARG;  // NaN, < 0, inf
    c[size_t(i)] = cost[i];
  }
  deal(batch, c);
  // the kernel (and a captured graph) reads the schedule through the same
  // device arrays, so the new one takes effect from the next launch
  if (upload_schedule(batch) != cudaSuccess) return KERDOCK_ERR_CUDA;
  return KERDOCK_OK;
}

int kerdock_debug_batch_schedule(const void* const* plan_ids, const uint32_t* row_bytes,
                                 const double* cost, int64_t count, int32_t grid,
                                 int32_t* order_out, int64_t* cta_start_out) {
  if (plan_ids == nullptr || row_bytes == nullptr || cost == nullptr || order_out == nullptr ||
      cta_start_out == nullptr || count < 1 || count > (int64_t(1) << 31) - 1 || grid < 1)
    return KERDOCK_ERR_INVALID_ARG;
  for (int64_t i = 0; i < count; ++i)
    if (!(cost[i] >= 0.0) || !(cost[i] <= 1e300)) return KERDOCK_ERR_INVALID_ARG;
  std::vector<int32_t> order;
  std::vector<int64_t> cta_start;
  plan_major_schedule(plan_ids, row_bytes, cost, count, grid, order, cta_start);
  std::copy(order.begin(), order.end(), order_out);
  std::copy(cta_start.begin(), cta_start.end(), cta_start_out);
  return KERDOCK_OK;
}

int32_t kerdock_batch_ctas(kerdock_batch_t batch) { return batch == nullptr ? 0 : batch->grid; }

int kerdock_batch_set_schedule(kerdock_batch_t batch, const int32_t* order,
                               const int64_t* cta_start, int32_t ctas) {
  if (batch == nullptr || order == nullptr || cta_start == nullptr || ctas < 1 ||
      ctas > batch->grid)
    return KERDOCK_ERR_INVALID_ARG;
  const int64_t count = int64_t(batch->descs.size());
  if (cta_start[0] != 0 || cta_start[ctas] != count) return KERDOCK_ERR_INVALID_ARG;
  for (int32_t c = 0; c < ctas; ++c)
    if (cta_start[c + 1] < cta_start[c]) return KERDOCK_ERR_INVALID_ARG;
  std::vector<char> seen(static_cast<size_t>(count), 0);  // order must be a permutation
  for (int64_t i = 0; i < count; ++i) {
    if (order[i] < 0 || order[i] >= count || seen[size_t(order[i])]) return KERDOCK_ERR_INVALID_ARG;
    seen[size_t(order[i])] = 1;
  }
  batch->order.assign(order, order + count);
  batch->cta_start.assign(size_t(batch->grid) + 1, count);  // CTAs past ctas get no queries
  for (int32_t c = 0; c <= ctas; ++c) batch->cta_start[size_t(c)] = cta_start[c];
  if (upload_schedule(batch) != cudaSuccess) return KERDOCK_ERR_CUDA;
  return KERDOCK_OK;
}

int kerdock_batch_tune(kerdock_batch_t batch, int32_t reps, int32_t* ring_kb, int32_t* crows,
                       float* best_ms) {
  if (batch == nullptr || reps < 1) return KERDOCK_ERR_INVALID_ARG;
  const bool graph = batch->use_graph;
  batch->use_graph = false;  // time plain launches; capture once at the end
  float best = -1.f;
  kd::Tuning best_tu;
  for (int rk : kTuneRingKb) {
    for (int cr : kTuneCrows) {
      kd::Tuning tu;
      tu.ring_kb = rk;
      tu.crows = cr;
      if (configure(batch, tu) != KERDOCK_OK) continue;
      float ms = 0.f;
      const int rc = time_runs(batch->stream, reps, [&] { return launch(batch); }, &ms);
      if (rc != KERDOCK_OK) {
        batch->use_graph = graph;
        return rc;
      }
      if (best < 0.f || ms < best) {
        best = ms;
        best_tu = tu;
      }
    }
  }
  batch->use_graph = graph;
  if (best < 0.f) return KERDOCK_ERR_UNSUPPORTED;
  const int rc = configure(batch, best_tu);
  if (rc != KERDOCK_OK) return rc;
  if (ring_kb) *ring_kb = best_tu.ring_kb;
  if (crows) *crows = best_tu.crows;
  if (best_ms) *best_ms = best;
  return KERDOCK_OK;
}

int kerdock_batch_sync(kerdock_batch_t batch) {
  if (batch == nullptr) return KERDOCK_ERR_INVALID_ARG;
  uint32_t status = 0;
  KD_CUDA_TRY(cudaMemcpyAsync(&status, batch->status, sizeof(status), cudaMemcpyDeviceToHost,
                              batch->stream));
  KD_CUDA_TRY(cudaStreamSynchronize(batch->stream));
  if (status != kd::kStatusOk) {
    KD_CUDA_TRY(cudaMemsetAsync(batch->status, 0, sizeof(uint32_t), batch->stream));
    KD_CUDA_TRY(cudaStreamSynchronize(batch->stream));
    return status == kd::kStatusTimeout ? KERDOCK_ERR_DEVICE_TIMEOUT : KERDOCK_ERR_INVALID_ARG;
  }
  return KERDOCK_OK;
}

int kerdock_batch_destroy(kerdock_batch_t batch) {
  if (batch == nullptr) return KERDOCK_OK;
  destroy_graph(batch);
  delete batch;
  return KERDOCK_OK;
}

int kerdock_plan_set_tuning(kerdock_plan_t plan, int32_t ring_kb, int32_t crows) {
  if (plan == nullptr || ring_kb < 0 || crows < 0 ||
      (crows != 0 && crows != 1 && crows != 2 && crows != 4 && crows != 8))
    return KERDOCK_ERR_INVALID_ARG;
  kd::Plan& p = plan->p;
  kd::Tuning tu;
  tu.ring_kb = ring_kb;
  tu.crows = crows;
  const kd::Dims dm = kd::plan_dims(p);
  kd::LaunchCfg cfg{};
  if (!kd::make_cfg(dm, tu, kd::means_fit_smem(dm), cfg)) return KERDOCK_ERR_UNSUPPORTED;
  p.tuning = tu;
  return KERDOCK_OK;
}

int kerdock_plan_tune(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx, float eps,
                      uint64_t seed, int32_t* out_idx, float* out_val, int32_t* out_count,
                      void* ws_dev, size_t ws_bytes, int32_t reps, int32_t* ring_kb,
                      int32_t* crows, float* best_ms) {
  if (plan == nullptr || reps < 1 || q < 1) return KERDOCK_ERR_INVALID_ARG;
  kd::Plan& p = plan->p;
  const kd::Tuning saved = p.tuning;
  float best = -1.f;
  kd::Tuning best_tu;
  for (int rk : kTuneRingKb) {
    for (int cr : kTuneCrows) {
      if (kerdock_plan_set_tuning(plan, rk, cr) != KERDOCK_OK) continue;
      float ms = 0.f;
      const int rc = time_runs(p.stream, reps,
                               [&] {
                                 return kerdock_apply(plan, X_dev, q, ldx, eps, seed, 0, out_idx,
                                                      out_val, out_count, ws_dev, ws_bytes);
                               },
                               &ms);
      if (rc != KERDOCK_OK) {
        p.tuning = saved;
        return rc;
      }
      if (best < 0.f || ms < best) {
        best = ms;
        best_tu = p.tuning;
      }
    }
  }
  if (best < 0.f) {
    p.tuning = saved;
    return KERDOCK_ERR_UNSUPPORTED;
  }
  p.tuning = best_tu;
  if (ring_kb) *ring_kb = best_tu.ring_kb;
  if (crows) *crows = best_tu.crows;
  if (best_ms) *best_ms = best;
  return KERDOCK_OK;
}

}  // extern "C"
