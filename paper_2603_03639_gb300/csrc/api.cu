// Host runtime of the tnrc C ABI: validation, one device arena per context,
// slot layout, launch order (noise -> gates -> trajectories -> reduction).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/tnrc.h"
#include "plan.h"
#include "tnrc_device.cuh"

extern "C" cudaError_t tnrc_launch_traj(const tnrc::TrajParams* p, int grid, size_t smem, cudaStream_t st);
extern "C" cudaError_t tnrc_traj_prepare();
extern "C" cudaError_t tnrc_plain_prepare();
extern "C" cudaError_t tnrc_launch_plain(const tnrc::TrajParams* p, int op, const unsigned char* a,
                                         unsigned char* b, int s, int l, int t, size_t smem, cudaStream_t st);
extern "C" cudaError_t tnrc_traj_occupancy(int phys_dim, int min_blocks, int warps, size_t smem, int* per_sm);
extern "C" cudaError_t tnrc_launch_layer_gates(int N, int K, int C, int M, int terms, int order, int nsub,
                                               int L, int R, int first_parity, double dt, const double* u,
                                               const unsigned char* mask, const double* gfix, const double* J,
                                               const int* layer_off, tnrc::LayerGate* out, int* status,
                                               cudaStream_t st);
extern "C" cudaError_t tnrc_launch_noise(unsigned long long seed, int dist, double scale, int M, int nb, double* J,
                                         cudaStream_t st);
extern "C" cudaError_t tnrc_launch_reduce(const double2* O, int T, double* F, double* per_traj, const double* gsp,
                                          int X, double* grad, cudaStream_t st);
extern "C" cudaError_t tnrc_launch_canon(const tnrc::CanonArgs* a, int nmps, cudaStream_t st);

using namespace tnrc_host;

namespace {
// An NVTX range over a host-side phase (launches are asynchronous, so a range
// marks when the phase was issued); a no-op unless a profiler is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};
}  // namespace

struct tnrc_ctx {
  Plan plan;
  double dt, eps;
  cudaStream_t stream = nullptr;
  unsigned char* arena = nullptr;
  bool have_u = false, have_J = false, gates_dirty = true, broken = false;
  int last_status = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> tev;   // pairs around trajectory-kernel launches
  size_t tev_used = 0;
  // the forward history of the costate sweep is kept packed at the actual bond
  // dimensions in each CTA's work region when it fits (else checkpoints)
  int packed_history = 1;
  long long history_cap = (long long)1 << 62;
  // CUDA graphs of tnrc_evaluate_dev, one per (gradient?, outputs, gate rebuild?)
  struct GraphEntry {
    bool grad, gates;
    double *dF, *dgrad, *dper;
    cudaGraphExec_t exec;
  };
  bool use_graphs = false;
  // pooled launch (one CTA per trajectory, work regions from a pool), with
  // the dynamic shared memory that keeps the resident CTAs within the pool
  bool pooled = false;
  size_t pooled_smem = 0;
  int pair_svd = 1;               // matrix shape: two small SVDs per warp (1) or one (0)
  bool timed_last = false;        // ev0/ev1 bracket the last evaluation (not a graph replay)
  std::vector<GraphEntry> graphs;
  char err[256] = {0};            // the CUDA failure that made the context unusable
  // buffers of the plain one-trajectory-at-a-time path (made on first use)
  unsigned char* plain = nullptr;
  tnrc_stats stats{};
  int n_sm = 0;
  template <class T>
  T* at(int64_t off) {
    return reinterpret_cast<T*>(arena + off);
  }
};

namespace {

tnrc_status fail_cuda(tnrc_ctx* c, cudaError_t e, int line) {
  if (c) {
    c->broken = true;
    snprintf(c->err, sizeof(c->err), "api.cu:%d: %s: %s", line, cudaGetErrorName(e), cudaGetErrorString(e));
  }
  return TNRC_E_CUDA;
}

#define CK(x)                                                   \
  do {                                                          \
    const cudaError_t ck_e_ = (x);                              \
    if (ck_e_ != cudaSuccess) return fail_cuda(ctx, ck_e_, __LINE__); \
  } while (0)

// Trajectory-kernel parameters of a context (the persistent launch's arena
// regions; other launch forms override what differs).
tnrc::TrajParams traj_params(tnrc_ctx* ctx, bool grad) {
  Plan& P = ctx->plan;
  tnrc::TrajParams tp{};
  tp.N = P.N;
  tp.K = P.K;
  tp.C = P.C;
  tp.P = P.P;
  tp.M = P.M;
  tp.chi = P.chi;
  tp.T = P.T;
  tp.dt = ctx->dt;
  tp.eps = ctx->eps;
  tp.want_grad = grad ? 1 : 0;
  tp.warps = P.warps;
  tp.slab_elems = P.slab_elems;
  tp.min_blocks = P.d == 4 ? 1 : P.min_blocks;
  tp.phys_dim = P.d;
  tp.full.L = P.L;
  tp.full.site_off = ctx->at<int>(P.off_siteoff);
  tp.full.dcap = ctx->at<int>(P.off_dcap);
  tp.full.seg = P.seg;
  tp.full.nseg = P.nseg;
  tp.packed_history = ctx->packed_history;
  tp.history_cap = ctx->history_cap;
  tp.in_slots = ctx->at<unsigned char>(P.off_in);
  tp.tg_slots = ctx->at<unsigned char>(P.off_tg);
  tp.work = ctx->at<unsigned char>(P.off_work);
  tp.work_stride = P.work_stride;
  tp.warp_scratch = ctx->at<double2>(P.off_scratch);
  tp.scratch_elems = P.scratch_elems;
  tp.env_scratch = ctx->at<double2>(P.off_env);
  tp.lgates = ctx->at<tnrc::LayerGate>(P.off_gates);
  tp.layer_off = ctx->at<int>(P.off_loff);
  tp.n_layers = P.n_layers;
  tp.first_parity = P.first_parity;
  tp.recs_per_sample = P.recs;
  tp.mask = ctx->at<unsigned char>(P.off_mask);
  tp.O = ctx->at<double2>(P.off_O);
  tp.gsp = ctx->at<double>(P.off_gsp);
  tp.disc = ctx->at<double>(P.off_disc);
  tp.counters = ctx->at<unsigned long long>(P.off_counters);
  tp.status = ctx->at<int>(P.off_status);
  tp.work_counter = ctx->at<int>(P.off_wc);
  tp.pair_svd = ctx->pair_svd;
  return tp;
}

tnrc_status launch_eval(tnrc_ctx* ctx, bool grad, double* dF, double* dgrad, double* dper, bool capturing = false) {
  Plan& P = ctx->plan;
  cudaStream_t st = ctx->stream;
  if (!capturing) CK(cudaEventRecord(ctx->ev0, st));
  ctx->timed_last = !capturing;
  Range eval_range(grad ? "tnrc:evaluate(F, grad)" : "tnrc:evaluate(F)");
  if (ctx->gates_dirty) {
    Range r("tnrc:layer gates");
    CK(tnrc_launch_layer_gates(P.N, P.K, P.C, P.M, P.terms, P.order, P.nsub, P.n_layers, P.recs, P.first_parity,
                               ctx->dt, ctx->at<double>(P.off_u), ctx->at<unsigned char>(P.off_mask),
                               ctx->at<double>(P.off_gfix), ctx->at<double>(P.off_J), ctx->at<int>(P.off_loff),
                               ctx->at<tnrc::LayerGate>(P.off_gates), ctx->at<int>(P.off_status), st));
    ctx->gates_dirty = false;
  }
  CK(cudaMemsetAsync(ctx->at<int>(P.off_wc), 0, sizeof(int), st));
  CK(cudaMemsetAsync(ctx->at<unsigned long long>(P.off_counters), 0, tnrc::kNumCounters * 8, st));
  CK(cudaMemsetAsync(ctx->at<unsigned long long>(P.off_counters) + tnrc::kCtrGap, 0xff, 8, st));
  tnrc::TrajParams tp = traj_params(ctx, grad);
  size_t smem = tnrc_traj_smem(P.warps, P.slab_elems);
  int grid = P.grid;
  if (ctx->pooled) {
    tp.pooled = 1;
    tp.n_regions = P.grid;
    tp.region_owner = ctx->at<int>(P.off_owner);
    CK(cudaMemsetAsync(tp.region_owner, 0, (size_t)P.grid * 4, st));
    smem = ctx->pooled_smem;
    grid = P.T;
  }
  const bool timed = !capturing && ctx->tev_used + 2 <= ctx->tev.size();
  if (timed) CK(cudaEventRecord(ctx->tev[ctx->tev_used], st));
  {
    Range r("tnrc:trajectories");
    CK(tnrc_launch_traj(&tp, grid, smem, st));
  }
  if (timed) {
    CK(cudaEventRecord(ctx->tev[ctx->tev_used + 1], st));
    ctx->tev_used += 2;
  }
  const int X = P.K * P.C * P.N;
  Range red_range("tnrc:reduce");
  CK(tnrc_launch_reduce(ctx->at<double2>(P.off_O), P.T, dF ? dF : ctx->at<double>(P.off_F), dper,
                        grad ? ctx->at<double>(P.off_gsp) : nullptr, X,
                        grad ? (dgrad ? dgrad : ctx->at<double>(P.off_grad)) : nullptr, st));
  if (!capturing) CK(cudaEventRecord(ctx->ev1, st));
  return TNRC_OK;
}

// tnrc_evaluate_dev through a CUDA graph captured on first use for these
// outputs and replayed afterwards (the launch sequence and every kernel
// argument are fixed per context, so a replay is the same work).
tnrc_status launch_eval_graph(tnrc_ctx* ctx, bool grad, double* dF, double* dgrad, double* dper) {
  const bool gates = ctx->gates_dirty;
  for (auto& g : ctx->graphs) {
    if (g.grad == grad && g.gates == gates && g.dF == dF && g.dgrad == dgrad && g.dper == dper) {
      CK(cudaGraphLaunch(g.exec, ctx->stream));
      ctx->gates_dirty = false;
      ctx->timed_last = false;
      return TNRC_OK;
    }
  }
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  const tnrc_status s = launch_eval(ctx, grad, dF, dgrad, dper, true);
  const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
  if (s != TNRC_OK) return s;
  CK(e);
  tnrc_ctx::GraphEntry g{grad, gates, dF, dgrad, dper, nullptr};
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(ei);
  ctx->graphs.push_back(g);
  CK(cudaGraphLaunch(g.exec, ctx->stream));
  ctx->timed_last = false;
  return TNRC_OK;
}

tnrc_status finish(tnrc_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  int status = 0;
  CK(cudaMemcpy(&status, ctx->at<int>(ctx->plan.off_status), sizeof(int), cudaMemcpyDeviceToHost));
  if (status) {
    CK(cudaMemset(ctx->at<int>(ctx->plan.off_status), 0, sizeof(int)));
    ctx->last_status = status;
    return (status & tnrc::kStatusTimeout) ? TNRC_E_TIMEOUT : TNRC_E_NUMERIC;
  }
  float ms = 0.f;
  if (ctx->timed_last) CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  ctx->stats.last_ms = ctx->timed_last ? ms : 0.0;
  return TNRC_OK;
}

tnrc_status evaluate_host(tnrc_ctx* ctx, bool grad, double* F, double* grad_out, double* per_traj) {
  if (!ctx || !F || (grad && !grad_out)) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  if (!ctx->have_u || !ctx->have_J) return TNRC_E_STATE;
  Plan& P = ctx->plan;
  tnrc_status s = launch_eval(ctx, grad, nullptr, nullptr, per_traj ? ctx->at<double>(P.off_per) : nullptr);
  if (s != TNRC_OK) return s;
  s = finish(ctx);
  if (s != TNRC_OK) return s;
  CK(cudaMemcpy(F, ctx->at<double>(P.off_F), 8, cudaMemcpyDeviceToHost));
  if (grad) CK(cudaMemcpy(grad_out, ctx->at<double>(P.off_grad), (size_t)P.K * P.C * P.N * 8, cudaMemcpyDeviceToHost));
  if (per_traj) CK(cudaMemcpy(per_traj, ctx->at<double>(P.off_per), (size_t)P.T * 8, cudaMemcpyDeviceToHost));
  return TNRC_OK;
}

}  // namespace

extern "C" {

size_t tnrc_footprint(const tnrc_problem* problem) {
  Plan P;
  int dev = 0, n_sm = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (!make_plan(problem, n_sm, 0, P, false)) return 0;
  return (size_t)P.total;
}

tnrc_status tnrc_create(const tnrc_problem* pb, const tnrc_mps* inputs, const tnrc_mps* targets, void* cuda_stream,
                        tnrc_ctx** out) {
  if (!out) return TNRC_E_INVALID;
  *out = nullptr;
  if (!pb || !inputs || !targets || pb->struct_size != sizeof(tnrc_problem)) return TNRC_E_INVALID;
  {
    Plan check;
    if (!make_plan(pb, 1, 0, check, false)) return TNRC_E_INVALID;
  }
  const int N = pb->n_sites;
  if (check_problem_arrays(pb, inputs, targets) != TNRC_OK) return TNRC_E_INVALID;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TNRC_E_CUDA;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TNRC_E_CUDA;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return TNRC_E_CUDA;
  tnrc_ctx* ctx = new (std::nothrow) tnrc_ctx();
  if (!ctx) return TNRC_E_NOMEM;
  if (!make_plan(pb, n_sm, 0, ctx->plan, false)) {
    delete ctx;
    return TNRC_E_INVALID;
  }
  if (!make_plan(pb, n_sm, free_b, ctx->plan, true)) {
    delete ctx;
    return TNRC_E_NOMEM;
  }
  Plan& P = ctx->plan;
  ctx->n_sm = n_sm;
  ctx->dt = pb->dt;
  ctx->eps = std::max(pb->sv_cutoff, tnrc::kZeroFloor);
  ctx->stream = (cudaStream_t)cuda_stream;
  if (cudaMalloc(&ctx->arena, (size_t)P.total) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return TNRC_E_NOMEM;
  }
  auto bail = [&](tnrc_status s) {
    tnrc_destroy(ctx);
    return s;
  };
  if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess)
    return bail(TNRC_E_CUDA);
  if (tnrc_traj_prepare() != cudaSuccess) return bail(TNRC_E_CUDA);
  ctx->tev.assign(512, nullptr);
  for (auto& e : ctx->tev)
    if (cudaEventCreate(&e) != cudaSuccess) return bail(TNRC_E_CUDA);
  cudaStream_t st = ctx->stream;
  // mask, g_fixed, site offsets, zeroed status
  const std::vector<unsigned char> mask = control_mask(pb);
  std::vector<double> gfix((size_t)P.K * (N - 1), 0.0);
  if (pb->g_fixed) std::memcpy(gfix.data(), pb->g_fixed, gfix.size() * 8);
  if (cudaMemcpyAsync(ctx->at<void>(P.off_mask), mask.data(), mask.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ctx->at<void>(P.off_gfix), gfix.data(), gfix.size() * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(ctx->at<void>(P.off_siteoff), P.site_off.data(), (size_t)N * 4, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(ctx->at<void>(P.off_dcap), P.dcap.data(), (size_t)(N + 1) * 4, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(ctx->at<void>(P.off_loff), P.layer_off.data(), (size_t)(P.n_layers + 1) * 4,
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(ctx->at<void>(P.off_status), 0, 16, st) != cudaSuccess ||
      cudaMemsetAsync(ctx->at<void>(P.off_in), 0, (size_t)P.P * P.L.bytes, st) != cudaSuccess ||
      cudaMemsetAsync(ctx->at<void>(P.off_tg), 0, (size_t)P.P * P.L.bytes, st) != cudaSuccess)
    return bail(TNRC_E_CUDA);
  // canonical inputs and targets
  {
    Range r("tnrc:canonical inputs and targets");
    const int nmps = 2 * P.P;
    std::vector<int> dims((size_t)nmps * (N + 1));
    std::vector<long long> offs(nmps);
    long long total = 0;
    int dmax = P.chi;
    for (int j = 0; j < nmps; ++j) {
      const tnrc_mps& m = (j < P.P) ? inputs[j] : targets[j - P.P];
      offs[j] = total;
      for (int i = 0; i <= N; ++i) {
        dims[(size_t)j * (N + 1) + i] = m.bond_dims[i];
        dmax = std::max(dmax, m.bond_dims[i]);
      }
      for (int i = 0; i < N; ++i) total += (long long)m.bond_dims[i] * P.d * m.bond_dims[i + 1];
    }
    std::vector<double> raw((size_t)total * 2);
    for (int j = 0; j < nmps; ++j) {
      const tnrc_mps& m = (j < P.P) ? inputs[j] : targets[j - P.P];
      long long cnt = 0;
      for (int i = 0; i < N; ++i) cnt += (long long)m.bond_dims[i] * P.d * m.bond_dims[i + 1];
      for (long long e = 0; e < 2 * cnt; ++e)
        if (!std::isfinite(m.data[e])) return bail(TNRC_E_INVALID);
      std::memcpy(raw.data() + offs[j] * 2, m.data, (size_t)cnt * 16);
    }
    const long long wstride = (long long)(N + 4) * P.d * dmax * dmax;
    void *d_dims = nullptr, *d_raw = nullptr, *d_offs = nullptr, *d_work = nullptr;
    bool ok = cudaMalloc(&d_dims, dims.size() * 4) == cudaSuccess && cudaMalloc(&d_raw, raw.size() * 8) == cudaSuccess &&
              cudaMalloc(&d_offs, offs.size() * 8) == cudaSuccess &&
              cudaMalloc(&d_work, (size_t)nmps * wstride * 16) == cudaSuccess;
    if (ok) {
      ok = cudaMemcpyAsync(d_dims, dims.data(), dims.size() * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(d_raw, raw.data(), raw.size() * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
           cudaMemcpyAsync(d_offs, offs.data(), offs.size() * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
    }
    if (ok) {
      tnrc::CanonArgs a{};
      a.N = N;
      a.chi = P.chi;
      a.d = P.d;
      a.eps = ctx->eps;
      a.dmax = dmax;
      a.raw_dims = (const int*)d_dims;
      a.raw_data = (const double2*)d_raw;
      a.raw_off = (const long long*)d_offs;
      a.work = (double2*)d_work;
      a.work_stride = wstride;
      a.slots = ctx->at<unsigned char>(P.off_in);  // inputs then targets: contiguous
      a.L = P.L;
      a.site_off = ctx->at<int>(P.off_siteoff);
      a.status = ctx->at<int>(P.off_status);
      ok = (P.off_tg == P.off_in + align_up((int64_t)P.P * P.L.bytes, 256)) &&
           tnrc_launch_canon(&a, nmps, st) == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
    }
    cudaFree(d_dims);
    cudaFree(d_raw);
    cudaFree(d_offs);
    cudaFree(d_work);
    if (!ok) {
      cudaGetLastError();
      return bail(TNRC_E_CUDA);
    }
    int status = 0;
    if (cudaMemcpy(&status, ctx->at<int>(P.off_status), 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return bail(TNRC_E_CUDA);
    if (status) return bail(TNRC_E_NUMERIC);
  }
  ctx->stats.hist_len = P.chi + 1;
  if (const char* e = getenv("TNRC_PACKED_HISTORY")) ctx->packed_history = atoi(e) != 0;
  if (const char* e = getenv("TNRC_HISTORY_CAP")) ctx->history_cap = std::max(0ll, atoll(e));
  *out = ctx;
  return TNRC_OK;
}

tnrc_status tnrc_set_controls(tnrc_ctx* ctx, const double* u, int64_t len) {
  if (!ctx || !u) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  const Plan& P = ctx->plan;
  if (len != (int64_t)P.K * P.C * P.N) return TNRC_E_INVALID;
  for (int64_t i = 0; i < len; ++i)
    if (!std::isfinite(u[i])) return TNRC_E_INVALID;
  CK(cudaMemcpyAsync(ctx->at<void>(P.off_u), u, (size_t)len * 8, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->have_u = true;
  ctx->gates_dirty = true;
  return TNRC_OK;
}

tnrc_status tnrc_set_controls_dev(tnrc_ctx* ctx, const double* d_u) {
  if (!ctx || !d_u) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  const Plan& P = ctx->plan;
  CK(cudaMemcpyAsync(ctx->at<void>(P.off_u), d_u, (size_t)P.K * P.C * P.N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  ctx->have_u = true;
  ctx->gates_dirty = true;
  return TNRC_OK;
}

tnrc_status tnrc_sample_noise(tnrc_ctx* ctx, uint64_t seed, int32_t dist, double scale) {
  if (!ctx || (dist != 0 && dist != 1) || !(scale >= 0.0) || !std::isfinite(scale)) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  const Plan& P = ctx->plan;
  CK(tnrc_launch_noise(seed, dist, scale, P.M, (P.N - 1) * P.terms, ctx->at<double>(P.off_J), ctx->stream));
  ctx->have_J = true;
  ctx->gates_dirty = true;
  return TNRC_OK;
}

tnrc_status tnrc_set_noise(tnrc_ctx* ctx, const double* J, int64_t len) {
  if (!ctx || !J) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  const Plan& P = ctx->plan;
  if (len != (int64_t)P.M * (P.N - 1) * P.terms) return TNRC_E_INVALID;
  for (int64_t i = 0; i < len; ++i)
    if (!std::isfinite(J[i])) return TNRC_E_INVALID;
  CK(cudaMemcpyAsync(ctx->at<void>(P.off_J), J, (size_t)len * 8, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->have_J = true;
  ctx->gates_dirty = true;
  return TNRC_OK;
}

tnrc_status tnrc_get_noise(tnrc_ctx* ctx, double* J, int64_t len) {
  if (!ctx || !J) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  if (!ctx->have_J) return TNRC_E_STATE;
  const Plan& P = ctx->plan;
  if (len != (int64_t)P.M * (P.N - 1) * P.terms) return TNRC_E_INVALID;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(J, ctx->at<void>(P.off_J), (size_t)len * 8, cudaMemcpyDeviceToHost));
  return TNRC_OK;
}

tnrc_status tnrc_fidelity(tnrc_ctx* ctx, double* F, double* per_traj) {
  return evaluate_host(ctx, false, F, nullptr, per_traj);
}

tnrc_status tnrc_fidelity_grad(tnrc_ctx* ctx, double* F, double* grad) {
  return evaluate_host(ctx, true, F, grad, nullptr);
}

tnrc_status tnrc_evaluate_dev(tnrc_ctx* ctx, double* d_F, double* d_grad, double* d_per_traj) {
  if (!ctx || !d_F) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  if (!ctx->have_u || !ctx->have_J) return TNRC_E_STATE;
  if (ctx->use_graphs) return launch_eval_graph(ctx, d_grad != nullptr, d_F, d_grad, d_per_traj);
  return launch_eval(ctx, d_grad != nullptr, d_F, d_grad, d_per_traj);
}

tnrc_status tnrc_set_graphs(tnrc_ctx* ctx, int32_t enable) {
  if (!ctx || (enable != 0 && enable != 1)) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  if (enable && ctx->stream == nullptr) return TNRC_E_INVALID;  // the legacy stream cannot be captured
  ctx->use_graphs = enable != 0;
  return TNRC_OK;
}

tnrc_status tnrc_fidelity_grad_plain(tnrc_ctx* ctx, double* F, double* grad) {
  if (!ctx || !F || !grad) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  if (!ctx->have_u || !ctx->have_J) return TNRC_E_STATE;
  Plan& P = ctx->plan;
  cudaStream_t st = ctx->stream;
  const int L = P.n_layers;
  const int64_t sb = P.L.bytes;
  int nbmax = 0;
  for (int par = 0; par < 2; ++par) nbmax = std::max(nbmax, (P.N - 1 - par + 1) / 2);
  const int nscr = std::max(nbmax, 2);
  // every layer state of the trajectory as a full slot, the costate slot,
  // per-CTA warp scratch and one environment region
  const int64_t off_hist = 0, off_c = off_hist + (int64_t)(L + 1) * sb, off_scr = align_up(off_c + sb, 256),
                off_env = align_up(off_scr + (int64_t)nscr * P.scratch_elems * 16, 256),
                total = off_env + P.env_elems * 16;
  if (!ctx->plain && cudaMalloc(&ctx->plain, (size_t)total) != cudaSuccess) {
    cudaGetLastError();
    return TNRC_E_NOMEM;
  }
  CK(tnrc_plain_prepare());
  unsigned char* hist = ctx->plain + off_hist;
  unsigned char* cslot = ctx->plain + off_c;
  if (ctx->gates_dirty) {
    CK(tnrc_launch_layer_gates(P.N, P.K, P.C, P.M, P.terms, P.order, P.nsub, P.n_layers, P.recs, P.first_parity,
                               ctx->dt, ctx->at<double>(P.off_u), ctx->at<unsigned char>(P.off_mask),
                               ctx->at<double>(P.off_gfix), ctx->at<double>(P.off_J), ctx->at<int>(P.off_loff),
                               ctx->at<tnrc::LayerGate>(P.off_gates), ctx->at<int>(P.off_status), st));
    ctx->gates_dirty = false;
  }
  CK(cudaMemsetAsync(ctx->at<unsigned long long>(P.off_counters), 0, tnrc::kNumCounters * 8, st));
  CK(cudaMemsetAsync(ctx->at<unsigned long long>(P.off_counters) + tnrc::kCtrGap, 0xff, 8, st));
  tnrc::TrajParams tp = traj_params(ctx, true);
  tp.warps = 2;   // the environment launch runs two warps; the others one
  tp.slab_elems = P.slab_elems;   // the batched launch's slab: the same bonds go as pairs
  tp.warp_scratch = reinterpret_cast<double2*>(ctx->plain + off_scr);
  tp.env_scratch = reinterpret_cast<double2*>(ctx->plain + off_env);
  const size_t smem = tnrc_traj_smem(2, tp.slab_elems);
  const unsigned char* in = ctx->at<unsigned char>(P.off_in);
  const unsigned char* tg = ctx->at<unsigned char>(P.off_tg);
  const int64_t KCN = (int64_t)P.K * P.C * P.N;
  CK(cudaEventRecord(ctx->ev0, st));
  Range plain_range("tnrc:plain path");
  for (int t = 0; t < P.T; ++t) {
    const int s = t / P.P, pi = t - s * P.P;
    CK(tnrc_launch_plain(&tp, 0, in + (size_t)pi * sb, hist, 0, 0, 0, 0, st));
    for (int l = 0; l < L; ++l) {
      CK(tnrc_launch_plain(&tp, 0, hist + (size_t)l * sb, hist + (size_t)(l + 1) * sb, 0, 0, 0, 0, st));
      CK(tnrc_launch_plain(&tp, 1, nullptr, hist + (size_t)(l + 1) * sb, s, l, t, smem, st));
    }
    CK(tnrc_launch_plain(&tp, 2, tg + (size_t)pi * sb, hist + (size_t)L * sb, 0, 0, t, smem, st));
    CK(tnrc_launch_plain(&tp, 0, tg + (size_t)pi * sb, cslot, 0, 0, 0, 0, st));
    CK(cudaMemsetAsync(ctx->at<double>(P.off_gsp) + (size_t)t * KCN, 0, (size_t)KCN * 8, st));
    for (int l = L - 1; l >= 0; --l) {
      CK(tnrc_launch_plain(&tp, 3, hist + (size_t)(l + 1) * sb, cslot, s, l, t, smem, st));
      CK(tnrc_launch_plain(&tp, 4, hist + (size_t)(l + 1) * sb, cslot, s, l, t, smem, st));
    }
  }
  const int X = (int)KCN;
  CK(tnrc_launch_reduce(ctx->at<double2>(P.off_O), P.T, ctx->at<double>(P.off_F), nullptr,
                        ctx->at<double>(P.off_gsp), X, ctx->at<double>(P.off_grad), st));
  CK(cudaEventRecord(ctx->ev1, st));
  ctx->timed_last = true;
  tnrc_status r = finish(ctx);
  if (r != TNRC_OK) return r;
  CK(cudaMemcpy(F, ctx->at<double>(P.off_F), 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(grad, ctx->at<double>(P.off_grad), (size_t)KCN * 8, cudaMemcpyDeviceToHost));
  return TNRC_OK;
}

tnrc_status tnrc_set_svd_shape(tnrc_ctx* ctx, int32_t pairs) {
  if (!ctx || (pairs != 0 && pairs != 1)) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  if (ctx->pair_svd != pairs) {
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);   // captured with the other shape
    ctx->graphs.clear();
  }
  ctx->pair_svd = pairs;
  return TNRC_OK;
}

tnrc_status tnrc_set_stream(tnrc_ctx* ctx, void* cuda_stream) {
  if (!ctx) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  if (ctx->use_graphs && cuda_stream == nullptr) return TNRC_E_INVALID;   // the legacy stream cannot be captured
  CK(cudaStreamSynchronize(ctx->stream));   // work already queued stays ordered before the switch
  ctx->stream = (cudaStream_t)cuda_stream;
  return TNRC_OK;
}

tnrc_status tnrc_set_pooled(tnrc_ctx* ctx, int32_t enable) {
  if (!ctx || (enable != 0 && enable != 1)) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  const Plan& P = ctx->plan;
  if (enable && !ctx->pooled) {
    // the pool holds P.grid regions: no more CTAs than that may be resident,
    // so ask for enough dynamic shared memory to keep the occupancy there
    int dev = 0, smem_sm = 0, occ = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const int tp_min_blocks = P.d == 4 ? 1 : P.min_blocks;
    const size_t base = tnrc_traj_smem(P.warps, P.slab_elems);
    const int per_sm_max = std::max(1, P.grid / std::max(1, ctx->n_sm));
    size_t smem = base;
    CK(tnrc_traj_occupancy(P.d, tp_min_blocks, P.warps, smem, &occ));
    if ((long long)occ * ctx->n_sm > P.grid && P.T > P.grid) {
      smem = std::max(base, (size_t)(smem_sm / per_sm_max) - 4096);
      smem = std::min<size_t>(smem, 226 * 1024);
      CK(tnrc_traj_occupancy(P.d, tp_min_blocks, P.warps, smem, &occ));
      if ((long long)occ * ctx->n_sm > P.grid) return TNRC_E_INVALID;
    }
    ctx->pooled_smem = smem;
  }
  if (ctx->pooled != (enable != 0)) {
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);   // captured with the other launch
    ctx->graphs.clear();
  }
  ctx->pooled = enable != 0;
  return TNRC_OK;
}

tnrc_status tnrc_sync(tnrc_ctx* ctx) {
  if (!ctx) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  return finish(ctx);
}

tnrc_status tnrc_get_overlaps(tnrc_ctx* ctx, double* overlaps, int64_t len) {
  if (!ctx || !overlaps) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  const Plan& P = ctx->plan;
  if (len != 2 * (int64_t)P.T) return TNRC_E_INVALID;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaMemcpy(overlaps, ctx->at<void>(P.off_O), (size_t)P.T * 16, cudaMemcpyDeviceToHost));
  return TNRC_OK;
}

tnrc_status tnrc_get_stats(tnrc_ctx* ctx, tnrc_stats* stats) {
  if (!ctx || !stats) return TNRC_E_INVALID;
  if (ctx->broken) return TNRC_E_CUDA;
  const Plan& P = ctx->plan;
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<unsigned long long> c(tnrc::kNumCounters);
  CK(cudaMemcpy(c.data(), ctx->at<void>(P.off_counters), c.size() * 8, cudaMemcpyDeviceToHost));
  std::vector<double> disc(P.T);
  CK(cudaMemcpy(disc.data(), ctx->at<void>(P.off_disc), (size_t)P.T * 8, cudaMemcpyDeviceToHost));
  tnrc_stats s{};
  s.updates = (int64_t)c[0];
  s.jacobi_sweeps = (int64_t)c[1];
  s.max_bond = (int32_t)c[2];
  s.hist_len = P.chi + 1;
  for (int d = 0; d <= P.chi; ++d) s.bond_hist[d] = (int64_t)c[5 + d];
  s.alg_flops = (double)c[3];
  s.restarts = (int64_t)c[4];
  for (int i = 0; i < tnrc::kNumPhases; ++i) s.phase_cycles[i] = (int64_t)c[tnrc::kCtrPhase + i];
  s.cap_truncations = (int64_t)c[tnrc::kCtrCapTrunc];
  {
    const unsigned long long g = c[tnrc::kCtrGap];
    double gv = -1.0;
    if (s.cap_truncations > 0 && g != ~0ull) std::memcpy(&gv, &g, 8);
    s.min_trunc_gap = gv;
  }
  double tms = 0.0;
  for (size_t i = 0; i + 1 < ctx->tev_used; i += 2) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->tev[i], ctx->tev[i + 1]));
    tms += ms;
  }
  s.traj_ms = tms;
  s.traj_launches = (int64_t)(ctx->tev_used / 2);
  ctx->tev_used = 0;
  double dw = 0.0;
  for (double v : disc) dw += v;
  s.discarded_weight = dw;
  s.last_ms = ctx->stats.last_ms;
  *stats = s;
  return TNRC_OK;
}

void tnrc_destroy(tnrc_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->plain) cudaFree(ctx->plain);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  for (auto e : ctx->tev)
    if (e) cudaEventDestroy(e);
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  delete ctx;
}

const char* tnrc_last_error(const tnrc_ctx* ctx) {
  if (!ctx) return "";
  return ctx->err;
}

const char* tnrc_status_string(tnrc_status s) {
  switch (s) {
    case TNRC_OK: return "TNRC_OK";
    case TNRC_E_INVALID: return "TNRC_E_INVALID: invalid argument";
    case TNRC_E_NOMEM: return "TNRC_E_NOMEM: not enough device memory";
    case TNRC_E_CUDA: return "TNRC_E_CUDA: CUDA error (context unusable)";
    case TNRC_E_STATE: return "TNRC_E_STATE: controls or noise not set";
    case TNRC_E_TIMEOUT: return "TNRC_E_TIMEOUT: device wait expired";
    case TNRC_E_NUMERIC: return "TNRC_E_NUMERIC: SVD did not converge or non-finite values";
    case TNRC_E_TOO_LARGE: return "TNRC_E_TOO_LARGE: problem exceeds the 32 MiB static scratch of tnrc_fidelity_static";
    default: return "unknown tnrc status";
  }
}

}  // extern "C"
