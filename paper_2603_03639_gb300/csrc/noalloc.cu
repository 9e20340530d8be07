// Fidelity evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host runtime that
// owns all device allocations (a memory pool that must not be bypassed, a
// sandbox without allocation rights) or a process that must not grow its
// device footprint after start-up.  For them tnrc_fidelity_static runs the
// same kernels as tnrc_create + tnrc_fidelity, but every buffer it needs --
// staged inputs, canonical states, the gate table, the trajectory working
// slots and per-warp scratch, the outputs before they are copied back --
// lives in one fixed static device array, kStaticBytes long, compiled into
// this library.  Every GPU that loads the library holds that array until the
// process exits.
//
// The array is shared by all calls: each call overwrites it and clears the
// parts that must start at zero.  Calls whose device work overlaps (two host
// threads, or two streams, at the same time) race on it; serialise them.
// Every call looks up the array's device address on the current device
// (cudaGetSymbolAddress, checked), so the address stays right after a device
// reset; the call synchronises its stream, so it is never stream-captured.
// With CUDA's lazy module loading (the default) the array is placed on a
// device at the first call there -- that call grows the device footprint by
// kStaticBytes -- or when the library loads, with CUDA_MODULE_LOADING=EAGER;
// callers that must not grow their footprint later make one small call at
// start-up.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/tnrc.h"
#include "plan.h"
#include "tnrc_device.cuh"

extern "C" cudaError_t tnrc_launch_traj(const tnrc::TrajParams* p, int grid, size_t smem, cudaStream_t st);
extern "C" cudaError_t tnrc_traj_prepare();
extern "C" cudaError_t tnrc_launch_layer_gates(int N, int K, int C, int M, int terms, int order, int nsub,
                                               int L, int R, int first_parity, double dt, const double* u,
                                               const unsigned char* mask, const double* gfix, const double* J,
                                               const int* layer_off, tnrc::LayerGate* out, int* status,
                                               cudaStream_t st);
extern "C" cudaError_t tnrc_launch_reduce(const double2* O, int T, double* F, double* per_traj, const double* gsp,
                                          int X, double* grad, cudaStream_t st);
extern "C" cudaError_t tnrc_launch_canon(const tnrc::CanonArgs* a, int nmps, cudaStream_t st);

namespace {

constexpr size_t kStaticBytes = size_t(32) << 20;   // 32 MiB per device
constexpr int kMaxInputDimStatic = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

// Device address of g_static_scratch on the current device.  Host code
// cannot use the array's name as a device address; the runtime maps it.
cudaError_t static_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

int64_t up(int64_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" tnrc_status tnrc_fidelity_static(const tnrc_problem* pb, const tnrc_mps* inputs,
                                            const tnrc_mps* targets, const double* u, const double* J,
                                            void* cuda_stream, double* F, double* per_traj) {
  // ---- validation (host only; the same rules as tnrc_create) ----
  if (!pb || !inputs || !targets || !u || !J || !F || pb->struct_size != sizeof(tnrc_problem))
    return TNRC_E_INVALID;
  tnrc_host::Plan plan;
  if (!tnrc_host::make_plan(pb, 1, 0, plan, false)) return TNRC_E_INVALID;
  if (tnrc_host::check_problem_arrays(pb, inputs, targets) != TNRC_OK) return TNRC_E_INVALID;
  const int N = plan.N, K = plan.K, chi = plan.chi, M = plan.M, P = plan.P, C = plan.C;
  const int terms = plan.terms, order = plan.order, nsub = plan.nsub, d = plan.d;
  const int n_layers = plan.n_layers, first_parity = plan.first_parity, recs = plan.recs;
  const std::vector<int>& layer_off = plan.layer_off;
  const std::vector<int>& dcap = plan.dcap;
  const std::vector<int>& site_off = plan.site_off;
  const tnrc::SlotLayout L = plan.L;
  const long long T = (long long)M * P;
  if (T > (1 << 24)) return TNRC_E_TOO_LARGE;
  int dmax = chi;
  for (int j = 0; j < 2 * P; ++j) {
    const tnrc_mps& m = (j < P) ? inputs[j] : targets[j - P];
    for (int i = 0; i <= N; ++i) {
      if (m.bond_dims[i] > kMaxInputDimStatic) return TNRC_E_TOO_LARGE;
      dmax = std::max(dmax, m.bond_dims[i]);
    }
  }
  const int64_t KCN = (int64_t)K * C * N;
  for (int64_t i = 0; i < KCN; ++i)
    if (!std::isfinite(u[i])) return TNRC_E_INVALID;
  for (int64_t i = 0; i < (int64_t)M * (N - 1) * terms; ++i)
    if (!std::isfinite(J[i])) return TNRC_E_INVALID;

  // ---- static scratch map ----
  std::vector<int> rdims((size_t)2 * P * (N + 1));
  std::vector<long long> roffs(2 * P);
  long long rtotal = 0;
  for (int j = 0; j < 2 * P; ++j) {
    const tnrc_mps& m = (j < P) ? inputs[j] : targets[j - P];
    roffs[j] = rtotal;
    for (int i = 0; i <= N; ++i) rdims[(size_t)j * (N + 1) + i] = m.bond_dims[i];
    for (int i = 0; i < N; ++i) rtotal += (long long)m.bond_dims[i] * d * m.bond_dims[i + 1];
  }
  const long long cwork = (long long)(N + 4) * d * dmax * dmax;
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    const int64_t o = off;
    off = up(off + std::max<int64_t>(bytes, 1));
    return o;
  };
  const int64_t o_mask = take((int64_t)C * N), o_gfix = take((int64_t)K * (N - 1) * 8), o_u = take(KCN * 8),
                o_J = take((int64_t)M * (N - 1) * terms * 8), o_site = take((int64_t)N * 4),
                o_dcap = take((int64_t)(N + 1) * 4),
                o_rdims = take((int64_t)rdims.size() * 4), o_roffs = take((int64_t)roffs.size() * 8),
                o_raw = take(rtotal * 16), o_cwork = take((int64_t)2 * P * cwork * 16),
                o_slots = take((int64_t)2 * P * L.bytes),
                o_gates = take((int64_t)M * recs * (int64_t)sizeof(tnrc::LayerGate)),
                o_loff = take((int64_t)(n_layers + 1) * 4), o_O = take(T * 16),
                o_disc = take(T * 8), o_per = take(T * 8), o_small = take(4096);
  int maxb = 0;
  for (int par = 0; par < 2; ++par) maxb = std::max(maxb, (N - 1 - par + 1) / 2);
  const int warps = std::max(2, std::min(tnrc::kWarps, maxb));
  const int slab = std::min(1024, d * d * chi * chi);
  const int64_t cc = (int64_t)chi * chi;
  const int64_t scratch_elems = (4 * (int64_t)d * d + d) * cc;   // the same per-warp layout as tnrc_create
  const int64_t env_elems = 2 * (int64_t)(N + 1) * cc;
  const int64_t per_cta = up(L.bytes) + up(warps * scratch_elems * 16) + up(env_elems * 16);
  if (off + per_cta > (int64_t)kStaticBytes) return TNRC_E_TOO_LARGE;
  int dev = 0, n_sm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TNRC_E_CUDA;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>({T, (int64_t)n_sm, ((int64_t)kStaticBytes - off) / per_cta}));
  const int64_t o_work = take((int64_t)grid * L.bytes), o_wscr = take((int64_t)grid * warps * scratch_elems * 16),
                o_env = take((int64_t)grid * env_elems * 16);
  if (off > (int64_t)kStaticBytes) return TNRC_E_TOO_LARGE;

  void* base_v = nullptr;
  if (static_scratch(&base_v) != cudaSuccess) return TNRC_E_CUDA;
  unsigned char* base = static_cast<unsigned char*>(base_v);
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // ---- stage inputs ----
  const std::vector<unsigned char> mask = tnrc_host::control_mask(pb);
  std::vector<double> gfix((size_t)K * (N - 1), 0.0);
  if (pb->g_fixed) std::memcpy(gfix.data(), pb->g_fixed, gfix.size() * 8);
  std::vector<double> raw((size_t)rtotal * 2);
  for (int j = 0; j < 2 * P; ++j) {
    const tnrc_mps& m = (j < P) ? inputs[j] : targets[j - P];
    long long cnt = 0;
    for (int i = 0; i < N; ++i) cnt += (long long)m.bond_dims[i] * d * m.bond_dims[i + 1];
    for (long long e = 0; e < 2 * cnt; ++e)
      if (!std::isfinite(m.data[e])) return TNRC_E_INVALID;
    std::memcpy(raw.data() + roffs[j] * 2, m.data, (size_t)cnt * 16);
  }
  bool ok = cudaMemcpyAsync(base + o_mask, mask.data(), mask.size(), cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(base + o_gfix, gfix.data(), gfix.size() * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(base + o_u, u, KCN * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(base + o_J, J, (size_t)M * (N - 1) * terms * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(base + o_site, site_off.data(), (size_t)N * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(base + o_dcap, dcap.data(), (size_t)(N + 1) * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(base + o_loff, layer_off.data(), layer_off.size() * 4, cudaMemcpyHostToDevice, st) ==
                cudaSuccess &&
            cudaMemcpyAsync(base + o_rdims, rdims.data(), rdims.size() * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(base + o_roffs, roffs.data(), roffs.size() * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(base + o_raw, raw.data(), raw.size() * 8, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            // the array keeps the previous call's contents: clear what must start at zero
            cudaMemsetAsync(base + o_slots, 0, (size_t)2 * P * L.bytes, st) == cudaSuccess &&
            cudaMemsetAsync(base + o_small, 0, 4096, st) == cudaSuccess;
  if (!ok) return TNRC_E_CUDA;
  int* status = reinterpret_cast<int*>(base + o_small);
  int* work_counter = reinterpret_cast<int*>(base + o_small + 256);
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(base + o_small + 512);
  double* dF = reinterpret_cast<double*>(base + o_small + 1536);
  const double eps = std::max(pb->sv_cutoff, tnrc::kZeroFloor);

  // ---- canonical inputs and targets ----
  tnrc::CanonArgs ca{};
  ca.N = N;
  ca.chi = chi;
  ca.eps = eps;
  ca.dmax = dmax;
  ca.d = d;
  ca.raw_dims = reinterpret_cast<const int*>(base + o_rdims);
  ca.raw_data = reinterpret_cast<const double2*>(base + o_raw);
  ca.raw_off = reinterpret_cast<const long long*>(base + o_roffs);
  ca.work = reinterpret_cast<double2*>(base + o_cwork);
  ca.work_stride = cwork;
  ca.slots = base + o_slots;
  ca.L = L;
  ca.site_off = reinterpret_cast<const int*>(base + o_site);
  ca.status = status;
  if (tnrc_launch_canon(&ca, 2 * P, st) != cudaSuccess) return TNRC_E_CUDA;
  // ---- gates ----
  if (tnrc_launch_layer_gates(N, K, C, M, terms, order, nsub, n_layers, recs, first_parity, pb->dt,
                              reinterpret_cast<const double*>(base + o_u), base + o_mask,
                              reinterpret_cast<const double*>(base + o_gfix),
                              reinterpret_cast<const double*>(base + o_J), reinterpret_cast<const int*>(base + o_loff),
                              reinterpret_cast<tnrc::LayerGate*>(base + o_gates), status, st) != cudaSuccess)
    return TNRC_E_CUDA;
  // ---- trajectories (forward and overlap only) ----
  tnrc::TrajParams tp{};
  tp.N = N;
  tp.K = K;
  tp.C = C;
  tp.P = P;
  tp.M = M;
  tp.chi = chi;
  tp.T = (int)T;
  tp.dt = pb->dt;
  tp.eps = eps;
  tp.want_grad = 0;
  tp.warps = warps;
  tp.slab_elems = slab;
  tp.min_blocks = 1;
  tp.phys_dim = d;
  tp.full.L = L;
  tp.full.site_off = reinterpret_cast<const int*>(base + o_site);
  tp.full.dcap = reinterpret_cast<const int*>(base + o_dcap);
  tp.full.seg = n_layers;
  tp.full.nseg = 1;
  tp.packed_history = 0;
  tp.history_cap = 0;
  tp.in_slots = base + o_slots;
  tp.tg_slots = base + o_slots + (size_t)P * L.bytes;
  tp.work = base + o_work;
  tp.work_stride = L.bytes;
  tp.warp_scratch = reinterpret_cast<double2*>(base + o_wscr);
  tp.scratch_elems = scratch_elems;
  tp.env_scratch = reinterpret_cast<double2*>(base + o_env);
  tp.lgates = reinterpret_cast<const tnrc::LayerGate*>(base + o_gates);
  tp.layer_off = reinterpret_cast<const int*>(base + o_loff);
  tp.n_layers = n_layers;
  tp.first_parity = first_parity;
  tp.recs_per_sample = recs;
  tp.mask = base + o_mask;
  tp.O = reinterpret_cast<double2*>(base + o_O);
  tp.gsp = nullptr;
  tp.disc = reinterpret_cast<double*>(base + o_disc);
  tp.counters = counters;
  tp.status = status;
  tp.work_counter = work_counter;
  if (tnrc_traj_prepare() != cudaSuccess) return TNRC_E_CUDA;
  if (tnrc_launch_traj(&tp, grid, tnrc_traj_smem(warps, slab), st) != cudaSuccess) return TNRC_E_CUDA;
  if (tnrc_launch_reduce(tp.O, (int)T, dF, per_traj ? reinterpret_cast<double*>(base + o_per) : nullptr, nullptr, 0,
                         nullptr, st) != cudaSuccess)
    return TNRC_E_CUDA;
  // ---- results ----
  int hstatus = 0;
  double hF = 0.0;
  if (cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&hF, dF, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TNRC_E_CUDA;
  std::vector<double> hper(per_traj ? (size_t)T : 0);
  if (per_traj && cudaMemcpyAsync(hper.data(), base + o_per, (size_t)T * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TNRC_E_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TNRC_E_CUDA;
  if (hstatus) return TNRC_E_NUMERIC;
  *F = hF;
  if (per_traj) std::memcpy(per_traj, hper.data(), (size_t)T * 8);
  return TNRC_OK;
}
