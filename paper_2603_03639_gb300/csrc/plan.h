// Host-side problem plan of the tnrc library, shared by the allocating
// entry points (api.cu) and the allocation-free one (noalloc.cu): validation
// of a tnrc_problem, the slot layout of an MPS, the truncated-layer schedule
// and the device arena map of a context.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/tnrc.h"
#include "tnrc_device.cuh"

extern "C" size_t tnrc_traj_smem(int warps, int slab_elems);

namespace tnrc_host {

constexpr int kMaxN = 256;
constexpr int kMaxInputDim = 128;

inline int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Capacities min(d^i, d^(N-i), cap), site offsets and byte layout of a slot
// (physical dimension d = 2 for states, 4 for operators).
struct Layout {
  std::vector<int> dcap;      // [N+1] capacity of D[i]
  std::vector<int> site_off;  // [N]
  tnrc::SlotLayout L;
  int seg = 1, nseg = 1;
};

inline Layout make_layout(int N, int cap, int d) {
  Layout Y;
  Y.dcap.assign(N + 1, 1);
  const int lg = d == 4 ? 2 : 1;   // log2 d
  for (int i = 1; i < N; ++i) {
    const int a = i * lg >= 30 ? cap : std::min(1 << (i * lg), cap);
    const int b = (N - i) * lg >= 30 ? cap : std::min(1 << ((N - i) * lg), cap);
    Y.dcap[i] = std::min(a, b);
  }
  Y.site_off.resize(N);
  int64_t elems = 0;
  for (int i = 0; i < N; ++i) {
    Y.site_off[i] = (int)elems;
    elems += (int64_t)Y.dcap[i] * d * Y.dcap[i + 1];
    elems = align_up(elems, 2);
  }
  Y.L.N = N;
  Y.L.chi = cap;
  Y.L.lam_off = align_up((int64_t)(N + 1) * 4, 16);
  Y.L.sites_off = align_up(Y.L.lam_off + (int64_t)(N - 1) * cap * 8, 256);
  Y.L.bytes = align_up(Y.L.sites_off + elems * 16, 256);
  return Y;
}

struct Plan {
  int N, K, C, chi, M, P, T, terms;
  int order, nsub;            // Trotter order (1 or 2), Trotter steps per control bin
  int d;                      // physical dimension: 2 (states) or 4 (operators)
  int n_layers, first_parity, recs;   // truncated layers, parity of layer 0, layer-gate records per sample
  std::vector<int> layer_off; // [n_layers + 1] first record of each layer within a sample
  int seg, nseg;
  int warps, slab_elems, min_blocks;
  int grid;
  std::vector<int> dcap;      // [N+1] capacity of D[i]
  std::vector<int> site_off;  // [N]
  tnrc::SlotLayout L;
  int64_t scratch_elems;      // per warp
  int64_t work_stride;        // bytes per CTA
  int64_t env_elems;          // per CTA
  // arena offsets (bytes)
  int64_t off_loff;
  int64_t off_u, off_mask, off_gfix, off_J, off_gates, off_in, off_tg, off_work, off_scratch, off_env, off_O,
      off_gsp, off_disc, off_counters, off_status, off_wc, off_F, off_grad, off_per, off_siteoff, off_dcap,
      off_owner, total;
};

inline bool make_plan(const tnrc_problem* pb, int n_sm, size_t free_bytes, Plan& P, bool limit_by_memory) {
  if (!pb || pb->struct_size != sizeof(tnrc_problem)) return false;
  const int N = pb->n_sites, K = pb->n_slices, chi = pb->chi_max;
  if (N < 2 || N > kMaxN || K < 1 || chi < 1 || chi > tnrc::kMaxChi) return false;
  if (!(pb->dt > 0.0) || !std::isfinite(pb->dt) || !(pb->sv_cutoff >= 0.0) || !(pb->sv_cutoff < 1.0)) return false;
  if (pb->n_samples < 1 || pb->n_inputs < 1 || (pb->n_controls != 2 && pb->n_controls != 3)) return false;
  if (pb->checkpoint_every < 0) return false;
  if (pb->crosstalk_terms != 0 && pb->crosstalk_terms != 1 && pb->crosstalk_terms != 3) return false;
  const long long T = (long long)pb->n_samples * pb->n_inputs;
  if (T > (1ll << 30)) return false;
  P.N = N;
  P.K = K;
  P.C = pb->n_controls;
  P.chi = chi;
  P.M = pb->n_samples;
  P.P = pb->n_inputs;
  P.T = (int)T;
  P.terms = pb->crosstalk_terms == 3 ? 3 : 1;
  if (pb->trotter_order < 0 || pb->trotter_order > 2 || pb->substeps < 0) return false;
  P.order = pb->trotter_order == 1 ? 1 : 2;
  if (pb->operator_form != 0 && pb->operator_form != 1) return false;
  P.d = pb->operator_form ? 4 : 2;
  if (P.d * chi > tnrc::kMaxDim) return false;   // theta sides d chi must fit the per-warp arrays
  P.nsub = pb->substeps > 0 ? pb->substeps : 1;
  if ((long long)K * P.nsub > (1 << 20)) return false;
  // truncated layers: 2S+1 (second order; A half steps merged at step
  // boundaries) or 2S (first order), S = K n_sub Trotter steps; parities alternate
  const int S = K * P.nsub;
  P.n_layers = (P.order == 2) ? 2 * S + 1 : 2 * S;
  P.first_parity = (P.order == 2) ? 0 : 1;
  P.layer_off.assign(P.n_layers + 1, 0);
  for (int l = 0; l < P.n_layers; ++l) {
    const int par = (l + P.first_parity) & 1;
    P.layer_off[l + 1] = P.layer_off[l] + (N - 1 - par + 1) / 2;
  }
  P.recs = P.layer_off[P.n_layers];
  // checkpoint segments in truncated layers
  const int L = P.n_layers;
  P.seg = pb->checkpoint_every > 0 ? (int)std::min<long long>(2ll * P.nsub * pb->checkpoint_every, L)
                                   : (int)std::ceil(std::sqrt((double)L));
  P.nseg = (L + P.seg - 1) / P.seg;
  {
    Layout Y = make_layout(N, chi, P.d);
    P.dcap = Y.dcap;
    P.site_off = Y.site_off;
    P.L = Y.L;
  }
  int maxb = 0;
  for (int par = 0; par < 2; ++par) maxb = std::max(maxb, (N - 1 - par + 1) / 2);
  P.warps = std::max(2, std::min(tnrc::kWarps, maxb));
  if (pb->warps_per_cta < 0 || pb->warps_per_cta == 1 || pb->warps_per_cta > tnrc::kWarps) return false;
  if (pb->ctas_per_sm < 0 || pb->ctas_per_sm > 4) return false;
  if (pb->warps_per_cta > 0) P.warps = pb->warps_per_cta;
  if (const char* e = getenv("TNRC_WARPS")) {
    const int w = atoi(e);
    if (w >= 2 && w <= tnrc::kWarps) P.warps = w;
  }
  // the register file holds 8 warps of the 255-register build per SM and 16 of
  // the 128-register build; more than 8 warps per SM select the latter
  const int ctas_per_sm =
      std::max(1, std::min(pb->ctas_per_sm > 0 ? pb->ctas_per_sm : 1, (P.d == 4 ? 1 : 2) * tnrc::kWarps / P.warps));
  P.min_blocks = (P.warps * ctas_per_sm > tnrc::kWarps) ? 2 : 1;
  // each warp's shared slab holds theta^dagger up to slab_elems complex values
  // (wider thetas use global scratch): split what the resident CTAs of an SM
  // leave after the per-warp arrays, within the 227 KB a CTA may use
  {
    const int per_sm = 220 * 1024 / ctas_per_sm;
    const int small = (int)tnrc_traj_smem(P.warps, 0) + 1024;
    const int per_warp = std::max(0, per_sm - small) / P.warps / 16;
    P.slab_elems = std::max(256, std::min(P.d * P.d * chi * chi, per_warp / 32 * 32));
  }
  const int64_t cc = (int64_t)chi * chi;
  // per warp: Phi (d chi)^2, theta (d chi)^2, then the gradient's three
  // intermediates (at most (d + 2 d^2) chi^2) past 2 (d chi)^2
  P.scratch_elems = (4 * (int64_t)P.d * P.d + P.d) * cc;
  P.env_elems = 2 * (int64_t)(N + 1) * cc;
  P.work_stride = (int64_t)(2 + P.nseg + P.seg) * P.L.bytes;
  const int64_t per_cta = P.work_stride + (P.scratch_elems * P.warps + P.env_elems) * 16;
  int grid = (int)std::min<long long>(T, (long long)n_sm * ctas_per_sm);
  if (const char* e = getenv("TNRC_GRID")) {
    const int g = atoi(e);
    if (g >= 1) grid = (int)std::min<long long>(T, g);
  }
  // fixed parts
  int64_t off = 0;
  auto take = [&](int64_t bytes) {
    const int64_t o = off;
    off = align_up(off + std::max<int64_t>(bytes, 1), 256);
    return o;
  };
  const int64_t KCN = (int64_t)K * P.C * N;
  P.off_u = take(KCN * 8);
  P.off_mask = take((int64_t)P.C * N);
  P.off_gfix = take((int64_t)K * (N - 1) * 8);
  P.off_J = take((int64_t)P.M * (N - 1) * P.terms * 8);
  P.off_gates = take((int64_t)P.M * P.recs * (int64_t)sizeof(tnrc::LayerGate));
  P.off_loff = take((int64_t)(P.n_layers + 1) * 4);
  P.off_in = take((int64_t)P.P * P.L.bytes);
  P.off_tg = take((int64_t)P.P * P.L.bytes);
  P.off_O = take(T * 16);
  P.off_gsp = take(T * KCN * 8);
  P.off_disc = take(T * 8);
  P.off_counters = take(tnrc::kNumCounters * 8);
  P.off_status = take(16);
  P.off_wc = take(16);
  P.off_F = take(8);
  P.off_grad = take(KCN * 8);
  P.off_per = take(T * 8);
  P.off_siteoff = take((int64_t)N * 4);
  P.off_dcap = take((int64_t)(N + 1) * 4);

  const int64_t fixed = off;
  if (limit_by_memory && free_bytes > 0) {
    const int64_t budget = (int64_t)(free_bytes * 0.85) - fixed;
    if (budget < per_cta) return false;
    grid = (int)std::min<int64_t>(grid, budget / per_cta);
  }
  P.grid = std::max(1, grid);
  P.off_work = take((int64_t)P.grid * P.work_stride);
  P.off_scratch = take((int64_t)P.grid * P.warps * P.scratch_elems * 16);
  P.off_env = take((int64_t)P.grid * P.env_elems * 16);
  P.off_owner = take((int64_t)P.grid * 4);   // region pool of the pooled launch
  P.total = off;
  return true;
}

inline bool valid_mps(const tnrc_mps& m, int N) {  // the data size follows from bond_dims and d
  if (m.n_sites != N || !m.bond_dims || !m.data) return false;
  if (m.bond_dims[0] != 1 || m.bond_dims[N] != 1) return false;
  for (int i = 0; i <= N; ++i)
    if (m.bond_dims[i] < 1 || m.bond_dims[i] > kMaxInputDim) return false;
  return true;
}


// Checks of a problem's host arrays beyond make_plan: every input and target
// MPS well formed, mask entries 0 or 1, g_fixed finite.  Returns TNRC_OK or
// TNRC_E_INVALID.
inline tnrc_status check_problem_arrays(const tnrc_problem* pb, const tnrc_mps* inputs, const tnrc_mps* targets) {
  const int N = pb->n_sites;
  for (int p = 0; p < pb->n_inputs; ++p)
    if (!valid_mps(inputs[p], N) || !valid_mps(targets[p], N)) return TNRC_E_INVALID;
  if (pb->control_mask) {
    for (int c = 0; c < pb->n_controls; ++c)
      for (int i = 0; i < N; ++i)
        if (pb->control_mask[c * N + i] > 1) return TNRC_E_INVALID;
  }
  if (pb->g_fixed) {
    for (int64_t i = 0; i < (int64_t)pb->n_slices * (N - 1); ++i)
      if (!std::isfinite(pb->g_fixed[i])) return TNRC_E_INVALID;
  }
  return TNRC_OK;
}

// The control mask the kernels read: [C][N] bytes, the caller's or the
// default (every x, y; for C = 3 every bond's g), with the g slot of the last
// site (which has no bond) always off.
inline std::vector<unsigned char> control_mask(const tnrc_problem* pb) {
  const int N = pb->n_sites, C = pb->n_controls;
  std::vector<unsigned char> mask((size_t)C * N, 1);
  if (pb->control_mask) {
    std::memcpy(mask.data(), pb->control_mask, mask.size());
  } else if (C == 3) {
    for (int i = 0; i < N; ++i) mask[2 * N + i] = (i < N - 1) ? 1 : 0;
  }
  if (C == 3) mask[2 * N + N - 1] = 0;
  return mask;
}

}  // namespace tnrc_host
