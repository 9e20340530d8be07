// Persistent trajectory kernel: one CTA evaluates one trajectory (noise sample
// s, input p) at a time and takes the next one from a device work counter.
//
//   forward  (Sec. II): the truncated layers of the time discretisation, each
//            a set of disjoint two-site gates with their parity alternating --
//            for the second-order split A(dt/2) B(dt) A(dt/2) per Trotter step
//            the 2S+1 layers A_0, B_0, A_0A_1, B_1, ..., B_{S-1}, A_{S-1} (half
//            layers at a step boundary merged into one gate: the state is
//            compressed once per time step), for the first-order slice of
//            Eq. circuit two layers per step (odd bonds; even bonds with the
//            single-site rotations folded in).  Every two-site gate is
//            followed by the truncated SVD; the warps of the CTA share the
//            disjoint bonds of a layer, largest first.
//   overlap  (Sec. II state form): O = <t_p | a(T)> by a transfer-matrix sweep.
//   gradient (App. A): the costate b_l = L_{l+1}^dag .. L_L^dag t is propagated
//            backwards with the same truncated update; for every gate of layer
//            l, dO/du += tr(Q_u rho) with rho the mixed two-site density of
//            <b_l|.|a_l> from left/right environments and Q_u from the layer
//            gate table; the forward states a_l come from the packed history
//            of the forward pass (or are recomputed segment by segment from
//            checkpoints when the history does not fit).
// Each trajectory writes its own O and its own gradient row, so results do not
// depend on which CTA ran it or on what else ran in the launch.
#include "svd_warp.cuh"

namespace tnrc {

// device counters: [0] updates [1] Jacobi sweeps [2] max bond [3] algorithmic
// FP64 flops [4] trajectories whose packed history did not fit and that were
// redone with checkpoints [5 + d] forward updates that left bond dimension d
constexpr int kCtrHist = 5;

struct WarpCtx {
  double2* slab;       // shared, slab_elems
  double2* scratch;    // global, scratch_elems
  double* sig2;        // shared, kMaxDim
  double* qn;          // shared, kMaxDim (column norms of the pivoted QR)
  int* perm;           // shared, kMaxDim
  int* piv;            // shared, kMaxDim (column pivots of the QR)
  double2* small;      // shared, 64 complex (four 4x4 matrices)
  int lane;
  long long sweeps;
  long long updates;
  double disc;
  int maxk;
  unsigned long long alg;   // algorithmic flops counted by lane 0
  long long capcuts;        // cuts decided by the cap chi (forward and costate updates)
  long long ph[kNumPhases]; // phase cycles (TNRC_PHASE_TIMERS builds)
  int* order;               // shared, CTA-wide: bonds of the current layer by decreasing cost
  int* next;                // shared, CTA-wide: next entry of `order` to take
  int region;               // the CTA's work region (scratch, environments, slots)
};

// Algorithmic flops of one two-site update with theta of m x n (m = 2 Dl,
// n = 2 Dr), inner bond Dc and k kept values: contraction 8 m Dc n, gate
// 128 Dl Dr, thin SVD 4 (14 a b^2 + 8 b^3) (a = max(m, n), b = min(m, n);
// Golub-Van Loan count, x4 for complex), split 8 m n k.
__device__ __forceinline__ unsigned long long update_flops(int m, int n, int Dc, int k) {
  const unsigned long long a = m > n ? m : n, b = m > n ? n : m;
  return 8ull * m * Dc * n + 32ull * m * n + 4ull * (14ull * a * b * b + 8ull * b * b * b) + 8ull * m * n * k;
}

// Bonds of truncated layer l have parity (l + first_parity) & 1; the record of
// bond b in layer l of sample s is layer_off[l] + b / 2 within the sample.
__device__ __forceinline__ int layer_parity(const TrajParams& p, int l) { return (l + p.first_parity) & 1; }

__device__ __forceinline__ const LayerGate& layer_rec(const TrajParams& p, int s, int l, int b) {
  return p.lgates[(size_t)s * p.recs_per_sample + p.layer_off[l] + (b >> 1)];
}

// Where the two-site update of a theta with n_theta elements keeps theta:
// the warp's shared slab when it fits, else its global scratch past Phi's
// room.
__device__ __forceinline__ double2* theta_home(const TrajParams& p, int kDD, int n_theta, WarpCtx& w) {
  return (n_theta <= p.slab_elems) ? w.slab : (w.scratch + (size_t)kDD * p.chi * p.chi);
}

// ---------------------------------------------------------------------------
// Physical dimension kD: 2 for qubit states; 4 for operators written as
// vectors (site index s = 2 out + in, the MPO of Sec. II), where the 4x4 gate
// acts on the two out indices and leaves the in indices alone.  With
// kI = kD / 2, s = o kI + i.
// ---------------------------------------------------------------------------
// Two-site update of bond b: theta = lam_{b-1} G (B_b B_{b+1}), truncated SVD,
// B_{b+1} <- Y_k^dag, B_b <- Phi Y_k / |S_k|, lam_b <- S_k / |S_k|.
// The SVD: theta P = Q R by pivoted QR (Q not formed; R has r rows, r the
// numerical rank), then one-sided Jacobi on the r columns of R^dagger:
// R^dagger V = Z S, so theta = (Q V) S (P Z)^dagger and Y = P Z.
// ---------------------------------------------------------------------------
// Per-matrix work arrays of the SVD (shared, per warp): squared singular
// values, column norms (later 1 / sigma), rank order, QR column pivots.
struct SvdBufs {
  double* sig2;
  double* qn;
  int* perm;
  int* piv;
};

// Phase 1 of a two-site update of bond b: Phi = G (B_b B_{b+1}) and theta =
// lam_{b-1} Phi, both row-major: row (al s1), column (s2 ga).  With `pre` the
// product B_b B_{b+1} is given ([Dl][kD^2][Dr], the layout of theta itself,
// so pre may be T: each item reads and writes only its own kD^2 entries).
// Returns |theta|_F^2 (the same in every lane).
template <int kD>
__device__ double theta_build(const TrajParams& p, const Lay& Y, unsigned char* slot, int b, const double2* G,
                              bool adjoint, WarpCtx& w, double2* T, double2* Phi, const double2* pre) {
  constexpr int kI = kD / 2;
  const int lane = w.lane;
  const int lstride = Y.L.chi;
  const int* D = slot_dims(slot);
  const int Dl = D[b], Dc = D[b + 1], Dr = D[b + 2];
  const int n = kD * Dr;
  const double2* sites = slot_sites(slot, Y.L);
  const double* lam = slot_lam(slot, Y.L);
  const double2* A = sites + Y.site_off[b];
  const double2* Bt = sites + Y.site_off[b + 1];

  double2 g[16];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) g[r * 4 + c] = adjoint ? cconj(G[c * 4 + r]) : G[r * 4 + c];

  double fro = 0.0;
  for (int it = lane; it < Dl * Dr; it += 32) {
    const int al = it / Dr, ga = it - al * Dr;
    double2 acc[kD * kD];   // (B_b B_{b+1})[al][s1][s2][ga] at s1 kD + s2
    if (pre) {
#pragma unroll
      for (int q = 0; q < kD * kD; ++q) acc[q] = pre[((size_t)al * kD * kD + q) * Dr + ga];
    } else {
#pragma unroll
      for (int q = 0; q < kD * kD; ++q) acc[q] = make_double2(0.0, 0.0);
      const double2* ap = A + (size_t)(al * kD) * Dc;
      for (int be = 0; be < Dc; ++be) {
        double2 av[kD], bv[kD];
#pragma unroll
        for (int q = 0; q < kD; ++q) {
          av[q] = ap[(size_t)q * Dc + be];
          bv[q] = Bt[(size_t)(be * kD + q) * Dr + ga];
        }
#pragma unroll
        for (int q1 = 0; q1 < kD; ++q1)
#pragma unroll
          for (int q2 = 0; q2 < kD; ++q2) cfma(acc[q1 * kD + q2], av[q1], bv[q2]);
      }
    }
    const double ll = (b > 0) ? lam[(size_t)(b - 1) * lstride + al] : 1.0;
#pragma unroll
    for (int s1 = 0; s1 < kD; ++s1)
#pragma unroll
      for (int s2 = 0; s2 < kD; ++s2) {
        const int o1 = s1 / kI, i1 = s1 % kI, o2 = s2 / kI, i2 = s2 % kI;
        const int row = o1 * 2 + o2;
        double2 v = make_double2(0.0, 0.0);
#pragma unroll
        for (int p1 = 0; p1 < 2; ++p1)
#pragma unroll
          for (int p2 = 0; p2 < 2; ++p2)
            cfma(v, g[row * 4 + p1 * 2 + p2], acc[(p1 * kI + i1) * kD + p2 * kI + i2]);
        const size_t idx = (size_t)(al * kD + s1) * n + s2 * Dr + ga;
        Phi[idx] = v;
        const double2 th = cscale(v, ll);
        T[idx] = th;
        fro += cabs2(th);
      }
  }
  fro = warp_sum(fro);
  __syncwarp();
  return fro;
}

// The split after the second QR: Z = Q2 Z2 (T holds Q2, n x r; Z2 the
// rotated columns of R2, r x r) formed while B_{b+1} = Y_k^dag is written,
// then B_b = Phi Y_k / |S_k| from B_{b+1} (Y[piv[c]][i] = conj(B_{b+1}[i][
// piv[c]])).  Out of line: the common path of theta_finish stays as it is.
static __device__ __noinline__ void split_q2(const double2* T, const double2* Z2, const double2* Phi, double2* Bt,
                                      double2* A, const int* perm, const int* piv, const double* isig, int m,
                                      int n, int r, int k, double inv_kn, int lane) {
  for (int it = lane; it < k * n; it += 32) {
    const int i = it / n, c = it - i * n;
    const double2* z2 = Z2 + (size_t)perm[i] * r;
    double2 z = make_double2(0.0, 0.0);
    for (int l = 0; l < r; ++l) cfma(z, T[(size_t)l * n + c], z2[l]);
    Bt[(size_t)i * n + piv[c]] = cscale(cconj(z), isig[i]);
  }
  __syncwarp();
  for (int it = lane; it < m * k; it += 32) {
    const int row = it / k, i = it - row * k;
    const double2* ph = Phi + (size_t)row * n;
    const double2* bt = Bt + (size_t)i * n;
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < n; ++c) cfmac(acc, bt[c], ph[c]);
    A[it] = cscale(acc, inv_kn);
  }
  __syncwarp();
}

// Phases 3 and 4 of a two-site update of bond b, after the SVD left R^dagger
// V = Z S in T (r columns of length n; QR pivots in bf.piv): rank and
// truncate, then lam_b <- S_k / |S_k|, B_{b+1} <- Y_k^dag, B_b <- Phi Y_k /
// |S_k|, where Y[piv[c]][i] = Z[c][i] = T[perm[i] n + c] / sigma_i.  After
// the second QR (Z2 given) T holds Q2 (n x r) and Z2 (r x r) the rotated
// columns of R2, so that Z[c][i] = sum_l T[l n + c] Z2[perm[i] r + l] /
// sigma_i.
template <int kD>
__device__ void theta_finish(const TrajParams& p, const Lay& Y, unsigned char* slot, int b, double2* T,
                             const double2* Phi, int r, int sw, bool record, bool count, WarpCtx& w, SvdBufs bf,
                             const double2* Z2 = nullptr) {
  const int lane = w.lane;
  const int lstride = Y.L.chi;
  int* D = slot_dims(slot);
  const int Dl = D[b], Dc = D[b + 1], Dr = D[b + 2];
  const int m = kD * Dl, n = kD * Dr;
  double2* sites = slot_sites(slot, Y.L);
  double* lam = slot_lam(slot, Y.L);
  double2* A = sites + Y.site_off[b];
  double2* Bt = sites + Y.site_off[b + 1];

  TNRC_TIC(t_r);
  double kept2, tot2, gap;
  int k = warp_rank_truncate(Z2 ? Z2 : T, Z2 ? r : n, r, p.chi, p.eps, bf.sig2, bf.perm, lane, kept2, tot2, gap);
  if (k > Y.dcap[b + 1]) {  // cannot happen (k <= min(m, n, chi)); keeps memory in bounds regardless
    k = Y.dcap[b + 1];
    if (lane == 0) atomicOr(p.status, kStatusBadDims);
  }
  if (lane == 0) {
    if (sw < 0) atomicOr(p.status, kStatusNoConverge);
    if (!(tot2 >= 0.0) || !(tot2 < 1e300) || !(kept2 > 0.0)) atomicOr(p.status, kStatusNaN);
  }
  w.sweeps += (sw < 0) ? -sw : sw;
  w.updates += 1;
  if (record) {
    w.disc += fmax(0.0, tot2 - kept2) / tot2;   // rounding can make tot2 - kept2 slightly negative
    if (k > w.maxk) w.maxk = k;
    if (lane == 0) atomicAdd(&p.counters[kCtrHist + k], 1ull);
  }
  if (count) {
    w.alg += update_flops(m, n, Dc, k);
    if (gap >= 0.0) {   // the cap chi_max decided this cut
      w.capcuts += 1;
      if (lane == 0) atomicMin(&p.counters[kCtrGap], (unsigned long long)__double_as_longlong(gap));
    }
  }
  const double inv_kn = rsqrt(kept2);
  TNRC_TOC(w, 2, t_r);

  // 1 / sigma once per kept value, in qn, which the Jacobi no longer needs
  TNRC_TIC(t_w);
  double* lamw = lam + (size_t)b * lstride;
  const int* piv = bf.piv;
  double* isig = bf.qn;
  for (int i = lane; i < k; i += 32) {
    lamw[i] = sqrt(bf.sig2[bf.perm[i]]) * inv_kn;
    isig[i] = rsqrt(bf.sig2[bf.perm[i]]);
  }
  __syncwarp();
  if (Z2) {
    split_q2(T, Z2, Phi, Bt, A, bf.perm, piv, isig, m, n, r, k, inv_kn, lane);
    if (lane == 0) D[b + 1] = k;
    __syncwarp();
    TNRC_TOC(w, 3, t_w);
    return;
  }
  for (int it = lane; it < k * n; it += 32) {
    const int i = it / n, c = it - i * n;
    const int j = bf.perm[i];
    Bt[(size_t)i * n + piv[c]] = cscale(cconj(T[(size_t)j * n + c]), isig[i]);
  }
  for (int it = lane; it < m * k; it += 32) {
    const int row = it / k, i = it - row * k;
    const int j = bf.perm[i];
    const double2* ph = Phi + (size_t)row * n;
    const double2* z = T + (size_t)j * n;
    double2 acc = make_double2(0.0, 0.0);
    for (int c = 0; c < n; ++c) cfma(acc, ph[piv[c]], z[c]);
    A[it] = cscale(acc, isig[i] * inv_kn);
  }
  __syncwarp();
  if (lane == 0) D[b + 1] = k;
  __syncwarp();
  TNRC_TOC(w, 3, t_w);
}

template <int kD>
__device__ void two_site_update(const TrajParams& p, const Lay& Y, unsigned char* slot, int b, const double2* G,
                                bool adjoint, bool record, bool count, WarpCtx& w, const double2* pre = nullptr) {
  const int lane = w.lane;
  const int* D = slot_dims(slot);
  const int m = kD * D[b], n = kD * D[b + 2];
  // theta (then R^dagger) and Phi in the warp's shared slab when they fit
  double2* T = theta_home(p, kD * kD, m * n, w);
  double2* Phi = (2 * m * n <= p.slab_elems) ? w.slab + m * n : w.scratch;
  TNRC_TIC(t_c);
  const double fro = theta_build<kD>(p, Y, slot, b, G, adjoint, w, T, Phi, pre);
  TNRC_TOC(w, 0, t_c);

  // Phase 2: pivoted QR of theta, then one-sided Jacobi on the r columns of
  // R^dagger (column j = conjugated row j of R, contiguous at T + j n).
  TNRC_TIC(t_j);
  const double zthr = kJacobiZero * kJacobiZero * fro;
  int r = warp_qrcp<kD == 4>(T, m, n, zthr, w.piv, w.qn, lane);
  if (r < 1) r = 1;  // theta == 0 (or not finite): keep one column; the NaN check reports it
  for (int e = lane; e < r * n; e += 32) T[e] = cconj(T[e]);
  __syncwarp();
  // columns of R^dagger much longer than their number: the second QR, after
  // which the Jacobi runs on r x r (Z2 in theta's home past R^dagger when it
  // fits there, else in the warp's scratch past theta's room)
  double2* Z2 = nullptr;
  if (r >= kRowQrMinRank && 2 * n >= 5 * r) {
    Z2 = (T == w.slab && (size_t)(m - r) * n >= (size_t)r * r) ? T + (size_t)r * n
                                                              : w.scratch + (size_t)2 * kD * kD * p.chi * p.chi;
    warp_qr_rows<kD == 4>(T, n, r, Z2, w.small, w.sig2, lane);
  }
  TNRC_TOC(w, 1, t_j);
  TNRC_TIC(t_s);
  const int sw = warp_jacobi<kD == 4>(Z2 ? Z2 : T, Z2 ? r : n, r, fro, w.qn, lane);   // qn is free after the QR
  TNRC_TOC(w, 8, t_s);
  theta_finish<kD>(p, Y, slot, b, T, Phi, r, sw, record, count, w, SvdBufs{w.sig2, w.qn, w.perm, w.piv}, Z2);
}

// Whether bonds b1 and b2 of one layer are updated as a pair: pairing is on
// for the context (the matrix shape the autotuner picks), both thetas and
// both Phis fit the warp's shared slab side by side, and every side is at
// most 64 (the per-warp SVD arrays are split in halves).
template <int kD>
__device__ __forceinline__ bool pair_fits(const TrajParams& p, const int* D, int b1, int b2) {
  const int m1 = kD * D[b1], n1 = kD * D[b1 + 2], m2 = kD * D[b2], n2 = kD * D[b2 + 2];
  return p.pair_svd && 2 * (m1 * n1 + m2 * n2) <= p.slab_elems && m1 <= 64 && n1 <= 64 && m2 <= 64 &&
         n2 <= 64;
}

// Where a pair update keeps its two thetas in the slab: T1 at 0, Phi1 at
// m1 n1, T2 at 2 m1 n1, Phi2 after T2.
template <int kD>
__device__ __forceinline__ double2* pair_theta(const TrajParams& p, const int* D, int b1, int which, WarpCtx& w) {
  const int mn1 = kD * D[b1] * kD * D[b1 + 2];
  return which == 0 ? w.slab : w.slab + 2 * mn1;
}

// Two two-site updates (bonds b1, b2 of one layer, disjoint sites) by one
// warp: thetas built one after the other, then the pivoted QR and the Jacobi
// of both at once on the two half-warps, then ranks and splits one after the
// other.  The same arithmetic per bond as two_site_update, in another lane
// arrangement (so the same results up to the order of sums).
template <int kD>
__device__ void two_site_update_pair(const TrajParams& p, const Lay& Y, unsigned char* slot, int b1,
                                     const double2* G1, int b2, const double2* G2, bool adjoint, bool record,
                                     bool count, WarpCtx& w, const double2* pre1 = nullptr,
                                     const double2* pre2 = nullptr) {
  const int lane = w.lane;
  const int* D = slot_dims(slot);
  const int m1 = kD * D[b1], n1 = kD * D[b1 + 2], m2 = kD * D[b2], n2 = kD * D[b2 + 2];
  double2* T1 = w.slab;
  double2* Phi1 = w.slab + m1 * n1;
  double2* T2 = w.slab + 2 * m1 * n1;
  double2* Phi2 = T2 + m2 * n2;
  TNRC_TIC(t_c);
  const double fro1 = theta_build<kD>(p, Y, slot, b1, G1, adjoint, w, T1, Phi1, pre1);
  const double fro2 = theta_build<kD>(p, Y, slot, b2, G2, adjoint, w, T2, Phi2, pre2);
  TNRC_TOC(w, 0, t_c);
  const SvdBufs bf1{w.sig2, w.qn, w.perm, w.piv};
  const SvdBufs bf2{w.sig2 + 64, w.qn + 64, w.perm + 64, w.piv + 64};
  const bool hi = lane >= 16;
  TNRC_TIC(t_j);
  int rh = half_qrcp<kD == 4>(hi ? T2 : T1, hi ? m2 : m1, hi ? n2 : n1,
                              kJacobiZero * kJacobiZero * (hi ? fro2 : fro1), hi ? bf2.piv : bf1.piv,
                              hi ? bf2.qn : bf1.qn, lane);
  int r1 = __shfl_sync(0xffffffffu, rh, 0), r2 = __shfl_sync(0xffffffffu, rh, 16);
  if (r1 < 1) r1 = 1;
  if (r2 < 1) r2 = 1;
  for (int e = lane; e < r1 * n1; e += 32) T1[e] = cconj(T1[e]);
  for (int e = lane; e < r2 * n2; e += 32) T2[e] = cconj(T2[e]);
  __syncwarp();
  TNRC_TOC(w, 1, t_j);
  TNRC_TIC(t_s);
  const int swh = half_jacobi<kD == 4>(hi ? T2 : T1, hi ? n2 : n1, hi ? r2 : r1, hi ? fro2 : fro1,
                                       hi ? bf2.qn : bf1.qn, lane);
  const int sw1 = __shfl_sync(0xffffffffu, swh, 0), sw2 = __shfl_sync(0xffffffffu, swh, 16);
  TNRC_TOC(w, 8, t_s);
  theta_finish<kD>(p, Y, slot, b1, T1, Phi1, r1, sw1, record, count, w, bf1);
  theta_finish<kD>(p, Y, slot, b2, T2, Phi2, r2, sw2, record, count, w, bf2);
}

// ---------------------------------------------------------------------------
// Read-only view of a stored state: a slot of a layout, or a packed record.
// A packed record holds D[N+1], the site offsets off[N] (complex elements) and
// the site tensors at their actual dimensions -- the layer history of the
// costate sweep is kept in this form.
// ---------------------------------------------------------------------------
struct StateView {
  const int* D;
  const int* off;
  const double2* sites;
};

__device__ __forceinline__ StateView slot_view(const unsigned char* slot, const Lay& Y) {
  return StateView{slot_dims(slot), Y.site_off, slot_sites(slot, Y.L)};
}

__device__ __forceinline__ size_t packed_header(int N) { return ((size_t)(2 * N + 1) * 4 + 15) / 16 * 16; }

__device__ __forceinline__ StateView packed_view(const unsigned char* rec, int N) {
  const int* D = reinterpret_cast<const int*>(rec);
  return StateView{D, D + N + 1, reinterpret_cast<const double2*>(rec + packed_header(N))};
}

// Bytes of the packed record of a slot (same value in every thread).
template <int kD>
__device__ __forceinline__ size_t packed_bytes(const int* D, int N) {
  size_t e = 0;
  for (int i = 0; i < N; ++i) e += (size_t)D[i] * kD * D[i + 1];
  return packed_header(N) + e * 16;
}

// CTA-wide: write the packed record of `slot` to `rec`.
template <int kD>
__device__ void pack_state(const TrajParams& p, const Lay& Y, const unsigned char* slot, unsigned char* rec) {
  const int N = p.N;
  const int* D = slot_dims(slot);
  int* hd = reinterpret_cast<int*>(rec);
  double2* out = reinterpret_cast<double2*>(rec + packed_header(N));
  const double2* src = slot_sites(slot, Y.L);
  if (threadIdx.x == 0) {
    int o = 0;
    for (int i = 0; i <= N; ++i) hd[i] = D[i];
    for (int i = 0; i < N; ++i) {
      hd[N + 1 + i] = o;
      o += D[i] * kD * D[i + 1];
    }
  }
  size_t o = 0;
  for (int i = 0; i < N; ++i) {
    const int cnt = D[i] * kD * D[i + 1];
    const double2* a = src + Y.site_off[i];
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) out[o + e] = a[e];
    o += cnt;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Transfer-matrix steps of <c| . |a>.
// Left:  Eout[b'][a'] = sum_{b,s,a} conj(c[b][s][b']) Ein[b][a] a[a][s][a']
// Right: Eout[b][a]   = sum_{s,b',a'} conj(c[b][s][b']) Ein[b'][a'] a[a][s][a']
// Run by a team of nt threads (thread ti of the team): one warp (nt = 32,
// bar < 0: the warp synchronises itself) or several warps meeting at the
// named barrier `bar`.  Every output element is summed by one thread in the
// same order whatever the team, so the result does not depend on it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void team_sync(int bar, int nt) {
  if (bar < 0)
    __syncwarp();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
}

template <int kD>
__device__ void env_left_step(const double2* Ein, int Dcl, int Dal, const double2* c, int Dcr,
                              const double2* a, int Dar, double2* tmp, double2* Eout, int ti, int nt = 32,
                              int bar = -1) {
  const int w2 = kD * Dar;
  for (int it = ti; it < Dcl * w2; it += nt) {
    const int be = it / w2, rest = it - be * w2;
    double2 acc = make_double2(0.0, 0.0);
    for (int al = 0; al < Dal; ++al) cfma(acc, Ein[be * Dal + al], a[(size_t)al * w2 + rest]);
    tmp[it] = acc;
  }
  team_sync(bar, nt);
  for (int it = ti; it < Dcr * Dar; it += nt) {
    const int bp = it / Dar, ap = it - bp * Dar;
    double2 acc = make_double2(0.0, 0.0);
    for (int be = 0; be < Dcl; ++be)
#pragma unroll
      for (int s = 0; s < kD; ++s)
        cfmac(acc, c[(size_t)be * kD * Dcr + s * Dcr + bp], tmp[(size_t)be * w2 + s * Dar + ap]);
    Eout[it] = acc;
  }
  team_sync(bar, nt);
}

template <int kD>
__device__ void env_right_step(const double2* Ein, int Dcr, int Dar, const double2* c, int Dcl,
                               const double2* a, int Dal, double2* tmp, double2* Eout, int ti, int nt = 32,
                               int bar = -1) {
  const int w2 = kD * Dal;
  for (int it = ti; it < Dcr * w2; it += nt) {
    const int bp = it / w2, rest = it - bp * w2;
    const int s = rest / Dal, al = rest - s * Dal;
    double2 acc = make_double2(0.0, 0.0);
    for (int ap = 0; ap < Dar; ++ap) cfma(acc, Ein[bp * Dar + ap], a[(size_t)al * kD * Dar + s * Dar + ap]);
    tmp[it] = acc;
  }
  team_sync(bar, nt);
  for (int it = ti; it < Dcl * Dal; it += nt) {
    const int be = it / Dal, al = it - be * Dal;
    double2 acc = make_double2(0.0, 0.0);
    for (int bp = 0; bp < Dcr; ++bp)
#pragma unroll
      for (int s = 0; s < kD; ++s)
        cfmac(acc, c[(size_t)be * kD * Dcr + s * Dcr + bp], tmp[(size_t)bp * w2 + s * Dal + al]);
    Eout[it] = acc;
  }
  team_sync(bar, nt);
}

// <t|a> by one warp.
template <int kD>
__device__ double2 warp_overlap(const TrajParams& p, const Lay& Yt, const unsigned char* tslot, const Lay& Ya,
                                const unsigned char* aslot, WarpCtx& w) {
  const int* Dt = slot_dims(tslot);
  const int* Da = slot_dims(aslot);
  const double2* ts = slot_sites(tslot, Yt.L);
  const double2* as = slot_sites(aslot, Ya.L);
  const size_t cc = (size_t)p.chi * p.chi;
  double2* E0 = w.scratch;
  double2* E1 = w.scratch + cc;
  double2* tmp = w.scratch + 2 * cc;
  if (w.lane == 0) E0[0] = make_double2(1.0, 0.0);
  __syncwarp();
  for (int i = 0; i < p.N; ++i) {
    env_left_step<kD>(E0, Dt[i], Da[i], ts + Yt.site_off[i], Dt[i + 1], as + Ya.site_off[i], Da[i + 1], tmp, E1,
                      w.lane);
    double2* x = E0;
    E0 = E1;
    E1 = x;
  }
  return E0[0];
}

// Cost of a two-site update with theta of (2 Dl) x (2 Dr): the Jacobi work
// grows as m n min(m, n).
__device__ __forceinline__ long long update_cost(int Dl, int Dr) {
  const long long m = 2 * Dl, n = 2 * Dr;
  return m * n * (m < n ? m : n);
}

// One warp: the bonds of parity `parity` in decreasing order of update cost
// into w.order, and the shared counter reset.
__device__ inline void order_layer(const TrajParams& p, const int* D, int parity, WarpCtx& w) {
  const int nb = (p.N - 1 - parity + 1) / 2;
  const int lane = w.lane;
  for (int j = lane; j < nb; j += 32) {
    const long long cj = update_cost(D[parity + 2 * j], D[parity + 2 * j + 2]);
    int rk = 0;
    for (int i = 0; i < nb; ++i) {
      const long long ci = update_cost(D[parity + 2 * i], D[parity + 2 * i + 2]);
      rk += (ci > cj || (ci == cj && i < j)) ? 1 : 0;
    }
    w.order[rk] = parity + 2 * j;
  }
  if (lane == 0) *w.next = 0;
}

// ---------------------------------------------------------------------------
// Gradient of one layer (App. A), split so that each bond's gradient and its
// costate update run back to back on one warp:
//   layer_envs    left/right environments of <c|.|a> for the layer (warps 0
//                 and 1) and the bonds ordered by cost (the last warp);
//   bond_gradient the mixed two-site density rho of bond b and dO/du =
//                 tr(Q_u rho) for every control u of its gate, added to the
//                 trajectory's gradient row as 2 Re(conj(O) dO/du); it leaves
//                 the costate's two-site product c_b c_{b+1} where the costate
//                 update of the bond takes theta, which then skips its own
//                 contraction.
// ---------------------------------------------------------------------------
template <int kD>
__device__ void layer_envs(const TrajParams& p, const Lay& Y, const unsigned char* cslot, const StateView av,
                           WarpCtx& w, int warp) {
  const int N = p.N, chi = p.chi;
  const size_t cc = (size_t)chi * chi;
  const int* Dc = slot_dims(cslot);
  const int* Da = av.D;
  const double2* cs = slot_sites(cslot, Y.L);
  const double2* as = av.sites;
  const int* so = Y.site_off;   // costate slot offsets
  const int* ao = av.off;       // forward-state offsets
  double2* Lbuf = p.env_scratch + (size_t)w.region * 2 * (N + 1) * cc;
  double2* Rbuf = Lbuf + (size_t)(N + 1) * cc;
  const int lane = w.lane;

  // left environments L_i (sites < i) for i <= N-2 by the even warps, right
  // R_i (sites >= i) for i >= 2 by the odd warps: each sweep is sequential
  // over the sites, so each step is shared by its team of warps (named
  // barriers 1 and 2); the step's intermediate (at most Dc x kD Da) sits in
  // the team's first warp's shared slab when it fits, else in its scratch
  TNRC_TIC(t_e);
  const int team = warp & 1;                               // 0: left, 1: right
  const int nt = 32 * (team == 0 ? (p.warps + 1) / 2 : p.warps / 2);
  const int ti = (warp >> 1) * 32 + lane;
  double2* lead_slab = w.slab - (size_t)(warp - team) * p.slab_elems;
  double2* lead_scratch = w.scratch - (size_t)(warp - team) * p.scratch_elems;
  const bool lead = warp == team;
  if (team == 0) {
    for (int i = 0; i + 1 <= N - 2; ++i) {
      double2* tmp = (Dc[i] * kD * Da[i + 1] <= p.slab_elems) ? lead_slab : lead_scratch;
      env_left_step<kD>(Lbuf + i * cc, Dc[i], Da[i], cs + so[i], Dc[i + 1], as + ao[i], Da[i + 1],
                        tmp, Lbuf + (i + 1) * cc, ti, nt, 1);
      if (lead) w.alg += 8ull * kD * Da[i + 1] * (unsigned long long)(Dc[i] * Da[i] + Dc[i + 1] * Dc[i]);
    }
  } else {
    for (int i = N - 1; i >= 2; --i) {
      double2* tmp = (Dc[i + 1] * kD * Da[i] <= p.slab_elems) ? lead_slab : lead_scratch;
      env_right_step<kD>(Rbuf + (size_t)(i + 1) * cc, Dc[i + 1], Da[i + 1], cs + so[i], Dc[i],
                         as + ao[i], Da[i], tmp, Rbuf + (size_t)i * cc, ti, nt, 2);
      if (lead) w.alg += 8ull * kD * Da[i] * (unsigned long long)(Dc[i + 1] * Da[i + 1] + Dc[i] * Dc[i + 1]);
    }
  }
  TNRC_TOC(w, 4, t_e);
}

template <int kD>
__device__ void bond_gradient(const TrajParams& p, const Lay& Y, const unsigned char* cslot, const StateView av,
                              int s, int l, int b, double2 wO, double* gsp_row, WarpCtx& w, double2* Wc) {
  constexpr int kDD = kD * kD, kI = kD / 2;
  const int N = p.N, chi = p.chi;
  const size_t cc = (size_t)chi * chi;
  const int* Dc = slot_dims(cslot);
  const int* Da = av.D;
  const double2* cs = slot_sites(cslot, Y.L);
  const double2* as = av.sites;
  const int* so = Y.site_off;
  const int* ao = av.off;
  const double2* Lbuf = p.env_scratch + (size_t)w.region * 2 * (N + 1) * cc;
  const double2* Rbuf = Lbuf + (size_t)(N + 1) * cc;
  const int lane = w.lane;
  TNRC_TIC(t_g);
  const int dcl = Dc[b], dcm = Dc[b + 1], dcr = Dc[b + 2];
  const int dal = Da[b], dam = Da[b + 1], dar = Da[b + 2];
  const double2* L = Lbuf + (size_t)b * cc;
  const double2* R = Rbuf + (size_t)(b + 2) * cc;
  const double2* a0 = as + ao[b];
  const double2* a1 = as + ao[b + 1];
  const double2* c0 = cs + so[b];
  const double2* c1 = cs + so[b + 1];
  // the costate product c_b c_{b+1} is shared with the bond's costate update
  // (counted there)
  w.alg += 8ull * dcl * (kD * dam * dal + kDD * dar * dam + kDD * dcr * dar +
                         (unsigned long long)kDD * kDD * dcr) + 2048ull;
  // Wc = c_b c_{b+1} [dcl][kD^2][dcr] at Wc (theta's home); the other three
  // intermediates packed at their actual sizes right after it in the warp's
  // shared slab when they fit there, else in its global scratch past theta's
  // room
  const int n1 = dcl * kD * dam, n2 = dcl * kDD * dar, n3 = dcl * kDD * dcr;
  const bool wc_in_slab = Wc >= w.slab && Wc < w.slab + p.slab_elems;
  double2* U1 = (wc_in_slab && (Wc - w.slab) + n3 + n1 + n2 + n3 <= p.slab_elems)
                    ? Wc + n3
                    : w.scratch + (size_t)2 * kDD * chi * chi;   // [dcl][kD][dam]
  double2* U2 = U1 + n1;                          // [dcl][kD^2][dar]
  double2* U3 = U2 + n2;                          // [dcl][kD^2][dcr]
  for (int it = lane; it < dcl * kD * dam; it += 32) {
    const int be = it / (kD * dam), rest = it - be * kD * dam;
    double2 acc = make_double2(0.0, 0.0);
    for (int al = 0; al < dal; ++al) cfma(acc, L[be * dal + al], a0[(size_t)al * kD * dam + rest]);
    U1[it] = acc;
  }
  for (int it = lane; it < dcl * kDD * dcr; it += 32) {
    const int be = it / (kDD * dcr), rest = it - be * kDD * dcr;
    const int ss = rest / dcr, b2 = rest - ss * dcr;
    const int s1 = ss / kD, s2 = ss % kD;
    double2 acc = make_double2(0.0, 0.0);
    for (int b1 = 0; b1 < dcm; ++b1)
      cfma(acc, c0[(size_t)be * kD * dcm + s1 * dcm + b1], c1[(size_t)b1 * kD * dcr + s2 * dcr + b2]);
    Wc[it] = acc;
  }
  __syncwarp();
  for (int it = lane; it < dcl * kDD * dar; it += 32) {
    const int be = it / (kDD * dar), rest = it - be * kDD * dar;
    const int ss = rest / dar, a2 = rest - ss * dar;
    const int s1 = ss / kD, s2 = ss % kD;
    double2 acc = make_double2(0.0, 0.0);
    for (int a1i = 0; a1i < dam; ++a1i)
      cfma(acc, U1[(size_t)be * kD * dam + s1 * dam + a1i], a1[(size_t)a1i * kD * dar + s2 * dar + a2]);
    U2[it] = acc;
  }
  __syncwarp();
  for (int it = lane; it < dcl * kDD * dcr; it += 32) {
    const int be = it / (kDD * dcr), rest = it - be * kDD * dcr;
    const int ss = rest / dcr, b2 = rest - ss * dcr;
    double2 acc = make_double2(0.0, 0.0);
    const double2* u2 = U2 + (size_t)be * kDD * dar + ss * dar;
    const double2* rr = R + (size_t)b2 * dar;
    for (int a2 = 0; a2 < dar; ++a2) cfma(acc, u2[a2], rr[a2]);
    U3[it] = acc;
  }
  __syncwarp();
  // rho[o'][o] = sum_{i1,i2} sum_{be,b2} U3[be][s'][b2] conj(Wc[be][s][b2]) over the
  // two-site out indices o (the in indices, if any, traced out: the gate acts
  // as Q (x) I); lane = (o', o) pair, 16 lanes x 2 halves
  double2* rho = w.small;
  {
    const int o = lane & 15, half = lane >> 4;
    const int op = o >> 2, oq = o & 3;
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll
    for (int i1 = 0; i1 < kI; ++i1)
#pragma unroll
      for (int i2 = 0; i2 < kI; ++i2) {
        const int sp = ((op >> 1) * kI + i1) * kD + (op & 1) * kI + i2;
        const int sq = ((oq >> 1) * kI + i1) * kD + (oq & 1) * kI + i2;
        for (int be = half; be < dcl; be += 2) {
          const double2* u = U3 + (size_t)be * kDD * dcr + sp * dcr;
          const double2* wv = Wc + (size_t)be * kDD * dcr + sq * dcr;
          for (int b2 = 0; b2 < dcr; ++b2) cfmac(acc, wv[b2], u[b2]);
        }
      }
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 16);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 16);
    if (lane < 16) rho[o] = acc;
  }
  __syncwarp();
  // dO/du_q = tr(Q_q rho) = sum_ij Q_q[i][j] rho[j][i]: lane q takes control q
  const LayerGate& lg = layer_rec(p, s, l, b);
  const int nq = lg.nq;
  if (lane < nq) {
    const double2* Q = lg.Q[lane];
    double2 v = make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) cfma(v, Q[i * 4 + j], rho[j * 4 + i]);
    // explicit fma: this function is inlined into both history modes, which
    // must round identically
    gsp_row[lg.slot[lane]] += 2.0 * fma(wO.x, v.x, wO.y * v.y);
  }
  __syncwarp();
  TNRC_TOC(w, 5, t_g);
}

// ---------------------------------------------------------------------------
// Copy the used part of a state slot; src and dst may use different layouts.
// Returns 1 (and copies nothing) when a dimension exceeds dst's capacity.
template <int kD>
__device__ int copy_slot(const TrajParams& p, const Lay& Ys, const unsigned char* src, const Lay& Yd,
                         unsigned char* dst) {
  __syncthreads();
  const int* Ds = slot_dims(src);
  int* Dd = slot_dims(dst);
  const int tid = threadIdx.x, nt = blockDim.x;
  int bad = 0;
  for (int i = tid; i <= p.N; i += nt) bad |= (Ds[i] > Yd.dcap[i]) ? 1 : 0;
  if (__syncthreads_or(bad)) return 1;
  for (int i = tid; i <= p.N; i += nt) Dd[i] = Ds[i];
  const double* ls = slot_lam(src, Ys.L);
  double* ld = slot_lam(dst, Yd.L);
  for (int b = 0; b < p.N - 1; ++b) {
    const int d = Ds[b + 1];
    for (int j = tid; j < d; j += nt) ld[(size_t)b * Yd.L.chi + j] = ls[(size_t)b * Ys.L.chi + j];
  }
  const double2* ss = slot_sites(src, Ys.L);
  double2* sd = slot_sites(dst, Yd.L);
  for (int i = 0; i < p.N; ++i) {
    const int cnt = Ds[i] * kD * Ds[i + 1];
    const double2* a = ss + Ys.site_off[i];
    double2* b = sd + Yd.site_off[i];
    for (int e = tid; e < cnt; e += nt) b[e] = a[e];
  }
  __syncthreads();
  return 0;
}

// Entries e and e+1 of the layer's bond order (w.order, nb entries): one
// warp updates both, as a pair when both are small (two_site_update_pair),
// else one after the other.  The grouping depends only on the order and the
// bond dimensions, not on which warp or CTA takes it, so every launch form
// computes the same thing.
template <int kD>
__device__ void forward_group(const TrajParams& p, const Lay& Y, unsigned char* slot, int s, int l, int e, int nb,
                              bool adjoint, bool record, bool count, WarpCtx& w) {
  const int b1 = w.order[e];
  const int b2 = (e + 1 < nb) ? w.order[e + 1] : -1;
  if (b2 >= 0 && pair_fits<kD>(p, slot_dims(slot), b1, b2)) {
    two_site_update_pair<kD>(p, Y, slot, b1, layer_rec(p, s, l, b1).G, b2, layer_rec(p, s, l, b2).G, adjoint,
                             record, count, w);
    return;
  }
  two_site_update<kD>(p, Y, slot, b1, layer_rec(p, s, l, b1).G, adjoint, record, count, w);
  if (b2 >= 0) two_site_update<kD>(p, Y, slot, b2, layer_rec(p, s, l, b2).G, adjoint, record, count, w);
}

// All bonds of truncated layer l.  The warps take bonds from a shared counter
// in decreasing order of cost (largest SVD first), so that they reach the
// layer barrier together; a bond's result does not depend on which warp
// computes it.
template <int kD>
__device__ void apply_layer(const TrajParams& p, const Lay& Y, unsigned char* slot, int s, int l, bool adjoint,
                            bool record, bool count, WarpCtx& w, int warp) {
  const int parity = layer_parity(p, l);
  const int nb = (p.N - 1 - parity + 1) / 2;
  const int lane = w.lane;
  if (warp == 0) order_layer(p, slot_dims(slot), parity, w);
  __syncthreads();
  for (;;) {   // two bonds at a time
    int e = 0;
    if (lane == 0) e = atomicAdd(w.next, 2);
    e = __shfl_sync(0xffffffffu, e, 0);
    if (e >= nb) break;
    forward_group<kD>(p, Y, slot, s, l, e, nb, adjoint, record, count, w);
  }
  TNRC_TIC(t_b);
  __syncthreads();
  TNRC_TOC(w, 7, t_b);
}

// Entries e and e+1 of the layer's bond order: each bond's gradient and its
// costate update, the two updates as a pair when both bonds are small (the
// grouping rule of forward_group).
template <int kD>
__device__ void costate_group(const TrajParams& p, const Lay& Y, unsigned char* cslot, const StateView av, int s,
                              int l, int e, int nb, double2 wO, double* gsp_row, WarpCtx& w) {
  constexpr int kDD = kD * kD;
  const int* Dc = slot_dims(cslot);
  const int b1 = w.order[e];
  const int b2 = (e + 1 < nb) ? w.order[e + 1] : -1;
  if (b2 >= 0 && pair_fits<kD>(p, Dc, b1, b2)) {
    double2* th1 = pair_theta<kD>(p, Dc, b1, 0, w);
    double2* th2 = pair_theta<kD>(p, Dc, b1, 1, w);
    bond_gradient<kD>(p, Y, cslot, av, s, l, b1, wO, gsp_row, w, th1);
    bond_gradient<kD>(p, Y, cslot, av, s, l, b2, wO, gsp_row, w, th2);
    two_site_update_pair<kD>(p, Y, cslot, b1, layer_rec(p, s, l, b1).G, b2, layer_rec(p, s, l, b2).G, true, false,
                             true, w, th1, th2);
    return;
  }
  for (int q = 0; q < 2; ++q) {
    const int b = q == 0 ? b1 : b2;
    if (b < 0) break;
    double2* th = theta_home(p, kDD, kDD * Dc[b] * Dc[b + 2], w);
    bond_gradient<kD>(p, Y, cslot, av, s, l, b, wO, gsp_row, w, th);
    two_site_update<kD>(p, Y, cslot, b, layer_rec(p, s, l, b).G, true, false, true, w, th);
  }
}

// One layer of the costate sweep (App. A): the environments of <c_l|.|a_l>
// (warps 0 and 1), then every bond of layer l -- largest first from the
// shared counter -- its gradient and at once its costate update
// c_{l-1} = G^dag c_l, which reuses the product c_b c_{b+1} the gradient
// formed.  A bond's gradient reads only its own two costate sites and the
// environments; its update rewrites those two sites, which no other bond of
// the layer touches.  (Starting bonds while the environment sweeps still run
// -- as soon as both are past the bond's sites -- measured slower: the sweeps
// then share the FP64 pipes and the edge bonds wait for them all the same.)
template <int kD>
__device__ void costate_layer(const TrajParams& p, const Lay& Y, unsigned char* cslot, const StateView av, int s,
                              int l, double2 wO, double* gsp_row, WarpCtx& w, int warp) {
  constexpr int kDD = kD * kD;
  const int parity = layer_parity(p, l);
  const int nb = (p.N - 1 - parity + 1) / 2;
  const int lane = w.lane;
  const int* Dc = slot_dims(cslot);
  const size_t cc = (size_t)p.chi * p.chi;
  if (warp == p.warps - 1) order_layer(p, Dc, parity, w);
  if (lane == 0 && warp == 0) {
    double2* Lbuf = p.env_scratch + (size_t)w.region * 2 * (p.N + 1) * cc;
    Lbuf[0] = make_double2(1.0, 0.0);
    Lbuf[(size_t)(2 * p.N + 1) * cc] = make_double2(1.0, 0.0);   // R_N
  }
  __syncthreads();
  layer_envs<kD>(p, Y, cslot, av, w, warp);
  __syncthreads();
  for (;;) {   // two bonds at a time
    int e = 0;
    if (lane == 0) e = atomicAdd(w.next, 2);
    e = __shfl_sync(0xffffffffu, e, 0);
    if (e >= nb) break;
    costate_group<kD>(p, Y, cslot, av, s, l, e, nb, wO, gsp_row, w);
  }
  TNRC_TIC(t_b);
  __syncthreads();
  TNRC_TOC(w, 7, t_b);
}

// One trajectory (sample s, input pi) with the CTA's work region `base`.
//   packed = true : every layer state of the forward pass is kept as a packed
//                   record in the region (no recomputation in the costate
//                   sweep); returns 1 if the history outgrows the region.
//   packed = false: checkpoints every Y.seg layers and recomputation of each
//                   segment (fits by construction).
template <int kD>
__device__ int run_trajectory(const TrajParams& p, bool packed, unsigned char* base, int t, int s, int pi,
                              WarpCtx& w, int warp, double* s_disc, int* s_maxk, double2* s_O) {
  const Lay& Y = p.full;
  const int lane = w.lane;
  const size_t sb = (size_t)Y.L.bytes;
  const int L = p.n_layers;  // truncated layers
  unsigned char* a_slot = base;
  unsigned char* c_slot = base + sb;
  unsigned char* ckpt = base + 2 * sb;
  unsigned char* segs = ckpt + (size_t)Y.nseg * sb;
  long long* hpos = reinterpret_cast<long long*>(base + 2 * sb);  // packed mode: record offsets
  unsigned char* harena = base + 2 * sb + (((size_t)L * 8 + 255) / 256) * 256;
  const size_t hbytes = min((size_t)p.work_stride - (size_t)(harena - base), (size_t)p.history_cap);
  const int KCN = p.K * p.C * p.N;
  w.disc = 0.0;
  w.maxk = 0;
  copy_slot<kD>(p, Y, p.in_slots + (size_t)pi * sb, Y, a_slot);
  // ---- forward ----
  size_t pos = 0;
  for (int l = 0; l < L; ++l) {
    const int q = l / Y.seg;
    if (p.want_grad && !packed && (l % Y.seg) == 0 && q < Y.nseg - 1) copy_slot<kD>(p, Y, a_slot, Y, ckpt + (size_t)q * sb);
    apply_layer<kD>(p, Y, a_slot, s, l, false, true, true, w, warp);
    if (p.want_grad) {
      if (packed) {
        const size_t need = packed_bytes<kD>(slot_dims(a_slot), p.N);
        if (pos + need > hbytes) return 1;
        TNRC_TIC(t_h);
        pack_state<kD>(p, Y, a_slot, harena + pos);
        TNRC_TOC(w, 6, t_h);
        if (threadIdx.x == 0) hpos[l] = (long long)pos;
        pos += (need + 255) / 256 * 256;
      } else if (q == Y.nseg - 1) {
        copy_slot<kD>(p, Y, a_slot, Y, segs + (size_t)(l - q * Y.seg) * sb);
      }
    }
  }
  const unsigned char* tg = p.tg_slots + (size_t)pi * sb;
  if (warp == 0) {
    const double2 O = warp_overlap<kD>(p, Y, tg, Y, a_slot, w);
    if (lane == 0) *s_O = O;
    const int* Dt = slot_dims(tg);
    const int* Da = slot_dims(a_slot);
    for (int i = 0; i < p.N; ++i)
      w.alg += 8ull * kD * Da[i + 1] * (unsigned long long)(Dt[i] * Da[i] + Dt[i + 1] * Dt[i]);
  }
  if (lane == 0) {
    s_disc[warp] = w.disc;
    s_maxk[warp] = w.maxk;
  }
  __syncthreads();
  const double2 O = *s_O;
  if (threadIdx.x == 0) {
    p.O[t] = O;
    double d = 0.0;
    int mk = 0;
    for (int i = 0; i < p.warps; ++i) {
      d += s_disc[i];
      mk = max(mk, s_maxk[i]);
    }
    p.disc[t] = d;
    atomicMax(&p.counters[2], (unsigned long long)mk);
  }
  if (!p.want_grad) return 0;
  // ---- costate sweep ----
  double* grow = p.gsp + (size_t)t * KCN;
  for (int i = threadIdx.x; i < KCN; i += blockDim.x) grow[i] = 0.0;
  copy_slot<kD>(p, Y, tg, Y, c_slot);
  if (packed) {
    for (int l = L - 1; l >= 0; --l)
      costate_layer<kD>(p, Y, c_slot, packed_view(harena + hpos[l], p.N), s, l, O, grow, w, warp);
    return 0;
  }
  for (int q = Y.nseg - 1; q >= 0; --q) {
    const int l0 = q * Y.seg;
    const int l1 = min(L, l0 + Y.seg);
    if (q != Y.nseg - 1) {
      unsigned char* ck = ckpt + (size_t)q * sb;
      for (int l = l0; l < l1; ++l) {
        apply_layer<kD>(p, Y, ck, s, l, false, false, false, w, warp);
        copy_slot<kD>(p, Y, ck, Y, segs + (size_t)(l - l0) * sb);
      }
    }
    for (int l = l1 - 1; l >= l0; --l)
      costate_layer<kD>(p, Y, c_slot, slot_view(segs + (size_t)(l - l0) * sb, Y), s, l, O, grow, w, warp);
  }
  return 0;
}

// Compiled twice: kMinBlocks = 1 lets a thread use up to 255 registers (at
// most 8 warps per SM); kMinBlocks = 2 caps it at 128 so that 16 warps fit an
// SM, trading a few spilled values for twice the warps to hide FP64 latency.
template <int kMinBlocks, int kD>
__global__ void __launch_bounds__(kWarps * 32, kMinBlocks) traj_kernel(TrajParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  __shared__ double s_disc[kWarps];
  __shared__ int s_maxk[kWarps];
  __shared__ double2 s_O;
  __shared__ int s_order[128];
  __shared__ int s_next;
  __shared__ int s_region;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  double2* slabs = reinterpret_cast<double2*>(smem_raw);
  double* sig = reinterpret_cast<double*>(slabs + (size_t)p.warps * p.slab_elems);
  double* qns = sig + (size_t)p.warps * kMaxDim;
  int* perms = reinterpret_cast<int*>(qns + (size_t)p.warps * kMaxDim);
  int* pivs = perms + (size_t)p.warps * kMaxDim;
  double2* smalls = reinterpret_cast<double2*>(pivs + (size_t)p.warps * kMaxDim);

  // pooled launch: take a free work region (bounded scan; a full pool cannot
  // happen while n_regions covers the CTAs that can be resident at once)
  int region = blockIdx.x;
  if (p.pooled) {
    if (blockIdx.x >= p.T) return;
    if (threadIdx.x == 0) {
      int got = -1;
      for (int attempt = 0; attempt < kRegionTries && got < 0; ++attempt) {
        for (int i = 0; i < p.n_regions; ++i) {
          const int r = (int)((blockIdx.x + (unsigned)i) % (unsigned)p.n_regions);
          if (atomicCAS(&p.region_owner[r], 0, 1) == 0) {
            got = r;
            break;
          }
        }
        if (got < 0) __nanosleep(16000);
      }
      s_region = got;
    }
    __syncthreads();
    region = s_region;
    if (region < 0) {
      if (threadIdx.x == 0) atomicOr(p.status, kStatusTimeout);
      return;
    }
  }
  WarpCtx w;
  w.region = region;
  w.slab = slabs + (size_t)warp * p.slab_elems;
  w.scratch = p.warp_scratch + ((size_t)region * p.warps + warp) * p.scratch_elems;
  w.sig2 = sig + (size_t)warp * kMaxDim;
  w.perm = perms + (size_t)warp * kMaxDim;
  w.qn = qns + (size_t)warp * kMaxDim;
  w.piv = pivs + (size_t)warp * kMaxDim;
  w.small = smalls + (size_t)warp * 64;
  w.lane = lane;
  w.sweeps = 0;
  w.updates = 0;
  w.alg = 0;
  w.capcuts = 0;
  for (int i = 0; i < kNumPhases; ++i) w.ph[i] = 0;
  w.order = s_order;
  w.next = &s_next;
  unsigned char* base = p.work + (size_t)region * p.work_stride;

  for (int iter = 0;; ++iter) {
    if (threadIdx.x == 0) s_item = p.pooled ? (iter == 0 ? (int)blockIdx.x : p.T) : atomicAdd(p.work_counter, 1);
    __syncthreads();
    const int t = s_item;
    __syncthreads();
    if (t >= p.T) break;
    const int s = t / p.P, pi = t - s * p.P;
    bool redo = true;
    if (p.want_grad && p.packed_history) {
      const long long sw0 = w.sweeps, up0 = w.updates, cc0 = w.capcuts;
      const unsigned long long al0 = w.alg;
      redo = run_trajectory<kD>(p, true, base, t, s, pi, w, warp, s_disc, s_maxk, &s_O) != 0;
      if (redo) {  // history outgrew the region: discard the attempt's counts, count the fallback
        w.sweeps = sw0;
        w.updates = up0;
        w.alg = al0;
        w.capcuts = cc0;
        if (threadIdx.x == 0) atomicAdd(&p.counters[4], 1ull);
      }
    }
    if (redo) run_trajectory<kD>(p, false, base, t, s, pi, w, warp, s_disc, s_maxk, &s_O);
  }
  if (lane == 0) {
    atomicAdd(&p.counters[0], (unsigned long long)w.updates);
    atomicAdd(&p.counters[1], (unsigned long long)w.sweeps);
    atomicAdd(&p.counters[3], w.alg);
    atomicAdd(&p.counters[kCtrCapTrunc], (unsigned long long)w.capcuts);
#ifdef TNRC_PHASE_TIMERS
    for (int i = 0; i < kNumPhases; ++i) atomicAdd(&p.counters[kCtrPhase + i], (unsigned long long)w.ph[i]);
#endif
  }
  if (p.pooled) {   // hand the region back once every thread is done with it
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicExch(&p.region_owner[region], 0);
    }
  }
}

// ---------------------------------------------------------------------------
// The plain GPU path: one trajectory at a time, one launch per step, the
// bonds of a layer spread over CTAs of one warp each (the whole GPU for one
// trajectory, as far as its layers have bonds).  It runs the same device
// functions as the batched kernel and gives bitwise the same results; it is
// the baseline that the persistent batched launch is measured against.
// ---------------------------------------------------------------------------
struct PlainShared {
  double2* slab;
  double* sig;
  double* qn;
  int* perm;
  int* piv;
  double2* small;
};

__device__ inline void plain_warp(const TrajParams& p, WarpCtx& w, int scratch_index, int* order, int* next,
                                  int warp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* slabs = reinterpret_cast<double2*>(smem_raw);
  double* sig = reinterpret_cast<double*>(slabs + (size_t)p.warps * p.slab_elems);
  double* qns = sig + (size_t)p.warps * kMaxDim;
  int* perms = reinterpret_cast<int*>(qns + (size_t)p.warps * kMaxDim);
  int* pivs = perms + (size_t)p.warps * kMaxDim;
  double2* smalls = reinterpret_cast<double2*>(pivs + (size_t)p.warps * kMaxDim);
  w.region = 0;   // the one environment region
  w.slab = slabs + (size_t)warp * p.slab_elems;
  w.scratch = p.warp_scratch + (size_t)scratch_index * p.scratch_elems;
  w.sig2 = sig + (size_t)warp * kMaxDim;
  w.perm = perms + (size_t)warp * kMaxDim;
  w.qn = qns + (size_t)warp * kMaxDim;
  w.piv = pivs + (size_t)warp * kMaxDim;
  w.small = smalls + (size_t)warp * 64;
  w.lane = threadIdx.x & 31;
  w.sweeps = w.updates = w.capcuts = 0;
  w.alg = 0;
  w.disc = 0.0;
  w.maxk = 0;
  for (int i = 0; i < kNumPhases; ++i) w.ph[i] = 0;
  w.order = order;
  w.next = next;
}

// Copy a full slot (one CTA).
template <int kD>
__global__ void plain_copy_kernel(TrajParams p, const unsigned char* src, unsigned char* dst) {
  copy_slot<kD>(p, p.full, src, p.full, dst);
}

// Forward layer l of trajectory (s, .) on `slot`: CTA j updates the j-th
// group of two bonds of the layer's bond order (the grouping of the batched
// launch, so the results are the same).
template <int kD>
__global__ void __launch_bounds__(32) plain_fwd_kernel(TrajParams p, unsigned char* slot, int s, int l) {
  __shared__ int s_order[128], s_next;
  WarpCtx w;
  plain_warp(p, w, blockIdx.x, s_order, &s_next, 0);
  const int parity = layer_parity(p, l);
  const int nb = (p.N - 1 - parity + 1) / 2;
  order_layer(p, slot_dims(slot), parity, w);   // reads outer bond dimensions only, which no update changes
  __syncwarp();
  forward_group<kD>(p, p.full, slot, s, l, 2 * (int)blockIdx.x, nb, false, true, true, w);
  if (w.lane == 0) atomicAdd(&p.counters[1], (unsigned long long)w.sweeps);
}

// O_t = <t_p | a_t> (one warp).
template <int kD>
__global__ void __launch_bounds__(32) plain_overlap_kernel(TrajParams p, const unsigned char* tg,
                                                           const unsigned char* a, int t) {
  __shared__ int s_order[1], s_next;
  WarpCtx w;
  plain_warp(p, w, 0, s_order, &s_next, 0);
  const double2 O = warp_overlap<kD>(p, p.full, tg, p.full, a, w);
  if (w.lane == 0) p.O[t] = O;
}

// Environments of <c|.|a_l> for layer l (two warps: left and right sweeps).
template <int kD>
__global__ void __launch_bounds__(64) plain_envs_kernel(TrajParams p, const unsigned char* cslot,
                                                        const unsigned char* aslot) {
  __shared__ int s_order[1], s_next;
  WarpCtx w;
  const int warp = threadIdx.x >> 5;
  plain_warp(p, w, warp, s_order, &s_next, warp);
  const size_t cc = (size_t)p.chi * p.chi;
  if (threadIdx.x == 0) {
    p.env_scratch[0] = make_double2(1.0, 0.0);
    p.env_scratch[(size_t)(2 * p.N + 1) * cc] = make_double2(1.0, 0.0);
  }
  __syncthreads();
  layer_envs<kD>(p, p.full, cslot, slot_view(aslot, p.full), w, warp);
}

// Gradient and costate update of the bonds of layer l (CTA j: the j-th
// group of two bonds, as in the batched launch).
template <int kD>
__global__ void __launch_bounds__(32) plain_bwd_kernel(TrajParams p, unsigned char* cslot, const unsigned char* aslot,
                                                       int s, int l, int t) {
  __shared__ int s_order[128], s_next;
  WarpCtx w;
  plain_warp(p, w, blockIdx.x, s_order, &s_next, 0);
  const int parity = layer_parity(p, l);
  const int nb = (p.N - 1 - parity + 1) / 2;
  order_layer(p, slot_dims(cslot), parity, w);
  __syncwarp();
  costate_group<kD>(p, p.full, cslot, slot_view(aslot, p.full), s, l, 2 * (int)blockIdx.x, nb, p.O[t],
                    p.gsp + (size_t)t * p.K * p.C * p.N, w);
  if (w.lane == 0) atomicAdd(&p.counters[1], (unsigned long long)w.sweeps);
}

}  // namespace tnrc

// Host launchers of the plain path (see above).  `op`: 0 copy, 1 forward
// layer, 2 overlap, 3 environments, 4 gradient and costate update.
extern "C" cudaError_t tnrc_launch_plain(const tnrc::TrajParams* p, int op, const unsigned char* a,
                                         unsigned char* b, int s, int l, int t, size_t smem, cudaStream_t st) {
  (void)cudaGetLastError();
  const int nb = (p->N - 1 - ((l + p->first_parity) & 1) + 1) / 2;
  const int ng = (nb + 1) / 2;   // groups of two bonds
  const bool d4 = p->phys_dim == 4;
  switch (op) {
    case 0:
      if (d4) tnrc::plain_copy_kernel<4><<<1, 256, 0, st>>>(*p, a, b);
      else tnrc::plain_copy_kernel<2><<<1, 256, 0, st>>>(*p, a, b);
      break;
    case 1:
      if (d4) tnrc::plain_fwd_kernel<4><<<ng, 32, smem, st>>>(*p, b, s, l);
      else tnrc::plain_fwd_kernel<2><<<ng, 32, smem, st>>>(*p, b, s, l);
      break;
    case 2:
      if (d4) tnrc::plain_overlap_kernel<4><<<1, 32, smem, st>>>(*p, a, b, t);
      else tnrc::plain_overlap_kernel<2><<<1, 32, smem, st>>>(*p, a, b, t);
      break;
    case 3:
      if (d4) tnrc::plain_envs_kernel<4><<<1, 64, smem, st>>>(*p, b, a);
      else tnrc::plain_envs_kernel<2><<<1, 64, smem, st>>>(*p, b, a);
      break;
    case 4:
      if (d4) tnrc::plain_bwd_kernel<4><<<ng, 32, smem, st>>>(*p, b, a, s, l, t);
      else tnrc::plain_bwd_kernel<2><<<ng, 32, smem, st>>>(*p, b, a, s, l, t);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

extern "C" cudaError_t tnrc_plain_prepare() {
  cudaError_t e = cudaSuccess;
  const int lim = 226 * 1024;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tnrc::plain_fwd_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tnrc::plain_fwd_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tnrc::plain_overlap_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tnrc::plain_overlap_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tnrc::plain_envs_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tnrc::plain_envs_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tnrc::plain_bwd_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(tnrc::plain_bwd_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e;
}

// host-side launcher; tnrc_create (and the allocation-free entry point) raise
// the shared-memory limit with tnrc_traj_prepare before any launch or capture
extern "C" cudaError_t tnrc_traj_prepare() {
  cudaError_t e = cudaFuncSetAttribute(tnrc::traj_kernel<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tnrc::traj_kernel<2, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tnrc::traj_kernel<1, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 226 * 1024);
  return e;
}

// Resident CTAs per SM of the trajectory kernel for this launch shape (the
// size of a pooled launch's region pool is SMs times this).
extern "C" cudaError_t tnrc_traj_occupancy(int phys_dim, int min_blocks, int warps, size_t smem, int* per_sm) {
  if (phys_dim == 4)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, tnrc::traj_kernel<1, 4>, warps * 32, smem);
  if (min_blocks == 2)
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, tnrc::traj_kernel<2, 2>, warps * 32, smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, tnrc::traj_kernel<1, 2>, warps * 32, smem);
}

extern "C" cudaError_t tnrc_launch_traj(const tnrc::TrajParams* p, int grid, size_t smem, cudaStream_t st) {
  (void)cudaGetLastError();  // report only this launch below
  // operators (physical dimension 4) run the 255-register build only
  if (p->phys_dim == 4)
    tnrc::traj_kernel<1, 4><<<grid, p->warps * 32, smem, st>>>(*p);
  else if (p->min_blocks == 2)
    tnrc::traj_kernel<2, 2><<<grid, p->warps * 32, smem, st>>>(*p);
  else
    tnrc::traj_kernel<1, 2><<<grid, p->warps * 32, smem, st>>>(*p);
  return cudaGetLastError();
}

extern "C" size_t tnrc_traj_smem(int warps, int slab_elems) {
  return (size_t)warps * slab_elems * sizeof(double2) + (size_t)warps * tnrc::kMaxDim * 2 * (sizeof(double) + sizeof(int)) +
         (size_t)warps * 64 * sizeof(double2);
}
