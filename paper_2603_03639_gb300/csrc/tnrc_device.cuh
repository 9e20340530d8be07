// Device-side data layout and helpers of the tnrc library (sm_103a).
//
// A "state slot" holds one MPS in right-canonical form with Schmidt values
// (the form the TEBD two-site update of Sec. II keeps):
//   int    D[N+1]            bond dimensions, D[0] = D[N] = 1; bond b <-> D[b+1]
//   double lam[(N-1)*chi]    Schmidt values of bond b at lam[b*chi .. b*chi+D[b+1])
//   double2 sites[...]       site i at site_off[i]: row-major [D[i]][2][D[i+1]]
// Every site region is sized for the largest dimensions the site can reach,
// Dcap_b = min(2^(b+1), 2^(N-1-b), chi), and holds the tensor packed with its
// actual dimensions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tnrc {

constexpr int kMaxChi = 64;
constexpr int kMaxDim = 2 * kMaxChi;        // largest theta side
constexpr int kWarps = 8;                   // warps per trajectory CTA (upper bound)
constexpr int kMaxSweeps = 60;              // Jacobi sweep limit
constexpr double kZeroFloor = 1e-13;        // relative numerical-zero level of singular values
constexpr double kJacobiZero = 5e-15;       // columns below this x ||theta||_F are left alone
constexpr double kJacobiQuad = 1e-20;       // |<a,b>|^2 / (|a|^2 |b|^2) of a rotation that counts as
                                            // large: a sweep with none is the last (quadratic convergence)
constexpr int kRowQrMinRank = 8;            // second QR of R^dagger from this rank on, when n >= 2.5 r

// device status bits (OR-ed into *status)
constexpr int kStatusNoConverge = 1;
constexpr int kStatusNaN = 2;
constexpr int kStatusBadDims = 4;
constexpr int kStatusTimeout = 8;            // a bounded device wait gave up (no free work region)
constexpr int kRegionTries = 1 << 16;        // region-pool scans before giving up (about a second)
constexpr int kCtrPhase = 5 + kMaxChi + 1;      // first of kNumPhases cycle counters
constexpr int kNumPhases = 9;
constexpr int kCtrCapTrunc = kCtrPhase + kNumPhases;  // truncations whose cut the cap chi_max decided
constexpr int kCtrGap = kCtrCapTrunc + 1;              // smallest relative gap at such a cut (double bits;
                                                       // starts as all ones, lowered by atomicMin)
constexpr int kNumCounters = kCtrGap + 1;              // device counters of one evaluation

// Per-phase cycle counters (lane 0 of every warp, clock64), compiled in only
// with -DTNRC_PHASE_TIMERS: 0 contraction, 1 pivoted QR, 2 rank/truncate,
// 3 split and write-back, 4 environment sweeps, 5 mixed densities and gate
// gradients, 6 history and slot copies, 7 waiting at layer barriers,
// 8 Jacobi sweeps.
#ifdef TNRC_PHASE_TIMERS
#define TNRC_TIC(v) const long long v = clock64()
#define TNRC_TOC(w, idx, v) \
  do {                      \
    (w).ph[idx] += clock64() - (v); \
  } while (0)
#else
#define TNRC_TIC(v) \
  do {              \
  } while (0)
#define TNRC_TOC(w, idx, v) \
  do {                      \
  } while (0)
#endif

struct SlotLayout {
  int N, chi;
  int64_t lam_off;    // bytes from slot start
  int64_t sites_off;  // bytes from slot start
  int64_t bytes;      // slot stride
};

// The gate of one bond in one truncated layer for one noise sample, with
// what the costate gradient needs of it.  The gate is a product of factors
// G = G_F ... G_1 (one factor, or the two half steps merged at a step
// boundary, or the interaction and the folded single-site rotations of the
// first-order slice); for every control u it depends on,
//   Q_u = sum over the factors f containing u of L_f (dG_f/du) G_f^dag L_f^dag,
//   L_f = G_F ... G_{f+1},
// so that dO/du = tr(Q_u rho) with rho the mixed two-site density of the
// costate and the state after the layer (App. A).
constexpr int kMaxLayerParams = 10;
struct LayerGate {
  double2 G[16];                       // row-major, basis |s_b s_b+1>
  double2 Q[kMaxLayerParams][16];      // row-major
  int slot[kMaxLayerParams];           // gradient index k C N + c N + site
  int nq;                              // number of controls the gate depends on
  int pad_[5];
};

// One slot layout: byte layout, site offsets, capacities and the checkpoint
// segmentation that fits the per-CTA work region in this layout.
struct Lay {
  SlotLayout L;
  const int* site_off;         // [N] complex-element offsets of the sites in a slot
  const int* dcap;             // [N+1] capacity of D[i]
  int seg, nseg;               // checkpoint segment length and count, in truncated layers
};

struct TrajParams {
  int N, K, C, P, M, chi, T;
  double dt, eps;              // eps = max(cutoff, kZeroFloor)
  int want_grad;
  int warps;                   // warps per CTA
  int phys_dim;                // 2: qubit states; 4: operators as vectors (s = 2 out + in)
  int min_blocks;              // register budget of the launch: 1 = up to 8 warps per SM
                               // (255 registers), 2 = up to 16 warps per SM (128 registers)
  int slab_elems;              // complex elements of each warp's shared slab
  Lay full;                    // capacities min(2^i, 2^(N-i), chi)
  int packed_history;          // keep the forward history packed (no recomputation)
  long long history_cap;       // upper bound on a CTA's packed-history bytes
  const unsigned char* in_slots;   // P canonical input slots (full layout)
  const unsigned char* tg_slots;   // P canonical target slots (full layout)
  unsigned char* work;             // per CTA: 2 working slots, then packed history or checkpoints
  int64_t work_stride;             // bytes per CTA
  double2* warp_scratch;           // per warp: scratch_elems complex
  int64_t scratch_elems;
  double2* env_scratch;            // per CTA: 2*(N+1)*chi*chi complex
  const LayerGate* lgates;         // [M][recs_per_sample]: layer l's bonds at layer_off[l]
  const int* layer_off;            // [n_layers + 1]
  int n_layers;                    // truncated layers of one trajectory
  int first_parity;                // bond parity of layer 0 (they alternate)
  int recs_per_sample;
  const unsigned char* mask;       // [C][N]
  double2* O;                      // [T]
  double* gsp;                     // [T][K*C*N] or null
  double* disc;                    // [T]
  unsigned long long* counters;    // see kCtrHist in traj.cu
  int* status;
  int* work_counter;
  // launch mode: 0 = persistent (grid <= resident CTAs; each CTA takes
  // trajectories from work_counter and uses the work region of its index);
  // 1 = pooled (one CTA per trajectory, t = blockIdx.x; the CTA holds one of
  // n_regions work regions from region_owner while it runs, so the block
  // scheduler can interleave CTAs of other launches between trajectories)
  int pair_svd;                    // 1: two small SVDs per warp on the half-warps (see traj.cu)
  int pooled;
  int n_regions;
  int* region_owner;               // [n_regions], 0 = free
};

struct CanonArgs {
  int N, chi;
  int d;                       // physical dimension (2 or 4)
  double eps;
  int dmax;
  const int* raw_dims;         // [nmps][N+1]
  const double2* raw_data;     // packed site-major
  const long long* raw_off;    // [nmps] element offsets into raw_data
  double2* work;               // per MPS: (N + 4) * 2 * dmax^2 complex
  long long work_stride;       // complex elements per MPS
  unsigned char* slots;        // nmps slots
  SlotLayout L;
  const int* site_off;
  int* status;
};

// ---- small complex helpers (double2 = re, im) ----
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }

__device__ __forceinline__ double warp_sum(double v, unsigned mask = 0xffffffffu) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// slot accessors
__device__ __forceinline__ int* slot_dims(unsigned char* s) { return reinterpret_cast<int*>(s); }
__device__ __forceinline__ const int* slot_dims(const unsigned char* s) { return reinterpret_cast<const int*>(s); }
__device__ __forceinline__ double* slot_lam(unsigned char* s, const SlotLayout& L) {
  return reinterpret_cast<double*>(s + L.lam_off);
}
__device__ __forceinline__ const double* slot_lam(const unsigned char* s, const SlotLayout& L) {
  return reinterpret_cast<const double*>(s + L.lam_off);
}
__device__ __forceinline__ double2* slot_sites(unsigned char* s, const SlotLayout& L) {
  return reinterpret_cast<double2*>(s + L.sites_off);
}
__device__ __forceinline__ const double2* slot_sites(const unsigned char* s, const SlotLayout& L) {
  return reinterpret_cast<const double2*>(s + L.sites_off);
}

}  // namespace tnrc
