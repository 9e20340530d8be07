// Canonical form of the input and target states (costate initialisation of
// App. A needs the target in the same right-canonical form with Schmidt values
// that the TEBD update keeps; Sec. IV gives the targets as arbitrary MPS).
//
// One warp per MPS (physical dimension d = 2 for states, 4 for operators):
//   left sweep : site i as (d D_i) x D_{i+1}; SVD -> U S W^dag; site i <- U_r
//                (left isometry, numerically-zero values dropped), site i+1 <- (U_r^dag M) site i+1;
//   right sweep: with everything to the left left-isometric, site i (times the
//                carry from the right) as D_i x (d D_{i+1}); SVD -> U S Y^dag;
//                B_i <- Y_k^dag, lam_{i-1} <- S_k/|S_k|, carry <- M Y_k/|S_k| = U_k S_k/|S_k|;
//   B_0 <- site 0 times the carry, normalised.
#include "svd_warp.cuh"

namespace tnrc {

__global__ void canon_kernel(CanonArgs a) {
  __shared__ double sig2[256];
  __shared__ double cn[256];
  __shared__ int perm[256];
  __shared__ int D[257];
  const int lane = threadIdx.x;
  const int mi = blockIdx.x;
  const int N = a.N, dm = a.dmax, d = a.d;
  const size_t sz = (size_t)d * dm * dm;
  double2* W = a.work + (size_t)mi * a.work_stride;   // N sites, each sz
  double2* Mb = W + (size_t)N * sz;
  double2* T = Mb + sz;
  double2* carry = T + sz;
  double2* tmp = carry + sz;
  const int* rd = a.raw_dims + (size_t)mi * (N + 1);
  for (int i = lane; i <= N; i += 32) D[i] = rd[i];
  __syncwarp();
  {  // unpack
    const double2* src = a.raw_data + a.raw_off[mi];
    size_t off = 0;
    for (int i = 0; i < N; ++i) {
      const int cnt = D[i] * d * D[i + 1];
      for (int e = lane; e < cnt; e += 32) W[(size_t)i * sz + e] = src[off + e];
      off += cnt;
    }
  }
  __syncwarp();
  double kept2, tot2;
  // ---- left sweep ----
  for (int i = 0; i + 1 < N; ++i) {
    const int dl = D[i], dr = D[i + 1], dn = D[i + 2];
    const int n = d * dl, m = dr;
    double2* Wi = W + (size_t)i * sz;
    double fro = 0.0;
    for (int e = lane; e < n * m; e += 32) {
      const int row = e / m, col = e - row * m;  // row (al s), col be
      const double2 v = Wi[e];
      Mb[e] = v;
      T[(size_t)col * n + row] = v;
      fro += cabs2(v);
    }
    fro = warp_sum(fro);
    __syncwarp();
    const int sw = warp_jacobi(T, n, m, fro, cn, lane);
    double gap;
    int r = warp_rank_truncate(T, n, m, m, a.eps, sig2, perm, lane, kept2, tot2, gap);
    if (r > n) r = n;
    if (lane == 0 && sw < 0) atomicOr(a.status, kStatusNoConverge);
    // U_r into site i
    for (int e = lane; e < n * r; e += 32) {
      const int row = e / r, j = e - row * r;
      Wi[e] = cscale(T[(size_t)perm[j] * n + row], rsqrt(sig2[perm[j]]));
    }
    __syncwarp();
    // carry[j][be] = sum_row conj(U[row][j]) M[row][be]
    for (int e = lane; e < r * m; e += 32) {
      const int j = e / m, be = e - j * m;
      double2 acc = make_double2(0.0, 0.0);
      for (int row = 0; row < n; ++row) cfmac(acc, Wi[(size_t)row * r + j], Mb[(size_t)row * m + be]);
      carry[e] = acc;
    }
    __syncwarp();
    // site i+1 <- carry . site i+1
    double2* Wn = W + (size_t)(i + 1) * sz;
    for (int e = lane; e < r * d * dn; e += 32) {
      const int j = e / (d * dn), rest = e - j * d * dn;
      double2 acc = make_double2(0.0, 0.0);
      for (int be = 0; be < m; ++be) cfma(acc, carry[(size_t)j * m + be], Wn[(size_t)be * d * dn + rest]);
      tmp[e] = acc;
    }
    __syncwarp();
    for (int e = lane; e < r * d * dn; e += 32) Wn[e] = tmp[e];
    if (lane == 0) D[i + 1] = r;
    __syncwarp();
  }
  {  // normalise the last site
    double2* Wl = W + (size_t)(N - 1) * sz;
    const int cnt = D[N - 1] * d;
    double s = 0.0;
    for (int e = lane; e < cnt; e += 32) s += cabs2(Wl[e]);
    s = warp_sum(s);
    const double inv = rsqrt(s);
    for (int e = lane; e < cnt; e += 32) Wl[e] = cscale(Wl[e], inv);
    __syncwarp();
  }
  // ---- right sweep ----
  unsigned char* slot = a.slots + (size_t)mi * a.L.bytes;
  int* SD = slot_dims(slot);
  double* lam = slot_lam(slot, a.L);
  double2* sites = slot_sites(slot, a.L);
  int cr = 1;  // carry columns (new right dim)
  if (lane == 0) carry[0] = make_double2(1.0, 0.0);
  __syncwarp();
  for (int i = N - 1; i >= 1; --i) {
    const int dl = D[i], dr = D[i + 1];
    double2* Wi = W + (size_t)i * sz;
    const int n = d * cr, m = dl;
    // M[al][s][c] = sum_r Wi[al][s][r] carry[r][c]
    double fro = 0.0;
    for (int e = lane; e < dl * d * cr; e += 32) {
      const int al = e / (d * cr), rest = e - al * d * cr;
      const int s = rest / cr, c = rest - s * cr;
      double2 acc = make_double2(0.0, 0.0);
      for (int r = 0; r < dr; ++r) cfma(acc, Wi[(size_t)al * d * dr + s * dr + r], carry[(size_t)r * cr + c]);
      Mb[e] = acc;
      T[e] = cconj(acc);  // column al of M^dagger, row (s c)
      fro += cabs2(acc);
    }
    fro = warp_sum(fro);
    __syncwarp();
    const int sw = warp_jacobi(T, n, m, fro, cn, lane);
    double gap;
    int k = warp_rank_truncate(T, n, m, a.chi, a.eps, sig2, perm, lane, kept2, tot2, gap);
    if (k > n) k = n;
    if (lane == 0 && sw < 0) atomicOr(a.status, kStatusNoConverge);
    const double inv_kn = rsqrt(kept2);
    double2* Bi = sites + a.site_off[i];
    for (int e = lane; e < k * n; e += 32) {
      const int j = e / n, r = e - j * n;
      Bi[e] = cscale(cconj(T[(size_t)perm[j] * n + r]), rsqrt(sig2[perm[j]]));
    }
    for (int j = lane; j < k; j += 32) lam[(size_t)(i - 1) * a.chi + j] = sqrt(sig2[perm[j]]) * inv_kn;
    // new carry[al][j] = sum_r M[al][r] y_j[r] / |S_k|
    for (int e = lane; e < m * k; e += 32) {
      const int al = e / k, j = e - al * k;
      double2 acc = make_double2(0.0, 0.0);
      for (int r = 0; r < n; ++r) cfma(acc, Mb[(size_t)al * n + r], T[(size_t)perm[j] * n + r]);
      tmp[e] = cscale(acc, rsqrt(sig2[perm[j]]) * inv_kn);
    }
    __syncwarp();
    for (int e = lane; e < m * k; e += 32) carry[e] = tmp[e];
    if (lane == 0) SD[i] = k;
    cr = k;
    __syncwarp();
  }
  {  // B_0 = site 0 . carry, normalised
    const int dr = D[1];
    double2* W0 = W;
    double2* B0 = sites + a.site_off[0];
    double s = 0.0;
    for (int e = lane; e < d * cr; e += 32) {
      const int sidx = e / cr, c = e - sidx * cr;
      double2 acc = make_double2(0.0, 0.0);
      for (int r = 0; r < dr; ++r) cfma(acc, W0[(size_t)sidx * dr + r], carry[(size_t)r * cr + c]);
      tmp[e] = acc;
      s += cabs2(acc);
    }
    s = warp_sum(s);
    const double inv = rsqrt(s);
    __syncwarp();
    for (int e = lane; e < d * cr; e += 32) B0[e] = cscale(tmp[e], inv);
    if (lane == 0) {
      SD[0] = 1;
      SD[N] = 1;
      if (!(s > 0.0) || !(s < 1e300)) atomicOr(a.status, kStatusNaN);
    }
  }
}

}  // namespace tnrc

extern "C" cudaError_t tnrc_launch_canon(const tnrc::CanonArgs* a, int nmps, cudaStream_t st) {
  (void)cudaGetLastError();  // report only this launch below
  tnrc::canon_kernel<<<nmps, 32, 0, st>>>(*a);
  return cudaGetLastError();
}
