// Warp-level one-sided (Hestenes) Jacobi SVD in FP64 -- the truncated SVD of
// the TEBD compression step (Sec. II: "compressed after each time step ...
// using truncated singular-value decomposition").
//
// The matrix is held column-major (column j at T + j*n, n rows).  Its m
// columns are orthogonalised by plane rotations in the round-robin (circle)
// ordering, m/2 disjoint pairs per round, so that a whole round runs in
// parallel: each pair gets g lanes (g * pairs <= 32), each lane owns rows
// lig, lig+g, ...; the three inner products of a pair are reduced over its g
// lanes by shuffles (bitwise identical in every lane, so every lane takes the
// same decision).  After convergence column j equals
// sigma_j y_j with y_j orthonormal: for T = M^dagger, y_j are the right
// singular vectors of M and sigma_j its singular values.
#pragma once
#include "tnrc_device.cuh"

namespace tnrc {

__device__ __forceinline__ void rr_pair(int mp, int r, int q, int& i, int& j) {
  if (q == 0) {
    i = r;
    j = mp - 1;
  } else {
    const int m1 = mp - 1;
    i = (r + q) % m1;
    j = (r - q + m1) % m1;
  }
}

// Sum of v over the g lanes gb .. gb+g-1 of this lane's group (lig = lane -
// gb, gmask = those lanes); every lane of the group receives the same value.
// A power-of-two g uses an xor butterfly; any other g a shift-down tree into
// lane gb and a broadcast from it (a source lane outside the group is never
// added).
__device__ __forceinline__ double group_sum(double v, int g, int lig, int gb, unsigned gmask) {
  if ((g & (g - 1)) == 0) {
    for (int o = g >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(gmask, v, o);
    return v;
  }
  int o = 1;
  while (2 * o < g) o <<= 1;
  for (; o > 0; o >>= 1) {
    const double x = __shfl_down_sync(gmask, v, o);
    if (lig + o < g) v += x;
  }
  return __shfl_sync(gmask, v, gb);
}

__device__ __forceinline__ unsigned group_mask(int g, int gb) {
  return (g >= 32) ? 0xffffffffu : (((1u << g) - 1u) << gb);
}

// FP64 warp instructions of a unit loop that gives g lanes to each of
// `units` units (the trailing columns of a QR step, the pairs of a Jacobi
// round) of `rows` rows on `lanes` lanes: iterations x (rows per lane x
// per_row + fixed + per_level x reduction levels).
__device__ __forceinline__ int unit_loop_cost(int units, int rows, int g, int lanes, int per_row, int fixed,
                                              int per_level) {
  const int gpw = lanes / g;
  const int iters = (units + gpw - 1) / gpw;
  int lv = 0;
  while ((1 << lv) < g) ++lv;
  return iters * (((rows + g - 1) / g) * per_row + fixed + per_level * lv);
}

// Lanes per unit.  With units <= lanes / 2 every unit gets floor(lanes /
// units) lanes in one iteration.  Beyond that one lane per unit leaves lanes
// idle (or takes a second, partly idle iteration), and groups of 2..8 lanes
// over more iterations can cost fewer FP64 warp instructions -- 41 columns
// of 80 rows: 2 iterations of 80 rows on single lanes, or 6 of 20 rows on
// groups of 4 -- so the cheapest by unit_loop_cost is taken when it beats one
// lane per unit by more than 1/16.  The choice depends only on the sizes.
__device__ __forceinline__ int pick_lanes(int units, int rows, int lanes, int per_row, int fixed, int per_level) {
  if (units < 1) return lanes;
  if (2 * units <= lanes) return lanes / units;
  int best = 1;
  int bc = unit_loop_cost(units, rows, 1, lanes, per_row, fixed, per_level);
  const int c1 = bc;
  for (int g = 2; g <= 8; ++g) {
    const int c = unit_loop_cost(units, rows, g, lanes, per_row, fixed, per_level);
    if (c < bc && 16 * c < 15 * c1) {
      bc = c;
      best = g;
    }
  }
  return best;
}

// Per-unit FP64 instruction counts of the two loops (rows: per row of the
// unit; fixed: scalars per unit; level: per level of the group reduction).
constexpr int kQrRow = 11, kQrFixed = 2, kQrLevel = 3;      // QR step: <v, x>, x -= v s, |x|^2
constexpr int kJacRow = 16, kJacFixed = 40, kJacLevel = 2;  // Jacobi round: <a, b>, rotation

// Lanes per unit: one iteration with floor(lanes / units) lanes each (one
// lane per unit from `lanes` units on), or, with kModel, the pick_lanes
// choice.  The qubit-state kernels keep the first (their theta are at most
// 32 rows on the benchmark, where the model's choices measured slower); the
// operator kernels, whose theta are 40 to 80 rows wide, take the model.
template <bool kModel>
__device__ __forceinline__ int lanes_per_unit(int units, int rows, int lanes, int per_row, int fixed,
                                              int per_level) {
  if (kModel) return pick_lanes(units, rows, lanes, per_row, fixed, per_level);
  return units >= lanes ? 1 : lanes / units;
}

// out[c] = |column c|^2 for the m columns of length n of T (column-major),
// with g = 32 / m lanes per column (any g), so that short columns keep most
// lanes busy.
__device__ inline void warp_col_norms(const double2* T, int n, int m, double* out, int lane) {
  const int g = (m >= 32 || m < 1) ? 1 : 32 / m;
  const int gi = lane / g, lig = lane - gi * g, gb = gi * g;
  const int groups = 32 / g;
  const unsigned gmask = group_mask(g, gb);
  for (int c = gi; c < m && gi < groups; c += groups) {
    const double2* col = T + (size_t)c * n;
    double s = 0.0;
    for (int row = lig; row < n; row += g) s = fma(col[row].x, col[row].x, fma(col[row].y, col[row].y, s));
    if (g > 1) s = group_sum(s, g, lig, gb, gmask);
    if (lig == 0) out[c] = s;
  }
  __syncwarp();
}

// Returns the number of sweeps (the last one made no rotation, or only
// rotations with |cos| <= 1e-10 between the pair's columns), or -kMaxSweeps
// when the sweep limit was reached.  fro2 = squared Frobenius norm of T;
// cn: shared scratch of m doubles holding the column norms squared.
//
// Lanes per pair: an odd m is padded with a zero column, which the circle
// ordering pairs with a different real column in every round (pair q = 0);
// that pair needs no work, so the Pe = floor(m / 2) real pairs of a round
// share the 32 lanes, g = lanes_per_unit(Pe, n) each (floor(32 / Pe), or
// the instruction-count choice with kModel; not necessarily a power of two).
// Each lane then owns ceil(n / g) rows of its pair.
//
// The norms are computed exactly before the first sweep and in the first
// round of every sweep (where the pair's lanes form all three inner
// products); in the other rounds only <a, b> is formed and the norms are
// carried through each rotation by |a'|^2 = |a|^2 - t |<a,b>|,
// |b'|^2 = |b|^2 + t |<a,b>| (t = tan theta), recomputed from the rotated
// column should a norm fall below 1/16 of its old value (cancellation).
template <bool kModel = false>
__device__ inline int warp_jacobi(double2* T, int n, int m, double fro2, double* cn, int lane) {
  const int mp = m + (m & 1);
  if (mp < 2 || n < 1) return 0;
  const int P = mp >> 1;
  const int q0 = m & 1;          // pair 0 holds the padding column of an odd m
  const int Pe = P - q0;         // real pairs per round
  if (Pe < 1) return 1;          // a single column is already orthogonal
  const int g = lanes_per_unit<kModel>(Pe, n, 32, kJacRow, kJacFixed, kJacLevel);
  const int groups = 32 / g;
  const int gi = lane / g, lig = lane - gi * g, gb = gi * g;
  const unsigned gmask = group_mask(g, gb);
  const double thr = kJacobiZero * kJacobiZero * fro2;
  const double tol = 2.0 * (double)(m > n ? m : n) * 2.220446049250313e-16;
  const double tol2 = tol * tol;
  warp_col_norms(T, n, m, cn, lane);
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    int rotated = 0, large = 0;
    for (int r = 0; r < mp - 1; ++r) {
      for (int q = q0 + gi; q < P && gi < groups; q += groups) {
        int i, j;
        rr_pair(mp, r, q, i, j);
        double2* a = T + (size_t)i * n;
        double2* b = T + (size_t)j * n;
        double aa, bb;
        double2 ab = make_double2(0.0, 0.0);
        if (r == 0) {
          aa = 0.0;
          bb = 0.0;
          for (int row = lig; row < n; row += g) {
            const double2 x = a[row], y = b[row];
            aa = fma(x.x, x.x, fma(x.y, x.y, aa));
            bb = fma(y.x, y.x, fma(y.y, y.y, bb));
            cfmac(ab, x, y);
          }
          if (g > 1) {
            aa = group_sum(aa, g, lig, gb, gmask);
            bb = group_sum(bb, g, lig, gb, gmask);
            ab.x = group_sum(ab.x, g, lig, gb, gmask);
            ab.y = group_sum(ab.y, g, lig, gb, gmask);
          }
        } else {
          aa = cn[i];
          bb = cn[j];
          for (int row = lig; row < n; row += g) cfmac(ab, a[row], b[row]);
          if (g > 1) {
            ab.x = group_sum(ab.x, g, lig, gb, gmask);
            ab.y = group_sum(ab.y, g, lig, gb, gmask);
          }
        }
        double na = aa, nb = bb;
        const double ab2 = cabs2(ab);
        const double pab = aa * bb;
        if (aa > thr && bb > thr && ab2 > tol2 * pab) {
          rotated = 1;
          large |= (ab2 > kJacobiQuad * pab) ? 1 : 0;
          // Real rotation of the pair after the phase of <a,b> is divided out,
          // cot(2 theta) = (|b|^2 - |a|^2) / (2 |<a,b>|).  With d = |b|^2 - |a|^2
          // and w = 1 / sqrt(d^2 + 4 |<a,b>|^2): cos 2theta = |d| w,
          // sin 2theta = 2 |<a,b>| w, c = sqrt((1 + cos 2theta) / 2) and
          // s e^{i phi} = sign(d) w / sqrt((1 + cos 2theta) / 2) <a,b> -- two
          // reciprocal square roots, no division, no cancellation.
          const double d = bb - aa;
          const double w = rsqrt(fma(d, d, 4.0 * ab2));
          const double hq = fma(0.5, fabs(d) * w, 0.5);   // c^2
          const double rc = rsqrt(hq);
          const double c = hq * rc;
          const double f = copysign(w * rc, d);
          const double2 sp = make_double2(f * ab.x, f * ab.y);  // s e^{i phi}
          // a <- c a - conj(sp) b ;  b <- c b + sp a
          for (int row = lig; row < n; row += g) {
            const double2 x = a[row], y = b[row];
            double2 na_ = cscale(x, c);
            na_.x = fma(-sp.x, y.x, na_.x);
            na_.x = fma(-sp.y, y.y, na_.x);
            na_.y = fma(-sp.x, y.y, na_.y);
            na_.y = fma(sp.y, y.x, na_.y);
            double2 nb_ = cscale(y, c);
            cfma(nb_, sp, x);
            a[row] = na_;
            b[row] = nb_;
          }
          // t |<a,b>| = sign(d) 2 |<a,b>|^2 w; c^2 = hq, s^2 = 1 - hq
          const double dl = copysign(2.0 * ab2 * w, d);
          na = fma(hq, aa, fma(1.0 - hq, bb, -dl));
          nb = fma(hq, bb, fma(1.0 - hq, aa, dl));
          if (na < 0.0625 * aa) {
            na = 0.0;
            for (int row = lig; row < n; row += g) na = fma(a[row].x, a[row].x, fma(a[row].y, a[row].y, na));
            if (g > 1) na = group_sum(na, g, lig, gb, gmask);
          }
          if (nb < 0.0625 * bb) {
            nb = 0.0;
            for (int row = lig; row < n; row += g) nb = fma(b[row].x, b[row].x, fma(b[row].y, b[row].y, nb));
            if (g > 1) nb = group_sum(nb, g, lig, gb, gmask);
          }
        }
        if (lig == 0) {
          cn[i] = na;
          cn[j] = nb;
        }
      }
      __syncwarp();
    }
    // converged: a sweep without rotations -- or one whose rotations all had
    // |cos| <= 1e-10 between the pair's columns, after which (the cyclic
    // method converging quadratically) the next sweep would find every
    // |cos| near 1e-20, far below tol, and rotate nothing
    if (!__any_sync(0xffffffffu, rotated) || !__any_sync(0xffffffffu, large)) return sweep + 1;
  }
  return -kMaxSweeps;
}

// Householder QR with column pivoting, W P = Q R, of the m x n matrix W held
// row-major (row i at W + i*n), by one warp; Q is not formed.  This is the
// preconditioner of Drmac and Veselic ("New fast and accurate Jacobi SVD
// algorithm", SIAM J. Matrix Anal. Appl. 29, 2008): one-sided Jacobi applied
// to the columns of R^dagger converges in fewer sweeps than on the original
// matrix, and R^dagger has only r columns where r is the numerical rank.
//
// Step j takes the remaining column of largest norm as pivot; when that norm
// squared is <= thr, every remaining column is below it and the
// factorisation stops with r = j.  The trailing columns of a step are shared
// out to groups of G = lanes_per_unit(columns, rows) lanes (floor(32 /
// columns), or the instruction-count choice with kModel), each group's lanes
// splitting the rows; the trailing column norms are recomputed exactly while
// the reflector is applied,
// so the pivot choice needs no norm downdating.  Reductions within a group
// leave the same sums in every lane of the group, and the pivot
// reduction (integer comparisons of the non-negative norms' bit patterns, ties
// to the smaller index) gives every lane the same pivot.
//
// On return rows 0..r-1 of W hold R (zeros below the diagonal; row j is the
// j-th row of R in the pivoted column order), piv[c] is the original index of
// pivoted column c (c < n), and qn (n doubles) has been used as scratch.
template <bool kModel = false>
__device__ inline int warp_qrcp(double2* W, int m, int n, double thr, int* piv, double* qn, int lane) {
  {
    const int G = n >= 32 ? 1 : 32 / n;
    const int groups = 32 / G;
    const int gi = lane / G, lig = lane - gi * G, gb = gi * G;
    const unsigned gmask = group_mask(G, gb);
    for (int c = gi; c < n && gi < groups; c += groups) {
      double q = 0.0;
      for (int i = lig; i < m; i += G) q += cabs2(W[(size_t)i * n + c]);
      if (G > 1) q = group_sum(q, G, lig, gb, gmask);
      if (lig == 0) {
        qn[c] = q;
        piv[c] = c;
      }
    }
  }
  __syncwarp();
  const int steps = m < n ? m : n;
  for (int j = 0; j < steps; ++j) {
    // pivot: the column c >= j of largest remaining norm
    long long best = -1;
    int bi = n;
    for (int c = j + lane; c < n; c += 32) {
      const long long v = __double_as_longlong(qn[c]);
      if (v > best) {
        best = v;
        bi = c;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    const double xn2 = __longlong_as_double(best);
    if (!(xn2 > thr)) return j;
    if (bi != j) {
      for (int i = lane; i < m; i += 32) {
        const double2 t = W[(size_t)i * n + j];
        W[(size_t)i * n + j] = W[(size_t)i * n + bi];
        W[(size_t)i * n + bi] = t;
      }
      if (lane == 0) {
        const int tp = piv[j];
        piv[j] = piv[bi];
        piv[bi] = tp;
        qn[bi] = qn[j];
        qn[j] = xn2;
      }
      __syncwarp();
    }
    // reflector H = I - beta v v^dag mapping column j (rows j..m-1) to alpha e_j:
    // alpha = -e^{i arg x0} |x|, v = x - alpha e_j, beta = 1 / (|x| (|x| + |x0|))
    const double2 x0 = W[(size_t)j * n + j];
    const double xn = sqrt(xn2);
    const double ax0 = sqrt(cabs2(x0));
    const double2 ph = (ax0 > 0.0) ? cscale(x0, 1.0 / ax0) : make_double2(1.0, 0.0);
    const double2 v0 = cscale(ph, ax0 + xn);
    const double beta = 1.0 / (xn * (xn + ax0));
    // the na = n - j - 1 trailing columns share the 32 lanes, G =
    // lanes_per_unit(na, m - j) lanes each (any G), so that the lanes stay busy
    // as the columns run out
    const int na = n - j - 1;
    if (na > 0) {
      const int G = lanes_per_unit<kModel>(na, m - j, 32, kQrRow, kQrFixed, kQrLevel);
      const int groups = 32 / G;
      const int gi = lane / G, lig = lane - gi * G, gb = gi * G;
      const unsigned gmask = group_mask(G, gb);
      for (int c = j + 1 + gi; c < n && gi < groups; c += groups) {
        double2 s = make_double2(0.0, 0.0);
        for (int i = j + lig; i < m; i += G) {
          const double2 vi = (i == j) ? v0 : W[(size_t)i * n + j];
          cfmac(s, vi, W[(size_t)i * n + c]);
        }
        if (G > 1) {
          s.x = group_sum(s.x, G, lig, gb, gmask);
          s.y = group_sum(s.y, G, lig, gb, gmask);
        }
        s = cscale(s, beta);
        double q = 0.0;
        for (int i = j + lig; i < m; i += G) {
          const double2 vi = (i == j) ? v0 : W[(size_t)i * n + j];
          double2 x = W[(size_t)i * n + c];
          x.x = fma(-vi.x, s.x, x.x);
          x.x = fma(vi.y, s.y, x.x);
          x.y = fma(-vi.x, s.y, x.y);
          x.y = fma(-vi.y, s.x, x.y);
          W[(size_t)i * n + c] = x;
          if (i > j) q += cabs2(x);
        }
        if (G > 1) q = group_sum(q, G, lig, gb, gmask);
        if (lig == 0) qn[c] = q;
      }
    }
    __syncwarp();
    for (int i = j + lane; i < m; i += 32)
      W[(size_t)i * n + j] = (i == j) ? make_double2(-xn * ph.x, -xn * ph.y) : make_double2(0.0, 0.0);
    __syncwarp();
  }
  return steps;
}

// The second QR of the Drmac-Veselic preconditioner, taken here to shorten
// the columns the Jacobi works on.  X = R^dagger (n x r, column-major, column
// j at X + j n) is factorised X = Q2 R2 by Householder reflections without
// pivoting; R2 (r x r, upper triangular) is written column-major to R2 with
// zeros below the diagonal, and Q2 (n x r, orthonormal columns) overwrites X.
// X and R2 have the same Gram matrix (X^dag X = R2^dag R2), so one-sided
// Jacobi on the r columns of R2 makes the same rotations as on X, on columns
// of length r instead of n: R2 V = Z2 S gives X V = (Q2 Z2) S.  vh (r
// complex) and beta (r doubles) are shared scratch.
template <bool kModel>
static __device__ __noinline__ void warp_qr_rows(double2* X, int n, int r, double2* R2, double2* vh, double* beta,
                                                int lane) {
  for (int j = 0; j < r; ++j) {
    double2* xj = X + (size_t)j * n;
    double s = 0.0;
    for (int i = j + lane; i < n; i += 32) s += cabs2(xj[i]);
    const double xn2 = warp_sum(s);
    // reflector H_j = I - beta v v^dag mapping rows j..n-1 of column j to
    // alpha e_j: alpha = -e^{i arg x0} |x|, v = x - alpha e_j
    const double2 x0 = xj[j];
    const double xn = sqrt(xn2);
    const double ax0 = sqrt(cabs2(x0));
    const double2 ph = (ax0 > 0.0) ? cscale(x0, 1.0 / ax0) : make_double2(1.0, 0.0);
    const double2 v0 = cscale(ph, ax0 + xn);
    const double bt = (xn > 0.0) ? 1.0 / (xn * (xn + ax0)) : 0.0;
    const int na = r - j - 1;
    if (na > 0) {
      const int G = lanes_per_unit<kModel>(na, n - j, 32, kQrRow - 3, kQrFixed, 2);
      const int groups = 32 / G;
      const int gi = lane / G, lig = lane - gi * G, gb = gi * G;
      const unsigned gmask = group_mask(G, gb);
      for (int c = j + 1 + gi; c < r && gi < groups; c += groups) {
        double2* xc = X + (size_t)c * n;
        double2 sc = make_double2(0.0, 0.0);
        for (int i = j + lig; i < n; i += G) cfmac(sc, (i == j) ? v0 : xj[i], xc[i]);
        if (G > 1) {
          sc.x = group_sum(sc.x, G, lig, gb, gmask);
          sc.y = group_sum(sc.y, G, lig, gb, gmask);
        }
        sc = cscale(sc, bt);
        for (int i = j + lig; i < n; i += G) {
          const double2 vi = (i == j) ? v0 : xj[i];
          double2 x = xc[i];
          x.x = fma(-vi.x, sc.x, x.x);
          x.x = fma(vi.y, sc.y, x.x);
          x.y = fma(-vi.x, sc.y, x.y);
          x.y = fma(-vi.y, sc.x, x.y);
          xc[i] = x;
        }
      }
    }
    __syncwarp();
    if (lane == 0) {
      vh[j] = v0;
      beta[j] = bt;
      xj[j] = make_double2(-xn * ph.x, -xn * ph.y);   // R2[j][j]; rows below keep v's tail
    }
    __syncwarp();
  }
  for (int e = lane; e < r * r; e += 32) {
    const int c = e / r, i = e - c * r;
    R2[e] = (i <= c) ? X[(size_t)c * n + i] : make_double2(0.0, 0.0);
  }
  __syncwarp();
  // Q2 = H_0 H_1 ... H_{r-1} [I_r; 0] in place, from the last reflector back:
  // before step j, column c > j holds H_{j+1} .. H_{r-1} e_c (zero above row
  // j+1) and column j still holds v's tail; step j applies H_j to the columns
  // c > j, then writes H_j e_j over column j.
  for (int j = r - 1; j >= 0; --j) {
    double2* xj = X + (size_t)j * n;
    const double2 v0 = vh[j];
    const double bt = beta[j];
    const int na = r - j - 1;
    if (na > 0) {
      const int G = lanes_per_unit<kModel>(na, n - j, 32, kQrRow - 3, kQrFixed, 2);
      const int groups = 32 / G;
      const int gi = lane / G, lig = lane - gi * G, gb = gi * G;
      const unsigned gmask = group_mask(G, gb);
      for (int c = j + 1 + gi; c < r && gi < groups; c += groups) {
        double2* xc = X + (size_t)c * n;
        double2 sc = make_double2(0.0, 0.0);
        for (int i = j + lig; i < n; i += G) cfmac(sc, (i == j) ? v0 : xj[i], xc[i]);
        if (G > 1) {
          sc.x = group_sum(sc.x, G, lig, gb, gmask);
          sc.y = group_sum(sc.y, G, lig, gb, gmask);
        }
        sc = cscale(sc, bt);
        for (int i = j + lig; i < n; i += G) {
          const double2 vi = (i == j) ? v0 : xj[i];
          double2 x = xc[i];
          x.x = fma(-vi.x, sc.x, x.x);
          x.x = fma(vi.y, sc.y, x.x);
          x.y = fma(-vi.x, sc.y, x.y);
          x.y = fma(-vi.y, sc.x, x.y);
          xc[i] = x;
        }
      }
    }
    __syncwarp();
    // H_j e_j = e_j - beta v conj(v_j): zero above row j
    for (int i = lane; i < n; i += 32) {
      double2 q = make_double2(0.0, 0.0);
      if (i == j) {
        q = make_double2(1.0 - bt * cabs2(v0), 0.0);
      } else if (i > j) {
        const double2 vi = xj[i];
        q = make_double2(-bt * (vi.x * v0.x + vi.y * v0.y), -bt * (vi.y * v0.x - vi.x * v0.y));
      }
      xj[i] = q;
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Two matrices per warp.  For small matrices a Jacobi round costs mostly its
// per-pair scalars (inner products reduced, two reciprocal square roots, the
// norm updates), which every lane of a pair's group computes: with few pairs
// per round most of a round's FP64 instructions are that fixed part.  Two
// matrices on the two half-warps share those instructions -- the halves run
// the same instruction stream on different data -- at the price of twice
// the rows per lane.  Lane hb + ll (hb = 0 or 16, ll < 16) works on the
// matrix of its half; every loop containing a warp-wide barrier runs to the
// larger of the two trip counts, the half that is done idling.
// ---------------------------------------------------------------------------

__device__ inline void half_col_norms(const double2* T, int n, int m, double* out, int ll, int hb) {
  const int g = (m >= 16 || m < 1) ? 1 : 16 / m;
  const int gi = ll / g, lig = ll - gi * g, gb = hb + gi * g;
  const int groups = 16 / g;
  const unsigned gmask = group_mask(g, gb);
  for (int c = gi; c < m && gi < groups; c += groups) {
    const double2* col = T + (size_t)c * n;
    double s = 0.0;
    for (int row = lig; row < n; row += g) s = fma(col[row].x, col[row].x, fma(col[row].y, col[row].y, s));
    if (g > 1) s = group_sum(s, g, lig, gb, gmask);
    if (lig == 0) out[c] = s;
  }
}

// warp_qrcp on each half's matrix (W m x n row-major, thr, piv, qn its own);
// returns this half's numerical rank.
template <bool kModel = false>
__device__ inline int half_qrcp(double2* W, int m, int n, double thr, int* piv, double* qn, int lane) {
  const int hb = lane & 16, ll = lane & 15;
  const unsigned hmask = 0xffffu << hb;
  {
    const int G = n >= 16 ? 1 : 16 / n;
    const int groups = 16 / G;
    const int gi = ll / G, lig = ll - gi * G, gb = hb + gi * G;
    const unsigned gmask = group_mask(G, gb);
    for (int c = gi; c < n && gi < groups; c += groups) {
      double q = 0.0;
      for (int i = lig; i < m; i += G) q += cabs2(W[(size_t)i * n + c]);
      if (G > 1) q = group_sum(q, G, lig, gb, gmask);
      if (lig == 0) {
        qn[c] = q;
        piv[c] = c;
      }
    }
  }
  __syncwarp();
  const int steps_own = m < n ? m : n;
  const int steps = __reduce_max_sync(0xffffffffu, (unsigned)steps_own);
  int rank = steps_own;
  bool done = false;
  for (int j = 0; j < steps; ++j) {
    done = done || (j >= steps_own);
    // pivot: the column c >= j of largest remaining norm (within the half)
    long long best = -1;
    int bi = n;
    if (!done) {
      for (int c = j + ll; c < n; c += 16) {
        const long long v = __double_as_longlong(qn[c]);
        if (v > best) {
          best = v;
          bi = c;
        }
      }
    }
    for (int o = 8; o > 0; o >>= 1) {
      const long long ov = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    const double xn2 = __longlong_as_double(best);
    if (!done && !(xn2 > thr)) {
      rank = j;
      done = true;
    }
    if (!done && bi != j) {
      for (int i = ll; i < m; i += 16) {
        const double2 t = W[(size_t)i * n + j];
        W[(size_t)i * n + j] = W[(size_t)i * n + bi];
        W[(size_t)i * n + bi] = t;
      }
      if (ll == 0) {
        const int tp = piv[j];
        piv[j] = piv[bi];
        piv[bi] = tp;
        qn[bi] = qn[j];
        qn[j] = xn2;
      }
    }
    __syncwarp();
    double xn = 0.0;
    double2 ph = make_double2(1.0, 0.0);
    if (!done) {
      const double2 x0 = W[(size_t)j * n + j];
      xn = sqrt(xn2);
      const double ax0 = sqrt(cabs2(x0));
      ph = (ax0 > 0.0) ? cscale(x0, 1.0 / ax0) : make_double2(1.0, 0.0);
      const double2 v0 = cscale(ph, ax0 + xn);
      const double beta = 1.0 / (xn * (xn + ax0));
      const int na = n - j - 1;
      if (na > 0) {
        const int G = lanes_per_unit<kModel>(na, m - j, 16, kQrRow, kQrFixed, kQrLevel);
        const int groups = 16 / G;
        const int gi = ll / G, lig = ll - gi * G, gb = hb + gi * G;
        const unsigned gmask = group_mask(G, gb);
        for (int c = j + 1 + gi; c < n && gi < groups; c += groups) {
          double2 sacc = make_double2(0.0, 0.0);
          for (int i = j + lig; i < m; i += G) {
            const double2 vi = (i == j) ? v0 : W[(size_t)i * n + j];
            cfmac(sacc, vi, W[(size_t)i * n + c]);
          }
          if (G > 1) {
            sacc.x = group_sum(sacc.x, G, lig, gb, gmask);
            sacc.y = group_sum(sacc.y, G, lig, gb, gmask);
          }
          sacc = cscale(sacc, beta);
          double q = 0.0;
          for (int i = j + lig; i < m; i += G) {
            const double2 vi = (i == j) ? v0 : W[(size_t)i * n + j];
            double2 x = W[(size_t)i * n + c];
            x.x = fma(-vi.x, sacc.x, x.x);
            x.x = fma(vi.y, sacc.y, x.x);
            x.y = fma(-vi.x, sacc.y, x.y);
            x.y = fma(-vi.y, sacc.x, x.y);
            W[(size_t)i * n + c] = x;
            if (i > j) q += cabs2(x);
          }
          if (G > 1) q = group_sum(q, G, lig, gb, gmask);
          if (lig == 0) qn[c] = q;
        }
      }
    }
    __syncwarp();
    if (!done)
      for (int i = j + ll; i < m; i += 16)
        W[(size_t)i * n + j] = (i == j) ? make_double2(-xn * ph.x, -xn * ph.y) : make_double2(0.0, 0.0);
    __syncwarp();
  }
  (void)hmask;
  return rank;
}

// warp_jacobi on each half's matrix (T n x m column-major, fro2, cn its own);
// returns this half's sweep count (or -kMaxSweeps).
template <bool kModel = false>
__device__ inline int half_jacobi(double2* T, int n, int m, double fro2, double* cn, int lane) {
  const int hb = lane & 16, ll = lane & 15;
  const unsigned hmask = 0xffffu << hb;
  const int mp = m + (m & 1);
  const int P = mp >> 1;
  const int q0 = m & 1;
  const int Pe = P - q0;
  const bool trivial = (mp < 2 || n < 1 || Pe < 1);
  const int g = trivial ? 1 : lanes_per_unit<kModel>(Pe, n, 16, kJacRow, kJacFixed, kJacLevel);
  const int groups = 16 / g;
  const int gi = ll / g, lig = ll - gi * g, gb = hb + gi * g;
  const unsigned gmask = group_mask(g, gb);
  const double thr = kJacobiZero * kJacobiZero * fro2;
  const double tol = 2.0 * (double)(m > n ? m : n) * 2.220446049250313e-16;
  const double tol2 = tol * tol;
  if (!trivial) half_col_norms(T, n, m, cn, ll, hb);
  __syncwarp();
  const int rounds = __reduce_max_sync(0xffffffffu, (unsigned)(trivial ? 0 : mp - 1));
  bool active = !trivial;
  int result = trivial ? ((mp < 2 || n < 1) ? 0 : 1) : -kMaxSweeps;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    if (!__any_sync(0xffffffffu, active)) break;
    int rotated = 0, large = 0;
    for (int r = 0; r < rounds; ++r) {
      if (active && r < mp - 1) {
        for (int q = q0 + gi; q < P && gi < groups; q += groups) {
          int i, j;
          rr_pair(mp, r, q, i, j);
          double2* a = T + (size_t)i * n;
          double2* b = T + (size_t)j * n;
          double aa, bb;
          double2 ab = make_double2(0.0, 0.0);
          if (r == 0) {
            aa = 0.0;
            bb = 0.0;
            for (int row = lig; row < n; row += g) {
              const double2 x = a[row], y = b[row];
              aa = fma(x.x, x.x, fma(x.y, x.y, aa));
              bb = fma(y.x, y.x, fma(y.y, y.y, bb));
              cfmac(ab, x, y);
            }
            if (g > 1) {
              aa = group_sum(aa, g, lig, gb, gmask);
              bb = group_sum(bb, g, lig, gb, gmask);
              ab.x = group_sum(ab.x, g, lig, gb, gmask);
              ab.y = group_sum(ab.y, g, lig, gb, gmask);
            }
          } else {
            aa = cn[i];
            bb = cn[j];
            for (int row = lig; row < n; row += g) cfmac(ab, a[row], b[row]);
            if (g > 1) {
              ab.x = group_sum(ab.x, g, lig, gb, gmask);
              ab.y = group_sum(ab.y, g, lig, gb, gmask);
            }
          }
          double na = aa, nb = bb;
          const double ab2 = cabs2(ab);
          const double pab = aa * bb;
          if (aa > thr && bb > thr && ab2 > tol2 * pab) {
            rotated = 1;
            large |= (ab2 > kJacobiQuad * pab) ? 1 : 0;
            const double d = bb - aa;
            const double w = rsqrt(fma(d, d, 4.0 * ab2));
            const double hq = fma(0.5, fabs(d) * w, 0.5);   // c^2
            const double rc = rsqrt(hq);
            const double c = hq * rc;
            const double f = copysign(w * rc, d);
            const double2 sp = make_double2(f * ab.x, f * ab.y);
            for (int row = lig; row < n; row += g) {
              const double2 x = a[row], y = b[row];
              double2 na_ = cscale(x, c);
              na_.x = fma(-sp.x, y.x, na_.x);
              na_.x = fma(-sp.y, y.y, na_.x);
              na_.y = fma(-sp.x, y.y, na_.y);
              na_.y = fma(sp.y, y.x, na_.y);
              double2 nb_ = cscale(y, c);
              cfma(nb_, sp, x);
              a[row] = na_;
              b[row] = nb_;
            }
            const double dl = copysign(2.0 * ab2 * w, d);
            na = fma(hq, aa, fma(1.0 - hq, bb, -dl));
            nb = fma(hq, bb, fma(1.0 - hq, aa, dl));
            if (na < 0.0625 * aa) {
              na = 0.0;
              for (int row = lig; row < n; row += g) na = fma(a[row].x, a[row].x, fma(a[row].y, a[row].y, na));
              if (g > 1) na = group_sum(na, g, lig, gb, gmask);
            }
            if (nb < 0.0625 * bb) {
              nb = 0.0;
              for (int row = lig; row < n; row += g) nb = fma(b[row].x, b[row].x, fma(b[row].y, b[row].y, nb));
              if (g > 1) nb = group_sum(nb, g, lig, gb, gmask);
            }
          }
          if (lig == 0) {
            cn[i] = na;
            cn[j] = nb;
          }
        }
      }
      __syncwarp();
    }
    // per half: converged after a sweep without rotations, or with only tiny ones
    const unsigned rot = __ballot_sync(0xffffffffu, rotated) & hmask;
    const unsigned big = __ballot_sync(0xffffffffu, large) & hmask;
    if (active && (rot == 0u || big == 0u)) {
      active = false;
      result = sweep + 1;
    }
  }
  return result;
}

// Column norms, ranking and the truncation decision after warp_jacobi.
// sig2[j] = |column j|^2 (j < m); perm[i] = column of rank i (i <= k, i < m),
// ranks by decreasing sigma with ties broken by the smaller index.  Returns
// k = max(1, min(kcap, #{sigma_j > eps sigma_max})); kept2 / tot2 receive the
// squared norms of the kept values and of all values.  When the cap decided
// the cut (more than kcap values above the cutoff), gap = (sigma_(k) -
// sigma_(k+1)) / sigma_max, the relative distance between the last kept and
// the first dropped value; otherwise gap = -1.
__device__ inline int warp_rank_truncate(const double2* T, int n, int m, int kcap, double eps, double* sig2,
                                  int* perm, int lane, double& kept2, double& tot2, double& gap) {
  warp_col_norms(T, n, m, sig2, lane);
  double mx = 0.0, tot = 0.0;
  for (int j = lane; j < m; j += 32) {
    mx = fmax(mx, sig2[j]);
    tot += sig2[j];
  }
  mx = warp_max(mx);
  tot = warp_sum(tot);
  const double cut2 = eps * eps * mx;
  int cnt = 0;
  for (int j = lane; j < m; j += 32) cnt += (sig2[j] > cut2) ? 1 : 0;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  int k = cnt < kcap ? cnt : kcap;
  if (k > n) k = n;  // at most n orthogonal columns of length n
  if (k < 1) k = 1;
  for (int j = lane; j < m; j += 32) {
    const long long vj = __double_as_longlong(sig2[j]);
    int rk = 0;
    for (int i = 0; i < m; ++i) {
      const long long vi = __double_as_longlong(sig2[i]);
      rk += (vi > vj || (vi == vj && i < j)) ? 1 : 0;
    }
    if (rk <= k) perm[rk] = j;
  }
  __syncwarp();
  double kn = 0.0;
  for (int i = lane; i < k; i += 32) kn += sig2[perm[i]];
  kept2 = warp_sum(kn);
  tot2 = tot;
  gap = (cnt > k && k < m) ? (sqrt(sig2[perm[k - 1]]) - sqrt(sig2[perm[k]])) / sqrt(mx) : -1.0;
  return k;
}

}  // namespace tnrc
