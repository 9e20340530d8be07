// Layer gate table of the truncated TEBD layers, and the noise realisations.
//
// layer_gate_kernel: one thread per (sample s, truncated layer l, bond b of
// that layer).  The layer's gate on bond b is a product of factors
// exp(-i tau h_f) (time order f = 1..F), each h_f Hermitian and linear in the
// controls it contains:
//   second order  (A(dts/2) B(dts) A(dts/2) per Trotter step, dts = dt/n_sub):
//     one factor h_b = c ZZ + J^x XX + J^y YY + wL (x_b X + y_b Y) (x) I
//                      + wR I (x) (x_{b+1} X + y_{b+1} Y)          (Eq. sysH, Eq. Hp)
//     with tau = dts (odd bonds) or dts/2 (even bonds), or two such half-step
//     factors where a step boundary merges them;
//   first order   (Eq. circuit): the interaction c ZZ + J^x XX + J^y YY with
//     tau = dts, followed on the bond that carries them by the single-site
//     rotations y Y then x X of its sites;
// c = g_b (if a control) + gfix_{k,b} + J^z(s)_b.  Each factor is diagonalised
// by cyclic complex Jacobi rotations (FP64); the gate is the product and, for
// every control u, Q_u = sum_f L_f (dG_f/du) G_f^dag L_f^dag (L_f the factors
// after f) with dG_f/du by the Daleckii-Krein formula
//   dG = V (Gam o (V^dag P V)) V^dag,  Gam_jk = -i tau e^{-i tau (l_j + l_k)/2} sinc(tau (l_j - l_k)/2),
// P = dh_f/du.  The trajectory kernel then needs only tr(Q_u rho) per control.
//
// noise_kernel: J^(s)_b from the counter-based SplitMix64 generator (Steele,
// Lea, Flood 2014): out(i) = mix(seed + (i+1) * 0x9E3779B97F4A7C15).
#include "tnrc_device.cuh"

namespace tnrc {

__device__ __forceinline__ void herm_rotate(double2 (&h)[16], double2 (&V)[16], int p, int q) {
  const double2 z = h[p * 4 + q];
  const double az2 = cabs2(z);
  if (az2 == 0.0) return;
  const double inv = rsqrt(az2);
  const double2 ph = make_double2(z.x * inv, z.y * inv);  // e^{i phi}
  const double a = h[p * 4 + p].x, d = h[q * 4 + q].x;
  const double zeta = (d - a) * 0.5 * inv;
  double t;
  if (fabs(zeta) > 1e150)
    t = 0.5 / zeta;
  else
    t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
  const double c = rsqrt(fma(t, t, 1.0));
  const double s = c * t;
  // U = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on (p, q):  h <- U^dag h U,  V <- V U
  const double2 u00 = make_double2(c, 0.0), u01 = make_double2(s, 0.0);
  const double2 u10 = make_double2(-s * ph.x, s * ph.y);
  const double2 u11 = make_double2(c * ph.x, -c * ph.y);
#pragma unroll
  for (int r = 0; r < 4; ++r) {  // columns
    const double2 hp = h[r * 4 + p], hq = h[r * 4 + q];
    double2 np = cmul(hp, u00), nq = cmul(hp, u01);
    cfma(np, hq, u10);
    cfma(nq, hq, u11);
    h[r * 4 + p] = np;
    h[r * 4 + q] = nq;
    const double2 vp = V[r * 4 + p], vq = V[r * 4 + q];
    double2 wp = cmul(vp, u00), wq = cmul(vp, u01);
    cfma(wp, vq, u10);
    cfma(wq, vq, u11);
    V[r * 4 + p] = wp;
    V[r * 4 + q] = wq;
  }
#pragma unroll
  for (int cidx = 0; cidx < 4; ++cidx) {  // rows
    const double2 hp = h[p * 4 + cidx], hq = h[q * 4 + cidx];
    double2 np = make_double2(0.0, 0.0), nq = make_double2(0.0, 0.0);
    cfmac(np, u00, hp);
    cfmac(np, u10, hq);
    cfmac(nq, u01, hp);
    cfmac(nq, u11, hq);
    h[p * 4 + cidx] = np;
    h[q * 4 + cidx] = nq;
  }
  h[p * 4 + q] = make_double2(0.0, 0.0);
  h[q * 4 + p] = make_double2(0.0, 0.0);
  h[p * 4 + p].y = 0.0;
  h[q * 4 + q].y = 0.0;
}

// Hermitian 4x4 eigendecomposition h = V diag(lam) V^dag by cyclic Jacobi
// rotations; h is overwritten.  Returns false if it did not converge.
__device__ bool herm_eig4(double2 (&h)[16], double2 (&V)[16], double (&lam)[4]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) V[i] = make_double2((i % 5 == 0) ? 1.0 : 0.0, 0.0);
  double scale2 = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) scale2 += cabs2(h[i]);
  const double stop2 = 1e-32 * scale2;
  bool ok = false;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off2 = 0.0;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = p + 1; q < 4; ++q) off2 += cabs2(h[p * 4 + q]);
    if (off2 <= stop2) {
      ok = true;
      break;
    }
    herm_rotate(h, V, 0, 1);
    herm_rotate(h, V, 2, 3);
    herm_rotate(h, V, 0, 2);
    herm_rotate(h, V, 1, 3);
    herm_rotate(h, V, 0, 3);
    herm_rotate(h, V, 1, 2);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) lam[j] = h[j * 5].x;
  return ok;
}

// Generators in the bond basis |s_b s_{b+1}> (index 2 s_b + s_{b+1}), scaled by w:
// 0: X (x) I, 1: Y (x) I, 2: I (x) X, 3: I (x) Y, 4: Z (x) Z.
__device__ void generator4(int code, double w, double2 (&P)[16]) {
#pragma unroll
  for (int i = 0; i < 16; ++i) P[i] = make_double2(0.0, 0.0);
  switch (code) {
    case 0:
      P[0 * 4 + 2].x = w; P[1 * 4 + 3].x = w; P[2 * 4 + 0].x = w; P[3 * 4 + 1].x = w;
      break;
    case 1:
      P[0 * 4 + 2].y = -w; P[1 * 4 + 3].y = -w; P[2 * 4 + 0].y = w; P[3 * 4 + 1].y = w;
      break;
    case 2:
      P[0 * 4 + 1].x = w; P[1 * 4 + 0].x = w; P[2 * 4 + 3].x = w; P[3 * 4 + 2].x = w;
      break;
    case 3:
      P[0 * 4 + 1].y = -w; P[1 * 4 + 0].y = w; P[2 * 4 + 3].y = -w; P[3 * 4 + 2].y = w;
      break;
    default:
      P[0].x = w; P[5].x = -w; P[10].x = -w; P[15].x = w;
      break;
  }
}

struct LayerGateArgs {
  int N, K, C, M, terms, order, nsub, L, R, first_parity;
  double dt;
  const double* u;            // [K][C][N]
  const unsigned char* mask;  // [C][N]
  const double* gfix;         // [K][N-1] or null
  const double* J;            // [M][N-1][terms]: (J^z) or (J^x, J^y, J^z)
  const int* layer_off;       // [L + 1]
  LayerGate* out;             // [M][R]
  int* status;
};

// factor kinds
constexpr int kFBond = 0, kFInter = 1, kFXl = 2, kFYl = 3, kFXr = 4, kFYr = 5;
constexpr int kMaxFactors = 5;

__global__ void layer_gate_kernel(LayerGateArgs a) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)a.M * a.R) return;
  const int s = (int)(idx / a.R);
  const int r = (int)(idx - (long long)s * a.R);
  int lo = 0, hi = a.L;  // largest l with layer_off[l] <= r
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.layer_off[mid] <= r) lo = mid; else hi = mid;
  }
  const int l = lo;
  const int parity = (l + a.first_parity) & 1;
  const int b = parity + 2 * (r - a.layer_off[l]);
  const int N = a.N, nb = N - 1;
  const int S = a.K * a.nsub;
  const double dts = a.dt / a.nsub;

  // the layer's factors on bond b, first in time first
  int fk[kMaxFactors], fkind[kMaxFactors];
  double ftau[kMaxFactors];
  int nf = 0;
  if (a.order == 2) {
    if (l & 1) {
      fkind[nf] = kFBond; fk[nf] = ((l - 1) >> 1) / a.nsub; ftau[nf++] = dts;
    } else if (l == 0) {
      fkind[nf] = kFBond; fk[nf] = 0; ftau[nf++] = 0.5 * dts;
    } else if (l == 2 * S) {
      fkind[nf] = kFBond; fk[nf] = (S - 1) / a.nsub; ftau[nf++] = 0.5 * dts;
    } else {
      const int st = (l >> 1) - 1;
      fkind[nf] = kFBond; fk[nf] = st / a.nsub; ftau[nf++] = 0.5 * dts;
      fkind[nf] = kFBond; fk[nf] = (st + 1) / a.nsub; ftau[nf++] = 0.5 * dts;
    }
  } else {
    const int k = (l >> 1) / a.nsub;
    fkind[nf] = kFInter; fk[nf] = k; ftau[nf++] = dts;
    if (l & 1) {  // even bonds: both sites' rotations, Y before X
      fkind[nf] = kFYl; fk[nf] = k; ftau[nf++] = dts;
      fkind[nf] = kFYr; fk[nf] = k; ftau[nf++] = dts;
      fkind[nf] = kFXl; fk[nf] = k; ftau[nf++] = dts;
      fkind[nf] = kFXr; fk[nf] = k; ftau[nf++] = dts;
    } else if ((N & 1) && b == N - 2) {  // the last site of an odd chain
      fkind[nf] = kFYr; fk[nf] = k; ftau[nf++] = dts;
      fkind[nf] = kFXr; fk[nf] = k; ftau[nf++] = dts;
    }
  }

  const double* Jb = a.J + ((size_t)s * nb + b) * a.terms;
  const double jz = Jb[a.terms - 1];
  const double jx = (a.terms == 3) ? Jb[0] : 0.0;
  const double jy = (a.terms == 3) ? Jb[1] : 0.0;
  const double wl = (b == 0) ? 1.0 : 0.5;
  const double wr = (b + 1 == N - 1) ? 1.0 : 0.5;

  // eigendecomposition and exponential of every factor
  double2 Vf[kMaxFactors][16], Gf[kMaxFactors][16];
  double lamf[kMaxFactors][4];
  for (int f = 0; f < nf; ++f) {
    const int k = fk[f];
    const double* uk = a.u + (size_t)k * a.C * N;
    const unsigned char* mk = a.mask;
    const double xl = uk[b] * mk[b];
    const double yl = uk[N + b] * mk[N + b];
    const double xr = uk[b + 1] * mk[b + 1];
    const double yr = uk[N + b + 1] * mk[N + b + 1];
    double c = jz;
    if (a.C == 3) c += uk[2 * N + b] * mk[2 * N + b];
    if (a.gfix) c += a.gfix[(size_t)k * nb + b];
    double2 h[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) h[i] = make_double2(0.0, 0.0);
    if (fkind[f] == kFBond || fkind[f] == kFInter) {
      h[0].x = c;
      h[5].x = -c;
      h[10].x = -c;
      h[15].x = c;
      // J^x XX + J^y YY: <00|.|11> = jx - jy, <01|.|10> = jx + jy
      h[0 * 4 + 3].x += jx - jy;
      h[3 * 4 + 0].x += jx - jy;
      h[1 * 4 + 2].x += jx + jy;
      h[2 * 4 + 1].x += jx + jy;
      if (fkind[f] == kFBond) {
        // (x X + y Y) on a site couples |0> <-> |1> with <0|.|1> = x - i y
        const double2 lz = make_double2(wl * xl, -wl * yl);
        const double2 rz = make_double2(wr * xr, -wr * yr);
        for (int q = 0; q < 2; ++q) {
          h[(0 + q) * 4 + (2 + q)] = lz;
          h[(2 + q) * 4 + (0 + q)] = cconj(lz);
          h[(2 * q) * 4 + (2 * q + 1)] = rz;
          h[(2 * q + 1) * 4 + (2 * q)] = cconj(rz);
        }
      }
    } else {
      const int code = fkind[f] - kFXl;  // 0 X(x)I, 1 Y(x)I, 2 I(x)X, 3 I(x)Y
      const double amp = (code == 0) ? xl : (code == 1) ? yl : (code == 2) ? xr : yr;
      generator4(code, amp, h);
    }
    if (!herm_eig4(h, Vf[f], lamf[f])) atomicOr(a.status, kStatusNoConverge);
    double2 E[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      double sn, cs;
      sincos(ftau[f] * lamf[f][j], &sn, &cs);
      E[j] = make_double2(cs, -sn);
    }
#pragma unroll
    for (int rr = 0; rr < 4; ++rr)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        double2 g = make_double2(0.0, 0.0);
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(g, Vf[f][rr * 4 + j], cmulc(E[j], Vf[f][cc * 4 + j]));
        Gf[f][rr * 4 + cc] = g;
      }
  }

  // walk the factors backwards: Lt = product of the factors after f
  LayerGate& out = a.out[idx];
  double2 Lt[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) Lt[i] = make_double2((i % 5 == 0) ? 1.0 : 0.0, 0.0);
  int nq = 0;
  for (int f = nf - 1; f >= 0; --f) {
    const int k = fk[f];
    // the controls of this factor: (generator code, weight, c, site)
    int pc[5], pcc[5], psite[5];
    double pw[5];
    int np = 0;
    const unsigned char* mk = a.mask;
    if (fkind[f] == kFBond) {
      if (mk[b]) { pc[np] = 0; pw[np] = wl; pcc[np] = 0; psite[np++] = b; }
      if (mk[N + b]) { pc[np] = 1; pw[np] = wl; pcc[np] = 1; psite[np++] = b; }
      if (mk[b + 1]) { pc[np] = 2; pw[np] = wr; pcc[np] = 0; psite[np++] = b + 1; }
      if (mk[N + b + 1]) { pc[np] = 3; pw[np] = wr; pcc[np] = 1; psite[np++] = b + 1; }
    }
    if ((fkind[f] == kFBond || fkind[f] == kFInter) && a.C == 3 && mk[2 * N + b]) {
      pc[np] = 4; pw[np] = 1.0; pcc[np] = 2; psite[np++] = b;
    }
    if (fkind[f] >= kFXl) {
      const int code = fkind[f] - kFXl;
      const int cidx = code & 1, site = b + (code >> 1);
      if (mk[cidx * N + site]) { pc[np] = code; pw[np] = 1.0; pcc[np] = cidx; psite[np++] = site; }
    }
    // Gam_ij e^{i tau lam_j} = -i tau e^{-i tau (lam_i - lam_j)/2} sinc(tau (lam_i - lam_j)/2):
    // one sincos per entry, shared by every control of the factor
    double2 GE[16];
    {
      const double tau = ftau[f];
      const double* lam = lamf[f];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const double x = 0.5 * tau * (lam[i] - lam[j]);
          double sn, cs;
          sincos(x, &sn, &cs);
          const double sinc = (fabs(x) < 1e-8) ? 1.0 - x * x / 6.0 : sn / x;
          // -i tau sinc (cs - i sn) = tau sinc (-sn - i cs)
          GE[i * 4 + j] = make_double2(-tau * sinc * sn, -tau * sinc * cs);
        }
    }
    for (int q = 0; q < np; ++q) {
      // Q_f = V (Gam o (V^dag P V)) e^{i tau Lam} V^dag  (= dG_f G_f^dag)
      double2 P[16], T1[16], T2[16];
      generator4(pc[q], pw[q], P);
      const double2* V = Vf[f];
#pragma unroll
      for (int i = 0; i < 4; ++i)       // T1 = P V
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double2 acc = make_double2(0.0, 0.0);
#pragma unroll
          for (int m = 0; m < 4; ++m) cfma(acc, P[i * 4 + m], V[m * 4 + j]);
          T1[i * 4 + j] = acc;
        }
#pragma unroll
      for (int i = 0; i < 4; ++i)       // T2 = (Gam o (V^dag T1)) e^{i tau Lam}
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double2 acc = make_double2(0.0, 0.0);
#pragma unroll
          for (int m = 0; m < 4; ++m) cfmac(acc, V[m * 4 + i], T1[m * 4 + j]);
          T2[i * 4 + j] = cmul(GE[i * 4 + j], acc);
        }
#pragma unroll
      for (int i = 0; i < 4; ++i)       // T1 = T2 V^dag
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double2 acc = make_double2(0.0, 0.0);
#pragma unroll
          for (int m = 0; m < 4; ++m) cfma(acc, T2[i * 4 + m], cconj(V[j * 4 + m]));
          T1[i * 4 + j] = acc;
        }
#pragma unroll
      for (int i = 0; i < 4; ++i)       // T2 = V T1  (= dG_f G_f^dag)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double2 acc = make_double2(0.0, 0.0);
#pragma unroll
          for (int m = 0; m < 4; ++m) cfma(acc, V[i * 4 + m], T1[m * 4 + j]);
          T2[i * 4 + j] = acc;
        }
#pragma unroll
      for (int i = 0; i < 4; ++i)       // T1 = T2 Lt^dag
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double2 acc = make_double2(0.0, 0.0);
#pragma unroll
          for (int m = 0; m < 4; ++m) cfma(acc, T2[i * 4 + m], cconj(Lt[j * 4 + m]));
          T1[i * 4 + j] = acc;
        }
#pragma unroll
      for (int i = 0; i < 4; ++i)       // T2 = Lt T1
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          double2 acc = make_double2(0.0, 0.0);
#pragma unroll
          for (int m = 0; m < 4; ++m) cfma(acc, Lt[i * 4 + m], T1[m * 4 + j]);
          T2[i * 4 + j] = acc;
        }
      const int slot = (k * a.C + pcc[q]) * N + psite[q];
      int at = -1;
      for (int e = 0; e < nq; ++e)
        if (out.slot[e] == slot) at = e;
      if (at < 0 && nq < kMaxLayerParams) {
        at = nq++;
        out.slot[at] = slot;
#pragma unroll
        for (int i = 0; i < 16; ++i) out.Q[at][i] = T2[i];
      } else if (at >= 0) {
#pragma unroll
        for (int i = 0; i < 16; ++i) out.Q[at][i] = make_double2(out.Q[at][i].x + T2[i].x, out.Q[at][i].y + T2[i].y);
      } else {
        atomicOr(a.status, kStatusBadDims);   // cannot happen: at most 10 distinct controls
      }
    }
    // Lt <- Lt G_f
    double2 T[16];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int m = 0; m < 4; ++m) cfma(acc, Lt[i * 4 + m], Gf[f][m * 4 + j]);
        T[i * 4 + j] = acc;
      }
#pragma unroll
    for (int i = 0; i < 16; ++i) Lt[i] = T[i];
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) out.G[i] = Lt[i];
  out.nq = nq;
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void noise_kernel(unsigned long long seed, int dist, double scale, int M, int nb, double* J) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)M * nb) return;
  const double two53 = 1.0 / 9007199254740992.0;
  if (dist == 0) {
    const double u = (double)(splitmix64(seed, idx) >> 11) * two53;
    J[idx] = scale * (2.0 * u - 1.0);
  } else {
    const double u1 = (double)((splitmix64(seed, 2 * idx) >> 11) + 1ull) * two53;
    const double u2 = (double)(splitmix64(seed, 2 * idx + 1) >> 11) * two53;
    J[idx] = scale * sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
  }
}

// F = (1/T) sum_t |O_t|^2 ; per_traj[t] = |O_t|^2 ; grad[x] = (1/T) sum_t gsp[t][x]
// (fixed summation order: independent of launch configuration and timing).
__global__ void reduce_fidelity_kernel(const double2* O, int T, double* F, double* per_traj) {
  __shared__ double part[256];
  double s = 0.0;
  for (int t = threadIdx.x; t < T; t += blockDim.x) {
    const double v = cabs2(O[t]);
    if (per_traj) per_traj[t] = v;
    s += v;
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *F = part[0] / (double)T;
}

__global__ void reduce_grad_kernel(const double* gsp, int T, int X, double* grad) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= X) return;
  double s = 0.0;
  for (int t = 0; t < T; ++t) s += gsp[(size_t)t * X + x];
  grad[x] = s / (double)T;
}

}  // namespace tnrc

extern "C" cudaError_t tnrc_launch_layer_gates(int N, int K, int C, int M, int terms, int order, int nsub,
                                               int L, int R, int first_parity, double dt, const double* u,
                                               const unsigned char* mask, const double* gfix, const double* J,
                                               const int* layer_off, tnrc::LayerGate* out, int* status,
                                               cudaStream_t st) {
  tnrc::LayerGateArgs a{N, K, C, M, terms, order, nsub, L, R, first_parity, dt, u, mask, gfix, J, layer_off, out,
                        status};
  const long long total = (long long)M * R;
  const int threads = 64;
  const long long blocks = (total + threads - 1) / threads;
  (void)cudaGetLastError();  // report only this launch below
  tnrc::layer_gate_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

extern "C" cudaError_t tnrc_launch_noise(unsigned long long seed, int dist, double scale, int M, int nb, double* J,
                                         cudaStream_t st) {
  const long long total = (long long)M * nb;
  const int threads = 256;
  (void)cudaGetLastError();  // report only this launch below
  tnrc::noise_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(seed, dist, scale, M, nb, J);
  return cudaGetLastError();
}

extern "C" cudaError_t tnrc_launch_reduce(const double2* O, int T, double* F, double* per_traj, const double* gsp,
                                          int X, double* grad, cudaStream_t st) {
  (void)cudaGetLastError();  // report only this launch below
  tnrc::reduce_fidelity_kernel<<<1, 256, 0, st>>>(O, T, F, per_traj);
  if (gsp && grad) tnrc::reduce_grad_kernel<<<(X + 127) / 128, 128, 0, st>>>(gsp, T, X, grad);
  return cudaGetLastError();
}
