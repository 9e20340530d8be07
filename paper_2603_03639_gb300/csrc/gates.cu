// Bond gates of the second-order TEBD slice, and the noise realisations.
//
// gate_kernel: one thread per (sample s, slice k, bond b).  Builds the bond
// Hamiltonian of Eq. sysH with ZZ crosstalk,
//   h = c ZZ + wL (x_b X + y_b Y) (x) I + wR I (x) (x_{b+1} X + y_{b+1} Y),
//   c = g_b (if a control) + gfix_{k,b} + J^z(s)_b, plus J^x XX + J^y YY for
//   the Heisenberg-type crosstalk of Eq. Hp,
// diagonalises it by cyclic complex Jacobi rotations (FP64), and stores
//   G = V e^{-i tau Lam} V^dag            (tau = dt/2 on even bonds, dt on odd)
//   Gam_jk = -i tau e^{-i tau (l_j + l_k)/2} sinc(tau (l_j - l_k)/2)
// (the divided differences of x -> e^{-i tau x}, used by the Daleckii-Krein
// derivative of the gate in the gradient), and E_j = e^{-i tau l_j}.
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

struct GateArgs {
  int N, K, C, M, terms;
  double dt;
  const double* u;            // [K][C][N]
  const unsigned char* mask;  // [C][N]
  const double* gfix;         // [K][N-1] or null
  const double* J;            // [M][N-1][terms]: (J^z) or (J^x, J^y, J^z)
  GateEntry* out;             // [M][K][N-1]
  int* status;
};

__global__ void gate_kernel(GateArgs a) {
  const int nb = a.N - 1;
  const long long total = (long long)a.M * a.K * nb;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int b = (int)(idx % nb);
  const int k = (int)((idx / nb) % a.K);
  const int s = (int)(idx / ((long long)nb * a.K));
  const double* uk = a.u + (size_t)k * a.C * a.N;
  const unsigned char* mk = a.mask;
  const double xl = uk[b] * mk[b];
  const double yl = uk[a.N + b] * mk[a.N + b];
  const double xr = uk[b + 1] * mk[b + 1];
  const double yr = uk[a.N + b + 1] * mk[a.N + b + 1];
  const double* Jb = a.J + ((size_t)s * nb + b) * a.terms;
  double c = Jb[a.terms - 1];
  const double jx = (a.terms == 3) ? Jb[0] : 0.0;
  const double jy = (a.terms == 3) ? Jb[1] : 0.0;
  if (a.C == 3) c += uk[2 * a.N + b] * mk[2 * a.N + b];
  if (a.gfix) c += a.gfix[(size_t)k * nb + b];
  const double wl = (b == 0) ? 1.0 : 0.5;
  const double wr = (b + 1 == a.N - 1) ? 1.0 : 0.5;
  const double tau = (b & 1) ? a.dt : 0.5 * a.dt;

  double2 h[16], V[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    h[i] = make_double2(0.0, 0.0);
    V[i] = make_double2((i % 5 == 0) ? 1.0 : 0.0, 0.0);
  }
  // ZZ diagonal (+1, -1, -1, +1)
  h[0].x = c;
  h[5].x = -c;
  h[10].x = -c;
  h[15].x = c;
  // left site: (xl X + yl Y) (x) I couples |0 s2> <-> |1 s2>; <0|.|1> = xl - i yl
  const double2 lz = make_double2(wl * xl, -wl * yl);
  const double2 rz = make_double2(wr * xr, -wr * yr);
  for (int s2 = 0; s2 < 2; ++s2) {
    h[(0 + s2) * 4 + (2 + s2)] = lz;
    h[(2 + s2) * 4 + (0 + s2)] = cconj(lz);
  }
  for (int s1 = 0; s1 < 2; ++s1) {
    h[(2 * s1) * 4 + (2 * s1 + 1)] = rz;
    h[(2 * s1 + 1) * 4 + (2 * s1)] = cconj(rz);
  }
  // crosstalk J^x XX + J^y YY: <00|.|11> = jx - jy, <01|.|10> = jx + jy
  h[0 * 4 + 3].x += jx - jy;
  h[3 * 4 + 0].x += jx - jy;
  h[1 * 4 + 2].x += jx + jy;
  h[2 * 4 + 1].x += jx + jy;
  double scale2 = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) scale2 += cabs2(h[i]);
  const double stop2 = 1e-32 * scale2;
  int sweep = 0;
  for (; sweep < 30; ++sweep) {
    double off2 = 0.0;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = p + 1; q < 4; ++q) off2 += cabs2(h[p * 4 + q]);
    if (off2 <= stop2) break;
    herm_rotate(h, V, 0, 1);
    herm_rotate(h, V, 2, 3);
    herm_rotate(h, V, 0, 2);
    herm_rotate(h, V, 1, 3);
    herm_rotate(h, V, 0, 3);
    herm_rotate(h, V, 1, 2);
  }
  if (sweep == 30) atomicOr(a.status, kStatusNoConverge);
  double lam[4];
  double2 E[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    lam[j] = h[j * 5].x;
    double sn, cs;
    sincos(tau * lam[j], &sn, &cs);
    E[j] = make_double2(cs, -sn);
  }
  GateEntry& ge = a.out[idx];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      double2 g = make_double2(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < 4; ++j) cfma(g, V[r * 4 + j], cmulc(E[j], V[cc * 4 + j]));
      ge.G[r * 4 + cc] = g;
      ge.V[r * 4 + cc] = V[r * 4 + cc];
      // Gam_rc = -i tau e^{-i tau (l_r + l_c)/2} sinc(tau (l_r - l_c)/2)
      const double x = 0.5 * tau * (lam[r] - lam[cc]);
      const double sinc = (fabs(x) < 1e-8) ? 1.0 - x * x / 6.0 : sin(x) / x;
      double sn, cs;
      sincos(0.5 * tau * (lam[r] + lam[cc]), &sn, &cs);
      // -i tau (cs - i sn) sinc = tau sinc (-sn - i cs)
      ge.Gam[r * 4 + cc] = make_double2(-tau * sinc * sn, -tau * sinc * cs);
    }
#pragma unroll
  for (int j = 0; j < 4; ++j) ge.E[j] = E[j];
}

// Merged half-step gates of the even bonds: Gm[s][k][b] = G[s][k+1][b] G[s][k][b]
// (k = 0..K-2), the A(dt/2) that ends slice k followed by the one that starts
// slice k+1, applied as one gate before one truncation.
__global__ void merge_kernel(int N, int K, int M, const GateEntry* g, double2* gm) {
  const int nb = N - 1;
  const int ne = (nb + 1) / 2;  // even bonds
  const long long total = (long long)M * (K - 1) * ne * 16;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int e = (int)(idx & 15);
  const long long rest = idx >> 4;
  const int b = 2 * (int)(rest % ne);
  const int k = (int)((rest / ne) % (K - 1));
  const int s = (int)(rest / ((long long)ne * (K - 1)));
  const GateEntry& g1 = g[((size_t)s * K + k) * nb + b];
  const GateEntry& g2 = g[((size_t)s * K + k + 1) * nb + b];
  const int r = e >> 2, c = e & 3;
  double2 acc = make_double2(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < 4; ++j) cfma(acc, g2.G[r * 4 + j], g1.G[j * 4 + c]);
  gm[(((size_t)s * (K - 1) + k) * nb + b) * 16 + e] = acc;
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

extern "C" cudaError_t tnrc_launch_gates(int N, int K, int C, int M, int terms, double dt, const double* u,
                                         const unsigned char* mask, const double* gfix, const double* J,
                                         tnrc::GateEntry* out, double2* merged, int* status, cudaStream_t st) {
  tnrc::GateArgs a{N, K, C, M, terms, dt, u, mask, gfix, J, out, status};
  const long long total = (long long)M * K * (N - 1);
  const int threads = 128;
  const long long blocks = (total + threads - 1) / threads;
  (void)cudaGetLastError();  // report only this launch below
  tnrc::gate_kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
  if (K > 1) {
    const long long tm = (long long)M * (K - 1) * (N / 2) * 16;
    tnrc::merge_kernel<<<(unsigned)((tm + 255) / 256), 256, 0, st>>>(N, K, M, out, merged);
  }
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
