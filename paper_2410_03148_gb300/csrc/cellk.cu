// Cell-level kernels: the ersatz map from the level set (§2.6), the nine
// right-hand sides (§2.2), reductions for the null-space projection and the
// homogenised tensors (Eqs. hom_C, hom_e, hom_kappa), and the element-wise
// sensitivity quadratic forms.
#include "kernels.cuh"

namespace cell {

namespace {

constexpr int kB = 256;
constexpr int kWarps = kB / 32;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < kWarps ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// rho_e = 1 - (1 - rho_void) H_eta(phi_e), phi_e = mean of the 8 nodal values.
template <typename Tin>
__global__ void k_ersatz(const Tin* __restrict__ phi, int nx, int ny, int nz, double rho_void,
                         double eta, float* __restrict__ r32, double* __restrict__ r64,
                         double* __restrict__ drho) {
  const i64 nxy = (i64)nx * ny, nn = nxy * nz;
  const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / nxy);
  const int i1 = i + 1 == nx ? 0 : i + 1, j1 = j + 1 == ny ? 0 : j + 1, k1 = k + 1 == nz ? 0 : k + 1;
  double s = 0.0;
  const int xs[2] = {i, i1}, ys[2] = {j, j1}, zs[2] = {k, k1};
#pragma unroll
  for (int c = 0; c < 8; ++c)
    s += (double)phi[xs[c & 1] + nx * (ys[(c >> 1) & 1] + (i64)ny * zs[c >> 2])];
  s *= 0.125;
  double H, dH = 0.0;
  if (s < -eta) H = 0.0;
  else if (s > eta) H = 1.0;
  else {
    const double t = s / eta;
    H = 0.5 * (1.0 + t + sin(M_PI * t) / M_PI);
    dH = 0.5 * (1.0 + cos(M_PI * t)) / eta;
  }
  const double r = 1.0 - (1.0 - rho_void) * H;
  r64[e] = r;
  r32[e] = (float)r;
  if (drho) drho[e] = -(1.0 - rho_void) * dH;   // d rho_e / d phi_e
}

// Nodal level-set sensitivities from element ones: phi_e is the mean of the
// element's 8 nodal values, so dL/dphi_n = sum over the 8 elements e around
// n of (dL/drho_e)(drho_e/dphi_e) / 8.
template <typename T>
__global__ void k_chain_phi(const double* __restrict__ ge, const double* __restrict__ drho, int nx,
                            int ny, int nz, T* __restrict__ gn) {
  const i64 nxy = (i64)nx * ny, nn = nxy * nz;
  const i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / nxy);
  const int xs[2] = {i, i == 0 ? nx - 1 : i - 1}, ys[2] = {j, j == 0 ? ny - 1 : j - 1},
            zs[2] = {k, k == 0 ? nz - 1 : k - 1};
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const i64 e = xs[c & 1] + nx * (ys[(c >> 1) & 1] + (i64)ny * zs[c >> 2]);
    acc += ge[e] * drho[e];
  }
  gn[n] = (T)(0.125 * acc);
}

template <typename Tin>
__global__ void k_rho_copy(const Tin* __restrict__ in, i64 n, float* __restrict__ r32,
                           double* __restrict__ r64, int* bad) {
  const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double r = (double)in[e];
  if (!(r > 0.0) || !isfinite(r)) atomicAdd(bad, 1);
  r64[e] = r;
  r32[e] = (float)r;
}

// bhat^I_c(n) = -sgn_c sum_{e around n} rho_e F[4 a_e + c][I]; sgn = -1 for phi.
__global__ void __launch_bounds__(kB)
k_rhs9(const double* __restrict__ rho, const __grid_constant__ RhsParams P, int mask,
       double* __restrict__ b, int nx, int ny, int nz) {
  const i64 nxy = (i64)nx * ny, nn = nxy * nz;
  const i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / nxy);
  double acc[4][9];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int I = 0; I < 9; ++I) acc[c][I] = 0.0;
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
    const int la = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
    const int ei = ex ? i : (i == 0 ? nx - 1 : i - 1);
    const int ej = ey ? j : (j == 0 ? ny - 1 : j - 1);
    const int ek = ez ? k : (k == 0 ? nz - 1 : k - 1);
    const double r = rho[ei + nx * (ej + (i64)ny * ek)];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int I = 0; I < 9; ++I) acc[c][I] = fma(r, P.F[(4 * la + c) * 9 + I], acc[c][I]);
  }
#pragma unroll
  for (int I = 0; I < 9; ++I)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const double v = ((mask >> I) & 1) ? (c == 3 ? acc[c][I] : -acc[c][I]) : 0.0;
      b[((i64)I * 4 + c) * nn + n] = v;
    }
}

// grid (nblk, nrhs*4): partial sums of each (rhs, comp) plane.
__global__ void __launch_bounds__(kB)
k_comp_sums(const double* __restrict__ x, i64 nn, double* __restrict__ partial) {
  __shared__ double sh[kWarps];
  const int qc = blockIdx.y;
  const i64 chunk = (nn + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk, hi = lo + chunk < nn ? lo + chunk : nn;
  const double* X = x + (i64)qc * nn;
  double s = 0.0;
  for (i64 k = lo + threadIdx.x; k < hi; k += kB) s += X[k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[(i64)qc * gridDim.x + blockIdx.x] = s;
}

__global__ void k_sub_means(double* __restrict__ x, i64 nn, const double* __restrict__ sums) {
  const int qc = blockIdx.y;
  const double m = sums[qc] / (double)nn;
  double* X = x + (i64)qc * nn;
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < nn; k += (i64)gridDim.x * blockDim.x)
    X[k] -= m;
}

// grid (nblk, 9): row I of sum_c sgn_c <u^I_c, v^J_c>, J = 0..8.
__global__ void __launch_bounds__(kB)
k_gram9(const double* __restrict__ u, const double* __restrict__ v, i64 nn,
        double* __restrict__ partial) {
  __shared__ double sh[kWarps];
  const int I = blockIdx.y;
  const i64 len = 4 * nn;
  const i64 chunk = (len + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk, hi = lo + chunk < len ? lo + chunk : len;
  const double* U = u + (i64)I * len;
  double acc[9];
#pragma unroll
  for (int J = 0; J < 9; ++J) acc[J] = 0.0;
  for (i64 k = lo + threadIdx.x; k < hi; k += kB) {
    const double sg = (k >= 3 * nn) ? -1.0 : 1.0;
    const double uk = sg * U[k];
#pragma unroll
    for (int J = 0; J < 9; ++J) acc[J] = fma(uk, v[(i64)J * len + k], acc[J]);
  }
  for (int J = 0; J < 9; ++J) {
    const double s = block_sum(acc[J], sh);
    if (threadIdx.x == 0) partial[((i64)I * gridDim.x + blockIdx.x) * 9 + J] = s;
  }
}

template <bool SQ>
__global__ void __launch_bounds__(kB)
k_sum(const double* __restrict__ x, i64 n, double* __restrict__ partial) {
  __shared__ double sh[kWarps];
  const i64 chunk = (n + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  double s = 0.0;
  for (i64 k = lo + threadIdx.x; k < hi; k += kB) s += SQ ? x[k] * x[k] : x[k];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// Element sensitivities in the eigen-modes of the symmetric upstream weights
// (sym(G) = Q diag(lam) Q^T):  g_e = sum_IJ G_IJ W_e^I.K0 W_e^J
//                                 = sum_m lam_m X_e^m.K0 X_e^m,  X^m = sum_I Q_Im W^I.
// Pass 1 forms the fluctuation part of every mode at the nodes (reads the
// nine FP64 solutions once, coalesced) and stores it as an FP32 pair
// (hi, lo = v - hi) or in FP64.  Pass 2 gives each thread one element.  K0
// annihilates a constant value per component (rigid translations, uniform
// potential), so the element's values are first taken relative to its local
// node 0: the nodal values are up to ~N times their variation across one
// element, and forming the quadratic form from them directly in FP32 would
// cancel that many digits.  The differences come from the pairs
// (hi_a - hi_0) + (lo_a - lo_0); the affine part of the loads (Zbar Q, zero at
// local node 0) is added, and the symmetric quadratic form is evaluated with
// the upper triangle of K0 (528 multiply-adds per mode, the coefficients at
// compile-time offsets of the parameter bank).
template <typename T>
__global__ void __launch_bounds__(kB)
k_sens_modes(const double* __restrict__ y, const __grid_constant__ SensQ Q, T* __restrict__ X,
             i64 nn) {
  const i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int c = blockIdx.y;
  double w[9];
#pragma unroll
  for (int I = 0; I < 9; ++I) w[I] = y[((i64)I * 4 + c) * nn + n];
  for (int m = 0; m < Q.R; ++m) {
    double v = 0.0;
#pragma unroll
    for (int I = 0; I < 9; ++I) v = fma(Q.q[I * 9 + m], w[I], v);
    if constexpr (sizeof(T) == 4) {
      const float hi = (float)v;
      X[((i64)m * 8 + c) * nn + n] = hi;                       // hi parts: planes 0..3
      X[((i64)m * 8 + 4 + c) * nn + n] = (float)(v - (double)hi);   // lo parts: planes 4..7
    } else {
      X[((i64)m * 4 + c) * nn + n] = (T)v;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kB, sizeof(T) == 4 ? 2 : 1)
k_sens_elem(const T* __restrict__ X, const double* __restrict__ rho,
            const __grid_constant__ SensModes<T> P, T* __restrict__ g, int nx, int ny, int nz,
            int times_rho) {
  const i64 nxy = (i64)nx * ny, nn = nxy * nz;
  const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / nxy);
  // 32-bit node offsets: cell_setup admits at most 4e8 nodes, so 8 nn < 2^32
  const unsigned xo[2] = {(unsigned)i, (unsigned)(i + 1 == nx ? 0 : i + 1)};
  const unsigned yo[2] = {(unsigned)(j * nx), (unsigned)((j + 1 == ny ? 0 : j + 1) * nx)};
  const unsigned nxy32 = (unsigned)nxy;
  const unsigned zo[2] = {(unsigned)k * nxy32, (unsigned)(k + 1 == nz ? 0 : k + 1) * nxy32};
  const unsigned nn32 = (unsigned)nn;
  T acc = T(0);
  for (int m = 0; m < P.R; ++m) {
    T x[32];
    if constexpr (sizeof(T) == 4) {
      const T* Xh = X + (i64)m * 8 * nn;
      const T* Xl = Xh + 4 * (i64)nn;
      float h0[4], l0[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        h0[c] = __ldg(Xh + (c * nn32 + zo[0] + yo[0] + xo[0]));
        l0[c] = __ldg(Xl + (c * nn32 + zo[0] + yo[0] + xo[0]));
      }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const unsigned node = xo[a & 1] + yo[(a >> 1) & 1] + zo[a >> 2];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float dh = a ? __ldg(Xh + (c * nn32 + node)) - h0[c] : 0.f;
          const float dl = a ? __ldg(Xl + (c * nn32 + node)) - l0[c] : 0.f;
          x[4 * a + c] = (dh + dl) + P.zq[(4 * a + c) * 9 + m];
        }
      }
    } else {
      const T* Xm = X + (i64)m * 4 * nn;
      T x0[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) x0[c] = __ldg(Xm + (c * nn32 + zo[0] + yo[0] + xo[0]));
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const unsigned node = xo[a & 1] + yo[(a >> 1) & 1] + zo[a >> 2];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          x[4 * a + c] = (a ? __ldg(Xm + (c * nn32 + node)) - x0[c] : T(0)) + P.zq[(4 * a + c) * 9 + m];
      }
    }
    T q = T(0);
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      T t = P.ku[a * 32 + a] * x[a];
#pragma unroll
      for (int b = a + 1; b < 32; ++b) t = fma(P.ku[a * 32 + b], x[b], t);
      q = fma(x[a], t, q);
    }
    acc = fma(P.lam[m], q, acc);
  }
  g[e] = times_rho ? (T)(acc * rho[e]) : acc;
}

// Energy difference of two solutions by the polarisation identity
// B(W1, W1) - B(W2, W2) = B(W1 + W2, W1 - W2) for the symmetric bilinear form
// B(U, V) = sum_IJ G_IJ U^I.K0 V^J = sum_m lam_m (Q^T U)_m.K0 (Q^T V)_m (FP64):
// the difference field is formed first, so its rounding scales with the
// difference, not with the energies.  Pass 1: the mode fields of the sum and
// of the difference of the two fluctuation sets; pass 2: per element, both
// taken relative to local node 0 (K0 annihilates constants), the sum gets
// twice the affine part, and q = S.K0 D.
__global__ void __launch_bounds__(kB)
k_sens_modes_pair(const double* __restrict__ y1, const double* __restrict__ y2, const __grid_constant__ SensQ Q,
                  double* __restrict__ XS, double* __restrict__ XD, i64 nn) {
  const i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int c = blockIdx.y;
  double ws[9], wd[9];
#pragma unroll
  for (int I = 0; I < 9; ++I) {
    const double a = y1[((i64)I * 4 + c) * nn + n], b = y2[((i64)I * 4 + c) * nn + n];
    ws[I] = a + b;
    wd[I] = a - b;
  }
  for (int m = 0; m < Q.R; ++m) {
    double vs = 0.0, vd = 0.0;
#pragma unroll
    for (int I = 0; I < 9; ++I) {
      vs = fma(Q.q[I * 9 + m], ws[I], vs);
      vd = fma(Q.q[I * 9 + m], wd[I], vd);
    }
    XS[((i64)m * 4 + c) * nn + n] = vs;
    XD[((i64)m * 4 + c) * nn + n] = vd;
  }
}

__global__ void __launch_bounds__(kB)
k_sens_elem_pair(const double* __restrict__ XS, const double* __restrict__ XD,
                 const __grid_constant__ SensPair P, double* __restrict__ g, int nx, int ny, int nz) {
  const i64 nxy = (i64)nx * ny, nn = nxy * nz;
  const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  const int i = (int)(e % nx), j = (int)((e / nx) % ny), k = (int)(e / nxy);
  const i64 xo[2] = {i, i + 1 == nx ? 0 : i + 1};
  const i64 yo[2] = {(i64)j * nx, (i64)(j + 1 == ny ? 0 : j + 1) * nx};
  const i64 zo[2] = {(i64)k * nxy, (i64)(k + 1 == nz ? 0 : k + 1) * nxy};
  double acc = 0.0;
  for (int m = 0; m < P.R; ++m) {
    const double* S = XS + (i64)m * 4 * nn;
    const double* D = XD + (i64)m * 4 * nn;
    double sv[32], dv[32];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const i64 node = xo[a & 1] + yo[(a >> 1) & 1] + zo[a >> 2];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        sv[4 * a + c] = S[c * nn + node];
        dv[4 * a + c] = D[c * nn + node];
      }
    }
#pragma unroll
    for (int a = 31; a >= 0; --a) {
      const int c = a & 3;
      sv[a] = sv[a] - sv[c] + 2.0 * P.zq[a * 9 + m];
      dv[a] = dv[a] - dv[c];
    }
    double q = 0.0;
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      double t = 0.0;
#pragma unroll
      for (int b = 0; b < 32; ++b) t = fma(P.k[a * 32 + b], dv[b], t);
      q = fma(sv[a], t, q);
    }
    acc = fma(P.lam[m], q, acc);
  }
  g[e] = acc;
}

inline unsigned nb(i64 n) { return (unsigned)((n + kB - 1) / kB); }

}  // namespace

// One explicit step of phi_t + v |grad phi| = 0 (Eq. HJ) on the periodic
// node grid with the first-order Godunov upwind Hamiltonian: one-sided
// differences D-/D+ per axis, the outward-moving norm built from
// max(D-, 0) and min(D+, 0), the inward one from min(D-, 0) and max(D+, 0).
template <typename T>
__global__ void k_hj_step(const T* __restrict__ phi, const T* __restrict__ v, int nx, int ny, int nz,
                          double dt, T* __restrict__ out) {
  const i64 nxy = (i64)nx * ny, nn = nxy * nz;
  const i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / nxy);
  const double p0 = (double)phi[n];
  const i64 nb[3][2] = {
      {n - i + (i == 0 ? nx - 1 : i - 1), n - i + (i == nx - 1 ? 0 : i + 1)},
      {n + ((j == 0 ? ny - 1 : j - 1) - j) * (i64)nx, n + ((j == ny - 1 ? 0 : j + 1) - j) * (i64)nx},
      {n + ((k == 0 ? nz - 1 : k - 1) - k) * nxy, n + ((k == nz - 1 ? 0 : k + 1) - k) * nxy}};
  const double hinv[3] = {(double)nx, (double)ny, (double)nz};
  double gp = 0.0, gm = 0.0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double dm = (p0 - (double)phi[nb[d][0]]) * hinv[d];
    const double dp = ((double)phi[nb[d][1]] - p0) * hinv[d];
    const double a = fmax(dm, 0.0), b = fmin(dp, 0.0), c = fmin(dm, 0.0), e = fmax(dp, 0.0);
    gp += a * a + b * b;
    gm += c * c + e * e;
  }
  const double vn = (double)v[n];
  out[n] = (T)(p0 - dt * (fmax(vn, 0.0) * sqrt(gp) + fmin(vn, 0.0) * sqrt(gm)));
}

template <typename Tin>
void ersatz(const Tin* phi, int nx, int ny, int nz, double rho_void, double eta, float* rho32,
            double* rho64, double* drho, cudaStream_t s) {
  const i64 nn = (i64)nx * ny * nz;
  note_launch(), k_ersatz<Tin><<<nb(nn), kB, 0, s>>>(phi, nx, ny, nz, rho_void, eta, rho32, rho64, drho);
}

template <typename T>
void hj_step(const T* phi, const T* v, int nx, int ny, int nz, double dt, T* out, cudaStream_t s) {
  const i64 nn = (i64)nx * ny * nz;
  note_launch(), k_hj_step<T><<<nb(nn), kB, 0, s>>>(phi, v, nx, ny, nz, dt, out);
}

template <typename T>
void chain_phi(const double* ge, const double* drho, int nx, int ny, int nz, T* gn, cudaStream_t s) {
  const i64 nn = (i64)nx * ny * nz;
  note_launch(), k_chain_phi<T><<<nb(nn), kB, 0, s>>>(ge, drho, nx, ny, nz, gn);
}

template <typename Tin>
void rho_copy(const Tin* in, i64 n, float* rho32, double* rho64, int* bad, cudaStream_t s) {
  note_launch(), k_rho_copy<Tin><<<nb(n), kB, 0, s>>>(in, n, rho32, rho64, bad);
}

void rhs9(const double* rho, const RhsParams& F, int mask, double* b, int nx, int ny, int nz,
          cudaStream_t s) {
  const i64 nn = (i64)nx * ny * nz;
  note_launch(), k_rhs9<<<nb(nn), kB, 0, s>>>(rho, F, mask, b, nx, ny, nz);
}

void comp_sums(const double* x, i64 nn, int nrhs, double* partial, int nblk, double* out,
               cudaStream_t s) {
  note_launch(), k_comp_sums<<<dim3(nblk, nrhs * 4), kB, 0, s>>>(x, nn, partial);
  reduce_partials(partial, nblk, 1, 1, out, 0, nrhs * 4, nullptr, s);
}

void sub_means(double* x, i64 nn, int nrhs, const double* sums, cudaStream_t s) {
  unsigned g = nb(nn);
  if (g > 2048) g = 2048;
  note_launch(), k_sub_means<<<dim3(g, nrhs * 4), kB, 0, s>>>(x, nn, sums);
}

void gram9(const double* u, const double* v, i64 nn, double* partial, int nblk, double* out,
           cudaStream_t s) {
  note_launch(), k_gram9<<<dim3(nblk, 9), kB, 0, s>>>(u, v, nn, partial);
  reduce_partials(partial, nblk, 9, 9, out, 0, 9, nullptr, s);
}

void sum_reduce(const double* x, i64 n, double* partial, int nblk, double* out, cudaStream_t s,
                int squares) {
  if (squares) note_launch(), k_sum<true><<<nblk, kB, 0, s>>>(x, n, partial);
  else note_launch(), k_sum<false><<<nblk, kB, 0, s>>>(x, n, partial);
  reduce_partials(partial, nblk, 1, 1, out, 0, 1, nullptr, s);
}

template <typename T>
void sensitivity(const double* y, const double* rho, const SensQ& Q, const SensModes<T>& P, T* xwork,
                 T* g, int nx, int ny, int nz, int times_rho, cudaStream_t s) {
  const i64 nn = (i64)nx * ny * nz;
  if (Q.R > 0) note_launch(), k_sens_modes<T><<<dim3(nb(nn), 4), kB, 0, s>>>(y, Q, xwork, nn);
  note_launch(), k_sens_elem<T><<<nb(nn), kB, 0, s>>>(xwork, rho, P, g, nx, ny, nz, times_rho);
}

void energy_difference(const double* y1, const double* y2, const SensQ& Q, const SensPair& P, double* xwork,
                       double* g, int nx, int ny, int nz, cudaStream_t s) {
  const i64 nn = (i64)nx * ny * nz;
  double* XS = xwork;
  double* XD = xwork + (i64)9 * 4 * nn;
  if (Q.R > 0) note_launch(), k_sens_modes_pair<<<dim3(nb(nn), 4), kB, 0, s>>>(y1, y2, Q, XS, XD, nn);
  note_launch(), k_sens_elem_pair<<<nb(nn), kB, 0, s>>>(XS, XD, P, g, nx, ny, nz);
}

template void ersatz<float>(const float*, int, int, int, double, double, float*, double*, double*, cudaStream_t);
template void ersatz<double>(const double*, int, int, int, double, double, float*, double*, double*, cudaStream_t);
template void chain_phi<float>(const double*, const double*, int, int, int, float*, cudaStream_t);
template void hj_step<float>(const float*, const float*, int, int, int, double, float*, cudaStream_t);
template void hj_step<double>(const double*, const double*, int, int, int, double, double*, cudaStream_t);
template void chain_phi<double>(const double*, const double*, int, int, int, double*, cudaStream_t);
template void rho_copy<float>(const float*, i64, float*, double*, int*, cudaStream_t);
template void rho_copy<double>(const double*, i64, float*, double*, int*, cudaStream_t);
template void sensitivity<float>(const double*, const double*, const SensQ&, const SensModes<float>&,
                                 float*, float*, int, int, int, int, cudaStream_t);
template void sensitivity<double>(const double*, const double*, const SensQ&, const SensModes<double>&,
                                  double*, double*, int, int, int, int, cudaStream_t);

}  // namespace cell
