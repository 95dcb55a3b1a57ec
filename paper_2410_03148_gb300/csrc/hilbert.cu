// Hilbertian extension-regularisation and projection of the shape velocity
// (§2.6) on the device.
//
// The velocity space is periodic H^1 on the unit cell, <u, v>_H =
// int alpha^2 grad u . grad v + u v, discretised with the Q1 node basis:
// <u, v>_H = u^T A v, A = alpha^2 K + M.  On the structured periodic grid A is
// a constant 27-point stencil, the sum of tensor products of the 1D Q1
// stencils S = [-1, 2, -1] / h and M = h [1, 4, 1] / 6.  A nodal sensitivity
// d (a dual vector) has the Riesz representer g = A^-1 d, computed by a
// Chebyshev iteration: A's eigenvalues are the symbol values on the grid's
// Fourier modes, a multilinear function of the per-axis cosines, so its
// extremes (corners of the cosine box) bound the spectrum exactly and the
// iteration count for a given reduction follows in advance.  The objective and
// constraint representers are solved together (one launch per step, one
// vector per grid z slice).
//
// Projection (null-space method): with the H Gram matrix G_ab = <g_a, g_b>_H
// = g_a . d_b, the constraint block factors as R^T R (R = the Gram-Schmidt
// coefficients of the constraint representers), theta = g R^-1 is their
// H-orthonormal basis, P g_J = g_J - sum_k <g_J, theta_k> theta_k, mu solves
// R^T mu = w_C C, and the velocity v = w_J P g_J / ||P g_J||_H + sum_k mu_k
// theta_k is formed as one linear combination of the representers.  To first
// order one step of Eq. HJ then lowers J (<g_J, v>_H = w_J ||P g_J||_H) and
// moves each constraint by -dt w_C C_i.
#include <cmath>
#include <vector>

#include "cell.h"
#include "kernels.cuh"

namespace cell {

namespace {

constexpr int kB = 256;
constexpr int kMaxVec = 1 + kHilbertMaxCons;

struct Stencil {
  double c[27];   // coefficient of neighbour (dx, dy, dz) at (dx + 1) + 3 (dy + 1) + 9 (dz + 1)
};

// x = 0 (implicit), r = d, p = d / theta for every vector (grid y = vector)
__global__ void k_cheb_init(const double* const* __restrict__ rhs, double* __restrict__ r,
                            double* __restrict__ p, double* __restrict__ x, i64 nn, double inv_theta) {
  const int v = blockIdx.y;
  const double* d = rhs[v];
  for (i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += (i64)gridDim.x * blockDim.x) {
    const double b = d[n];
    r[v * nn + n] = b;
    p[v * nn + n] = b * inv_theta;
    x[v * nn + n] = 0.0;
  }
}

// One Chebyshev step per node: x += p, r -= A p, p_new = a p + b r_new
// (p read from pin, written to pout: neighbours read the old direction).
__global__ void __launch_bounds__(kB)
k_cheb_step(const __grid_constant__ Stencil S, const double* __restrict__ pin, double* __restrict__ pout,
            double* __restrict__ r, double* __restrict__ x, int nx, int ny, int nz, double ca, double cb) {
  const i64 nxy = (i64)nx * ny, nn = nxy * nz;
  const i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int v = blockIdx.y;
  const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / nxy);
  const int xo[3] = {i == 0 ? nx - 1 : i - 1, i, i == nx - 1 ? 0 : i + 1};
  const i64 yo[3] = {(i64)(j == 0 ? ny - 1 : j - 1) * nx, (i64)j * nx, (i64)(j == ny - 1 ? 0 : j + 1) * nx};
  const i64 zo[3] = {(i64)(k == 0 ? nz - 1 : k - 1) * nxy, (i64)k * nxy, (i64)(k == nz - 1 ? 0 : k + 1) * nxy};
  const double* P = pin + v * nn;
  double ap = 0.0;
#pragma unroll
  for (int q = 0; q < 27; ++q) ap = fma(S.c[q], P[xo[q % 3] + yo[(q / 3) % 3] + zo[q / 9]], ap);
  const i64 o = v * nn + n;
  const double pn = P[n];
  x[o] += pn;
  const double rn = r[o] - ap;
  r[o] = rn;
  pout[o] = ca * pn + cb * rn;
}

// partial[(a * nblk + blk) * kNvMax + b] = block sum of g_a . d_b
__global__ void __launch_bounds__(kB)
k_gram(const double* __restrict__ g, const double* const* __restrict__ d, int nvec, i64 nn,
       double* __restrict__ partial) {
  __shared__ double sh[kB / 32][kMaxVec];
  const int a = blockIdx.y;
  const i64 chunk = (nn + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk, hi = lo + chunk < nn ? lo + chunk : nn;
  double acc[kMaxVec];
#pragma unroll
  for (int b = 0; b < kMaxVec; ++b) acc[b] = 0.0;
  for (i64 n = lo + threadIdx.x; n < hi; n += kB) {
    const double ga = g[a * nn + n];
#pragma unroll
    for (int b = 0; b < kMaxVec; ++b)
      if (b < nvec) acc[b] = fma(ga, d[b][n], acc[b]);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int b = 0; b < kMaxVec; ++b) {
    double v = acc[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w][b] = v;
  }
  __syncthreads();
  if (threadIdx.x < kMaxVec && (int)threadIdx.x < nvec) {
    double s = 0.0;
    for (int ww = 0; ww < kB / 32; ++ww) s += sh[ww][threadIdx.x];
    partial[((i64)a * gridDim.x + blockIdx.x) * kNvMax + threadIdx.x] = s;
  }
}

struct Coef {
  double c[kMaxVec];
};

__global__ void k_lincomb_vec(const double* __restrict__ g, const __grid_constant__ Coef C, int nvec, i64 nn,
                              double* __restrict__ v) {
  for (i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += (i64)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int a = 0; a < nvec; ++a) s = fma(C.c[a], g[a * nn + n], s);
    v[n] = s;
  }
}

// 1D Q1 stencils at offsets -1, 0, +1 (periodic grid of spacing h)
void stencils_1d(double h, double s[3], double m[3]) {
  s[0] = -1.0 / h; s[1] = 2.0 / h; s[2] = -1.0 / h;
  m[0] = h / 6.0; m[1] = 4.0 * h / 6.0; m[2] = h / 6.0;
}

// Symbol of A at per-axis cosines (cx, cy, cz).
double symbol(double alpha, const double h[3], const double c[3]) {
  double s[3], m[3];
  for (int d = 0; d < 3; ++d) {
    s[d] = (2.0 - 2.0 * c[d]) / h[d];
    m[d] = h[d] * (4.0 + 2.0 * c[d]) / 6.0;
  }
  return alpha * alpha * (s[0] * m[1] * m[2] + m[0] * s[1] * m[2] + m[0] * m[1] * s[2]) + m[0] * m[1] * m[2];
}

}  // namespace

int hilbert_velocity(int nx, int ny, int nz, double alpha, const double* dJ, const double* const* dC,
                     const double* C, int ncons, double wJ, double wC, double* v, double* work,
                     const double** dptrs_dev, double* partial, int nblk, double* red, double* info,
                     cudaStream_t s) {
  const i64 nn = (i64)nx * ny * nz;
  const int nvec = 1 + ncons;
  const double h[3] = {1.0 / nx, 1.0 / ny, 1.0 / nz};
  // exact spectral bounds: corners of the box of available cosines per axis
  const int n3[3] = {nx, ny, nz};
  double cmin[3];
  for (int d = 0; d < 3; ++d) cmin[d] = std::cos(2.0 * M_PI * (n3[d] / 2) / n3[d]);
  double lmin = 1e300, lmax = 0.0;
  for (int corner = 0; corner < 8; ++corner) {
    const double c[3] = {(corner & 1) ? cmin[0] : 1.0, (corner & 2) ? cmin[1] : 1.0, (corner & 4) ? cmin[2] : 1.0};
    const double l = symbol(alpha, h, c);
    lmin = std::min(lmin, l);
    lmax = std::max(lmax, l);
  }
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
  // iterations for an A-norm error reduction of 1e-13: 2 q^k / (1 + q^2k) <= 1e-13
  const double kap = lmax / lmin;
  const double q = (std::sqrt(kap) - 1.0) / (std::sqrt(kap) + 1.0);
  int iters = q <= 0.0 ? 1 : (int)std::ceil(std::log(1e-13 / 2.0) / std::log(q));
  iters = std::max(1, std::min(iters, 20000));
  const bool flat = !(delta > 1e-14 * theta);   // one eigenvalue: x = d / theta in one step
  // stencil of A
  Stencil S;
  double sx[3], mx[3], sy[3], my[3], sz[3], mz[3];
  stencils_1d(h[0], sx, mx);
  stencils_1d(h[1], sy, my);
  stencils_1d(h[2], sz, mz);
  for (int dz = 0; dz < 3; ++dz)
    for (int dy = 0; dy < 3; ++dy)
      for (int dx = 0; dx < 3; ++dx)
        S.c[dx + 3 * dy + 9 * dz] = alpha * alpha * (sx[dx] * my[dy] * mz[dz] + mx[dx] * sy[dy] * mz[dz] +
                                                     mx[dx] * my[dy] * sz[dz]) +
                                    mx[dx] * my[dy] * mz[dz];
  // workspace: x (the representers), r, p, p2: nvec x nn doubles each
  double* x = work;
  double* r = x + nvec * nn;
  double* p = r + nvec * nn;
  double* p2 = p + nvec * nn;
  const double* hp[kMaxVec];
  hp[0] = dJ;
  for (int i = 0; i < ncons; ++i) hp[1 + i] = dC[i];
  cudaError_t e = cudaMemcpyAsync(dptrs_dev, hp, nvec * sizeof(double*), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return CELL_ECUDA;
  const unsigned nb = (unsigned)std::min<i64>((nn + kB - 1) / kB, 4096);
  note_launch(), k_cheb_init<<<dim3(nb, nvec), kB, 0, s>>>(dptrs_dev, r, p, x, nn, 1.0 / theta);
  const unsigned nbs = (unsigned)((nn + kB - 1) / kB);
  const double s1 = flat ? 1.0 : theta / delta;
  double rho0 = 1.0 / s1;
  for (int k = 0; k < (flat ? 1 : iters); ++k) {
    const double rho1 = flat ? 0.0 : 1.0 / (2.0 * s1 - rho0);
    const double ca = rho1 * rho0, cb = flat ? 0.0 : 2.0 * rho1 / delta;
    note_launch(), k_cheb_step<<<dim3(nbs, nvec), kB, 0, s>>>(S, p, p2, r, x, nx, ny, nz, ca, cb);
    std::swap(p, p2);
    rho0 = rho1;
  }
  if (flat) iters = 1;
  // the last direction is not added (x_k = x_{k-1} + p_{k-1} is already the iterate)
  note_launch(), k_gram<<<dim3(nblk, nvec), kB, 0, s>>>(x, dptrs_dev, nvec, nn, partial);
  reduce_partials(partial, nblk, nvec, kNvMax, red, 0, nvec, nullptr, s);
  std::vector<double> Gr((size_t)nvec * kNvMax);
  e = cudaMemcpyAsync(Gr.data(), red, Gr.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return CELL_ECUDA;
  // symmetric H Gram matrix of (g_J, g_1..g_N)
  double G[kMaxVec][kMaxVec];
  for (int a = 0; a < nvec; ++a)
    for (int b = 0; b < nvec; ++b) G[a][b] = 0.5 * (Gr[a * kNvMax + b] + Gr[b * kNvMax + a]);
  // constraint block = R^T R (Cholesky, R upper triangular), Rinv = R^-1
  const int N = ncons;
  double R[kMaxVec][kMaxVec] = {}, Ri[kMaxVec][kMaxVec] = {};
  for (int j = 0; j < N; ++j) {
    for (int i = 0; i <= j; ++i) {
      double sum = G[1 + i][1 + j];
      for (int k = 0; k < i; ++k) sum -= R[k][i] * R[k][j];
      if (i == j) {
        // constraint sensitivities linearly dependent (to rounding)
        if (!(sum > 1e-12 * G[1 + i][1 + i])) return CELL_EINVAL;
        R[i][i] = std::sqrt(sum);
      } else {
        R[i][j] = sum / R[i][i];
      }
    }
  }
  for (int j = 0; j < N; ++j) {   // upper-triangular inverse, column by column
    Ri[j][j] = 1.0 / R[j][j];
    for (int i = j - 1; i >= 0; --i) {
      double sum = 0.0;
      for (int k = i + 1; k <= j; ++k) sum += R[i][k] * Ri[k][j];
      Ri[i][j] = -sum / R[i][i];
    }
  }
  // p_k = <g_J, theta_k> with theta_k = sum_i Ri[i][k] g_i
  double pk[kMaxVec] = {}, mu[kMaxVec] = {}, t[kMaxVec] = {};
  double pn2 = G[0][0];
  for (int k = 0; k < N; ++k) {
    for (int i = 0; i <= k; ++i) pk[k] += Ri[i][k] * G[0][1 + i];
    pn2 -= pk[k] * pk[k];
  }
  // R^T mu = w_C C (forward substitution)
  for (int i = 0; i < N; ++i) {
    double sum = wC * C[i];
    for (int k = 0; k < i; ++k) sum -= R[k][i] * mu[k];
    mu[i] = sum / R[i][i];
  }
  const double nP = pn2 > 0.0 ? std::sqrt(pn2) : 0.0;
  const double cJ = nP > 1e-14 * std::sqrt(std::max(G[0][0], 0.0)) && nP > 0.0 ? wJ / nP : 0.0;
  for (int k = 0; k < N; ++k) t[k] = mu[k] - cJ * pk[k];
  Coef co{};
  co.c[0] = cJ;
  for (int i = 0; i < N; ++i) {
    double c = 0.0;
    for (int k = i; k < N; ++k) c += Ri[i][k] * t[k];
    co.c[1 + i] = c;
  }
  note_launch(), k_lincomb_vec<<<nb, kB, 0, s>>>(x, co, nvec, nn, v);
  if (info) {
    info[0] = nP;
    info[1] = iters;
    for (int i = 0; i < N; ++i) info[2 + i] = mu[i];
  }
  e = cudaGetLastError();
  return e == cudaSuccess ? CELL_OK : CELL_ECUDA;
}

}  // namespace cell
