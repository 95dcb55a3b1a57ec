// Homogenisation reduction that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// homogenised tensors: a framework whose caching allocator owns the whole
// device-memory budget and forbids allocation outside its pools, or a
// real-time loop that must not stall on the driver's allocator (cudaMalloc
// may synchronise the device).  cell_homogenise needs the workspace of a
// cell_handle (made by cell_setup, which allocates); cell_homogenise_noalloc
// instead takes every field from the caller and keeps its block partial sums
// in the fixed device array below.  It copies the three reductions to the
// host and synchronises the caller's stream before it returns.
//
// The array is part of the library image: every GPU that loads libcell.so
// holds it (kScratchDoubles = 83,195 doubles, 665,560 bytes) until the
// process exits.  All calls share it, so calls that overlap on the GPU
// (different streams or threads without ordering between them) race on it and
// give wrong results; calls ordered on one stream are safe.  Each call overwrites every scratch
// word it later reads, so nothing has to be cleared between calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "cell.h"
#include "hostmath.h"
#include "kernels.cuh"

namespace {

constexpr int kMaxBlocks = 1024;            // partial-sum slots per reduction
constexpr long long kChunk = 16384;         // vector entries per block
constexpr long long kScratchDoubles = (long long)kMaxBlocks * 81 + 3 * 81 + 8;
constexpr long long kMaxNodes = kMaxBlocks * kChunk / 4;   // 4,194,304 nodes (e.g. 161^3)
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device, looked up on the first
// call per device (host code must not pass the symbol itself to a kernel).
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CELL_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return CELL_ECUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return CELL_OK;
}

}  // namespace

extern "C" int cell_homogenise_noalloc(const cell_desc* d, const double* rho, const double* bhat,
                                       const double* y, const double* rhat, double CH[36],
                                       double eH[18], double kH[9]) {
  if (!d || !rho || !bhat || !y || !rhat || !CH || !eH || !kH) return CELL_EINVAL;
  if (d->nx < 2 || d->ny < 2 || d->nz < 2) return CELL_EINVAL;
  const long long nn = (long long)d->nx * d->ny * d->nz;
  if (nn > kMaxNodes) return CELL_EINVAL;
  for (int i = 0; i < 36; ++i) if (!std::isfinite(d->C[i])) return CELL_EINVAL;
  for (int i = 0; i < 18; ++i) if (!std::isfinite(d->e[i])) return CELL_EINVAL;
  for (int i = 0; i < 9; ++i) if (!std::isfinite(d->kappa[i])) return CELL_EINVAL;
  // host set-up of the affine-load energy Zbar^T K0 Zbar (no allocation)
  double Cn[36], en[18], kn[9], C0, k0;
  cellhost::nondimensionalise(d->C, d->e, d->kappa, Cn, en, kn, &C0, &k0);
  const double h[3] = {1.0 / d->nx, 1.0 / d->ny, 1.0 / d->nz};
  double K0[1024], Z[288];
  cellhost::element_matrix(Cn, en, kn, h, K0);
  cellhost::affine_loads(h, Z);
  double H0e[81];
  for (int I = 0; I < 9; ++I)
    for (int J = 0; J < 9; ++J) {
      double s = 0.0;
      for (int a = 0; a < 32; ++a) {
        double f = 0.0;
        for (int b = 0; b < 32; ++b) f += K0[a * 32 + b] * Z[b * 9 + J];
        s += Z[a * 9 + I] * f;
      }
      H0e[I * 9 + J] = s;
    }
  cudaStream_t s = static_cast<cudaStream_t>(d->stream);
  // the scratch address is per device: the stream must belong to the current one
  int cur = -1, sdev = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess) e = cudaStreamGetDevice(s, &sdev);
  if (e != cudaSuccess) {
    cell::report_error("cell_homogenise_noalloc: device of the stream", e);
    return CELL_ECUDA;
  }
  if (sdev != cur) {
    cell::report_error("cell_homogenise_noalloc: the stream belongs to another device than the current one",
                       cudaSuccess);
    return CELL_EINVAL;
  }
  double* scr = nullptr;
  const int st = scratch_address(&scr);
  if (st != CELL_OK) return st;
  double* partial = scr;                         // kMaxBlocks * 81
  double* g1 = scr + (long long)kMaxBlocks * 81; // 81
  double* g2 = g1 + 81;                          // 81
  double* srho = g2 + 81;                        // 1
  const int nblk = (int)std::min<long long>(kMaxBlocks, std::max<long long>(1, (4 * nn + kChunk - 1) / kChunk));
  cell::sum_reduce(rho, nn, partial, nblk, srho, s);
  cell::gram9(bhat, y, nn, partial, nblk, g1, s);
  cell::gram9(y, rhat, nn, partial, nblk, g2, s);
  // a failed launch is not sticky: without this check the copies below could
  // return another call's sums left in the shared array
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    cell::report_error("cell_homogenise_noalloc: reduction launch", e);
    return CELL_ECUDA;
  }
  double G1[81], G2[81], sr = 0.0;
  e = cudaMemcpyAsync(G1, g1, sizeof(G1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(G2, g2, sizeof(G2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&sr, srho, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cell::report_error("cell_homogenise_noalloc: copy of the reductions", e);
    return CELL_ECUDA;
  }
  // energy form H = (sum rho) Zbar^T K0 Zbar - b.y - y.r, symmetrised
  double H[81];
  for (int i = 0; i < 81; ++i) H[i] = sr * H0e[i] - G1[i] - G2[i];
  for (int I = 0; I < 9; ++I)
    for (int J = I + 1; J < 9; ++J) {
      const double v = 0.5 * (H[I * 9 + J] + H[J * 9 + I]);
      H[I * 9 + J] = H[J * 9 + I] = v;
    }
  const double se = std::sqrt(C0 * k0);
  for (int p = 0; p < 6; ++p)
    for (int q = 0; q < 6; ++q) CH[p * 6 + q] = C0 * H[p * 9 + q];
  for (int i = 0; i < 3; ++i)
    for (int p = 0; p < 6; ++p) eH[i * 6 + p] = -se * H[(6 + i) * 9 + p];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) kH[i * 3 + j] = -k0 * H[(6 + i) * 9 + 6 + j];
  return CELL_OK;
}
