// Batched GMRES building blocks (§2.5: right-preconditioned GMRES, one Krylov
// space per load case): block-partial dot products with FP64 accumulation,
// fused Gram-Schmidt updates, deterministic partial reductions, and the FP64
// Hessenberg / Givens least-squares recurrences on the device.
#include <cstdint>

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

// Block reduction of one value per thread; result valid in thread 0.
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

// Per-thread partial sums use the vector type T (FP32 for the mixed path:
// FP64 arithmetic runs at 1/64 of the FP32 rate on this part and would cap
// the reductions far below HBM bandwidth); block and grid sums are FP64.

// Reduce G per-thread values over the block; thread i < G gets total i.
template <int G>
__device__ __forceinline__ void block_sum_many(double (&v)[G], double (*sh)[G]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < G; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < G; ++i) sh[wid][i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < G) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t += sh[w][threadIdx.x];
    v[0] = t;
  }
}

constexpr int kGrp = 8;

// grid (nblk, nrhs, ceil(nv / G)); each block computes the partial dots of w
// with the G basis vectors of its group over a contiguous chunk of len.  The
// element loop is unrolled so that each thread keeps several elements' loads
// in flight (these kernels are bound by HBM latency and bandwidth).
template <typename T, int G>
__global__ void __launch_bounds__(kB)
k_multidot(const T* __restrict__ V, i64 vstride, i64 rstride, int nv, const T* __restrict__ w,
           i64 wstride, i64 len, double* __restrict__ partial, int nvmax, const int* active) {
  __shared__ double sh[kWarps][G];
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const int g0 = blockIdx.z * G;
  const int ng = nv - g0 < G ? nv - g0 : G;
  const i64 chunk = (len + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk;
  const i64 hi = lo + chunk < len ? lo + chunk : len;
  const T* W = w + q * wstride;
  const T* V0 = V + q * rstride + (i64)g0 * vstride;
  T acc[G];
#pragma unroll
  for (int i = 0; i < G; ++i) acc[i] = T(0);
#pragma unroll 2
  for (i64 k = lo + threadIdx.x; k < hi; k += kB) {
    const T wk = W[k];
#pragma unroll
    for (int i = 0; i < G; ++i)
      if (i < ng) acc[i] = fma(V0[(i64)i * vstride + k], wk, acc[i]);
  }
  double d[G];
#pragma unroll
  for (int i = 0; i < G; ++i) d[i] = (double)acc[i];
  block_sum_many<G>(d, sh);
  if (threadIdx.x < ng) partial[((i64)q * gridDim.x + blockIdx.x) * nvmax + g0 + threadIdx.x] = d[0];
}

// FP32 variants with 16-byte loads (all lengths and strides multiples of 4,
// 16-byte aligned bases): a quarter of the load instructions and four times
// the bytes in flight per thread.
__device__ __forceinline__ float dot4(const float4 a, const float4 b, float acc) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
}

template <int G>
__global__ void __launch_bounds__(kB)
k_multidot4(const float* __restrict__ V, i64 vstride, i64 rstride, int nv, const float* __restrict__ w,
            i64 wstride, i64 len, double* __restrict__ partial, int nvmax, const int* active) {
  __shared__ double sh[kWarps][G];
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const int g0 = blockIdx.z * G;
  const int ng = nv - g0 < G ? nv - g0 : G;
  const i64 len4 = len >> 2;
  const i64 chunk = (len4 + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk;
  const i64 hi = lo + chunk < len4 ? lo + chunk : len4;
  const float4* W = reinterpret_cast<const float4*>(w + q * wstride);
  const float* V0 = V + q * rstride + (i64)g0 * vstride;
  float acc[G];
#pragma unroll
  for (int i = 0; i < G; ++i) acc[i] = 0.f;
  for (i64 k = lo + threadIdx.x; k < hi; k += kB) {
    const float4 wk = W[k];
#pragma unroll
    for (int i = 0; i < G; ++i)
      if (i < ng) acc[i] = dot4(reinterpret_cast<const float4*>(V0 + (i64)i * vstride)[k], wk, acc[i]);
  }
  double d[G];
#pragma unroll
  for (int i = 0; i < G; ++i) d[i] = (double)acc[i];
  block_sum_many<G>(d, sh);
  if (threadIdx.x < ng) partial[((i64)q * gridDim.x + blockIdx.x) * nvmax + g0 + threadIdx.x] = d[0];
}

// w -= sum_i h_i V_i (FP32, 16-byte loads); mode 2 also writes |w_new|^2.
__global__ void __launch_bounds__(kB)
k_update4(const float* __restrict__ V, i64 vstride, i64 rstride, int nv, const double* __restrict__ h,
          int nvmax, float* __restrict__ w, i64 wstride, i64 len, int mode, double* __restrict__ partial,
          const int* active) {
  __shared__ double sh[kWarps][1];
  __shared__ float hs[64];
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  for (int i = threadIdx.x; i < 64; i += kB) hs[i] = i < nv ? (float)h[q * nvmax + i] : 0.f;
  __syncthreads();
  const i64 len4 = len >> 2;
  const i64 chunk = (len4 + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk;
  const i64 hi = lo + chunk < len4 ? lo + chunk : len4;
  float4* W = reinterpret_cast<float4*>(w + q * wstride);
  const float* V0 = V + q * rstride;
  float nrm = 0.f;
  for (i64 k = lo + threadIdx.x; k < hi; k += kB) {
    float4 x = W[k];
    int i = 0;
    for (; i + 2 <= nv; i += 2) {
      const float4 a0 = reinterpret_cast<const float4*>(V0 + (i64)i * vstride)[k];
      const float4 a1 = reinterpret_cast<const float4*>(V0 + (i64)(i + 1) * vstride)[k];
      const float h0 = -hs[i], h1 = -hs[i + 1];
      x.x = fmaf(h1, a1.x, fmaf(h0, a0.x, x.x));
      x.y = fmaf(h1, a1.y, fmaf(h0, a0.y, x.y));
      x.z = fmaf(h1, a1.z, fmaf(h0, a0.z, x.z));
      x.w = fmaf(h1, a1.w, fmaf(h0, a0.w, x.w));
    }
    if (i < nv) {
      const float4 a0 = reinterpret_cast<const float4*>(V0 + (i64)i * vstride)[k];
      const float h0 = -hs[i];
      x.x = fmaf(h0, a0.x, x.x);
      x.y = fmaf(h0, a0.y, x.y);
      x.z = fmaf(h0, a0.z, x.z);
      x.w = fmaf(h0, a0.w, x.w);
    }
    W[k] = x;
    nrm = dot4(x, x, nrm);
  }
  if (mode == 2) {
    double d[1] = {(double)nrm};
    block_sum_many<1>(d, sh);
    if (threadIdx.x == 0) partial[((i64)q * gridDim.x + blockIdx.x) * nvmax + 0] = d[0];
  }
}

// k_update_dots with 16-byte loads (FP32, nv <= G <= 16: the nv basis
// float4 values of the element stay in registers between the update and the
// dots).
template <int G>
__global__ void __launch_bounds__(kB)
k_update_dots4(const float* __restrict__ V, i64 vstride, i64 rstride, int nv, const double* __restrict__ h,
               int nvmax, float* __restrict__ w, i64 wstride, i64 len, double* __restrict__ partial,
               const int* active) {
  __shared__ double sh[kWarps][G + 1];
  __shared__ float hs[G];
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  for (int i = threadIdx.x; i < G; i += kB) hs[i] = i < nv ? (float)h[q * nvmax + i] : 0.f;
  __syncthreads();
  const i64 len4 = len >> 2;
  const i64 chunk = (len4 + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk;
  const i64 hi = lo + chunk < len4 ? lo + chunk : len4;
  float4* W = reinterpret_cast<float4*>(w + q * wstride);
  const float* V0 = V + q * rstride;
  float acc[G + 1];
#pragma unroll
  for (int i = 0; i <= G; ++i) acc[i] = 0.f;
  for (i64 k = lo + threadIdx.x; k < hi; k += kB) {
    float4 v[G];
#pragma unroll
    for (int i = 0; i < G; ++i)
      v[i] = i < nv ? reinterpret_cast<const float4*>(V0 + (i64)i * vstride)[k] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 x = W[k];
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const float hi_ = -hs[i];
      x.x = fmaf(hi_, v[i].x, x.x);
      x.y = fmaf(hi_, v[i].y, x.y);
      x.z = fmaf(hi_, v[i].z, x.z);
      x.w = fmaf(hi_, v[i].w, x.w);
    }
    W[k] = x;
#pragma unroll
    for (int i = 0; i < G; ++i) acc[i] = dot4(v[i], x, acc[i]);
    acc[G] = dot4(x, x, acc[G]);
  }
  double d[G + 1];
#pragma unroll
  for (int i = 0; i <= G; ++i) d[i] = (double)acc[i];
  block_sum_many<G + 1>(d, sh);
  const i64 base = ((i64)q * gridDim.x + blockIdx.x) * nvmax;
  if (threadIdx.x < nv) partial[base + threadIdx.x] = d[0];
  if (threadIdx.x == G) partial[base + nv] = d[0];
}

inline bool vec4_ok(const void* a, const void* b, i64 s1, i64 s2, i64 len) {
  return ((uintptr_t)a & 15u) == 0 && ((uintptr_t)b & 15u) == 0 && s1 % 4 == 0 && s2 % 4 == 0 && len % 4 == 0;
}

// Fused Gram-Schmidt step: w -= sum_i h_i V_i and, in the same pass, the
// partial dots <V_i, w_new> (the coefficients of the next classical pass)
// and |w_new|^2 -> partial[..*nvmax + i] (i < nv) and [..*nvmax + nv].  Each
// thread keeps the nv basis values of its element in registers, so the basis
// is read once for both.  nv <= G.
template <typename T, int G>
__global__ void __launch_bounds__(kB)
k_update_dots(const T* __restrict__ V, i64 vstride, i64 rstride, int nv, const double* __restrict__ h,
              int nvmax, T* __restrict__ w, i64 wstride, i64 len, double* __restrict__ partial,
              const int* active) {
  __shared__ double sh[kWarps][G + 1];
  __shared__ T hs[G];
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  for (int i = threadIdx.x; i < G; i += kB) hs[i] = i < nv ? (T)h[q * nvmax + i] : T(0);
  __syncthreads();
  const i64 chunk = (len + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk;
  const i64 hi = lo + chunk < len ? lo + chunk : len;
  T* W = w + q * wstride;
  const T* V0 = V + q * rstride;
  T acc[G + 1];
#pragma unroll
  for (int i = 0; i <= G; ++i) acc[i] = T(0);
  for (i64 k = lo + threadIdx.x; k < hi; k += kB) {
    T v[G];
#pragma unroll
    for (int i = 0; i < G; ++i) v[i] = i < nv ? V0[(i64)i * vstride + k] : T(0);
    T x = W[k];
#pragma unroll
    for (int i = 0; i < G; ++i) x = fma(-hs[i], v[i], x);
    W[k] = x;
#pragma unroll
    for (int i = 0; i < G; ++i) acc[i] = fma(v[i], x, acc[i]);
    acc[G] = fma(x, x, acc[G]);
  }
  double d[G + 1];
#pragma unroll
  for (int i = 0; i <= G; ++i) d[i] = (double)acc[i];
  block_sum_many<G + 1>(d, sh);
  const i64 base = ((i64)q * gridDim.x + blockIdx.x) * nvmax;
  if (threadIdx.x < nv) partial[base + threadIdx.x] = d[0];
  if (threadIdx.x == G) partial[base + nv] = d[0];
}

// One warp per (rhs, i): fixed-order sum over blocks.
__global__ void k_reduce_partials(const double* __restrict__ partial, int nblk, int nv, int nvmax,
                                  double* __restrict__ out, int accumulate, const int* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const int i = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partial[((i64)q * nblk + b) * nvmax + i];
  s = warp_sum(s);
  if (lane == 0) out[q * nvmax + i] = accumulate ? out[q * nvmax + i] + s : s;
}

// w -= sum_i h_i V_i; mode 2 also writes block-partial |w_new|^2.
template <typename T>
__global__ void __launch_bounds__(kB)
k_update(const T* __restrict__ V, i64 vstride, i64 rstride, int nv, const double* __restrict__ h,
         int nvmax, T* __restrict__ w, i64 wstride, i64 len, int mode, double* __restrict__ partial,
         const int* active) {
  __shared__ double sh[kWarps][1];
  __shared__ T hs[64];
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  for (int i = threadIdx.x; i < 64; i += kB) hs[i] = i < nv ? (T)h[q * nvmax + i] : T(0);
  __syncthreads();
  const i64 chunk = (len + gridDim.x - 1) / gridDim.x;
  const i64 lo = (i64)blockIdx.x * chunk;
  const i64 hi = lo + chunk < len ? lo + chunk : len;
  T* W = w + q * wstride;
  const T* V0 = V + q * rstride;
  T nrm = T(0);
#pragma unroll 2
  for (i64 k = lo + threadIdx.x; k < hi; k += kB) {
    T x = W[k];
    const T* vp = V0 + k;
    int i = 0;
    for (; i + 4 <= nv; i += 4) {
      const T a0 = vp[(i64)i * vstride], a1 = vp[(i64)(i + 1) * vstride];
      const T a2 = vp[(i64)(i + 2) * vstride], a3 = vp[(i64)(i + 3) * vstride];
      x = fma(-hs[i], a0, x);
      x = fma(-hs[i + 1], a1, x);
      x = fma(-hs[i + 2], a2, x);
      x = fma(-hs[i + 3], a3, x);
    }
    for (; i < nv; ++i) x = fma(-hs[i], vp[(i64)i * vstride], x);
    W[k] = x;
    nrm = fma(x, x, nrm);
  }
  if (mode == 2) {
    double d[1] = {(double)nrm};
    block_sum_many<1>(d, sh);
    if (threadIdx.x == 0) partial[((i64)q * gridDim.x + blockIdx.x) * nvmax + 0] = d[0];
  }
}

// Normalisation of the new basis vector, in the vector's own precision (an
// FP32 vector scaled through FP64 arithmetic and conversions would run at the
// FP64 rate); FP32 vectors move as 16-byte chunks when aligned.
template <typename T>
__global__ void k_scale(T* __restrict__ w, i64 wstride, i64 len, const double* __restrict__ sc) {
  const int q = blockIdx.y;
  const double f = sc[q];
  if (f == 1.0) return;
  T* W = w + q * wstride;
  const T ft = (T)f;
  if constexpr (sizeof(T) == 4) {
    if ((((uintptr_t)W) & 15) == 0 && (len & 3) == 0) {
      float4* W4 = reinterpret_cast<float4*>(W);
      for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < (len >> 2); k += (i64)gridDim.x * blockDim.x) {
        float4 v = W4[k];
        v.x *= ft; v.y *= ft; v.z *= ft; v.w *= ft;
        W4[k] = v;
      }
      return;
    }
  }
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (i64)gridDim.x * blockDim.x)
    W[k] *= ft;
}

template <typename T>
__global__ void k_lincomb(const T* __restrict__ V, i64 vstride, i64 rstride,
                          const double* __restrict__ y, const int* __restrict__ kcount, int nvmax,
                          T* __restrict__ u, i64 ustride, i64 len, const int* active) {
  __shared__ double ys[64];
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const int kq = kcount[q];
  for (int i = threadIdx.x; i < kq; i += blockDim.x) ys[i] = y[q * nvmax + i];
  __syncthreads();
  const T* V0 = V + q * rstride;
  T* U = u + q * ustride;
  // accumulate in the vector type: the basis is T already, and FP64
  // arithmetic (1/64 rate) would dominate this pass for FP32 vectors
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (i64)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int i = 0; i < kq; ++i) acc = fma((T)ys[i], V0[i * vstride + k], acc);
    U[k] = acc;
  }
}

// Column j of the Hessenberg matrix: hcol[0..j] from Gram-Schmidt and
// h_{j+1,j} = sqrt(hnorm2).  Applies the stored rotations, forms the new one,
// updates the least-squares right-hand side g and the residual estimate.
// H is stored per rhs column-major with leading dimension m+1.
__global__ void k_givens(double* H, double* cs, double* sn, double* g, const double* hcol,
                         const double* hnorm2, int j, int m, int nvmax, int* active, double* resid,
                         const double* tolabs, double* invscale, int* kcount, int nrhs) {
  const int q = threadIdx.x;
  if (q >= nrhs) return;
  if (!active[q]) {
    invscale[q] = 1.0;
    return;
  }
  double* Hq = H + (i64)q * (m + 1) * m + (i64)j * (m + 1);
  double* cq = cs + q * m;
  double* sq = sn + q * m;
  double* gq = g + q * (m + 1);
  for (int i = 0; i <= j; ++i) Hq[i] = hcol[q * nvmax + i];
  const double hn = sqrt(fmax(hnorm2[q * nvmax], 0.0));
  for (int i = 0; i < j; ++i) {
    const double a = Hq[i], b = Hq[i + 1];
    Hq[i] = cq[i] * a + sq[i] * b;
    Hq[i + 1] = -sq[i] * a + cq[i] * b;
  }
  const double a = Hq[j], b = hn;
  const double rr = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (rr > 0.0) {
    c = a / rr;
    s = b / rr;
  }
  cq[j] = c;
  sq[j] = s;
  Hq[j] = rr;
  Hq[j + 1] = 0.0;
  const double gj = gq[j];
  gq[j] = c * gj;
  gq[j + 1] = -s * gj;
  const double res = fabs(gq[j + 1]);
  resid[q] = res;
  kcount[q] = j + 1;
  // breakdown (invariant subspace) or convergence: this space is done
  const bool brk = !(hn > 1e-300) || !(hn > 1e-14 * fabs(rr));
  invscale[q] = brk ? 0.0 : 1.0 / hn;
  if (res <= tolabs[q] || brk || j + 1 >= m) active[q] = 0;
}

// Reorthogonalisation test ("twice is enough"): after one classical
// Gram-Schmidt pass, repeat it for load q only if the new norm fell below
// 1/sqrt(2) of the norm before the pass (hcol[j+1] holds |w|^2 before).
__global__ void k_reorth_flag(const double* hcol, const double* hnorm2, int j, int nvmax,
                              const int* active, int* reorth, int nrhs) {
  const int q = threadIdx.x;
  if (q >= nrhs) return;
  const double before = hcol[q * nvmax + j + 1];
  reorth[q] = (active[q] && hnorm2[q * nvmax] < 0.5 * before) ? 1 : 0;
}

// Solve the k x k upper-triangular R y = g per rhs (mask: rhs that ran this cycle).
__global__ void k_backsolve(const double* H, const double* g, const int* kcount, int m, double* y,
                            int nvmax, int nrhs, const int* mask) {
  const int q = threadIdx.x;
  if (q >= nrhs || !mask[q]) return;
  const int k = kcount[q];
  const double* Hq = H + (i64)q * (m + 1) * m;
  const double* gq = g + q * (m + 1);
  double* yq = y + q * nvmax;
  for (int i = k - 1; i >= 0; --i) {
    double t = gq[i];
    for (int l = i + 1; l < k; ++l) t -= Hq[(i64)l * (m + 1) + i] * yq[l];
    const double d = Hq[(i64)i * (m + 1) + i];
    yq[i] = d != 0.0 ? t / d : 0.0;
  }
}

// Start of a GMRES cycle: beta = ||r0||, g = beta e1, v0 scale = 1/beta.
__global__ void k_start_cycle(const double* beta2, double* g, int m, int nvmax, int* active,
                              const int* want, double* resid, double* invscale,
                              const double* tolabs, int* kcount, int nrhs) {
  const int q = threadIdx.x;
  if (q >= nrhs) return;
  const double beta = sqrt(fmax(beta2[q * nvmax], 0.0));
  double* gq = g + q * (m + 1);
  for (int i = 0; i <= m; ++i) gq[i] = 0.0;
  gq[0] = beta;
  resid[q] = beta;
  kcount[q] = 0;
  const bool go = want[q] && beta > tolabs[q] && beta > 0.0;
  active[q] = go ? 1 : 0;
  invscale[q] = go ? 1.0 / beta : 1.0;
}

__global__ void k_to_f32(const double* __restrict__ r, i64 rs, float* __restrict__ v, i64 vs,
                         i64 len, const double* __restrict__ sc, const int* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const double f = sc[q];
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (i64)gridDim.x * blockDim.x)
    v[q * vs + k] = (float)(r[q * rs + k] * f);
}

template <typename T>
__global__ void k_axpy_f64(double* __restrict__ x, i64 xs, const T* __restrict__ d, i64 ds, i64 len,
                           const double* __restrict__ sc, const int* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const double f = sc[q];
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (i64)gridDim.x * blockDim.x)
    x[q * xs + k] += f * (double)d[q * ds + k];
}

template <typename T>
__global__ void k_fill(T* p, i64 n, T v) {
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (i64)gridDim.x * blockDim.x) p[k] = v;
}

inline unsigned stream_blocks(i64 len) {
  i64 b = (len + kB - 1) / kB;
  if (b > 4096) b = 4096;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
void multidot(const T* V, i64 vstride, i64 rstride, int nv, const T* w, i64 wstride, i64 len,
              double* partial, int nblk, int nvmax, int nrhs, const int* active, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (vec4_ok(V, w, vstride, rstride, len) && wstride % 4 == 0) {
      const unsigned ng = (unsigned)((nv + 15) / 16);
      note_launch(), k_multidot4<16><<<dim3(nblk, nrhs, ng), kB, 0, s>>>(V, vstride, rstride, nv, w, wstride,
                                                                         len, partial, nvmax, active);
      return;
    }
  }
  // one vector (norms): a single accumulator; up to 16 vectors: one group
  // per block (w read once); else groups of 8
  if (nv == 1) {
    note_launch(), k_multidot<T, 1><<<dim3(nblk, nrhs, 1), kB, 0, s>>>(V, vstride, rstride, nv, w, wstride,
                                                                       len, partial, nvmax, active);
    return;
  }
  if (nv <= 16) {
    note_launch(), k_multidot<T, 16><<<dim3(nblk, nrhs, 1), kB, 0, s>>>(V, vstride, rstride, nv, w, wstride,
                                                                        len, partial, nvmax, active);
    return;
  }
  const unsigned ng = (unsigned)((nv + kGrp - 1) / kGrp);
  note_launch(), k_multidot<T, kGrp><<<dim3(nblk, nrhs, ng), kB, 0, s>>>(V, vstride, rstride, nv, w, wstride,
                                                                         len, partial, nvmax, active);
}

template <typename T>
void update_dots(const T* V, i64 vstride, i64 rstride, int nv, const double* h, int nvmax, T* w,
                 i64 wstride, i64 len, double* partial, int nblk, int nrhs, const int* active,
                 cudaStream_t s) {
  const dim3 g(nblk, nrhs);
  if constexpr (sizeof(T) == 4) {
    if (nv <= 16 && vec4_ok(V, w, vstride, rstride, len) && wstride % 4 == 0) {
      if (nv <= 8) note_launch(), k_update_dots4<8><<<g, kB, 0, s>>>(V, vstride, rstride, nv, h, nvmax, w, wstride, len, partial, active);
      else note_launch(), k_update_dots4<16><<<g, kB, 0, s>>>(V, vstride, rstride, nv, h, nvmax, w, wstride, len, partial, active);
      return;
    }
  }
  if (nv <= 8) note_launch(), k_update_dots<T, 8><<<g, kB, 0, s>>>(V, vstride, rstride, nv, h, nvmax, w, wstride, len, partial, active);
  else if (nv <= 16) note_launch(), k_update_dots<T, 16><<<g, kB, 0, s>>>(V, vstride, rstride, nv, h, nvmax, w, wstride, len, partial, active);
  else if (nv <= 32) note_launch(), k_update_dots<T, 32><<<g, kB, 0, s>>>(V, vstride, rstride, nv, h, nvmax, w, wstride, len, partial, active);
  else note_launch(), k_update_dots<T, 63><<<g, kB, 0, s>>>(V, vstride, rstride, nv, h, nvmax, w, wstride, len, partial, active);
}

void reduce_partials(const double* partial, int nblk, int nv, int nvmax, double* out, int accumulate,
                     int nrhs, const int* active, cudaStream_t s) {
  const int wpb = 4;
  note_launch(), k_reduce_partials<<<dim3((nv + wpb - 1) / wpb, nrhs), 32 * wpb, 0, s>>>(partial, nblk, nv, nvmax,
                                                                         out, accumulate, active);
}

template <typename T>
void update(const T* V, i64 vstride, i64 rstride, int nv, const double* h, int nvmax, T* w,
            i64 wstride, i64 len, int mode, double* partial, int nblk, int nrhs, const int* active,
            cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (mode != 1 && vec4_ok(V, w, vstride, rstride, len) && wstride % 4 == 0) {
      note_launch(), k_update4<<<dim3(nblk, nrhs), kB, 0, s>>>(V, vstride, rstride, nv, h, nvmax, w, wstride,
                                                               len, mode == 2 ? 2 : 0, partial, active);
      return;
    }
  }
  note_launch(), k_update<T><<<dim3(nblk, nrhs), kB, 0, s>>>(V, vstride, rstride, nv, h, nvmax, w,
                                                             wstride, len, mode == 2 ? 2 : 0,
                                                             partial, active);
  if (mode == 1) multidot<T>(V, vstride, rstride, nv, w, wstride, len, partial, nblk, nvmax, nrhs, active, s);
}

template <typename T>
void scale_vec(T* w, i64 wstride, i64 len, const double* sc, int nrhs, cudaStream_t s) {
  note_launch(), k_scale<T><<<dim3(stream_blocks(len), nrhs), kB, 0, s>>>(w, wstride, len, sc);
}

template <typename T>
void lincomb(const T* V, i64 vstride, i64 rstride, const double* y, const int* kcount, int nvmax,
             T* u, i64 ustride, i64 len, int nrhs, const int* active, cudaStream_t s) {
  note_launch(), k_lincomb<T><<<dim3(stream_blocks(len), nrhs), kB, 0, s>>>(V, vstride, rstride, y, kcount, nvmax,
                                                              u, ustride, len, active);
}

void givens_step(double* H, double* cs, double* sn, double* g, const double* hcol,
                 const double* hnorm2, int j, int m, int* active, double* resid,
                 const double* tolabs, double* invscale, int* kcount, int nrhs, cudaStream_t s) {
  note_launch(), k_givens<<<1, 32, 0, s>>>(H, cs, sn, g, hcol, hnorm2, j, m, 64, active, resid, tolabs, invscale,
                            kcount, nrhs);
}

void reorth_flag(const double* hcol, const double* hnorm2, int j, const int* active, int* reorth,
                 int nrhs, cudaStream_t s) {
  note_launch(), k_reorth_flag<<<1, 32, 0, s>>>(hcol, hnorm2, j, 64, active, reorth, nrhs);
}

void backsolve(const double* H, const double* g, const int* kcount, int m, double* y, int nrhs,
               const int* mask, cudaStream_t s) {
  note_launch(), k_backsolve<<<1, 32, 0, s>>>(H, g, kcount, m, y, 64, nrhs, mask);
}

void start_cycle(const double* beta2, double* g, int m, int* active, const int* want, double* resid,
                 double* invscale, const double* tolabs, int* kcount, int nrhs, cudaStream_t s) {
  note_launch(), k_start_cycle<<<1, 32, 0, s>>>(beta2, g, m, 64, active, want, resid, invscale, tolabs, kcount, nrhs);
}

void to_f32_scaled(const double* r, i64 rs, float* v, i64 vs, i64 len, const double* sc, int nrhs,
                   const int* active, cudaStream_t s) {
  note_launch(), k_to_f32<<<dim3(stream_blocks(len), nrhs), kB, 0, s>>>(r, rs, v, vs, len, sc, active);
}

template <typename T>
void axpy_f64(double* x, i64 xs, const T* d, i64 ds, i64 len, const double* sc, int nrhs,
              const int* active, cudaStream_t s) {
  note_launch(), k_axpy_f64<T><<<dim3(stream_blocks(len), nrhs), kB, 0, s>>>(x, xs, d, ds, len, sc, active);
}

template <typename T>
void fill(T* p, i64 n, T v, cudaStream_t s) {
  note_launch(), k_fill<T><<<stream_blocks(n), kB, 0, s>>>(p, n, v);
}

#define INST(T)                                                                                    \
  template void multidot<T>(const T*, i64, i64, int, const T*, i64, i64, double*, int, int, int,   \
                            const int*, cudaStream_t);                                             \
  template void update<T>(const T*, i64, i64, int, const double*, int, T*, i64, i64, int, double*, \
                          int, int, const int*, cudaStream_t);                                     \
  template void update_dots<T>(const T*, i64, i64, int, const double*, int, T*, i64, i64, double*, \
                               int, int, const int*, cudaStream_t);                                \
  template void scale_vec<T>(T*, i64, i64, const double*, int, cudaStream_t);                      \
  template void lincomb<T>(const T*, i64, i64, const double*, const int*, int, T*, i64, i64, int,  \
                           const int*, cudaStream_t);                                              \
  template void axpy_f64<T>(double*, i64, const T*, i64, i64, const double*, int, const int*,      \
                            cudaStream_t);                                                         \
  template void fill<T>(T*, i64, T, cudaStream_t);
INST(float)
INST(double)
template void fill<int>(int*, i64, int, cudaStream_t);
#undef INST

}  // namespace cell
