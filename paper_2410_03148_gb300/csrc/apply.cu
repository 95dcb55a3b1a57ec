// Matrix-free operator applies on the periodic Q1 grid (the hot loop of the
// solver): y = sum_e w_e P_e^T K P_e x, node-centric.
//
// Each thread owns one (node, load) pair and computes the rows of its node
// from the 8 elements around it, gathering the 27 neighbouring nodes once.
// No thread writes another node's value, so there are no atomics and results
// are bitwise reproducible.  For fixed-matrix operators (level 0: w_e = rho_e,
// K = a block of the 32x32 element matrix K0 or the 8x8 local Schur matrix S0)
// the matrix sits in a __constant__ slot (or, when all slots are taken, in a
// by-value kernel parameter), so every multiply-add reads its coefficient
// straight from the constant bank; the full operator pairs its multiply-adds
// (two FP32 FMAs per instruction).  Coarse multigrid levels carry one Galerkin
// matrix per element, stored entry-major (coalesced), or an assembled stencil.
//
// Operator definitions: Eq. (sym-piezo) and its nonsymmetric second form
// (potential rows negated), §2.5; block operators of P_SCP, §2.5.3.
#include <cstring>
#include <mutex>

#include "kernels.cuh"

namespace cell {

namespace {

constexpr int kBlock = 128;
constexpr long long kSplitMaxNodes = 4096;   // levels up to 16^3 use the four-lane stencil apply

struct NodeIdx {
  i64 xo[3], yo[3], zo[3];
  i64 n, nn;
};

// Grid (ceil(nx*ny / kBlock), nz, nrhs): thread -> node (i, j, k) with 32-bit
// index arithmetic; returns false past the end of the xy plane.
__device__ __forceinline__ bool node_index_at(int p, int k, int nx, int ny, int nz, NodeIdx& t) {
  if (p >= nx * ny) return false;
  const int j = p / nx;
  const int i = p - j * nx;
  const i64 nxy = (i64)nx * ny;
  t.nn = nxy * nz;
  t.n = (i64)k * nxy + p;
  t.xo[0] = i == 0 ? nx - 1 : i - 1;
  t.xo[1] = i;
  t.xo[2] = i == nx - 1 ? 0 : i + 1;
  t.yo[0] = (i64)(j == 0 ? ny - 1 : j - 1) * nx;
  t.yo[1] = (i64)j * nx;
  t.yo[2] = (i64)(j == ny - 1 ? 0 : j + 1) * nx;
  t.zo[0] = (i64)(k == 0 ? nz - 1 : k - 1) * nxy;
  t.zo[1] = (i64)k * nxy;
  t.zo[2] = (i64)(k == nz - 1 ? 0 : k + 1) * nxy;
  return true;
}

// Grid (plane blocks, planes, load groups).
__device__ __forceinline__ bool node_index(int nx, int ny, int nz, NodeIdx& t) {
  return node_index_at(blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y, nx, ny, nz, t);
}

// Store the NCO output components of one node according to MODE.
// acc = (A x)_node, dold = this node's own gathered input (CHEB modes).
template <typename T, int NCO, int MODE>
__device__ __forceinline__ void epilogue(const ApplyArgs<T>& a, int r, const NodeIdx& t,
                                         const T* acc, const T* dold) {
  T c1 = a.c1, c2 = a.c2;
  if (MODE != AM_LINEAR && a.cc) {
    c1 = a.cc[0];
    c2 = a.cc[1];
  }
#pragma unroll
  for (int c = 0; c < NCO; ++c) {
    const i64 o = (i64)c * t.nn + t.n;
    if (MODE == AM_LINEAR) {
      T v = a.alpha * acc[c];
      if (a.b) v += a.beta * a.b[r * a.bs + o];
      a.y[r * a.ys + o] = v;
    } else if (MODE == AM_CHEB || MODE == AM_CHEB_LAST) {
      const T rr = a.y[r * a.ys + o] - acc[c];
      a.y[r * a.ys + o] = rr;
      T* sp = a.sol + r * a.ss + o;
      *sp = (a.sol_zero ? T(0) : *sp) + dold[c];
      if (MODE == AM_CHEB) a.dout[r * a.ds + o] = c1 * dold[c] + c2 * a.dinv[o] * rr;
    } else {  // AM_RESID_CHEB0
      const T rr = a.b[r * a.bs + o] - acc[c];
      a.y[r * a.ys + o] = rr;
      a.dout[r * a.ds + o] = c2 * a.dinv[o] * rr;
    }
  }
}

// Constant-bank slots for the FP32 element matrices: a kernel instantiated
// for a slot reads its coefficients at compile-time offsets of a __constant__
// array, which the compiler can fold into the FMA instructions as operands.
// Slots are shared by handles with equal matrices (reference counted, per
// device); kernel parameters remain the fallback when all slots are taken.
constexpr int kSlots = 4;
__constant__ __align__(16) float c_k0[kSlots][1024];   // 16-byte rows: read as float2 pairs too
__constant__ float c_s0[kSlots][64];

template <typename T, int NCM>
struct ParamCoef {
  const FixedMat<T, NCM>& M;
  __device__ __forceinline__ T operator()(int i) const { return M.k[i]; }
};
template <int SLOT, int NCM>
struct ConstCoef {
  __device__ __forceinline__ float operator()(int i) const {
    if constexpr (NCM == 4) return c_k0[SLOT][i];
    else return c_s0[SLOT][i];
  }
};

// Fixed-matrix operator, FP32: the 27 neighbours are preloaded into registers
// and every coefficient index is a compile-time constant.  Neighbour offsets
// are 32-bit and each component plane has its own base pointer, so a load is
// one address multiply-add.
template <typename T, int NCM, int NCI, int NCO, int R0, int C0, bool NEGLAST, int MODE, int RG,
          typename COEF>
__device__ __forceinline__ void apply_fixed_pre_body(const ApplyArgs<T>& a, const COEF& Kc) {
  // RG loads per thread share the index arithmetic, the rho loads and every
  // coefficient fetch; grid z = ceil(nrhs / RG)
  const int r0 = blockIdx.z * RG;
  bool on[RG];
  bool any = false;
#pragma unroll
  for (int g = 0; g < RG; ++g) {
    on[g] = (r0 + g < a.nrhs) && !(a.active && !a.active[r0 + g]);
    any = any || on[g];
  }
  if (!any) return;
  const int nx = a.nx, ny = a.ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nx * ny) return;
  const int j = p / nx;
  const int i = p - j * nx;
  const int k = blockIdx.y;
  const int nxy = nx * ny;
  const int xo[3] = {i == 0 ? nx - 1 : i - 1, i, i == nx - 1 ? 0 : i + 1};
  const int yo[3] = {(j == 0 ? ny - 1 : j - 1) * nx, j * nx, (j == ny - 1 ? 0 : j + 1) * nx};
  const int zo[3] = {(k == 0 ? a.nz - 1 : k - 1) * nxy, k * nxy, (k == a.nz - 1 ? 0 : k + 1) * nxy};
  NodeIdx t;
  t.nn = (i64)nxy * a.nz;
  t.n = (i64)k * nxy + p;
  T xs[RG][27][NCI];
#pragma unroll
  for (int g = 0; g < RG; ++g) {
    const int r = on[g] ? r0 + g : r0;
    const T* X[NCI];
#pragma unroll
    for (int d = 0; d < NCI; ++d) X[d] = a.x + r * a.xs + d * t.nn;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const int m = xo[q % 3] + yo[(q / 3) % 3] + zo[q / 9];
#pragma unroll
      for (int d = 0; d < NCI; ++d) xs[g][q][d] = __ldg(X[d] + m);
    }
  }
  T acc[RG][NCO];
#pragma unroll
  for (int g = 0; g < RG; ++g)
#pragma unroll
    for (int c = 0; c < NCO; ++c) acc[g][c] = T(0);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
    const int la = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
    const T w = __ldg(a.rho + (xo[ex] + yo[ey] + zo[ez]));
    T tl[RG][NCO];
#pragma unroll
    for (int g = 0; g < RG; ++g)
#pragma unroll
      for (int c = 0; c < NCO; ++c) tl[g][c] = T(0);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int q = (ex + (b & 1)) + 3 * (ey + ((b >> 1) & 1)) + 9 * (ez + (b >> 2));
#pragma unroll
      for (int c = 0; c < NCO; ++c)
#pragma unroll
        for (int d = 0; d < NCI; ++d) {
          const T kv = Kc((la * NCM + R0 + c) * (8 * NCM) + b * NCM + C0 + d);
#pragma unroll
          for (int g = 0; g < RG; ++g) tl[g][c] = fma(kv, xs[g][q][d], tl[g][c]);
        }
    }
#pragma unroll
    for (int g = 0; g < RG; ++g)
#pragma unroll
      for (int c = 0; c < NCO; ++c) acc[g][c] = fma(w, tl[g][c], acc[g][c]);
  }
#pragma unroll
  for (int g = 0; g < RG; ++g) {
    if (!on[g]) continue;
    if (NEGLAST) acc[g][NCO - 1] = -acc[g][NCO - 1];
    T dold[NCO];
#pragma unroll
    for (int c = 0; c < NCO; ++c) dold[c] = (MODE == AM_CHEB || MODE == AM_CHEB_LAST) ? xs[g][13][c] : T(0);
    epilogue<T, NCO, MODE>(a, r0 + g, t, acc[g], dold);
  }
}

template <typename T, int NCM, int NCI, int NCO, int R0, int C0, bool NEGLAST, int MODE>
__global__ void __launch_bounds__(kBlock)
k_apply_fixed_pre(const ApplyArgs<T> a, const __grid_constant__ FixedMat<T, NCM> M) {
  apply_fixed_pre_body<T, NCM, NCI, NCO, R0, C0, NEGLAST, MODE, 1>(a, ParamCoef<T, NCM>{M});
}

template <int SLOT, int NCM, int NCI, int NCO, int R0, int C0, bool NEGLAST, int MODE>
__global__ void __launch_bounds__(kBlock) k_apply_fixed_cslot(const ApplyArgs<float> a) {
  // the single-component (local Schur) operator takes three loads per thread
  apply_fixed_pre_body<float, NCM, NCI, NCO, R0, C0, NEGLAST, MODE, (NCI == 1 ? 3 : 1)>(
      a, ConstCoef<SLOT, NCM>{});
}

// Packed-FP32 apply of K0 rows R0 .. R0+NCO-1 to all four input components
// (the full operator Ahat), one (node, load) per thread.  Blackwell's paired
// FMA (two FP32 multiply-adds per issued instruction) halves the issue cost of
// the 1024-term element contraction, which bounds the scalar kernel at ~86 %
// issue use.  Operand pairs are components (0, 1) and (2, 3) of a neighbour
// against the matching adjacent coefficients of a K0 row; each element's pair
// sum is scaled by rho_e with one paired FMA and the halves are added at the
// end.  Capped at 96 registers (five 128-thread blocks per SM).  The same
// pairing measured no gain for the three-component elastic block in its
// Chebyshev modes, which keep the scalar kernel.
template <int SLOT, int NCO, int R0, bool NEGLAST, int MODE>
__global__ void __launch_bounds__(kBlock, 5) k_apply_k0_pk(const ApplyArgs<float> a) {
  const int r = blockIdx.z;
  if (r >= a.nrhs || (a.active && !a.active[r])) return;
  const int nx = a.nx, ny = a.ny;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nx * ny) return;
  const int j = p / nx;
  const int i = p - j * nx;
  const int k = blockIdx.y;
  const int nxy = nx * ny;
  const int xo[3] = {i == 0 ? nx - 1 : i - 1, i, i == nx - 1 ? 0 : i + 1};
  const int yo[3] = {(j == 0 ? ny - 1 : j - 1) * nx, j * nx, (j == ny - 1 ? 0 : j + 1) * nx};
  const int zo[3] = {(k == 0 ? a.nz - 1 : k - 1) * nxy, k * nxy, (k == a.nz - 1 ? 0 : k + 1) * nxy};
  NodeIdx t;
  t.nn = (i64)nxy * a.nz;
  t.n = (i64)k * nxy + p;
  const float* X[4];
#pragma unroll
  for (int d = 0; d < 4; ++d) X[d] = a.x + r * a.xs + d * t.nn;
  float2 x01[27], x23[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int m = xo[q % 3] + yo[(q / 3) % 3] + zo[q / 9];
    x01[q] = make_float2(__ldg(X[0] + m), __ldg(X[1] + m));
    x23[q] = make_float2(__ldg(X[2] + m), __ldg(X[3] + m));
  }
  const float2* K = reinterpret_cast<const float2*>(c_k0[SLOT]);
  float2 acc[NCO];
#pragma unroll
  for (int c = 0; c < NCO; ++c) acc[c] = make_float2(0.f, 0.f);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
    const int la = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
    const float w = __ldg(a.rho + (xo[ex] + yo[ey] + zo[ez]));
    float2 tl[NCO];
#pragma unroll
    for (int c = 0; c < NCO; ++c) tl[c] = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int q = (ex + (b & 1)) + 3 * (ey + ((b >> 1) & 1)) + 9 * (ez + (b >> 2));
#pragma unroll
      for (int c = 0; c < NCO; ++c) {
        const int row = (la * 4 + R0 + c) * 16 + b * 2;   // float2 index of K0[4la+R0+c][4b]
        tl[c] = __ffma2_rn(K[row], x01[q], tl[c]);
        tl[c] = __ffma2_rn(K[row + 1], x23[q], tl[c]);
      }
    }
    const float2 w2 = make_float2(w, w);
#pragma unroll
    for (int c = 0; c < NCO; ++c) acc[c] = __ffma2_rn(w2, tl[c], acc[c]);
  }
  float out[NCO], dold[NCO];
#pragma unroll
  for (int c = 0; c < NCO; ++c) {
    out[c] = acc[c].x + acc[c].y;
    // this node's own input (neighbour 13), used by the Chebyshev modes
    dold[c] = (MODE == AM_CHEB || MODE == AM_CHEB_LAST) ? (c < 2 ? (c ? x01[13].y : x01[13].x)
                                                               : (c == 3 ? x23[13].y : x23[13].x))
                                                        : 0.f;
  }
  if (NEGLAST) out[NCO - 1] = -out[NCO - 1];
  epilogue<float, NCO, MODE>(a, r, t, out, dold);
}

// Fixed-matrix operator, FP64: neighbours are loaded per element (FP64
// arithmetic, not load bandwidth, bounds this variant on GB300).
template <typename T, int NCM, int NCI, int NCO, int R0, int C0, bool NEGLAST, int MODE>
__global__ void __launch_bounds__(kBlock)
k_apply_fixed_ld(const ApplyArgs<T> a, const __grid_constant__ FixedMat<T, NCM> M) {
  const int r = blockIdx.z;
  if (a.active && !a.active[r]) return;
  NodeIdx t;
  if (!node_index(a.nx, a.ny, a.nz, t)) return;
  const T* X = a.x + r * a.xs;
  T acc[NCO];
#pragma unroll
  for (int c = 0; c < NCO; ++c) acc[c] = T(0);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
    const int la = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
    const T w = __ldg(a.rho + t.xo[ex] + t.yo[ey] + t.zo[ez]);
    T tl[NCO];
#pragma unroll
    for (int c = 0; c < NCO; ++c) tl[c] = T(0);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const i64 m = t.xo[ex + (b & 1)] + t.yo[ey + ((b >> 1) & 1)] + t.zo[ez + (b >> 2)];
#pragma unroll
      for (int d = 0; d < NCI; ++d) {
        const T xv = __ldg(X + d * t.nn + m);
#pragma unroll
        for (int c = 0; c < NCO; ++c)
          tl[c] = fma(M.k[(la * NCM + R0 + c) * (8 * NCM) + b * NCM + C0 + d], xv, tl[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NCO; ++c) acc[c] = fma(w, tl[c], acc[c]);
  }
  if (NEGLAST) acc[NCO - 1] = -acc[NCO - 1];
  T dold[NCO];
#pragma unroll
  for (int c = 0; c < NCO; ++c)
    dold[c] = (MODE == AM_CHEB || MODE == AM_CHEB_LAST) ? X[c * t.nn + t.n] : T(0);
  epilogue<T, NCO, MODE>(a, r, t, acc, dold);
}

// Per-element (Galerkin) matrices on a coarse level.  One thread per node
// and group of RG loads (grid z = 9 / RG groups): each element row block
// (NC x 8NC values, entry-major in memory so a warp's loads coalesce) is read
// once per group and applied to the group's loads.  Large levels use RG = 3
// (fewer matrix reads), small levels RG = 1 (more parallelism).
template <typename T, int NC, int RG, int MODE>
__global__ void __launch_bounds__(kBlock) k_apply_elem(const ApplyArgs<T> a, int nrhs) {
  NodeIdx t;
  if (!node_index(a.nx, a.ny, a.nz, t)) return;
  const int r0 = blockIdx.z * RG;
  bool on[RG];
  bool any = false;
#pragma unroll
  for (int g = 0; g < RG; ++g) {
    on[g] = (r0 + g < nrhs) && !(a.active && !a.active[r0 + g]);
    any = any || on[g];
  }
  if (!any) return;
  const i64 ne = t.nn;
  constexpr int R = 8 * NC;
  T acc[RG][NC];
#pragma unroll
  for (int g = 0; g < RG; ++g)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[g][c] = T(0);
#pragma unroll 1
  for (int e = 0; e < 8; ++e) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
    const int la = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
    // neighbour offsets of this element's corners, by select (no local arrays)
    const i64 x0 = ex ? t.xo[1] : t.xo[0], x1 = ex ? t.xo[2] : t.xo[1];
    const i64 y0 = ey ? t.yo[1] : t.yo[0], y1 = ey ? t.yo[2] : t.yo[1];
    const i64 z0 = ez ? t.zo[1] : t.zo[0], z1 = ez ? t.zo[2] : t.zo[1];
    const i64 el = x0 + y0 + z0;
    const T* K = a.ke + (i64)(la * NC) * R * ne + el;
    T km[NC][R];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int b = 0; b < R; ++b) km[c][b] = __ldg(K + (i64)(c * R + b) * ne);
    int m[8];
#pragma unroll
    for (int b = 0; b < 8; ++b)
      m[b] = (int)(((b & 1) ? x1 : x0) + (((b >> 1) & 1) ? y1 : y0) + ((b >> 2) ? z1 : z0));
#pragma unroll
    for (int g = 0; g < RG; ++g) {
      if (!on[g]) continue;
      const T* X = a.x + (r0 + g) * a.xs;
#pragma unroll
      for (int b = 0; b < 8; ++b)
#pragma unroll
        for (int d = 0; d < NC; ++d) {
          const T xv = __ldg(X + d * t.nn + m[b]);
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[g][c] = fma(km[c][b * NC + d], xv, acc[g][c]);
        }
    }
  }
#pragma unroll
  for (int g = 0; g < RG; ++g) {
    if (!on[g]) continue;
    const int r = r0 + g;
    T dold[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c)
      dold[c] = (MODE == AM_CHEB || MODE == AM_CHEB_LAST) ? a.x[r * a.xs + c * t.nn + t.n] : T(0);
    epilogue<T, NC, MODE>(a, r, t, acc[g], dold);
  }
}

// Assembled block stencil on a coarse level: y_n = sum_q S_n[q] x_{n+q} over the
// 27 neighbours q (offsets in {-1,0,1}^3, q = dx + 3 dy + 9 dz).  One thread per
// node and group of RG loads; the node's stencil row (27 NC x NC blocks) is
// read once per group with coalesced loads.  Grid (load groups, plane blocks,
// planes): the groups of one block of nodes are adjacent in launch order and
// run at the same time, so the stencil rows that the first group brings from
// DRAM are L2 hits for the others (a level-1 stencil of a 128^3 cell, 255 MB,
// does not stay in L2 between groups launched a whole grid apart).
template <typename T, int NC, int RG, int MODE>
__global__ void __launch_bounds__(kBlock) k_apply_st(const ApplyArgs<T> a, int nrhs) {
  NodeIdx t;
  if (!node_index_at(blockIdx.y * blockDim.x + threadIdx.x, blockIdx.z, a.nx, a.ny, a.nz, t)) return;
  const int r0 = blockIdx.x * RG;
  bool on[RG];
  bool any = false;
#pragma unroll
  for (int g = 0; g < RG; ++g) {
    on[g] = (r0 + g < nrhs) && !(a.active && !a.active[r0 + g]);
    any = any || on[g];
  }
  if (!any) return;
  T acc[RG][NC], dold[RG][NC];
#pragma unroll
  for (int g = 0; g < RG; ++g)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[g][c] = dold[g][c] = T(0);
  const T* S = a.st + t.n;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int m = (int)(t.xo[q % 3] + t.yo[(q / 3) % 3] + t.zo[q / 9]);
    T sb[NC][NC];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int d = 0; d < NC; ++d) sb[c][d] = __ldg(S + (i64)((q * NC + c) * NC + d) * t.nn);
#pragma unroll
    for (int g = 0; g < RG; ++g) {
      if (!on[g]) continue;
      const T* X = a.x + (r0 + g) * a.xs;
#pragma unroll
      for (int d = 0; d < NC; ++d) {
        const T xv = __ldg(X + d * t.nn + m);
        if (q == 13) dold[g][d] = xv;
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[g][c] = fma(sb[c][d], xv, acc[g][c]);
      }
    }
  }
#pragma unroll
  for (int g = 0; g < RG; ++g) {
    if (!on[g]) continue;
    epilogue<T, NC, MODE>(a, r0 + g, t, acc[g], dold[g]);
  }
}

// Small coarse levels are bound by the latency of the 27 dependent neighbour
// rounds of k_apply_st, not by throughput: here four lanes share one (node,
// load), each taking the neighbours q = lane, lane + 4, ... (7 or 6 of the
// 27), and the partial sums meet by two butterfly shuffles.  Lane 0 of each
// group runs the epilogue.  Grid (ceil(4 nx ny / kBlock), nz, nrhs).
template <typename T, int NC, int MODE>
__global__ void __launch_bounds__(kBlock) k_apply_st_split(const ApplyArgs<T> a, int nrhs) {
  const int r = blockIdx.z;
  if (r >= nrhs || (a.active && !a.active[r])) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane4 = g & 3;
  const int p = g >> 2;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const bool valid = p < nx * ny;   // whole groups of 4 share p: shuffles stay full-warp
  NodeIdx t;
  T acc[NC], dold[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = dold[c] = T(0);
  if (valid) {
    const int j = p / nx, i = p - j * nx, k = blockIdx.y;
    const i64 nxy = (i64)nx * ny;
    t.nn = nxy * nz;
    t.n = (i64)k * nxy + p;
    t.xo[0] = i == 0 ? nx - 1 : i - 1;
    t.xo[1] = i;
    t.xo[2] = i == nx - 1 ? 0 : i + 1;
    t.yo[0] = (i64)(j == 0 ? ny - 1 : j - 1) * nx;
    t.yo[1] = (i64)j * nx;
    t.yo[2] = (i64)(j == ny - 1 ? 0 : j + 1) * nx;
    t.zo[0] = (i64)(k == 0 ? nz - 1 : k - 1) * nxy;
    t.zo[1] = (i64)k * nxy;
    t.zo[2] = (i64)(k == nz - 1 ? 0 : k + 1) * nxy;
    const T* X = a.x + r * a.xs;
    const T* S = a.st + t.n;
#pragma unroll
    for (int kk = 0; kk < 7; ++kk) {
      const int q = 4 * kk + lane4;
      if (q < 27) {
        const int qx = q % 3, qy = (q / 3) % 3, qz = q / 9;
        const i64 ox = qx == 0 ? t.xo[0] : (qx == 1 ? t.xo[1] : t.xo[2]);
        const i64 oy = qy == 0 ? t.yo[0] : (qy == 1 ? t.yo[1] : t.yo[2]);
        const i64 oz = qz == 0 ? t.zo[0] : (qz == 1 ? t.zo[1] : t.zo[2]);
        const i64 m = ox + oy + oz;
        T xv[NC];
#pragma unroll
        for (int d = 0; d < NC; ++d) xv[d] = __ldg(X + d * t.nn + m);
        if (q == 13) {
#pragma unroll
          for (int d = 0; d < NC; ++d) dold[d] = xv[d];
        }
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
          for (int d = 0; d < NC; ++d)
            acc[c] = fma(__ldg(S + (i64)((q * NC + c) * NC + d) * t.nn), xv[d], acc[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 1);
    acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 2);
    dold[c] = __shfl_sync(0xffffffffu, dold[c], (threadIdx.x & ~3) | 1);   // q = 13 is lane 1
  }
  if (!valid || lane4 != 0) return;
  epilogue<T, NC, MODE>(a, r, t, acc, dold);
}

// One thread per (node, output component c): accumulate the element blocks of
// the 8 elements around the node into its 27 neighbour blocks.
template <typename T, int NC>
__global__ void __launch_bounds__(kBlock) k_stencil(const T* __restrict__ ke, T* __restrict__ st,
                                                   int nx, int ny, int nz) {
  NodeIdx t;
  if (!node_index(nx, ny, nz, t)) return;
  const int c = blockIdx.z;
  constexpr int R = 8 * NC;
  T acc[27][NC];
#pragma unroll
  for (int q = 0; q < 27; ++q)
#pragma unroll
    for (int d = 0; d < NC; ++d) acc[q][d] = T(0);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
    const int la = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
    const i64 el = t.xo[ex] + t.yo[ey] + t.zo[ez];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int q = (ex + (b & 1)) + 3 * (ey + ((b >> 1) & 1)) + 9 * (ez + (b >> 2));
#pragma unroll
      for (int d = 0; d < NC; ++d)
        acc[q][d] += __ldg(ke + (i64)((la * NC + c) * R + b * NC + d) * t.nn + el);
    }
  }
#pragma unroll
  for (int q = 0; q < 27; ++q)
#pragma unroll
    for (int d = 0; d < NC; ++d) st[(i64)((q * NC + c) * NC + d) * t.nn + t.n] = acc[q][d];
}

// Paired (two-lane) double-float steps: exact product error, TwoSum.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ void two_sum2(float2& s, float2& lo, float2 p) {
  const float2 m1 = f2(-1.f, -1.f);
  const float2 t = __fadd2_rn(s, p);
  const float2 bb = __ffma2_rn(s, m1, t);                       // t - s
  const float2 e1 = __ffma2_rn(__ffma2_rn(bb, m1, t), m1, s);   // s - (t - bb)
  const float2 e2 = __ffma2_rn(bb, m1, p);                      // p - bb
  lo = __fadd2_rn(lo, __fadd2_rn(e1, e2));
  s = t;
}

// r = b - Ahat x with FP64-grade accuracy from FP32 arithmetic only.  One
// thread per (node, load) computes the four rows: each element's 32 nodal
// pairs (x = xh + xl) are loaded once and feed two row pairs, (0, 1) and
// (2, 3), as paired FP32 operations.  Every product is error-free (FMA
// residual) and every sum a TwoSum, per element and again after the rho_e
// scaling (rho = rho_h + rho_l): the result carries about 2^-46 of the term
// magnitudes, far below the residuals of the refinement loop.
__global__ void __launch_bounds__(kBlock)
k_resid_df(const float* __restrict__ xh, const float* __restrict__ xl, i64 xs,
           const double* __restrict__ b, i64 bs, double* __restrict__ r, i64 rs,
           const float* __restrict__ rho_h, const float* __restrict__ rho_l,
           const __grid_constant__ DFMat M, int nx, int ny, int nz, const int* active) {
  const int q = blockIdx.z;
  if (active && !active[q]) return;
  NodeIdx t;
  if (!node_index(nx, ny, nz, t)) return;
  const float* XH = xh + q * xs;
  const float* XL = xl + q * xs;
  const int nn32 = (int)t.nn;
  const int xo[3] = {(int)t.xo[0], (int)t.xo[1], (int)t.xo[2]};
  const int yo[3] = {(int)t.yo[0], (int)t.yo[1], (int)t.yo[2]};
  const int zo[3] = {(int)t.zo[0], (int)t.zo[1], (int)t.zo[2]};
  float2 ah[2] = {f2(0.f, 0.f), f2(0.f, 0.f)}, al[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll 1
  for (int e = 0; e < 8; ++e) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
    const int la = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
    // corner offsets of this element by select (no dynamically indexed arrays)
    const int x0 = ex ? xo[1] : xo[0], x1 = ex ? xo[2] : xo[1];
    const int y0 = ey ? yo[1] : yo[0], y1 = ey ? yo[2] : yo[1];
    const int z0 = ez ? zo[1] : zo[0], z1 = ez ? zo[2] : zo[1];
    const int el = x0 + y0 + z0;
    float2 sh[2] = {f2(0.f, 0.f), f2(0.f, 0.f)}, sl[2] = {f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll
    for (int bn = 0; bn < 8; ++bn) {
      const int m = ((bn & 1) ? x1 : x0) + (((bn >> 1) & 1) ? y1 : y0) + ((bn >> 2) ? z1 : z0);
#pragma unroll
      for (int d = 0; d < 4; ++d) {
        const float vh = __ldg(XH + (d * nn32 + m)), vl = __ldg(XL + (d * nn32 + m));
        const float2 vh2 = f2(vh, vh), vl2 = f2(vl, vl);
#pragma unroll
        for (int rp = 0; rp < 2; ++rp) {
          const float2 kh = M.kh[(la * 2 + rp) * 32 + bn * 4 + d];
          const float2 kl = M.kl[(la * 2 + rp) * 32 + bn * 4 + d];
          const float2 p = __fmul2_rn(kh, vh2);
          const float2 pe = __ffma2_rn(kh, vh2, f2(-p.x, -p.y));
          two_sum2(sh[rp], sl[rp], p);
          sl[rp] = __ffma2_rn(kh, vl2, __ffma2_rn(kl, vh2, __fadd2_rn(sl[rp], pe)));
        }
      }
    }
    const float wh = __ldg(rho_h + el), wl = __ldg(rho_l + el);
    const float2 wh2 = f2(wh, wh), wl2 = f2(wl, wl);
#pragma unroll
    for (int rp = 0; rp < 2; ++rp) {
      const float2 p = __fmul2_rn(sh[rp], wh2);
      const float2 pe = __ffma2_rn(sh[rp], wh2, f2(-p.x, -p.y));
      two_sum2(ah[rp], al[rp], p);
      al[rp] = __ffma2_rn(sh[rp], wl2, __ffma2_rn(sl[rp], wh2, __fadd2_rn(al[rp], pe)));
    }
  }
  const double v[4] = {(double)ah[0].x + (double)al[0].x, (double)ah[0].y + (double)al[0].y,
                       (double)ah[1].x + (double)al[1].x, -((double)ah[1].y + (double)al[1].y)};
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const i64 o = (i64)c * t.nn + t.n;
    r[q * rs + o] = b ? b[q * bs + o] - v[c] : v[c];
  }
}

__global__ void k_axpy_split_f(double* __restrict__ x, float* __restrict__ xh, float* __restrict__ xl,
                               i64 xs, const float* __restrict__ d, i64 ds, i64 len,
                               const double* __restrict__ sc, const int* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const double f = sc[q];
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (i64)gridDim.x * blockDim.x) {
    const double v = x[q * xs + k] + f * (double)d[q * ds + k];
    x[q * xs + k] = v;
    const float h = (float)v;
    xh[q * xs + k] = h;
    xl[q * xs + k] = (float)(v - (double)h);
  }
}

__global__ void k_axpy_split_d(double* __restrict__ x, float* __restrict__ xh, float* __restrict__ xl,
                               i64 xs, const double* __restrict__ d, i64 ds, i64 len,
                               const double* __restrict__ sc, const int* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const double f = sc[q];
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (i64)gridDim.x * blockDim.x) {
    const double v = x[q * xs + k] + f * d[q * ds + k];
    x[q * xs + k] = v;
    const float h = (float)v;
    xh[q * xs + k] = h;
    xl[q * xs + k] = (float)(v - (double)h);
  }
}

template <typename T>
inline dim3 grid_for(const ApplyArgs<T>& a, int nrhs) {
  const int plane = a.nx * a.ny;
  return dim3((unsigned)((plane + kBlock - 1) / kBlock), (unsigned)a.nz, (unsigned)nrhs);
}

template <int NCM, int NCI, int NCO, int R0, int C0, bool NEG, int MODE>
void launch_cslot(const ApplyArgs<float>& a0, int nrhs, cudaStream_t s) {
  constexpr int RG = NCI == 1 ? 3 : 1;
  ApplyArgs<float> a = a0;
  a.nrhs = nrhs;
  const int groups = (nrhs + RG - 1) / RG;
  const dim3 g = grid_for(a, groups);
  if constexpr (NCM == 4 && NCI == 4 && C0 == 0) {
    switch (a.cslot1 - 1) {
      case 0: note_launch(), k_apply_k0_pk<0, NCO, R0, NEG, MODE><<<g, kBlock, 0, s>>>(a); break;
      case 1: note_launch(), k_apply_k0_pk<1, NCO, R0, NEG, MODE><<<g, kBlock, 0, s>>>(a); break;
      case 2: note_launch(), k_apply_k0_pk<2, NCO, R0, NEG, MODE><<<g, kBlock, 0, s>>>(a); break;
      default: note_launch(), k_apply_k0_pk<3, NCO, R0, NEG, MODE><<<g, kBlock, 0, s>>>(a); break;
    }
    return;
  }
  switch (a.cslot1 - 1) {
    case 0: note_launch(), k_apply_fixed_cslot<0, NCM, NCI, NCO, R0, C0, NEG, MODE><<<g, kBlock, 0, s>>>(a); break;
    case 1: note_launch(), k_apply_fixed_cslot<1, NCM, NCI, NCO, R0, C0, NEG, MODE><<<g, kBlock, 0, s>>>(a); break;
    case 2: note_launch(), k_apply_fixed_cslot<2, NCM, NCI, NCO, R0, C0, NEG, MODE><<<g, kBlock, 0, s>>>(a); break;
    default: note_launch(), k_apply_fixed_cslot<3, NCM, NCI, NCO, R0, C0, NEG, MODE><<<g, kBlock, 0, s>>>(a); break;
  }
}

template <typename T, int NCM, int NCI, int NCO, int R0, int C0, bool NEG, int MODE>
void launch_fixed(const ApplyArgs<T>& a, const FixedMat<T, NCM>& M, int nrhs, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (a.cslot1 > 0) {
      launch_cslot<NCM, NCI, NCO, R0, C0, NEG, MODE>(a, nrhs, s);
    } else {
      ApplyArgs<T> b = a;
      b.nrhs = nrhs;
      note_launch(), k_apply_fixed_pre<T, NCM, NCI, NCO, R0, C0, NEG, MODE><<<grid_for(b, nrhs), kBlock, 0, s>>>(b, M);
    }
  } else
    note_launch(), k_apply_fixed_ld<T, NCM, NCI, NCO, R0, C0, NEG, MODE><<<grid_for(a, nrhs), kBlock, 0, s>>>(a, M);
}

template <typename T, int NCM, int NCI, int NCO, int R0, int C0, bool NEG>
void dispatch_fixed(const ApplyArgs<T>& a, const FixedMat<T, NCM>& M, int mode, int nrhs,
                    cudaStream_t s) {
  switch (mode) {
    case AM_LINEAR: launch_fixed<T, NCM, NCI, NCO, R0, C0, NEG, AM_LINEAR>(a, M, nrhs, s); break;
    case AM_CHEB: launch_fixed<T, NCM, NCI, NCO, R0, C0, NEG, AM_CHEB>(a, M, nrhs, s); break;
    case AM_CHEB_LAST: launch_fixed<T, NCM, NCI, NCO, R0, C0, NEG, AM_CHEB_LAST>(a, M, nrhs, s); break;
    default: launch_fixed<T, NCM, NCI, NCO, R0, C0, NEG, AM_RESID_CHEB0>(a, M, nrhs, s); break;
  }
}

}  // namespace

template <typename T>
void apply_full(const ApplyArgs<T>& a, const FixedMat<T, 4>& M, int mode, int nrhs, cudaStream_t s) {
  // only LINEAR is meaningful for the full (nonsymmetric) operator
  (void)mode;
  launch_fixed<T, 4, 4, 4, 0, 0, true, AM_LINEAR>(a, M, nrhs, s);
}

template <typename T>
void apply_uu(const ApplyArgs<T>& a, const FixedMat<T, 4>& M, int mode, int nrhs, cudaStream_t s) {
  dispatch_fixed<T, 4, 3, 3, 0, 0, false>(a, M, mode, nrhs, s);
}

template <typename T>
void apply_pu(const ApplyArgs<T>& a, const FixedMat<T, 4>& M, int nrhs, cudaStream_t s) {
  launch_fixed<T, 4, 3, 1, 3, 0, false, AM_LINEAR>(a, M, nrhs, s);
}

template <typename T>
void apply_ss(const ApplyArgs<T>& a, const FixedMat<T, 1>& M, int mode, int nrhs, cudaStream_t s) {
  dispatch_fixed<T, 1, 1, 1, 0, 0, false>(a, M, mode, nrhs, s);
}

template <typename T, int NC, int RG>
void launch_elem(const ApplyArgs<T>& a, int mode, int nrhs, cudaStream_t s) {
  const dim3 g = grid_for(a, (nrhs + RG - 1) / RG);
  switch (mode) {
    case AM_LINEAR: note_launch(), k_apply_elem<T, NC, RG, AM_LINEAR><<<g, kBlock, 0, s>>>(a, nrhs); break;
    case AM_CHEB: note_launch(), k_apply_elem<T, NC, RG, AM_CHEB><<<g, kBlock, 0, s>>>(a, nrhs); break;
    case AM_CHEB_LAST: note_launch(), k_apply_elem<T, NC, RG, AM_CHEB_LAST><<<g, kBlock, 0, s>>>(a, nrhs); break;
    default: note_launch(), k_apply_elem<T, NC, RG, AM_RESID_CHEB0><<<g, kBlock, 0, s>>>(a, nrhs); break;
  }
}

template <typename T, int NC>
void apply_elem(const ApplyArgs<T>& a, int mode, int nrhs, cudaStream_t s) {
  const long long nn = (long long)a.nx * a.ny * a.nz;
  if (nn >= 16384) launch_elem<T, NC, 3>(a, mode, nrhs, s);
  else launch_elem<T, NC, 1>(a, mode, nrhs, s);
}

template <typename T, int NC, int RG>
void launch_st(const ApplyArgs<T>& a, int mode, int nrhs, cudaStream_t s) {
  const dim3 g0 = grid_for(a, (nrhs + RG - 1) / RG);
  const dim3 g(g0.z, g0.x, g0.y);   // load groups fastest (see k_apply_st)
  switch (mode) {
    case AM_LINEAR: note_launch(), k_apply_st<T, NC, RG, AM_LINEAR><<<g, kBlock, 0, s>>>(a, nrhs); break;
    case AM_CHEB: note_launch(), k_apply_st<T, NC, RG, AM_CHEB><<<g, kBlock, 0, s>>>(a, nrhs); break;
    case AM_CHEB_LAST: note_launch(), k_apply_st<T, NC, RG, AM_CHEB_LAST><<<g, kBlock, 0, s>>>(a, nrhs); break;
    default: note_launch(), k_apply_st<T, NC, RG, AM_RESID_CHEB0><<<g, kBlock, 0, s>>>(a, nrhs); break;
  }
}

template <typename T, int NC>
void launch_st_split(const ApplyArgs<T>& a, int mode, int nrhs, cudaStream_t s) {
  const dim3 g((unsigned)((4 * a.nx * a.ny + kBlock - 1) / kBlock), (unsigned)a.nz, (unsigned)nrhs);
  switch (mode) {
    case AM_LINEAR: note_launch(), k_apply_st_split<T, NC, AM_LINEAR><<<g, kBlock, 0, s>>>(a, nrhs); break;
    case AM_CHEB: note_launch(), k_apply_st_split<T, NC, AM_CHEB><<<g, kBlock, 0, s>>>(a, nrhs); break;
    case AM_CHEB_LAST: note_launch(), k_apply_st_split<T, NC, AM_CHEB_LAST><<<g, kBlock, 0, s>>>(a, nrhs); break;
    default: note_launch(), k_apply_st_split<T, NC, AM_RESID_CHEB0><<<g, kBlock, 0, s>>>(a, nrhs); break;
  }
}

template <typename T, int NC>
void apply_stencil(const ApplyArgs<T>& a, int mode, int nrhs, cudaStream_t s, int rg) {
  const long long nn = (long long)a.nx * a.ny * a.nz;
  if (nn <= kSplitMaxNodes) {
    launch_st_split<T, NC>(a, mode, nrhs, s);
    return;
  }
  // loads per thread: the tuned value, else three on large levels (all nine
  // per thread chains 27 rounds of 36 loads per thread) and one below
  if (rg <= 0) rg = nn > 16384 ? 3 : 1;
  if (rg == 9) launch_st<T, NC, 9>(a, mode, nrhs, s);
  else if (rg == 3) launch_st<T, NC, 3>(a, mode, nrhs, s);
  else launch_st<T, NC, 1>(a, mode, nrhs, s);
}

// Loads per thread of the coarse stencil apply, timed on the caller's level
// buffers (a as for apply_stencil, in the given mode).  Every choice computes
// each (node, load) with the same operation sequence, so the results are
// bitwise the same; candidates 1, 3 and 9, one warm-up and three timed
// launches each between CUDA events on the stream.  Returns 0 (keep the
// default) on levels that use the four-lane kernel or if nothing was timed.
template <typename T, int NC>
int stencil_autotune(const ApplyArgs<T>& a, int mode, int nrhs, cudaStream_t s, float* best_us) {
  constexpr int kReps = 3;
  if (best_us) *best_us = 0.f;
  if ((long long)a.nx * a.ny * a.nz <= kSplitMaxNodes) return 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return 0;
  }
  int best = 0;
  float best_t = 3.0e38f;
  for (int rg : {1, 3, 9}) {
    apply_stencil<T, NC>(a, mode, nrhs, s, rg);
    cudaEventRecord(e0, s);
    for (int r = 0; r < kReps; ++r) apply_stencil<T, NC>(a, mode, nrhs, s, rg);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) continue;
    if (ms < best_t) {
      best_t = ms;
      best = rg;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best && best_us) *best_us = best_t * 1000.f / kReps;
  return best;
}

template <typename T, int NC>
void stencil_from_elem(const T* ke, T* st, int nx, int ny, int nz, cudaStream_t s) {
  ApplyArgs<T> a{};
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  note_launch(), k_stencil<T, NC><<<grid_for(a, NC), kBlock, 0, s>>>(ke, st, nx, ny, nz);
}

void resid_df(const float* xh, const float* xl, i64 xs, const double* b, i64 bs, double* r, i64 rs,
              const float* rho_h, const float* rho_l, const DFMat& M, int nx, int ny, int nz,
              int nrhs, const int* active, cudaStream_t s) {
  ApplyArgs<float> a{};
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  note_launch(), k_resid_df<<<grid_for(a, nrhs), kBlock, 0, s>>>(xh, xl, xs, b, bs, r, rs, rho_h, rho_l, M,
                                                                  nx, ny, nz, active);
}

__global__ void k_split(const double* __restrict__ x, float* __restrict__ xh, float* __restrict__ xl,
                        i64 n) {
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (i64)gridDim.x * blockDim.x) {
    const double v = x[k];
    const float h = (float)v;
    xh[k] = h;
    xl[k] = (float)(v - (double)h);
  }
}

void split_f64(const double* x, float* xh, float* xl, i64 n, cudaStream_t s) {
  i64 blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  note_launch(), k_split<<<(unsigned)blocks, 256, 0, s>>>(x, xh, xl, n);
}

template <typename T>
void axpy_split(double* x, float* xh, float* xl, i64 xs, const T* d, i64 ds, i64 len,
                const double* sc, int nrhs, const int* active, cudaStream_t s) {
  i64 blocks = (len + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if constexpr (sizeof(T) == 4)
    note_launch(), k_axpy_split_f<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(x, xh, xl, xs, d, ds, len, sc, active);
  else
    note_launch(), k_axpy_split_d<<<dim3((unsigned)blocks, nrhs), 256, 0, s>>>(x, xh, xl, xs, d, ds, len, sc, active);
}
template void axpy_split<float>(double*, float*, float*, i64, const float*, i64, i64, const double*,
                                int, const int*, cudaStream_t);
template void axpy_split<double>(double*, float*, float*, i64, const double*, i64, i64,
                                 const double*, int, const int*, cudaStream_t);

// ---- constant-bank slot manager ---------------------------------------------
namespace {
struct SlotState {
  int refs = 0;
  float k0[1024];
  float s0[64];
};
std::mutex g_slot_mu;
SlotState g_slots[64][kSlots];
}  // namespace

int cslot_acquire(const float* K0f, const float* S0f) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(g_slot_mu);
  for (int i = 0; i < kSlots; ++i) {
    SlotState& st = g_slots[dev][i];
    if (st.refs > 0 && !std::memcmp(st.k0, K0f, sizeof(st.k0)) && !std::memcmp(st.s0, S0f, sizeof(st.s0))) {
      ++st.refs;
      return i + 1;
    }
  }
  for (int i = 0; i < kSlots; ++i) {
    SlotState& st = g_slots[dev][i];
    if (st.refs == 0) {
      if (cudaMemcpyToSymbol(c_k0, K0f, 1024 * sizeof(float), (size_t)i * 1024 * sizeof(float)) != cudaSuccess ||
          cudaMemcpyToSymbol(c_s0, S0f, 64 * sizeof(float), (size_t)i * 64 * sizeof(float)) != cudaSuccess)
        return 0;
      std::memcpy(st.k0, K0f, sizeof(st.k0));
      std::memcpy(st.s0, S0f, sizeof(st.s0));
      st.refs = 1;
      return i + 1;
    }
  }
  return 0;
}

void cslot_release(int slot1) {
  if (slot1 <= 0) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(g_slot_mu);
  SlotState& st = g_slots[dev][slot1 - 1];
  if (st.refs > 0) --st.refs;
}

#define INST(T)                                                                                   \
  template void apply_full<T>(const ApplyArgs<T>&, const FixedMat<T, 4>&, int, int, cudaStream_t); \
  template void apply_uu<T>(const ApplyArgs<T>&, const FixedMat<T, 4>&, int, int, cudaStream_t);   \
  template void apply_pu<T>(const ApplyArgs<T>&, const FixedMat<T, 4>&, int, cudaStream_t);        \
  template void apply_ss<T>(const ApplyArgs<T>&, const FixedMat<T, 1>&, int, int, cudaStream_t);   \
  template void apply_elem<T, 1>(const ApplyArgs<T>&, int, int, cudaStream_t);                     \
  template void apply_elem<T, 3>(const ApplyArgs<T>&, int, int, cudaStream_t);                     \
  template void apply_stencil<T, 1>(const ApplyArgs<T>&, int, int, cudaStream_t, int);             \
  template void apply_stencil<T, 3>(const ApplyArgs<T>&, int, int, cudaStream_t, int);             \
  template int stencil_autotune<T, 1>(const ApplyArgs<T>&, int, int, cudaStream_t, float*);        \
  template int stencil_autotune<T, 3>(const ApplyArgs<T>&, int, int, cudaStream_t, float*);        \
  template void stencil_from_elem<T, 1>(const T*, T*, int, int, int, cudaStream_t);                \
  template void stencil_from_elem<T, 3>(const T*, T*, int, int, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace cell
