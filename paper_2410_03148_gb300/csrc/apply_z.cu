// Fine-level smoother applies on the 5th-generation tensor cores, marching
// through the cell along z ("z-march" kernels).
//
// The operator is y_n = sum over the 8 elements e around node n of
// rho_e (K x_e)_n with K a fixed 32 x 32 matrix (a block of the element
// matrix K0 of Eq. (sym-piezo), or the local Schur matrix S0 of §2.5.3 acting
// on four loads at once).  For every element the product K x_e is one row of
// a dense GEMM  D[e][j] = sum_k A[e][k] B[j][k]  whose A rows are the
// element's nodal values.  No gather builds A: node values are staged in
// shared memory as 16-byte records (4 slots: the three displacement
// components plus either the potential, zero, or, for the Schur operator,
// four loads), one record per node, rows of nx+1 records along x (the last one
// repeats node 0, the periodic wrap).  For an M = 128 tile of elements
// (8 along x times 16 along y) and a fixed local-node shift (a, c) in x and z,
// the 8 K-values of an MMA are the records of the element's two nodes with
// b = 0, 1 (consecutive rows): the shared-memory matrix descriptor with both
// strides equal to the row pitch and its start address moved by a records and
// c planes addresses exactly those values.  Four tcgen05.mma (kind::tf32,
// K = 8) per tile and load cover the 32 element dofs.
//
// Element results are turned into node values without atomics: thread t of
// the 128 epilogue threads owns TMEM lane t, i.e. element (x0 + t % 8,
// y0 + t / 8).  After scaling by rho_e, the a = 1 halves move one lane up
// (x), the b = 1 halves eight lanes up (y; across warps through shared
// memory), and the c = 1 halves are carried to the next z plane in shared
// memory.  A node value is final once both z layers around it are done; the
// node-wise epilogue (plain product, Chebyshev step, residual) then runs as
// in the SIMT kernels.  The x-wrap of the first tile of a row is completed
// after the last tile (deferred column).
//
// A CTA owns one load (or group of four loads), a brick of 15 node rows in y
// (16 element rows: one halo row below) and a chunk of z planes (one halo
// layer below).  Node planes are fetched with cp.async into a ring of four
// buffers, three planes ahead.  TMEM holds 8 tiles (256 columns); larger rows
// run in several passes.
//
// Inputs are read as TF32 (the tensor core ignores the low 13 mantissa bits),
// B is rounded to TF32 on the host: the result carries TF32 rounding (about
// 1e-3 relative), which is what a multigrid smoother tolerates; the outer
// Krylov solver (flexible GMRES) applies the operator itself in FP32.
#include <cstring>

#include "kernels.cuh"
#include "tc.cuh"

namespace cell {

namespace {

constexpr int kThreads = 128;
constexpr int kERows = 16;             // element rows of an M tile
constexpr int kNRows = kERows + 1;     // staged node rows
constexpr int kOwnRows = kERows - 1;   // node rows a brick finalises
constexpr int kRing = 4;               // staged node planes
constexpr int kPassTiles = 8;          // M tiles per TMEM pass
constexpr int kTmemCols = 32 * kPassTiles;
constexpr int kMaxTiles = 16;          // nx <= 128
constexpr int kBFloats = 4 * 256;      // B: 4 (a, c) blocks of 32 x 8
constexpr int kMinSmem = 80 * 1024;    // at most two CTAs per SM (TMEM: 2 x 256 columns)
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr unsigned kFull = 0xFFFFFFFFu;

struct Geom {
  int nx, ny, nz;
  int T;        // tiles along x (nx / 8)
  int RS;       // bytes per staged node row ((nx + 1) * 16)
  int PS;       // bytes per staged plane (kNRows * RS)
  int L;        // owned planes per z chunk
  int off_b, off_zc, off_yb, off_bar, smem;
};

__device__ __forceinline__ void cp_async4(uint32_t saddr, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Operator kinds: which slots are read, which are written and where.
//  UU : slots 0..2 = u components of load r; slot 3 zero; writes slots 0..2.
//  PP4: slot s = potential-block vector of load r0 + s; writes all four.
template <int KIND>
struct Kind;
template <>
struct Kind<ZK_UU> {
  static constexpr int kUnitsPerLaunch = 1;
};
template <>
struct Kind<ZK_PP4> {
  static constexpr int kUnitsPerLaunch = 4;
};

// Node-wise epilogue of one output value (same arithmetic as the SIMT kernels).
template <int MODE>
__device__ __forceinline__ void epi_one(const ApplyArgs<float>& a, int r, i64 o, float acc, float dold,
                                        float c1, float c2) {
  if (MODE == AM_LINEAR) {
    float v = a.alpha * acc;
    if (a.b) v += a.beta * a.b[r * a.bs + o];
    a.y[r * a.ys + o] = v;
  } else if (MODE == AM_CHEB || MODE == AM_CHEB_LAST) {
    const float rr = a.y[r * a.ys + o] - acc;
    a.y[r * a.ys + o] = rr;
    float* sp = a.sol + r * a.ss + o;
    *sp = (a.sol_zero ? 0.f : *sp) + dold;
    if (MODE == AM_CHEB) a.dout[r * a.ds + o] = c1 * dold + c2 * a.dinv[o] * rr;
  } else {  // AM_RESID_CHEB0
    const float rr = a.b[r * a.bs + o] - acc;
    a.y[r * a.ys + o] = rr;
    a.dout[r * a.ds + o] = c2 * a.dinv[o] * rr;
  }
}

template <int KIND, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_zmarch(const ApplyArgs<float> a, const float* __restrict__ Btab, const Geom g, int nrhs, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int UPL = Kind<KIND>::kUnitsPerLaunch;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int xi = l & 7;              // x within the tile
  const int ey = 4 * w + (l >> 3);   // element row within the brick (0 = halo row)
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const i64 nxy = (i64)nx * ny, nn = nxy * nz;

  // ---- work unit -----------------------------------------------------------
  const int r0 = blockIdx.x * UPL;
  bool on[4];
  bool any = false;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    on[s] = (s < UPL) && (r0 + s < nrhs) && !(a.active && !a.active[r0 + s]);
    any = any || on[s];
  }
  if (!any) return;
  const int Y0 = blockIdx.y * kOwnRows;               // first owned node row
  const int Z0 = blockIdx.z * g.L;                    // first owned plane
  const int nown = min(g.L, nz - Z0);                 // owned planes
  const int nlayers = nown + 1;                       // + halo layer Z0 - 1

  unsigned char* planes = smem;
  float* sB = reinterpret_cast<float*>(smem + g.off_b);
  float4* zc = reinterpret_cast<float4*>(smem + g.off_zc);     // [T][128]
  float* yb = reinterpret_cast<float*>(smem + g.off_yb);       // [2][4][8][8]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + g.off_bar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + g.off_bar + 8);

  // ---- set-up: TMEM, barrier, B, zeroed planes -----------------------------
  if (w == 0) {
    tc::tmem_alloc(tslot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) tc::mbar_init(bar, 1);
  for (int i = tid; i < kBFloats; i += kThreads) sB[i] = Btab[i];
  {
    float4* p4 = reinterpret_cast<float4*>(planes);
    const int n4 = kRing * g.PS / 16;
    for (int i = tid; i < n4; i += kThreads) p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t splanes = tc::smem_u32(planes);
  const uint32_t sb_addr = tc::smem_u32(sB);

  // input slot base pointers (plane offset added per plane)
  const float* in[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    in[s] = nullptr;
    if (KIND == ZK_UU) {
      if (s < 3) in[s] = a.x + (i64)r0 * a.xs + (i64)s * nn;
    } else {
      if (on[s]) in[s] = a.x + (i64)(r0 + s) * a.xs;
    }
  }

  // stage node plane p (p = 0 is plane Z0 - 1) into ring buffer p % kRing
  auto load_plane = [&](int p) {
    if (p <= nown + 1) {  // planes Z0-1 .. Z0+nown
      const int gz = ((Z0 - 1 + p) % nz + nz) % nz;
      const uint32_t dst0 = splanes + (uint32_t)((p % kRing) * g.PS);
      const int W = nx + 1;
      const int per = kNRows * W;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (!in[s]) continue;
        const float* src = in[s] + (i64)gz * nxy;
        for (int i = tid; i < per; i += kThreads) {
          const int ry = i / W, x = i - ry * W;
          int gy = Y0 - 1 + ry;
          gy = gy < 0 ? gy + ny : (gy >= ny ? gy % ny : gy);
          const int gx = x == nx ? 0 : x;
          cp_async4(dst0 + (uint32_t)(ry * g.RS + x * 16 + s * 4), src + (i64)gy * nx + gx);
        }
      }
    }
    cp_async_commit();
  };

  const uint32_t idesc = tc::idesc_tf32(128, 32);
  uint32_t phase = 0;
  float c1 = a.c1, c2 = a.c2;
  if (MODE != AM_LINEAR && a.cc) {
    c1 = a.cc[0];
    c2 = a.cc[1];
  }

  load_plane(0);
  load_plane(1);
  load_plane(2);

  const bool row_owned = ey >= 1 && (Y0 - 1 + ey) < ny;
  const int gy_el = (Y0 - 1 + ey + ny) % ny;   // element row (periodic)
  int ypar = 0;
  bool aborted = false;

  for (int kk = 0; kk < nlayers; ++kk) {
    // planes kk and kk+1 must be resident; keep three in flight
    load_plane(kk + 3);
    cp_async_wait<2>();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    const int gz_el = ((Z0 - 1 + kk) % nz + nz) % nz;   // element layer = node plane kk of the chunk
    const bool finalize_layer = kk >= 1;                 // layer Z0-1 only feeds the carry
    const uint32_t pb0 = splanes + (uint32_t)((kk % kRing) * g.PS);
    const uint32_t pb1 = splanes + (uint32_t)(((kk + 1) % kRing) * g.PS);
    const unsigned char* pnode = planes + (kk % kRing) * g.PS;   // plane of the nodes finalised here

    float carryx[16], defer[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) carryx[i] = defer[i] = 0.f;

    // node epilogue for the node (8t + xi, ey) of plane kk, value V0 + carry
    auto finish = [&](int t, const float (&V)[2][4], bool pred) {
      float4* zp = zc + t * kThreads + tid;
      if (pred) {
        const float4 prev = *zp;
        *zp = make_float4(V[1][0], V[1][1], V[1][2], V[1][3]);
        if (finalize_layer && row_owned) {
          const float acc[4] = {V[0][0] + prev.x, V[0][1] + prev.y, V[0][2] + prev.z, V[0][3] + prev.w};
          const int x = 8 * t + xi;
          const i64 n = (i64)((Z0 - 1 + kk) % nz) * nxy + (i64)(Y0 - 1 + ey) * nx + x;
          const float* dsrc = reinterpret_cast<const float*>(pnode + ey * g.RS + x * 16);
          if (KIND == ZK_UU) {
#pragma unroll
            for (int s = 0; s < 3; ++s)
              epi_one<MODE>(a, r0, (i64)s * nn + n, acc[s], dsrc[s], c1, c2);
          } else {
#pragma unroll
            for (int s = 0; s < 4; ++s)
              if (on[s]) epi_one<MODE>(a, r0 + s, n, acc[s], dsrc[s], c1, c2);
          }
        }
      }
    };

    // y-combine of S (x-combined element halves) and node finish
    auto ycomb = [&](int t, const float (&S)[16], bool pred) {
      float* ybw = yb + ypar * 256;
      if ((l >> 3) == 3) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          ybw[(w * 8 + xi) * 8 + i] = S[4 + i];
          ybw[(w * 8 + xi) * 8 + 4 + i] = S[12 + i];
        }
      }
      __syncthreads();
      float V[2][4];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          float up = __shfl_up_sync(kFull, S[8 * c + 4 + s], 8);
          if ((l >> 3) == 0) up = w > 0 ? ybw[((w - 1) * 8 + xi) * 8 + 4 * c + s] : 0.f;
          V[c][s] = S[8 * c + s] + up;
        }
      ypar ^= 1;
      finish(t, V, pred);
    };

    for (int t0 = 0; t0 < g.T; t0 += kPassTiles) {
      const int nt = min(kPassTiles, g.T - t0);
      if (tid == 0) {
        tc::fence_after_sync();
        for (int tt = 0; tt < nt; ++tt) {
          const int t = t0 + tt;
#pragma unroll
          for (int ac = 0; ac < 4; ++ac) {
            const int aa = ac >> 1, cc = ac & 1;
            const uint32_t abase = (cc ? pb1 : pb0) + (uint32_t)((8 * t + aa) * 16);
            const uint64_t ad = tc::sdesc(abase, (uint32_t)g.RS, (uint32_t)g.RS);
            const uint64_t bd = tc::sdesc(sb_addr + (uint32_t)(ac * 1024), 128u, 256u);
            tc::mma_tf32(tmem + (uint32_t)(tt * 32), ad, bd, idesc, ac ? 1u : 0u);
          }
        }
        tc::mma_commit(bar);
      }
      // every thread waits for the MMAs; the outcome is made uniform
      const bool ok = tc::mbar_wait_bounded(bar, phase, kWaitLimit);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {  // uniform: every thread leaves together
        if (tid == 0) atomicAdd(err, 1);
        aborted = true;
        break;
      }
      tc::fence_after_sync();
      for (int tt = 0; tt < nt; ++tt) {
        const int t = t0 + tt;
        float G[32];
        tc::tmem_ld32(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)(tt * 32), G);
        const float re = __ldg(a.rho + (i64)gz_el * nxy + (i64)gy_el * nx + 8 * t + xi);
#pragma unroll
        for (int i = 0; i < 32; ++i) G[i] *= re;
        // x-combine: S = a=0 half + a=1 half of the element to the left
        float S[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float up = __shfl_up_sync(kFull, G[16 + i], 1);
          S[i] = G[i] + (xi ? up : carryx[i]);
          if (t == 0) defer[i] = G[i];
          carryx[i] = __shfl_sync(kFull, G[16 + i], (l & ~7) | 7);
        }
        ycomb(t, S, !(t == 0 && xi == 0));
      }
      tc::fence_before_sync();
      __syncthreads();
    }
    if (aborted) break;
    // deferred column: x = 0 of tile 0 with the wrap from the last tile
    {
      float S[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) S[i] = defer[i] + carryx[i];
      ycomb(0, S, xi == 0);
    }
    __syncthreads();  // plane kk - 1's buffer is refilled at the next layer
  }
  if (aborted) {
    // let any MMA still in flight finish before TMEM is released
    tc::mbar_wait_bounded(bar, phase ^ 1u, kWaitLimit);
  }
  cp_async_wait<0>();
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// TF32 rounding on the host (nearest, ties away from zero).
float tf32_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & ~0x1FFFu;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

Geom make_geom(int nx, int ny, int nz, int L) {
  Geom g{};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.T = nx / 8;
  g.RS = (nx + 1) * 16;
  g.PS = kNRows * g.RS;
  g.L = L;
  g.off_b = kRing * g.PS;
  g.off_zc = g.off_b + kBFloats * 4;
  g.off_yb = g.off_zc + g.T * kThreads * 16;
  g.off_bar = g.off_yb + 2 * 256 * 4;
  g.smem = g.off_bar + 16;
  if (g.smem < kMinSmem) g.smem = kMinSmem;
  return g;
}

// Owned planes per chunk: enough CTAs to fill the GPU twice over with the
// fewest halo layers.
int chunk_planes(int units, int nybrick, int nz) {
  int sms = 148;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_wave = units * nybrick;
  int chunks = (2 * sms) / per_wave;   // one wave at two CTAs per SM
  if (chunks < 1) chunks = 1;
  if (chunks > nz) chunks = nz;
  return (nz + chunks - 1) / chunks;
}

template <int KIND, int MODE>
void launch(const ApplyArgs<float>& a, const float* Btab, int nrhs, int* err, cudaStream_t s) {
  constexpr int UPL = Kind<KIND>::kUnitsPerLaunch;
  const int units = (nrhs + UPL - 1) / UPL;
  const int nyb = (a.ny + kOwnRows - 1) / kOwnRows;
  const int L = chunk_planes(units, nyb, a.nz);
  const Geom g = make_geom(a.nx, a.ny, a.nz, L);
  const dim3 grid((unsigned)units, (unsigned)nyb, (unsigned)((a.nz + L - 1) / L));
  note_launch(), k_zmarch<KIND, MODE><<<grid, kThreads, g.smem, s>>>(a, Btab, g, nrhs, err);
}

template <int KIND, int MODE>
void set_attr(int smem) {
  cudaFuncSetAttribute(k_zmarch<KIND, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace

bool zmarch_shape_ok(int nx, int ny, int nz) {
  return nx % 8 == 0 && nx >= 8 && nx <= 8 * kMaxTiles && ny >= 2 && nz >= 2 &&
         make_geom(nx, ny, nz, 1).smem <= 227 * 1024;
}

void zmarch_prepare() {
  // the attribute is an upper bound per kernel: set it for the widest grid
  // once, so handles of any supported width can launch
  const int smem = make_geom(8 * kMaxTiles, 2, 2, 1).smem;
  set_attr<ZK_UU, AM_LINEAR>(smem);
  set_attr<ZK_UU, AM_CHEB>(smem);
  set_attr<ZK_UU, AM_CHEB_LAST>(smem);
  set_attr<ZK_UU, AM_RESID_CHEB0>(smem);
  set_attr<ZK_PP4, AM_LINEAR>(smem);
  set_attr<ZK_PP4, AM_CHEB>(smem);
  set_attr<ZK_PP4, AM_CHEB_LAST>(smem);
  set_attr<ZK_PP4, AM_RESID_CHEB0>(smem);
}

// B operand of one kind in shared-memory order: for each local-node shift
// (a, c) of the input (block ac = 2a + c), a 32 x 8 K-major tile whose row j is
// the output (slot s = j % 4 of local node (a, b, c) = (j / 16, j / 4 % 2,
// j / 8 % 2)) and whose column k is the input (slot k % 4 of local node
// (a, k / 4, c)).  Local node index la = a + 2b + 4c (§2.5 element numbering).
void zmarch_build_b(int kind, const double* K0, const double* S0, float* out) {
  for (int ac = 0; ac < 4; ++ac) {
    const int ai = ac >> 1, ci = ac & 1;
    for (int j = 0; j < 32; ++j)
      for (int k = 0; k < 8; ++k) {
        const int so = j % 4, bo = (j / 4) % 2, co = (j / 8) % 2, ao = j / 16;
        const int si = k % 4, bi = k / 4;
        const int lo = ao + 2 * bo + 4 * co, li = ai + 2 * bi + 4 * ci;
        double v = 0.0;
        if (kind == ZK_UU) {
          if (so < 3 && si < 3) v = K0[(lo * 4 + so) * 32 + li * 4 + si];
        } else {
          if (so == si) v = S0[lo * 8 + li];
        }
        const int off = ac * 256 + (j / 8) * 64 + (k / 4) * 32 + (j % 8) * 4 + (k % 4);
        out[off] = tf32_host((float)v);
      }
  }
}

void apply_zmarch(int kind, const ApplyArgs<float>& a, const float* Btab, int mode, int nrhs, int* err,
                  cudaStream_t s) {
  if (kind == ZK_UU) {
    switch (mode) {
      case AM_LINEAR: launch<ZK_UU, AM_LINEAR>(a, Btab, nrhs, err, s); break;
      case AM_CHEB: launch<ZK_UU, AM_CHEB>(a, Btab, nrhs, err, s); break;
      case AM_CHEB_LAST: launch<ZK_UU, AM_CHEB_LAST>(a, Btab, nrhs, err, s); break;
      default: launch<ZK_UU, AM_RESID_CHEB0>(a, Btab, nrhs, err, s); break;
    }
  } else {
    switch (mode) {
      case AM_LINEAR: launch<ZK_PP4, AM_LINEAR>(a, Btab, nrhs, err, s); break;
      case AM_CHEB: launch<ZK_PP4, AM_CHEB>(a, Btab, nrhs, err, s); break;
      case AM_CHEB_LAST: launch<ZK_PP4, AM_CHEB_LAST>(a, Btab, nrhs, err, s); break;
      default: launch<ZK_PP4, AM_RESID_CHEB0>(a, Btab, nrhs, err, s); break;
    }
  }
}

}  // namespace cell
