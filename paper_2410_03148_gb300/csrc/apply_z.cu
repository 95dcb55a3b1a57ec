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
#include <cstdint>
#include <cstring>

#include "kernels.cuh"
#include "tc.cuh"

namespace cell {

namespace {

constexpr int kThreads = 256;          // two groups of four warps
constexpr int kERows = 16;             // element rows of an M tile
constexpr int kNRows = kERows + 1;     // staged node rows
constexpr int kOwnRows = kERows - 1;   // node rows a brick finalises
constexpr int kRing = 4;               // staged node planes
constexpr int kMaxTiles = 8;           // nx <= 64: two layers of 8 tiles fill TMEM
constexpr int kTmemCols = 512;
constexpr int kBFloats = 4 * 256;      // B: 4 (a, c) blocks of 32 x 8
constexpr int kMaxArr = 3;             // staged epilogue arrays
constexpr int kMinSmem = 120 * 1024;   // one CTA per SM: it holds all of TMEM
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr unsigned kFull = 0xFFFFFFFFu;

struct Geom {
  int nx, ny, nz;
  int T;        // tiles along x (nx / 8)
  int RS;       // bytes per staged node row ((nx + 1) * 16)
  int PS;       // bytes per staged plane (kNRows * RS)
  int L;        // owned planes per z chunk
  int P;        // floats per staged epilogue row (nx + 8: conflict-free rows)
  int OPS;      // floats per staged epilogue plane (kMaxArr * 4 slots * 15 rows * P)
  int off_ops, off_rho, off_b, off_zc, off_edge, off_def, off_yb, off_bar, smem;
};

__device__ __forceinline__ void cp_async4(uint32_t saddr, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void group_sync(int id) {
  asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
}

// Operator kinds: ZK_UU reads slots 0..2 (u components of one load, slot 3
// stays zero) and writes slots 0..2; ZK_PP4 reads and writes slot s = load
// r0 + s of a one-component vector.
template <int KIND>
struct Kind;
template <>
struct Kind<ZK_UU> {
  static constexpr int kUnits = 1;   // loads per CTA
  static constexpr int kSlots = 3;   // slots read and written
};
template <>
struct Kind<ZK_PP4> {
  static constexpr int kUnits = 4;
  static constexpr int kSlots = 4;
};

// Epilogue arrays staged in shared memory, per mode (nullptr = not used).
//   LINEAR: b;  CHEB: y, sol, dinv;  CHEB_LAST: y, sol;  RESID_CHEB0: b, dinv.
struct Staged {
  const float* p[kMaxArr];
  i64 rs[kMaxArr];   // stride between loads
  bool shared[kMaxArr];  // one array for all loads (dinv of the Schur block)
};

template <int MODE>
__device__ __forceinline__ Staged staged_arrays(const ApplyArgs<float>& a) {
  Staged st{};
  if (MODE == AM_LINEAR) {
    st.p[0] = a.b; st.rs[0] = a.bs;
  } else if (MODE == AM_CHEB || MODE == AM_CHEB_LAST) {
    st.p[0] = a.y; st.rs[0] = a.ys;
    st.p[1] = a.sol_zero ? nullptr : a.sol; st.rs[1] = a.ss;
    if (MODE == AM_CHEB) { st.p[2] = a.dinv; st.rs[2] = 0; st.shared[2] = true; }
  } else {
    st.p[0] = a.b; st.rs[0] = a.bs;
    st.p[1] = a.dinv; st.rs[1] = 0; st.shared[1] = true;
  }
  return st;
}

template <int KIND, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
k_zmarch(const ApplyArgs<float> a, const float* __restrict__ Btab, const Geom g, int nrhs, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int UPL = Kind<KIND>::kUnits;
  constexpr int NS = Kind<KIND>::kSlots;
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int grp = w >> 2, q = w & 3;     // warp group, TMEM lane quarter
  const int xi = l & 7;                  // x within the tile
  const int ey = 4 * q + (l >> 3);       // element row within the brick (0 = halo row)
  const int nx = g.nx, ny = g.ny, nz = g.nz, T = g.T;
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
  const int Y0 = blockIdx.y * kOwnRows;   // first owned node row
  const int Z0 = blockIdx.z * g.L;        // first owned plane
  const int nown = min(g.L, nz - Z0);     // owned planes
  const int nlayers = nown + 1;           // + halo layer Z0 - 1

  unsigned char* planes = smem;
  float* ops = reinterpret_cast<float*>(smem + g.off_ops);      // [2][kMaxArr][4][15][P]
  float* rho_s = reinterpret_cast<float*>(smem + g.off_rho);    // [2][16][nx]
  float* sB = reinterpret_cast<float*>(smem + g.off_b);
  float4* zc = reinterpret_cast<float4*>(smem + g.off_zc);      // [T][128]
  float* edge = reinterpret_cast<float*>(smem + g.off_edge);    // [T][16][16]
  float* defer = reinterpret_cast<float*>(smem + g.off_def);    // [T][16][16]
  float* yb = reinterpret_cast<float*>(smem + g.off_yb);        // [2 groups][2][4][8][8]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + g.off_bar); // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + g.off_bar + 16);

  // ---- set-up: TMEM, barriers, B, zeroed planes ----------------------------
  if (w == 0) {
    tc::tmem_alloc(tslot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::mbar_init(bar + 1, 1);
  }
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
  const uint32_t sops = tc::smem_u32(ops);
  const uint32_t srho = tc::smem_u32(rho_s);
  const uint32_t sb_addr = tc::smem_u32(sB);

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
  const Staged sta = staged_arrays<MODE>(a);

  // node plane p of the chunk (p = 0: plane Z0 - 1) -> ring slot p % kRing,
  // 16-byte records; warp w stages rows w, w + 8, w + 16
  auto stage_plane = [&](int p) {
    if (p > nown + 1) return;
    const int gz = (Z0 - 1 + p + nz) % nz;
    const uint32_t dst0 = splanes + (uint32_t)((p % kRing) * g.PS);
    for (int ry = w; ry < kNRows; ry += 8) {
      int gy = Y0 - 1 + ry;
      gy = gy < 0 ? gy + ny : (gy >= ny ? gy % ny : gy);
      const i64 rowoff = (i64)gz * nxy + (i64)gy * nx;
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        if (!in[s]) continue;
        const float* src = in[s] + rowoff;
        for (int x = l; x < nx; x += 32) cp_async4(dst0 + (uint32_t)(ry * g.RS + x * 16 + s * 4), src + x);
        if (l == 0) cp_async4(dst0 + (uint32_t)(ry * g.RS + nx * 16 + s * 4), src);   // periodic wrap
      }
    }
  };
  // epilogue inputs of the owned nodes of plane p -> buffer p % 2 (16-byte chunks)
  auto stage_ops = [&](int p) {
    if (p < 1 || p > nown) return;
    const int gz = Z0 - 1 + p;
    const uint32_t dst0 = sops + (uint32_t)((p & 1) * g.OPS * 4);
    const int C = nx >> 2;                     // chunks per row (<= 16)
    const int x4 = l & 15;
    // items (array, slot, row): two per warp pass
    for (int it = 2 * w + (l >> 4); it < kMaxArr * 4 * kOwnRows; it += 16) {
      const int arr = it / (4 * kOwnRows);
      const int rem = it - arr * 4 * kOwnRows;
      const int s = rem / kOwnRows, row = rem - s * kOwnRows;
      if (x4 >= C || !sta.p[arr] || s >= NS || Y0 + row >= ny) continue;
      if (sta.shared[arr] && KIND == ZK_PP4 && s > 0) continue;
      const float* src;
      if (KIND == ZK_UU) src = sta.p[arr] + (i64)r0 * sta.rs[arr] + (i64)s * nn;
      else src = sta.p[arr] + (sta.shared[arr] ? 0 : (i64)(r0 + s) * sta.rs[arr]);
      if (KIND == ZK_PP4 && !sta.shared[arr] && !on[s]) continue;
      src += (i64)gz * nxy + (i64)(Y0 + row) * nx + 4 * x4;
      cp_async16(dst0 + (uint32_t)((((arr * 4 + s) * kOwnRows + row) * g.P + 4 * x4) * 4), src);
    }
  };
  // rho of element layer p -> buffer p % 2
  auto stage_rho = [&](int p) {
    if (p > nown) return;
    const int gz = (Z0 - 1 + p + nz) % nz;
    const int C = nx >> 2;
    const int row = tid >> 4, x4 = tid & 15;
    if (x4 < C) {
      const int gy = (Y0 - 1 + row + ny) % ny;
      cp_async16(srho + (uint32_t)((((p & 1) * 16 + row) * nx + 4 * x4) * 4),
                 a.rho + (i64)gz * nxy + (i64)gy * nx + 4 * x4);
    }
  };

  const uint32_t idesc = tc::idesc_tf32(128, 32);
  auto issue_mma = [&](int layer) {
    const uint32_t pb0 = splanes + (uint32_t)((layer % kRing) * g.PS);
    const uint32_t pb1 = splanes + (uint32_t)(((layer + 1) % kRing) * g.PS);
    tc::fence_after_sync();
    for (int t = 0; t < T; ++t) {
#pragma unroll
      for (int ac = 0; ac < 4; ++ac) {
        const int aa = ac >> 1, cc = ac & 1;
        const uint32_t abase = (cc ? pb1 : pb0) + (uint32_t)((8 * t + aa) * 16);
        const uint64_t ad = tc::sdesc(abase, (uint32_t)g.RS, (uint32_t)g.RS);
        const uint64_t bd = tc::sdesc(sb_addr + (uint32_t)(ac * 1024), 128u, 256u);
        tc::mma_tf32(tmem + (uint32_t)((layer & 1) * 256 + t * 32), ad, bd, idesc, ac ? 1u : 0u);
      }
    }
    tc::mma_commit(bar + (layer & 1));
  };

  float c1 = a.c1, c2 = a.c2;
  if (MODE != AM_LINEAR && a.cc) {
    c1 = a.cc[0];
    c2 = a.cc[1];
  }

  // prologue: planes 0..2, epilogue inputs of plane 0 (unused: halo), rho of layer 0
  stage_plane(0);
  stage_plane(1);
  stage_plane(2);
  stage_rho(0);
  cp_async_commit();
  cp_async_wait<0>();
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0) issue_mma(0);

  int ypar = 0;
  bool aborted = false;
  int kfail = 0;
  for (int kk = 0; kk < nlayers; ++kk) {
    stage_plane(kk + 3);
    stage_ops(kk + 1);
    stage_rho(kk + 1);
    cp_async_commit();
    cp_async_wait<1>();          // everything but the group just issued
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0 && kk + 1 < nlayers) issue_mma(kk + 1);
    const bool ok = tc::mbar_wait_bounded(bar + (kk & 1), (uint32_t)((kk >> 1) & 1), kWaitLimit);
    if (__syncthreads_or(!ok)) {  // uniform: every thread leaves together
      if (tid == 0) atomicAdd(err, 1);
      aborted = true;
      kfail = kk;
      break;
    }
    tc::fence_after_sync();

    const bool fin_layer = kk >= 1;                       // layer Z0-1 only feeds the carry
    const i64 plane_off = (i64)(Z0 - 1 + kk) * nxy;       // valid when fin_layer
    const unsigned char* pnode = planes + (kk % kRing) * g.PS;
    const float* opsb = ops + (kk & 1) * g.OPS;
    const float* rhob = rho_s + (kk & 1) * 16 * nx;

    // node (x, row e) of plane kk: V0 + carry, then the node-wise epilogue
    auto finish = [&](int t, int zi, int e, int x, const float (&V)[2][4]) {
      float4* zp = zc + t * 128 + zi;
      const float4 prev = *zp;
      *zp = make_float4(V[1][0], V[1][1], V[1][2], V[1][3]);
      if (!fin_layer || e < 1 || Y0 - 1 + e >= ny) return;
      const float acc[4] = {V[0][0] + prev.x, V[0][1] + prev.y, V[0][2] + prev.z, V[0][3] + prev.w};
      const i64 n = plane_off + (i64)(Y0 - 1 + e) * nx + x;
      const float* dsrc = reinterpret_cast<const float*>(pnode + e * g.RS + x * 16);
      const int ro = (e - 1) * g.P + x;
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (KIND == ZK_PP4 && !on[s]) continue;
        const int r = KIND == ZK_UU ? r0 : r0 + s;
        const i64 o = KIND == ZK_UU ? (i64)s * nn + n : n;
        const float* o0 = opsb + (0 * 4 + s) * kOwnRows * g.P + ro;
        const float* o1 = opsb + (1 * 4 + s) * kOwnRows * g.P + ro;
        const int sd = KIND == ZK_PP4 ? 0 : s;            // slot of the shared dinv
        if (MODE == AM_LINEAR) {
          float v = a.alpha * acc[s];
          if (a.b) v += a.beta * *o0;
          a.y[r * a.ys + o] = v;
        } else if (MODE == AM_CHEB || MODE == AM_CHEB_LAST) {
          const float rr = *o0 - acc[s];
          a.y[r * a.ys + o] = rr;
          a.sol[r * a.ss + o] = (a.sol_zero ? 0.f : *o1) + dsrc[s];
          if (MODE == AM_CHEB) {
            const float dv = opsb[(2 * 4 + sd) * kOwnRows * g.P + ro];
            a.dout[r * a.ds + o] = c1 * dsrc[s] + c2 * dv * rr;
          }
        } else {  // AM_RESID_CHEB0
          const float rr = *o0 - acc[s];
          a.y[r * a.ys + o] = rr;
          const float dv = opsb[(1 * 4 + sd) * kOwnRows * g.P + ro];
          a.dout[r * a.ds + o] = c2 * dv * rr;
        }
      }
    };

    // tiles of this warp group: x-combine inside the tile, y-combine inside
    // the group, node epilogue for x % 8 != 0; x % 8 == 0 is deferred
    for (int t = grp; t < T; t += 2) {
      float G[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((kk & 1) * 256 + t * 32), G);
      const float re = rhob[ey * nx + 8 * t + xi];
#pragma unroll
      for (int i = 0; i < 32; ++i) G[i] *= re;
      float S[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) S[i] = G[i] + __shfl_up_sync(kFull, G[16 + i], 1);
      float4* ep = reinterpret_cast<float4*>(edge + (t * 16 + ey) * 16);
      float4* dp = reinterpret_cast<float4*>(defer + (t * 16 + ey) * 16);
      if (xi == 7) {
#pragma unroll
        for (int i = 0; i < 4; ++i) ep[i] = make_float4(G[16 + 4 * i], G[17 + 4 * i], G[18 + 4 * i], G[19 + 4 * i]);
      }
      if (xi == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) dp[i] = make_float4(G[4 * i], G[4 * i + 1], G[4 * i + 2], G[4 * i + 3]);
      }
      float* ybw = yb + (grp * 2 + ypar) * 256;
      if ((l >> 3) == 3) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          ybw[(q * 8 + xi) * 8 + i] = S[4 + i];
          ybw[(q * 8 + xi) * 8 + 4 + i] = S[12 + i];
        }
      }
      group_sync(1 + grp);
      float V[2][4];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          float up = __shfl_up_sync(kFull, S[8 * c + 4 + s], 8);
          if ((l >> 3) == 0) up = q > 0 ? ybw[((q - 1) * 8 + xi) * 8 + 4 * c + s] : 0.f;
          V[c][s] = S[8 * c + s] + up;
        }
      ypar ^= 1;
      if (xi != 0) finish(t, 32 * q + l, ey, 8 * t + xi, V);
    }
    tc::fence_before_sync();
    __syncthreads();
    // deferred column x = 8t of every tile: the a = 1 half of element 8t - 1
    // comes from the previous tile (periodic in x)
    if (tid < 16 * T) {
      const int t = tid >> 4, e = tid & 15;
      const int tl = t == 0 ? T - 1 : t - 1;
      const float* d0 = defer + (t * 16 + e) * 16;
      const float* e0 = edge + (tl * 16 + e) * 16;
      float V[2][4];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          float v = d0[8 * c + s] + e0[8 * c + s];
          if (e >= 1) v += d0[8 * c + 4 + s - 16] + e0[8 * c + 4 + s - 16];
          V[c][s] = v;
        }
      finish(t, 8 * e, e, 8 * t, V);
    }
    __syncthreads();   // buffers of layer kk - 1 are refilled by the next iteration
  }
  if (aborted) {
    // let the MMAs still in flight (layers kfail, kfail + 1) finish before
    // TMEM is released
    for (int lyr = kfail; lyr <= kfail + 1 && lyr < nlayers; ++lyr)
      tc::mbar_wait_bounded(bar + (lyr & 1), (uint32_t)((lyr >> 1) & 1), kWaitLimit);
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
  g.P = nx + 8;
  g.OPS = kMaxArr * 4 * kOwnRows * g.P;
  g.off_ops = kRing * g.PS;
  g.off_rho = g.off_ops + 2 * g.OPS * 4;
  g.off_b = g.off_rho + 2 * 16 * nx * 4;
  g.off_zc = g.off_b + kBFloats * 4;
  g.off_edge = g.off_zc + g.T * 128 * 16;
  g.off_def = g.off_edge + g.T * 16 * 16 * 4;
  g.off_yb = g.off_def + g.T * 16 * 16 * 4;
  g.off_bar = g.off_yb + 2 * 2 * 256 * 4;
  g.smem = g.off_bar + 32;
  if (g.smem < kMinSmem) g.smem = kMinSmem;
  return g;
}

// Owned planes per chunk: one wave of one CTA per SM with the fewest halo
// layers.
int chunk_planes(int units, int nybrick, int nz) {
  int sms = 148;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_wave = units * nybrick;
  int chunks = sms / per_wave;
  if (chunks < 1) chunks = 1;
  if (chunks > nz) chunks = nz;
  return (nz + chunks - 1) / chunks;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

template <int KIND, int MODE>
bool launch(const ApplyArgs<float>& a, const float* Btab, int nrhs, int* err, cudaStream_t s) {
  // the staged epilogue arrays and rho move in 16-byte chunks
  const bool al = aligned16(a.rho) && (!a.b || (aligned16(a.b) && a.bs % 4 == 0)) &&
                  (!a.y || (aligned16(a.y) && a.ys % 4 == 0)) && (!a.sol || (aligned16(a.sol) && a.ss % 4 == 0)) &&
                  (!a.dinv || aligned16(a.dinv));
  if (!al) return false;
  constexpr int UPL = Kind<KIND>::kUnits;
  const int units = (nrhs + UPL - 1) / UPL;
  const int nyb = (a.ny + kOwnRows - 1) / kOwnRows;
  const int L = chunk_planes(units, nyb, a.nz);
  const Geom g = make_geom(a.nx, a.ny, a.nz, L);
  const dim3 grid((unsigned)units, (unsigned)nyb, (unsigned)((a.nz + L - 1) / L));
  note_launch(), k_zmarch<KIND, MODE><<<grid, kThreads, g.smem, s>>>(a, Btab, g, nrhs, err);
  return true;
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

bool apply_zmarch(int kind, const ApplyArgs<float>& a, const float* Btab, int mode, int nrhs, int* err,
                  cudaStream_t s) {
  if (kind == ZK_UU) {
    switch (mode) {
      case AM_LINEAR: return launch<ZK_UU, AM_LINEAR>(a, Btab, nrhs, err, s);
      case AM_CHEB: return launch<ZK_UU, AM_CHEB>(a, Btab, nrhs, err, s);
      case AM_CHEB_LAST: return launch<ZK_UU, AM_CHEB_LAST>(a, Btab, nrhs, err, s);
      default: return launch<ZK_UU, AM_RESID_CHEB0>(a, Btab, nrhs, err, s);
    }
  }
  switch (mode) {
    case AM_LINEAR: return launch<ZK_PP4, AM_LINEAR>(a, Btab, nrhs, err, s);
    case AM_CHEB: return launch<ZK_PP4, AM_CHEB>(a, Btab, nrhs, err, s);
    case AM_CHEB_LAST: return launch<ZK_PP4, AM_CHEB_LAST>(a, Btab, nrhs, err, s);
    default: return launch<ZK_PP4, AM_RESID_CHEB0>(a, Btab, nrhs, err, s);
  }
}

}  // namespace cell
