// Fine-level smoother applies on the 5th-generation tensor cores, node-centric.
//
// The preconditioner blocks of §2.5.3 on the finest grid are
//   y_n = sum over the 8 elements e around node n of rho_e (K x_e)_n
// with K a fixed element matrix: the elastic block of the element matrix K0 of
// Eq. (sym-piezo) (3 components), or the local Schur matrix S0 (1 component).
// Split by the position o = (ex, ey, ez) of the element around the node (its
// lower corner is n + (ex - 1, ey - 1, ez - 1)):
//
//   y_n = sum_o rho_{e(n,o)} T_n[o],   T_n[o] = sum_q K[la(o), b(o,q)] x_{n+q},
//
// q running over the 27 neighbour offsets, la(o) the local index of n in that
// element and b(o,q) the one of n + q (zero where n + q is not a node of it).
// T is a dense GEMM with a FIXED right operand,
//   T[n][(o,c)] = sum_(q,d) X[n][(q,d)] B[(o,c)][(q,d)],
// rows = nodes, K = neighbours x 4 slots, N = 8 positions x 4 slots = 32.  Each
// row's epilogue sums its own 8 position columns weighted by rho: no thread
// writes another node's value (no scatter, no atomics, reproducible).
//
// A rows are never gathered.  Node values are staged in shared memory as
// 16-byte records (4 slots: u1, u2, u3, 0 of one load for the elastic block,
// or one component of four loads for the Schur block), in rows along x with a
// periodic halo record at each end.  An M = 128 tile is 8 nodes along x by 16
// rows along y.  In the no-swizzle K-major layout a core matrix is 8 rows of
// 16 bytes, i.e. 8 consecutive records; a descriptor whose row-group stride
// (SBO) is the staged row pitch and whose start address is moved by a
// neighbour offset (dx records, dy rows, dz planes) therefore addresses that
// neighbour's records for all 128 nodes.  One kind::tf32 MMA has K = 8 = two
// neighbours: the second one's address distance is the descriptor's K stride
// (LBO), chosen per MMA.  Per plane the pairs are dx = -1/+1 in each of the
// three rows, dy = -1/+1 at dx = 0, and the centre with a zero B half: 15 MMAs
// per tile and output plane (K = 120, 108 of it nonzero).
//
// A CTA owns XT x 16 nodes (XT = 8, 16 or 32; ragged edges masked) of one load
// (elastic) or four loads (Schur) and a chunk of L z-planes.  It stages node
// planes with 4-byte cp.async two planes ahead of use into a ring of six,
// issues the MMAs of plane k (one thread per M tile) into one of two TMEM
// buffers, and its eight warps run the epilogue of plane k - 1 meanwhile.
// The epilogue's node-wise operands (residual, iterate, inverse diagonal) and
// the 8 rho of each node are prefetched into registers one plane ahead, and
// into L2 two steps before that.
//
// Inputs enter the tensor core as TF32 (10 mantissa bits) and B is rounded to
// TF32 on the host, so results carry TF32 rounding (about 1e-3 relative),
// which a multigrid smoother inside flexible GMRES tolerates (the outer
// Krylov operator is applied in FP32).
#include <cstdint>
#include <cstring>

#include "kernels.cuh"
#include "tc.cuh"

namespace cell {

namespace {

constexpr int kThreads = 256;
constexpr int kTY = 16;                 // node rows (y) of an M tile
constexpr int kAhead = 2;               // planes staged beyond the three in use
constexpr int kRing = kAhead + 4;       // staged planes (see the ring argument below)
constexpr int kPairs = 5;               // MMAs per plane and tile
constexpr int kMmas = 3 * kPairs;
constexpr int kBFloats = kMmas * 256;   // B: kMmas tiles of 32 x 8
constexpr int kSmemPerSM = 228 * 1024;  // shared memory of an SM (1 KB of it reserved per CTA)
constexpr uint32_t kWaitLimit = 1u << 22;

// Neighbour (dx, dy) of K half h of pair p; half 1 of pair 4 is a dummy (zero B).
__host__ __device__ constexpr int pair_dx(int p, int h) { return p < 3 ? (h ? 1 : -1) : (p == 3 ? 0 : h); }
__host__ __device__ constexpr int pair_dy(int p, int h) { return p < 3 ? p - 1 : (p == 3 ? (h ? 1 : -1) : 0); }

struct NcGeom {
  int nx, ny, nz;
  int XT, TX;          // tile width in nodes, M tiles per plane (XT / 8)
  int gx, gy;          // CTAs along x and y
  int L, zchunks;      // planes per z chunk, chunks
  int RS, PS;          // staged row pitch and plane size (bytes)
  int off_b, off_bar, smem;
  int tcols;           // TMEM columns allocated (power of two)
};

// Widest tile for a grid: 32 nodes, or nx rounded up to a multiple of 8.
int max_xt(int nx) { return nx >= 32 ? 32 : ((nx + 7) / 8) * 8; }

NcGeom make_geom(int nx, int ny, int nz, int L, int XT) {
  NcGeom g{};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.XT = XT;
  g.TX = g.XT / 8;
  g.gx = (nx + g.XT - 1) / g.XT;
  g.gy = (ny + kTY - 1) / kTY;
  g.L = L;
  g.zchunks = (nz + L - 1) / L;
  g.RS = (g.XT + 2) * 16;
  g.PS = (kTY + 2) * g.RS;
  g.off_b = kRing * g.PS;
  g.off_bar = g.off_b + kBFloats * 4;
  g.smem = g.off_bar + 64 + 8 * (kMmas + kPairs);
  int c = 32;
  while (c < 2 * g.TX * 32) c <<= 1;
  g.tcols = c;
  // no more CTAs resident per SM than TMEM holds (512 columns): pad the
  // shared memory so that one more CTA would not fit
  const int max_ctas = 512 / g.tcols;
  const int min_smem = kSmemPerSM / (max_ctas + 1) + 1 - 1024;
  if (g.smem < min_smem) g.smem = min_smem;
  return g;
}

__device__ __forceinline__ void cp_async4(uint32_t saddr, const void* gp) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(gp) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ int wrap(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Node-wise output of one (node, slot) with the semantics of the SIMT kernels
// (ApplyMode); e0, e1, e2 are the prefetched operands of the mode.  y, sol and
// dout point at the slot's plane of the outputs, n is the node (32-bit index).
template <int MODE>
__device__ __forceinline__ void node_out(const ApplyArgs<float>& a, float* y, float* sol, float* dout, int n,
                                         float acc, float dold, float e0, float e1, float e2, float c1, float c2) {
  // explicit roundings: the result must not depend on how the compiler
  // contracts these expressions in each instantiation (tiles per warp, modes),
  // so that every CTA tile gives the same bits
  if (MODE == AM_LINEAR) {
    float v = __fmul_rn(a.alpha, acc);
    if (a.b) v = fmaf(a.beta, e0, v);
    y[n] = v;
  } else if (MODE == AM_CHEB || MODE == AM_CHEB_LAST) {
    const float rr = __fsub_rn(e0, acc);    // e0 = residual, e1 = iterate, e2 = dinv
    y[n] = rr;
    sol[n] = __fadd_rn(a.sol_zero ? 0.f : e1, dold);
    if (MODE == AM_CHEB) dout[n] = fmaf(c1, dold, __fmul_rn(__fmul_rn(c2, e2), rr));
  } else {                                   // AM_RESID_CHEB0: e0 = b, e2 = dinv
    const float rr = __fsub_rn(e0, acc);
    y[n] = rr;
    dout[n] = __fmul_rn(__fmul_rn(c2, e2), rr);
  }
}

// TPW = M tiles per warp in the epilogue: 2 for 32-node-wide CTA tiles (two
// CTAs per SM), 1 for narrower ones (up to four CTAs per SM, fewer registers).
template <int KIND, int MODE, int TPW>
__global__ void __launch_bounds__(kThreads, TPW == 2 ? 2 : 3)
k_nc(const ApplyArgs<float> a, const float* __restrict__ Btab, const NcGeom g, int nrhs, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int UPL = KIND == NK_UU ? 1 : 4;   // loads per CTA
  constexpr int NS = KIND == NK_UU ? 3 : 4;    // record slots read and written
  const int tid = threadIdx.x, w = tid >> 5, l = tid & 31;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  // 32-bit node indices within a load: the launcher checks that 4 nn and four
  // times every vector stride stay below 2^31; each load's 64-bit base is
  // formed once
  const int nxy = nx * ny, nn = nxy * nz;
  const int x0 = blockIdx.x * g.XT, y0 = blockIdx.y * kTY;
  const int zc = blockIdx.z % g.zchunks;
  const int r0 = (blockIdx.z / g.zchunks) * UPL;
  const int z0 = zc * g.L;
  const int L = min(g.L, nz - z0);
  bool on[4];
  bool any = false;
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    on[s] = (s < UPL) && (r0 + s < nrhs) && !(a.active && !a.active[r0 + s]);
    any = any || on[s];
  }
  if (!any) return;

  unsigned char* planes = smem;
  float* sB = reinterpret_cast<float*>(smem + g.off_b);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + g.off_bar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + g.off_bar + 16);
  uint64_t* dtab = reinterpret_cast<uint64_t*>(smem + g.off_bar + 64);   // [kMmas] B, [kPairs] A templates

  // ---- set-up: TMEM, barriers, B, zeroed ring (unused slots stay zero) ------
  if (w == 0) {
    tc::tmem_alloc(tslot, (uint32_t)g.tcols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(bar, (uint32_t)g.TX);       // one commit per M tile
    tc::mbar_init(bar + 1, (uint32_t)g.TX);
  }
  for (int i = tid; i < kBFloats; i += kThreads) sB[i] = Btab[i];
  {
    float4* p4 = reinterpret_cast<float4*>(planes);
    const int n4 = kRing * g.PS / 16;
    for (int i = tid; i < n4; i += kThreads) p4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t splanes = tc::smem_u32(planes);
  const uint32_t sb_addr = tc::smem_u32(sB);
  // descriptor tables: B per MMA, A templates per neighbour pair relative to a
  // plane base (the start-address field is the low 14 bits of a descriptor, so
  // adding a base address >> 4 moves it without carries: every shared-memory
  // address is below 2^18)
  if (tid < kMmas) {
    dtab[tid] = tc::sdesc(sb_addr + (uint32_t)(tid * 1024), 128u, 256u);
  } else if (tid < kMmas + kPairs) {
    const int p = tid - kMmas;
    const int o1 = (1 + pair_dy(p, 0)) * g.RS + (1 + pair_dx(p, 0)) * 16;
    const int o2 = (1 + pair_dy(p, 1)) * g.RS + (1 + pair_dx(p, 1)) * 16;
    dtab[tid] = tc::sdesc((uint32_t)o1, (uint32_t)(o2 - o1), (uint32_t)g.RS);
  }
  __syncthreads();

  const float* in[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    in[s] = nullptr;
    if (KIND == NK_UU) {
      if (s < 3) in[s] = a.x + (i64)r0 * a.xs + (i64)s * nn;
    } else if (on[s]) {
      in[s] = a.x + (i64)(r0 + s) * a.xs;
    }
  }

  // staged plane p (z = z0 - 1 + p) -> ring slot p % kRing; record (yy, xx)
  // of node (x0 - 1 + xx, y0 - 1 + yy) mod the grid, slot s at byte 4 s.  The
  // records of a thread are the same in every plane: their in-plane offsets
  // are computed once.
  const int RW = g.XT + 2;
  const int nrec = (kTY + 2) * RW;
  constexpr int kRecPerThread = ((kTY + 2) * 34 + kThreads - 1) / kThreads;   // XT <= 32
  int roff[kRecPerThread];
#pragma unroll
  for (int u = 0; u < kRecPerThread; ++u) {
    const int i = tid + u * kThreads;
    roff[u] = -1;
    if (i < nrec) {
      const int yy = i / RW, xx = i - yy * RW;
      roff[u] = wrap(y0 - 1 + yy, ny) * nx + wrap(x0 - 1 + xx, nx);
    }
  }
  auto stage_plane = [&](int p) {
    if (p > L + 1) return;
    int zs = z0 - 1 + p;
    zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
    const int zoff = zs * nxy;
    const uint32_t dst0 = splanes + (uint32_t)((p % kRing) * g.PS);
#pragma unroll
    for (int u = 0; u < kRecPerThread; ++u) {
      if (roff[u] < 0) continue;
      const uint32_t d = dst0 + (uint32_t)((tid + u * kThreads) * 16);
      const int off = zoff + roff[u];
#pragma unroll
      for (int s = 0; s < 4; ++s)
        if (in[s]) cp_async4(d + 4 * s, in[s] + off);
    }
  };

  // MMAs of M tile t of output plane k (planes k, k + 1, k + 2 of the ring)
  // into TMEM buffer k % 2.  Lane 0 of warp t issues tile t: the tiles'
  // accumulators are disjoint, so the issue work is spread over TX warps, and
  // each issuer's commit is one of the TX arrivals the plane's barrier expects.
  const uint32_t idesc = tc::idesc_tf32(128, 32);
  auto issue = [&](int k, int t) {
    tc::fence_after_sync();
    const uint32_t dcol = (uint32_t)((k & 1) * g.TX * 32 + t * 32);
#pragma unroll
    for (int pz = 0; pz < 3; ++pz) {
      // plane base and tile t (8 records of 16 bytes) in descriptor units
      const uint64_t pb = (uint64_t)(((splanes + (uint32_t)(((k + pz) % kRing) * g.PS)) >> 4) + 8 * t);
#pragma unroll
      for (int p = 0; p < kPairs; ++p)
        tc::mma_tf32(tmem + dcol, dtab[kMmas + p] + pb, dtab[pz * kPairs + p], idesc, (pz | p) ? 1u : 0u);
    }
    tc::mma_commit(bar + (k & 1));
  };

  float c1 = a.c1, c2 = a.c2;
  if (MODE != AM_LINEAR && a.cc) {
    c1 = a.cc[0];
    c2 = a.cc[1];
  }
  // this thread's M row: TMEM lane quarter of the warp, node (xi, yi) of a tile
  const int q = w & 3;
  const int row = 32 * q + l;
  const int xi = row & 7, yi = row >> 3;
  const int gy = y0 + yi;
  const int ym = gy == 0 ? ny - 1 : gy - 1;
  constexpr int kTilesPerWarp = TPW;   // TX <= 2 TPW tiles, two warps per lane quarter

  // Output and operand planes of slot s: the CTA's first load has 64-bit
  // bases; a slot adds a 32-bit offset (component plane for the elastic block,
  // load for the Schur block).
  float* const yB = a.y + (i64)r0 * a.ys;
  float* const solB = a.sol ? a.sol + (i64)r0 * a.ss : nullptr;
  float* const doutB = a.dout ? a.dout + (i64)r0 * a.ds : nullptr;
  const float* const bB = a.b ? a.b + (i64)r0 * a.bs : nullptr;
  auto soff = [&](int s, i64 stride) -> int { return KIND == NK_UU ? s * nn : s * (int)stride; };

  // Per tile j of the thread: the node's in-plane index and those of its 8
  // elements' (x, y) positions (o & 3 = ex + 2 ey), fixed for every plane.
  int pin[kTilesPerWarp], rin[kTilesPerWarp][4];
  bool valid[kTilesPerWarp];
#pragma unroll
  for (int j = 0; j < kTilesPerWarp; ++j) {
    const int t = (w >> 2) + 2 * j;
    const int gxn = x0 + 8 * t + xi;
    valid[j] = t < g.TX && gxn < nx && gy < ny;
    const int xm = gxn == 0 ? nx - 1 : gxn - 1;
    pin[j] = gy * nx + gxn;
    rin[j][0] = ym * nx + xm;
    rin[j][1] = ym * nx + gxn;
    rin[j][2] = gy * nx + xm;
    rin[j][3] = gy * nx + gxn;
  }


  // Epilogue of output plane k in two parts.  prefetch(k) loads the node-wise
  // operands and the 8 rho values of each of the thread's nodes into registers
  // one step ahead (they are inputs the MMAs do not depend on, and the y and sol
  // entries a thread reads are the ones it alone writes); finish(k) waits
  // (bounded) for the plane's MMAs and runs TMEM -> registers -> rho-weighted
  // sum -> output.
  float rho[kTilesPerWarp][8];
  float e0[kTilesPerWarp][NS], e1[kTilesPerWarp][NS], e2[kTilesPerWarp][NS];
  auto prefetch = [&](int k) {
    const int gz = z0 + k;
    const int zo = gz * nxy, zmo = (gz == 0 ? nz - 1 : gz - 1) * nxy;
#pragma unroll
    for (int j = 0; j < kTilesPerWarp; ++j) {
      if (!valid[j]) continue;
#pragma unroll
      for (int o = 0; o < 8; ++o) rho[j][o] = __ldg(a.rho + ((o >> 2) ? zo : zmo) + rin[j][o & 3]);
      const int n = zo + pin[j];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        e0[j][s] = e1[j][s] = e2[j][s] = 0.f;
        if (KIND == NK_SS4 && !on[s]) continue;
        const int nd = (KIND == NK_UU ? s * nn : 0) + n;   // inverse diagonal [NC][nn]
        if (MODE == AM_LINEAR) {
          if (bB) e0[j][s] = bB[soff(s, a.bs) + n];
        } else if (MODE == AM_CHEB || MODE == AM_CHEB_LAST) {
          e0[j][s] = yB[soff(s, a.ys) + n];
          if (!a.sol_zero) e1[j][s] = solB[soff(s, a.ss) + n];
          if (MODE == AM_CHEB) e2[j][s] = __ldg(a.dinv + nd);
        } else {
          e0[j][s] = bB[soff(s, a.bs) + n];
          e2[j][s] = __ldg(a.dinv + nd);
        }
      }
    }
  };
  // L2 prefetch of the node-wise operands of output plane k (two steps before
  // prefetch(k) loads them into registers, so that those loads hit L2)
  auto l2_prefetch = [&](int k) {
    if (k >= L) return;
    const int zo = (z0 + k) * nxy;
#pragma unroll
    for (int j = 0; j < kTilesPerWarp; ++j) {
      if (!valid[j]) continue;
      const int n = zo + pin[j];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (KIND == NK_SS4 && !on[s]) continue;
        const float* p0 = MODE == AM_LINEAR || MODE == AM_RESID_CHEB0 ? bB + soff(s, a.bs) : yB + soff(s, a.ys);
        if (MODE != AM_LINEAR || bB) prefetch_l2(p0 + n);
        if ((MODE == AM_CHEB || MODE == AM_CHEB_LAST) && !a.sol_zero) prefetch_l2(solB + soff(s, a.ss) + n);
        if (MODE == AM_CHEB || MODE == AM_RESID_CHEB0) prefetch_l2(a.dinv + (KIND == NK_UU ? s * nn : 0) + n);
      }
    }
  };
  auto finish = [&](int k) -> bool {
    if (!tc::mbar_wait_bounded(bar + (k & 1), (uint32_t)((k >> 1) & 1), kWaitLimit)) return false;
    tc::fence_after_sync();
    const int zo = (z0 + k) * nxy;
    const unsigned char* pl = planes + ((k + 1) % kRing) * g.PS;   // the output plane's records
#pragma unroll
    for (int j = 0; j < kTilesPerWarp; ++j) {
      const int t = (w >> 2) + 2 * j;
      if (t >= g.TX) continue;   // warp-uniform: every lane of the warp has the same t
      float T[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((k & 1) * g.TX * 32 + t * 32), T);
      if (!valid[j]) continue;
      const float4 rec = *reinterpret_cast<const float4*>(pl + ((yi + 1) * RW + 8 * t + xi + 1) * 16);
      const float dold[4] = {rec.x, rec.y, rec.z, rec.w};
      const int n = zo + pin[j];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if (KIND == NK_SS4 && !on[s]) continue;
        float acc = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o) acc = fmaf(rho[j][o], T[4 * o + s], acc);
        node_out<MODE>(a, yB + soff(s, a.ys), solB ? solB + soff(s, a.ss) : nullptr,
                       doutB ? doutB + soff(s, a.ds) : nullptr, n, acc, dold[s], e0[j][s], e1[j][s],
                       e2[j][s], c1, c2);
      }
    }
    return true;
  };

  // ---- pipeline --------------------------------------------------------------
  // One block barrier per step.  Ring argument: plane p_new = k + 2 + kAhead is
  // staged at step k into the slot of p_old = p_new - kRing = k - 2.  p_old is
  // read by the MMAs of output planes up to k - 2, whose completion this thread
  // awaited in the epilogue of plane k - 2 (step k - 1), and by the epilogue of
  // output plane k - 3 (step k - 2), which every thread finished before the
  // barrier of step k - 1.  TMEM buffer k % 2 is rewritten by the MMAs issued
  // at step k + 2, after the barrier that follows every thread's epilogue of
  // plane k (step k + 1).  A thread whose wait gives up skips its remaining
  // epilogues but keeps taking the barriers.  The operands of plane k are
  // loaded at the end of step k and used at step k + 1.
  for (int p = 0; p < 2 + kAhead; ++p) {
    stage_plane(p);
    cp_async_commit();
  }
  l2_prefetch(0);
  l2_prefetch(1);
  bool aborted = false;
  int issued = 0, waited = 0;
  for (int k = 0; k < L; ++k) {
    stage_plane(k + 2 + kAhead);
    cp_async_commit();
    cp_async_wait<kAhead>();      // planes 0 .. k + 2 have landed
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    if (l == 0 && w < g.TX) issue(k, w);
    ++issued;
    if (k >= 1 && !aborted) {
      if (finish(k - 1)) ++waited;
      else aborted = true;
    }
    prefetch(k);
    l2_prefetch(k + 2);
  }
  if (!aborted) {
    if (finish(L - 1)) ++waited;
    else aborted = true;
  }
  cp_async_wait<0>();
  if (aborted) {
    atomicAdd(err, 1);
    // let every committed MMA group finish (bounded) before TMEM is released
    for (int k = waited; k < issued; ++k)
      if (!tc::mbar_wait_bounded(bar + (k & 1), (uint32_t)((k >> 1) & 1), kWaitLimit)) break;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tmem, (uint32_t)g.tcols);
}

float tf32_rn(double v) {
  float x = (float)v;
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & ~0x1FFFu;
  std::memcpy(&x, &u, 4);
  return x;
}

int g_nsm[64] = {0};

int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!g_nsm[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    g_nsm[dev] = v;
  }
  return g_nsm[dev];
}

// Default tile: the widest XT, and the chunk length L with the smallest
// (waves x staged planes) for two resident CTAs per SM (the z halo costs two
// planes per chunk).
int choose_chunk(int units, const NcGeom& g0) {
  const int slots = 2 * num_sms();
  const int cand[] = {4, 8, 16, 32, 64, 128, 256};
  int best = g0.nz;
  double best_cost = 1e300;
  for (int L : cand) {
    if (L > g0.nz && L != cand[0]) break;
    const int Lc = L > g0.nz ? g0.nz : L;
    const long long ctas = (long long)g0.gx * g0.gy * ((g0.nz + Lc - 1) / Lc) * units;
    const double waves = (double)((ctas + slots - 1) / slots);
    const double cost = waves * (Lc + 2);
    if (cost < best_cost) {
      best_cost = cost;
      best = Lc;
    }
  }
  return best;
}

constexpr int units_of(int kind, int nrhs) { return kind == NK_UU ? nrhs : (nrhs + 3) / 4; }

NcGeom geom_for(int kind, const ApplyArgs<float>& a, int nrhs, NcTile tile) {
  const int xt = tile.xt ? tile.xt : max_xt(a.nx);
  const int L = tile.L ? (tile.L < a.nz ? tile.L : a.nz)
                       : choose_chunk(units_of(kind, nrhs), make_geom(a.nx, a.ny, a.nz, a.nz, xt));
  return make_geom(a.nx, a.ny, a.nz, L, xt);
}

template <int KIND, int MODE>
bool launch(const ApplyArgs<float>& a, const float* Btab, int nrhs, int* err, cudaStream_t s, NcTile tile) {
  const int units = units_of(KIND, nrhs);
  const NcGeom g = geom_for(KIND, a, nrhs, tile);
  if ((long long)g.zchunks * units > 65535 || g.gy > 65535) return false;
  // 32-bit node indices and slot offsets inside the kernel
  const long long nn = (long long)a.nx * a.ny * a.nz;
  const long long lim = 1ll << 31;
  if (4 * nn >= lim || 4 * a.xs >= lim || 4 * a.ys >= lim || 4 * a.ss >= lim || 4 * a.ds >= lim ||
      4 * a.bs >= lim)
    return false;
  const dim3 grid((unsigned)g.gx, (unsigned)g.gy, (unsigned)(g.zchunks * units));
  if (g.TX > 2)
    note_launch(), k_nc<KIND, MODE, 2><<<grid, kThreads, g.smem, s>>>(a, Btab, g, nrhs, err);
  else
    note_launch(), k_nc<KIND, MODE, 1><<<grid, kThreads, g.smem, s>>>(a, Btab, g, nrhs, err);
  return true;
}

template <int KIND, int MODE>
void set_attr(int smem) {
  cudaFuncSetAttribute(k_nc<KIND, MODE, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_nc<KIND, MODE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace

bool nc_shape_ok(int nx, int ny, int nz) {
  return nx >= 2 && ny >= 2 && nz >= 2 && make_geom(nx, ny, nz, 1, max_xt(nx)).smem <= 227 * 1024;
}

void nc_prepare() {
  const int smem = make_geom(32, 16, 2, 1, 32).smem;   // the widest tile
  set_attr<NK_UU, AM_LINEAR>(smem);
  set_attr<NK_UU, AM_CHEB>(smem);
  set_attr<NK_UU, AM_CHEB_LAST>(smem);
  set_attr<NK_UU, AM_RESID_CHEB0>(smem);
  set_attr<NK_SS4, AM_LINEAR>(smem);
  set_attr<NK_SS4, AM_CHEB>(smem);
  set_attr<NK_SS4, AM_CHEB_LAST>(smem);
  set_attr<NK_SS4, AM_RESID_CHEB0>(smem);
}

size_t nc_table_floats() { return (size_t)kBFloats; }

// B operand of one kind in shared-memory order: MMA m = 5 pz + p (plane
// dz = pz - 1, pair p) is a 32 x 8 K-major tile whose row n = 4 o + c is
// output slot c of element position o = ex + 2 ey + 4 ez, and whose column
// k = 4 h + d is input slot d of the neighbour (pair_dx(p, h), pair_dy(p, h),
// dz).  Entry = K[4 la + c][4 b + d] (elastic: c, d < 3) or S0[la][b] (Schur:
// c = d, each slot one load), la = local index of the node in element o and
// b = local index of the neighbour in it (local node = x + 2y + 4z).
void nc_build_b(int kind, const double* K0, const double* S0, float* out) {
  for (int pz = 0; pz < 3; ++pz)
    for (int p = 0; p < kPairs; ++p)
      for (int h = 0; h < 2; ++h) {
        const int dx = pair_dx(p, h), dy = pair_dy(p, h), dz = pz - 1;
        const bool dummy = p == 4 && h == 1;
        for (int o = 0; o < 8; ++o) {
          const int ex = o & 1, ey = (o >> 1) & 1, ez = o >> 2;
          const int la = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
          const int bx = dx + 1 - ex, by = dy + 1 - ey, bz = dz + 1 - ez;
          const bool in = !dummy && bx >= 0 && bx <= 1 && by >= 0 && by <= 1 && bz >= 0 && bz <= 1;
          const int b = bx + 2 * by + 4 * bz;
          for (int c = 0; c < 4; ++c)
            for (int d = 0; d < 4; ++d) {
              double v = 0.0;
              if (in) {
                if (kind == NK_UU) {
                  if (c < 3 && d < 3) v = K0[(4 * la + c) * 32 + 4 * b + d];
                } else if (c == d) {
                  v = S0[la * 8 + b];
                }
              }
              const int n = 4 * o + c, k = 4 * h + d;
              out[(pz * kPairs + p) * 256 + (n / 8) * 64 + (k / 4) * 32 + (n % 8) * 4 + (k % 4)] = tf32_rn(v);
            }
        }
      }
}

bool apply_nc(int kind, const ApplyArgs<float>& a, const float* Btab, int mode, int nrhs, int* err,
              cudaStream_t s, NcTile tile) {
  if (kind == NK_UU) {
    switch (mode) {
      case AM_LINEAR: return launch<NK_UU, AM_LINEAR>(a, Btab, nrhs, err, s, tile);
      case AM_CHEB: return launch<NK_UU, AM_CHEB>(a, Btab, nrhs, err, s, tile);
      case AM_CHEB_LAST: return launch<NK_UU, AM_CHEB_LAST>(a, Btab, nrhs, err, s, tile);
      default: return launch<NK_UU, AM_RESID_CHEB0>(a, Btab, nrhs, err, s, tile);
    }
  }
  switch (mode) {
    case AM_LINEAR: return launch<NK_SS4, AM_LINEAR>(a, Btab, nrhs, err, s, tile);
    case AM_CHEB: return launch<NK_SS4, AM_CHEB>(a, Btab, nrhs, err, s, tile);
    case AM_CHEB_LAST: return launch<NK_SS4, AM_CHEB_LAST>(a, Btab, nrhs, err, s, tile);
    default: return launch<NK_SS4, AM_RESID_CHEB0>(a, Btab, nrhs, err, s, tile);
  }
}

// Tile autotuner.  Every (XT, L) candidate computes bitwise the same result
// (a node's MMA sequence and epilogue arithmetic do not depend on the tiling),
// so the choice is free: each candidate is timed on the caller's buffers in
// the given mode (one warm-up launch, then kTuneReps launches between CUDA
// events on the stream, in two rounds of opposite order, the better round
// kept) and the fastest kept.  Candidates: XT in {8, 16, 32} up to the grid's
// widest tile, L in {4, 8, ..., 256} up to nz (and nz itself), within the
// launch limits.  Returns the default tile if nothing could be timed.
NcTile nc_autotune(int kind, const ApplyArgs<float>& a, const float* Btab, int mode, int nrhs, int* err,
                   cudaStream_t s, float* best_us) {
  constexpr int kTuneReps = 3;
  NcTile best{0, 0};
  float best_t = 3.0e38f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    if (best_us) *best_us = 0.f;
    return best;
  }
  const int xts[] = {8, 16, 32};
  const int Ls[] = {4, 8, 16, 32, 64, 128, 256};
  NcTile cand[24];
  int nc = 0;
  for (int xt : xts) {
    if (xt > max_xt(a.nx)) break;
    for (int i = 0; i <= 7; ++i) {
      int L = i < 7 ? Ls[i] : a.nz;
      if (i < 7 && L >= a.nz) continue;   // nz itself is the last candidate
      cand[nc++] = NcTile{xt, L};
    }
  }
  // the GPU warms up (clocks, caches) over the first launches: a few launches
  // of the default tile first, then two rounds over the candidates in opposite
  // orders, each candidate keeping its faster round, so that no candidate is
  // favoured by its place in the sequence
  for (int r = 0; r < 2 * kTuneReps; ++r) apply_nc(kind, a, Btab, mode, nrhs, err, s, NcTile{0, 0});
  float tbest[24];
  for (int c = 0; c < nc; ++c) tbest[c] = 3.0e38f;
  for (int round = 0; round < 2; ++round)
    for (int ci = 0; ci < nc; ++ci) {
      const int c = round == 0 ? ci : nc - 1 - ci;
      const NcTile t = cand[c];
      if (!apply_nc(kind, a, Btab, mode, nrhs, err, s, t)) continue;
      cudaEventRecord(e0, s);
      bool ok = true;
      for (int r = 0; r < kTuneReps && ok; ++r) ok = apply_nc(kind, a, Btab, mode, nrhs, err, s, t);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (!ok || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        continue;
      if (ms < tbest[c]) tbest[c] = ms;
    }
  for (int c = 0; c < nc; ++c)
    if (tbest[c] < best_t) {
      best_t = tbest[c];
      best = cand[c];
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_us) *best_us = best.xt ? best_t * 1000.f / kTuneReps : 0.f;
  return best;
}

}  // namespace cell
