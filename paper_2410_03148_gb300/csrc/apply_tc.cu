// Element-matrix operator applies on the 5th-generation tensor cores.
//
// y_n = sum over elements e around n of rho_e (K x_e)_n, with K a fixed
// (8NC x 8NC) block of the element matrix K0 (§2.5, Eq. sym-piezo): the
// contraction K x_e for all elements of a brick is one dense GEMM,
//   D[e][j] = sum_k A[e][k] B[j][k],  A[e][k] = x(node(e, k / NC), k % NC),
//   B[j][k] = K[j][k],
// run by tcgen05.mma (kind::tf32, FP32 accumulate in TMEM).  With the 3-term
// split x = xh + xl, K = Kh + Kl (each TF32) the products xh Kh + xh Kl + xl Kh
// recover FP32 accuracy ("3xTF32").
//
// Used for the full operator Ahat (NC = 4, potential rows negated).  One CTA
// (128 threads) owns a brick of 16 x 4 x 2 nodes and a group of
// loads.  Per load it stages the x values of the 18 x 6 x 4 halo nodes in
// shared memory and builds the gathered rows of the 17 x 5 x 3 = 255 elements
// touching the brick as a K-major no-swizzle operand (two M = 128 tiles).
// Each warp writes whole 128-byte core matrices (bank-conflict free), taking
// its gather indices from a precomputed table held in registers.  One thread
// issues the MMAs; after a bounded mbarrier wait, thread t reads rows t and
// 128 + t of D from TMEM, scales them by rho_e and adds the contributions to
// owned nodes in shared memory; the per-node epilogue (plain, residual or
// Chebyshev step) is the one of the SIMT kernels.  Face elements are computed
// by both bricks that share them (redundant tensor-core work), so every
// node's sum stays inside one CTA: no global atomics.
#include <cstring>

#include "kernels.cuh"
#include "tc.cuh"

namespace cell {

namespace {

constexpr int BX = 16, BY = 4, BZ = 2;                // owned nodes per brick
constexpr int HX = BX + 2, HY = BY + 2, HZ = BZ + 2;  // halo nodes
constexpr int EX = BX + 1, EY = BY + 1, EZ = BZ + 1;  // elements touching the brick
constexpr int NHALO = HX * HY * HZ;                   // 432
constexpr int NELEM = EX * EY * EZ;                   // 255
constexpr int NOWN = BX * BY * BZ;                    // 128
constexpr int kThreads = 128;
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr unsigned short kPad = 0xFFFF;

template <int NC>
struct Plan {
  static constexpr int K = 8 * NC;                 // element dofs of the block
  static constexpr int KG = K / 4;                 // core-matrix columns
  static constexpr int CM = 32 * KG;               // core matrices per 256-row operand
  static constexpr int ITER = CM / 4;              // core matrices per warp
  static constexpr int SBO = KG * 128;
  static constexpr int ABYTES = 256 * K * 4;
  static constexpr int BBYTES = 32 * K * 4;
  static constexpr int HLOAD = (NC * NHALO + kThreads - 1) / kThreads;
  static constexpr int OFF_AL = ABYTES;
  static constexpr int OFF_B = 2 * ABYTES;
  static constexpr int OFF_X = OFF_B + 2 * BBYTES;
  static constexpr int OFF_ACC = OFF_X + NC * NHALO * 4;
  static constexpr int OFF_BAR = (OFF_ACC + NC * NOWN * 4 + 15) / 16 * 16;
  static constexpr int SMEM = OFF_BAR + 32;
};

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

template <int NC, int MODE, bool NEG>
__global__ void __launch_bounds__(kThreads)
k_apply_tc(const ApplyArgs<float> a, const float* __restrict__ Btiles,
           const unsigned short* __restrict__ gsrc, int nrhs, int rg, int* err) {
  using P = Plan<NC>;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* sA = smem;
  unsigned char* sAl = smem + P::OFF_AL;
  unsigned char* sB = smem + P::OFF_B;
  float* xs = reinterpret_cast<float*>(smem + P::OFF_X);     // [NC][NHALO]
  float* acc = reinterpret_cast<float*>(smem + P::OFF_ACC);  // [NC][NOWN]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + P::OFF_BAR);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + P::OFF_BAR + 16);

  const int r_begin = blockIdx.z * rg;
  const int r_end = r_begin + rg < nrhs ? r_begin + rg : nrhs;
  bool any = false;
  for (int r = r_begin; r < r_end; ++r) any = any || !(a.active && !a.active[r]);
  if (!any) return;

  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int nbx = nx / BX;
  const int i0 = (blockIdx.x % nbx) * BX, j0 = (blockIdx.x / nbx) * BY, k0 = blockIdx.y * BZ;
  const i64 nn = (i64)nx * ny * nz;

  // B tiles (hi, lo), prepared on the host in the core-matrix layout
  {
    const float4* src = reinterpret_cast<const float4*>(Btiles);
    float4* dst = reinterpret_cast<float4*>(sB);
    for (int i = t; i < 2 * P::BBYTES / 16; i += kThreads) dst[i] = __ldg(src + i);
  }
  // gather indices of this thread's core-matrix slots
  unsigned short src_idx[P::ITER];
#pragma unroll
  for (int it = 0; it < P::ITER; ++it) src_idx[it] = __ldg(gsrc + (w + 4 * it) * 32 + lane);
  // global offsets of this thread's halo entries
  int hoff[P::HLOAD];
#pragma unroll
  for (int i = 0; i < P::HLOAD; ++i) {
    const int idx = t + kThreads * i;
    const int c = idx / NHALO, h = idx % NHALO;
    const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
    int gx = i0 + hx - 1, gy = j0 + hy - 1, gz = k0 + hz - 1;
    gx += gx < 0 ? nx : (gx >= nx ? -nx : 0);
    gy += gy < 0 ? ny : (gy >= ny ? -ny : 0);
    gz += gz < 0 ? nz : (gz >= nz ? -nz : 0);
    hoff[i] = idx < NC * NHALO ? (int)(c * nn + gx + (i64)nx * (gy + (i64)ny * gz)) : -1;
  }
  // this thread's two element rows: rho and position in the element brick
  float rho_e[2];
  int epos[2];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int e = t + 128 * half;
    const int ex = e % EX, ey = (e / EX) % EY, ez = e / (EX * EY);
    epos[half] = e < NELEM ? (ex | (ey << 8) | (ez << 16)) : -1;
    int gx = i0 + ex - 1, gy = j0 + ey - 1, gz = k0 + ez - 1;
    gx += gx < 0 ? nx : 0;
    gy += gy < 0 ? ny : 0;
    gz += gz < 0 ? nz : 0;
    rho_e[half] = e < NELEM ? __ldg(a.rho + gx + (i64)nx * (gy + (i64)ny * gz)) : 0.f;
  }
  // owned node of this thread for the epilogue
  const int ox = t % BX, oy = (t / BX) % BY, oz = t / (BX * BY);
  const i64 n_own = (i0 + ox) + (i64)nx * ((j0 + oy) + (i64)ny * (k0 + oz));
  const int h_own = (ox + 1) + HX * ((oy + 1) + HY * (oz + 1));

  if (t == 0) {
    tc::mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    tc::tmem_alloc(slot, 64);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = *slot;
  const uint32_t id = tc::idesc_tf32(128, 32);
  const uint32_t a0 = tc::smem_u32(sA), al0 = tc::smem_u32(sAl), b0 = tc::smem_u32(sB);
  const uint32_t bl0 = b0 + P::BBYTES;
  uint32_t phase = 0;
  bool timed_out = false;

  for (int r = r_begin; r < r_end; ++r) {
    if (a.active && !a.active[r]) continue;
    // x on the halo, zero node sums
    const float* X = a.x + r * a.xs;
#pragma unroll
    for (int i = 0; i < P::HLOAD; ++i)
      if (hoff[i] >= 0) xs[t + kThreads * i] = __ldg(X + hoff[i]);
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c * NOWN + t] = 0.f;
    __syncthreads();
    // gathered rows, split into TF32 high and low parts
#pragma unroll
    for (int it = 0; it < P::ITER; ++it) {
      const unsigned short s = src_idx[it];
      const float v = s == kPad ? 0.f : xs[s];
      const float vh = to_tf32(v);
      const int off = (w + 4 * it) * 128 + lane * 4;
      *reinterpret_cast<float*>(sA + off) = vh;
      *reinterpret_cast<float*>(sAl + off) = to_tf32(v - vh);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
#pragma unroll
      for (int tile = 0; tile < 2; ++tile)
#pragma unroll
        for (int s = 0; s < P::K / 8; ++s) {
          const uint32_t ao = tile * 16 * P::SBO + s * 256, bo = s * 256;
          const uint32_t d = tm + 32 * tile;
          tc::mma_tf32(d, tc::sdesc(a0 + ao, 128, P::SBO), tc::sdesc(b0 + bo, 128, P::SBO), id, s > 0);
          tc::mma_tf32(d, tc::sdesc(a0 + ao, 128, P::SBO), tc::sdesc(bl0 + bo, 128, P::SBO), id, 1);
          tc::mma_tf32(d, tc::sdesc(al0 + ao, 128, P::SBO), tc::sdesc(b0 + bo, 128, P::SBO), id, 1);
        }
      tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait_bounded(bar, phase, kWaitLimit);
    phase ^= 1u;
    tc::fence_after_sync();
    if (!ok) {
      timed_out = true;
    } else {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        float dv[32];
        tc::tmem_ld32(tm + ((uint32_t)(32 * w) << 16) + 32 * half, dv);
        const int p = epos[half];
        if (p >= 0) {
          const int ex = p & 0xFF, ey = (p >> 8) & 0xFF, ez = p >> 16;
#pragma unroll
          for (int b = 0; b < 8; ++b) {
            const int hx = ex + (b & 1), hy = ey + ((b >> 1) & 1), hz = ez + (b >> 2);
            if (hx >= 1 && hx <= BX && hy >= 1 && hy <= BY && hz >= 1 && hz <= BZ) {
              const int o = (hx - 1) + BX * ((hy - 1) + BY * (hz - 1));
#pragma unroll
              for (int c = 0; c < NC; ++c) atomicAdd(&acc[c * NOWN + o], rho_e[half] * dv[b * NC + c]);
            }
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    // per-node epilogue
    float c1 = a.c1, c2 = a.c2;
    if (MODE != AM_LINEAR && a.cc) {
      c1 = a.cc[0];
      c2 = a.cc[1];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float av = acc[c * NOWN + t];
      if (NEG && c == NC - 1) av = -av;
      const i64 o = (i64)c * nn + n_own;
      if (MODE == AM_LINEAR) {
        float v = a.alpha * av;
        if (a.b) v += a.beta * a.b[r * a.bs + o];
        a.y[r * a.ys + o] = v;
      } else if (MODE == AM_CHEB || MODE == AM_CHEB_LAST) {
        const float dold = xs[c * NHALO + h_own];
        const float rr = a.y[r * a.ys + o] - av;
        a.y[r * a.ys + o] = rr;
        float* sp = a.sol + r * a.ss + o;
        *sp = (a.sol_zero ? 0.f : *sp) + dold;
        if (MODE == AM_CHEB) a.dout[r * a.ds + o] = c1 * dold + c2 * a.dinv[o] * rr;
      } else {
        const float rr = a.b[r * a.bs + o] - av;
        a.y[r * a.ys + o] = rr;
        a.dout[r * a.ds + o] = c2 * a.dinv[o] * rr;
      }
    }
    __syncthreads();  // xs and acc are rewritten by the next load
  }
  if (timed_out && lane == 0) atomicAdd(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (w == 0) tc::tmem_dealloc(tm, 64);
}

template <int NC, int MODE, bool NEG>
void set_smem_attr() {
  cudaFuncSetAttribute(k_apply_tc<NC, MODE, NEG>, cudaFuncAttributeMaxDynamicSharedMemorySize, Plan<NC>::SMEM);
}

template <int NC, int MODE, bool NEG>
void launch(const ApplyArgs<float>& a, const TcTables& T, int nrhs, int* err, cudaStream_t s) {
  using P = Plan<NC>;
  const int rg = 3;
  const dim3 g((unsigned)((a.nx / BX) * (a.ny / BY)), (unsigned)(a.nz / BZ), (unsigned)((nrhs + rg - 1) / rg));
  const float* Bt = T.b_full;
  const unsigned short* gs = T.g_full;
  note_launch(), k_apply_tc<NC, MODE, NEG><<<g, kThreads, P::SMEM, s>>>(a, Bt, gs, nrhs, rg, err);
}

// TF32 rounding on the host, matching cvt.rna (nearest, ties away from zero).
float host_tf32(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & ~0x1FFFu;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

template <int NC>
void build_tables(const double* K0, float* btiles, unsigned short* gsrc) {
  using P = Plan<NC>;
  const int K = P::K;
  // B = rows j (output dof a*NC+c), columns k (input dof b*NC+d); rows >= K zero
  for (int j = 0; j < 32; ++j)
    for (int k = 0; k < K; ++k) {
      float v = 0.f;
      if (j < K) {
        const int ja = j / NC, jc = j % NC, kb = k / NC, kd = k % NC;
        v = (float)K0[(ja * 4 + jc) * 32 + kb * 4 + kd];
      }
      const float vh = host_tf32(v);
      const int off = tc::kmajor_off(j, k, K) / 4;
      btiles[off] = vh;
      btiles[P::BBYTES / 4 + off] = host_tf32(v - vh);
    }
  for (int cm = 0; cm < P::CM; ++cm)
    for (int l = 0; l < 32; ++l) {
      const int g = cm / P::KG, c = cm % P::KG;
      const int row = 8 * g + l / 4, col = 4 * c + l % 4;
      unsigned short v = kPad;
      if (row < NELEM) {
        const int ex = row % EX, ey = (row / EX) % EY, ez = row / (EX * EY);
        const int b = col / NC, d = col % NC;
        const int h = (ex + (b & 1)) + HX * ((ey + ((b >> 1) & 1)) + HY * (ez + (b >> 2)));
        v = (unsigned short)(d * NHALO + h);
      }
      gsrc[cm * 32 + l] = v;
    }
}

}  // namespace

// Opt the kernels into their dynamic shared memory (once per device, before
// any launch or graph capture).
void tc_prepare() { set_smem_attr<4, AM_LINEAR, true>(); }

bool tc_shape_ok(int nx, int ny, int nz) {
  return nx % BX == 0 && ny % BY == 0 && nz % BZ == 0 && nx >= BX && ny >= BY && nz >= BZ;
}

size_t tc_table_floats() { return 2 * Plan<4>::BBYTES / 4; }
size_t tc_table_idx() { return Plan<4>::CM * 32; }

void tc_build_tables_host(const double* K0, float* b_full, unsigned short* g_full) {
  build_tables<4>(K0, b_full, g_full);
}

void apply_tc_full(const ApplyArgs<float>& a, const TcTables& T, int nrhs, int* err, cudaStream_t s) {
  launch<4, AM_LINEAR, true>(a, T, nrhs, err, s);
}

}  // namespace cell
