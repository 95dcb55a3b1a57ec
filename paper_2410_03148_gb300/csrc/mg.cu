// Geometric multigrid on the periodic structured grid, used as the inner
// solver for the two diagonal blocks of the approximate Schur complement
// preconditioner (§2.5.3): Chebyshev-Jacobi smoothing, full-weighting
// restriction / trilinear prolongation, Galerkin coarse element matrices,
// Jacobi diagonals, element-wise bounds of lambda_max(D^-1 A) and the
// coarsest-level dense solve.
#include "kernels.cuh"

namespace cell {

namespace {

constexpr int kB = 256;

inline unsigned nblocks(i64 n, int b = kB) { return (unsigned)((n + b - 1) / b); }

template <typename T, int NC>
__global__ void k_cheb_init(const T* __restrict__ b, i64 bs, T* __restrict__ r, i64 rs,
                            T* __restrict__ d, i64 ds, const T* __restrict__ dinv,
                            const T* __restrict__ c2p, i64 nn, const int* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const T c2 = *c2p;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T v = b[q * bs + c * nn + n];
    r[q * rs + c * nn + n] = v;
    d[q * ds + c * nn + n] = c2 * dinv[c * nn + n] * v;
  }
}

template <typename T, int NC>
__global__ void k_axpy_view(T* __restrict__ x, i64 xs, const T* __restrict__ d, i64 ds, i64 nn,
                            const int* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) x[q * xs + c * nn + n] += d[q * ds + c * nn + n];
}

// Full weighting (transpose of trilinear interpolation) on a periodic grid
// whose fine sizes nx, ny, nz are even; coarse node I sits on fine node 2I.
// With r and d set, the coarse level's Chebyshev start is written in the
// same pass: r = b, d = c2 Dinv b (what cheb_init would do next).
template <typename T, int NC>
__global__ void k_restrict(const T* __restrict__ rf, i64 rs, T* __restrict__ bc, i64 bs, int nx,
                           int ny, int nz, const int* active, T* __restrict__ rc, T* __restrict__ dc,
                           const T* __restrict__ dinv, const T* __restrict__ c2p) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const i64 ncn = (i64)cx * cy * cz, nfn = (i64)nx * ny * nz;
  const i64 m = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ncn) return;
  const int I = (int)(m % cx);
  const int J = (int)((m / cx) % cy);
  const int K = (int)(m / ((i64)cx * cy));
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const T w = T((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0));
        const int i = (2 * I + dx + nx) % nx, j = (2 * J + dy + ny) % ny, k = (2 * K + dz + nz) % nz;
        const i64 f = i + (i64)nx * (j + (i64)ny * k);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += w * rf[q * rs + c * nfn + f];
      }
#pragma unroll
  for (int c = 0; c < NC; ++c) bc[q * bs + c * ncn + m] = acc[c];
  if (rc) {
    const T c2 = *c2p;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      rc[q * bs + c * ncn + m] = acc[c];
      dc[q * bs + c * ncn + m] = c2 * dinv[c * ncn + m] * acc[c];
    }
  }
}

// xf += P (xc [+ dc]): with dc set, the coarse level's last smoothing
// direction is folded in here instead of a separate xc += dc pass.
template <typename T, int NC>
__global__ void k_prolong_add(const T* __restrict__ xc, i64 cs, T* __restrict__ xf, i64 fs, int nx,
                              int ny, int nz, const int* active, const T* __restrict__ dc) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const int cx = nx / 2, cy = ny / 2, cz = nz / 2;
  const i64 ncn = (i64)cx * cy * cz, nfn = (i64)nx * ny * nz;
  const i64 f = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfn) return;
  const int i = (int)(f % nx);
  const int j = (int)((f / nx) % ny);
  const int k = (int)(f / ((i64)nx * ny));
  // per direction: one coarse node (even) or two with weight 1/2 (odd)
  const int i0 = i >> 1, i1 = (i & 1) ? ((i0 + 1) % cx) : i0;
  const int j0 = j >> 1, j1 = (j & 1) ? ((j0 + 1) % cy) : j0;
  const int k0 = k >> 1, k1 = (k & 1) ? ((k0 + 1) % cz) : k0;
  const T wx = (i & 1) ? T(0.5) : T(1), wy = (j & 1) ? T(0.5) : T(1), wz = (k & 1) ? T(0.5) : T(1);
  const int ii[2] = {i0, i1}, jj[2] = {j0, j1}, kk[2] = {k0, k1};
  const int nxs = (i & 1) ? 2 : 1, nys = (j & 1) ? 2 : 1, nzs = (k & 1) ? 2 : 1;
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  for (int c2 = 0; c2 < nzs; ++c2)
    for (int b2 = 0; b2 < nys; ++b2)
      for (int a2 = 0; a2 < nxs; ++a2) {
        const i64 m = ii[a2] + (i64)cx * (jj[b2] + (i64)cy * kk[c2]);
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[c] += xc[q * cs + c * ncn + m] + (dc ? dc[q * cs + c * ncn + m] : T(0));
      }
  const T w = wx * wy * wz;
#pragma unroll
  for (int c = 0; c < NC; ++c) xf[q * fs + c * nfn + f] += w * acc[c];
}

// Weight of coarse corner B for the fine local node a of child c (corner
// index = x + 2y + 4z); fine positions (c + a)/2 in {0, 1/2, 1}^3.
__device__ __forceinline__ float child_w(int c, int a, int B) {
  float w = 1.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int p2 = ((c >> d) & 1) + ((a >> d) & 1);
    const int Bd = (B >> d) & 1;
    if (p2 == 1) w *= 0.5f;
    else if ((p2 == 0) != (Bd == 0)) return 0.f;
  }
  return w;
}

// One thread per (coarse element, output row); K_E = sum_c P_c^T K_c P_c.
// blockIdx.y = output row (A, d).  Fine matrices: fixedm (8NC)^2 * rho[c]
// (level 0) or SoA kef (coarser levels).
template <typename T, int NC>
__global__ void k_galerkin(const T* __restrict__ fixedm, const T* __restrict__ rho,
                           const T* __restrict__ kef, T* __restrict__ kec, int ncx, int ncy, int ncz) {
  constexpr int R = 8 * NC;
  const i64 nce = (i64)ncx * ncy * ncz;
  const i64 E = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  const int row = blockIdx.y;
  const int A = row / NC, d = row % NC;
  if (E >= nce) return;
  const int nx = 2 * ncx, ny = 2 * ncy;
  const i64 nfe = nce * 8;
  const int I = (int)(E % ncx), J = (int)((E / ncx) % ncy), K = (int)(E / ((i64)ncx * ncy));
  T out[R];
#pragma unroll
  for (int col = 0; col < R; ++col) out[col] = T(0);
  for (int c = 0; c < 8; ++c) {
    const i64 fe = (2 * I + (c & 1)) + (i64)nx * ((2 * J + ((c >> 1) & 1)) + (i64)ny * (2 * K + (c >> 2)));
    const T rr = rho ? rho[fe] : T(1);
    for (int a = 0; a < 8; ++a) {
      const float wa = child_w(c, a, A);
      if (wa == 0.f) continue;
      // fine row (a, d) of K_c, contracted with the column weights
      for (int b = 0; b < 8; ++b) {
        T kb[NC];
#pragma unroll
        for (int dd = 0; dd < NC; ++dd) {
          const int entry = (a * NC + d) * R + b * NC + dd;
          kb[dd] = rho ? rr * fixedm[entry] : kef[(i64)entry * nfe + fe];
        }
#pragma unroll
        for (int B = 0; B < 8; ++B) {
          const float wb = child_w(c, b, B);
          if (wb == 0.f) continue;
          const T w = T(wa) * T(wb);
#pragma unroll
          for (int dd = 0; dd < NC; ++dd) out[B * NC + dd] += w * kb[dd];
        }
      }
    }
  }
#pragma unroll
  for (int col = 0; col < R; ++col) kec[(i64)(row * R + col) * nce + E] = out[col];
}

// Level-1 coarse element matrices when every fine element matrix is
// rho_e K: K_E = sum over the 8 children c of rho_c G_c with the fixed
// G_c = P_c^T K P_c (computed once per material and grid on the host).
// Thread per (coarse element, matrix entry); blockIdx.y = entry.
template <typename T, int NC>
__global__ void k_galerkin_child(const T* __restrict__ G, const T* __restrict__ rho, T* __restrict__ kec,
                                 int ncx, int ncy, int ncz) {
  constexpr int R = 8 * NC;
  const i64 nce = (i64)ncx * ncy * ncz;
  const i64 E = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  const int entry = blockIdx.y;
  if (E >= nce) return;
  const int nx = 2 * ncx, ny = 2 * ncy;
  const int I = (int)(E % ncx), J = (int)((E / ncx) % ncy), K = (int)(E / ((i64)ncx * ncy));
  T out = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const i64 fe = (2 * I + (c & 1)) + (i64)nx * ((2 * J + ((c >> 1) & 1)) + (i64)ny * (2 * K + (c >> 2)));
    out = fma(rho[fe], G[c * R * R + entry], out);
  }
  kec[(i64)entry * nce + E] = out;
}

template <typename T, int NC>
__global__ void k_diag_inv(const T* __restrict__ fixedm, const T* __restrict__ rho,
                           const T* __restrict__ ke, T* __restrict__ dinv, int nx, int ny, int nz) {
  constexpr int R = 8 * NC;
  const i64 nxy = (i64)nx * ny, nn = nxy * nz;
  const i64 n = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nn) return;
  const int i = (int)(n % nx), j = (int)((n / nx) % ny), k = (int)(n / nxy);
  T acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = T(0);
  for (int e = 0; e < 8; ++e) {
    const int ex = e & 1, ey = (e >> 1) & 1, ez = e >> 2;
    const int la = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
    const int ei = (i - 1 + ex + nx) % nx, ej = (j - 1 + ey + ny) % ny, ek = (k - 1 + ez + nz) % nz;
    const i64 el = ei + nx * (ej + (i64)ny * ek);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int entry = (la * NC + c) * R + la * NC + c;
      acc[c] += rho ? rho[el] * fixedm[entry] : ke[(i64)entry * nn + el];
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) dinv[c * nn + n] = acc[c] > T(0) ? T(1) / acc[c] : T(0);
}

// lambda_max(diag(K_e)^-1 K_e) per element by power iteration on the
// symmetric scaled matrix D^-1/2 K D^-1/2, max-reduced as float bits.
// (FP32 arithmetic: this is a bound for a smoother, not a result.)
template <typename T, int NC>
__global__ void k_elem_lmax(const T* __restrict__ ke, i64 ne, unsigned int* out) {
  constexpr int R = 8 * NC;
  const i64 e = (i64)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  float s[R], v[R], w[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const float dii = (float)ke[(i64)(i * R + i) * ne + e];
    s[i] = dii > 0.f ? rsqrtf(dii) : 0.f;
    v[i] = 1.f + 0.1f * i;
  }
  float lam = 0.f;
  for (int it = 0; it < 30; ++it) {
    float nv = 0.f, vv = 0.f, vw = 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < R; ++j) acc = fmaf((float)__ldg(ke + (i64)(i * R + j) * ne + e), s[j] * v[j], acc);
      w[i] = s[i] * acc;
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
      nv = fmaf(w[i], w[i], nv);
      vv = fmaf(v[i], v[i], vv);
      vw = fmaf(v[i], w[i], vw);
    }
    lam = vv > 0.f ? vw / vv : 0.f;
    const float inv = nv > 0.f ? rsqrtf(nv) : 0.f;
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = w[i] * inv;
  }
  if (lam > 0.f) atomicMax(out, __float_as_uint(lam));
}

// x = Ainv b per rhs and component block (nc comps of nn nodes, n = nc*nn).
// Ainv is symmetric, so thread t reads column t (coalesced across threads).
template <typename T>
__global__ void k_dense_solve(const T* __restrict__ Ainv, int n, const T* __restrict__ b, i64 bs,
                              T* __restrict__ x, i64 xs, const int* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  T acc = T(0);
  for (int j = 0; j < n; ++j) acc += Ainv[(i64)j * n + t] * b[q * bs + j];
  x[q * xs + t] = acc;
}

}  // namespace

template <typename T, int NC>
void cheb_init(const T* b, i64 bs, T* r, i64 rs, T* d, i64 ds, const T* dinv, const T* c2p, i64 nn,
               int nrhs, const int* active, cudaStream_t s) {
  note_launch(), k_cheb_init<T, NC><<<dim3(nblocks(nn), nrhs), kB, 0, s>>>(b, bs, r, rs, d, ds, dinv, c2p, nn, active);
}
template <typename T, int NC>
void axpy_view(T* x, i64 xs, const T* d, i64 ds, i64 nn, int nrhs, const int* active, cudaStream_t s) {
  note_launch(), k_axpy_view<T, NC><<<dim3(nblocks(nn), nrhs), kB, 0, s>>>(x, xs, d, ds, nn, active);
}
template <typename T, int NC>
void restrict_fw(const T* rf, i64 rs, T* bc, i64 bs, int nx, int ny, int nz, int nrhs,
                 const int* active, cudaStream_t s) {
  const i64 ncn = (i64)(nx / 2) * (ny / 2) * (nz / 2);
  note_launch(), k_restrict<T, NC><<<dim3(nblocks(ncn), nrhs), kB, 0, s>>>(rf, rs, bc, bs, nx, ny, nz, active,
                                                                          nullptr, nullptr, nullptr, nullptr);
}
template <typename T, int NC>
void restrict_init(const T* rf, i64 rs, T* bc, T* rc, T* dc, i64 cs, const T* dinv, const T* c2p, int nx,
                   int ny, int nz, int nrhs, const int* active, cudaStream_t s) {
  const i64 ncn = (i64)(nx / 2) * (ny / 2) * (nz / 2);
  note_launch(), k_restrict<T, NC><<<dim3(nblocks(ncn), nrhs), kB, 0, s>>>(rf, rs, bc, cs, nx, ny, nz, active,
                                                                          rc, dc, dinv, c2p);
}
template <typename T, int NC>
void prolong_add(const T* xc, i64 cs, T* xf, i64 fs, int nx, int ny, int nz, int nrhs,
                 const int* active, cudaStream_t s, const T* dc) {
  const i64 nfn = (i64)nx * ny * nz;
  note_launch(), k_prolong_add<T, NC><<<dim3(nblocks(nfn), nrhs), kB, 0, s>>>(xc, cs, xf, fs, nx, ny, nz, active,
                                                                              dc);
}
template <typename T, int NC>
void galerkin(const T* fixedm, const T* rho, const T* kef, T* kec, int ncx, int ncy, int ncz,
              cudaStream_t s) {
  const i64 nce = (i64)ncx * ncy * ncz;
  note_launch(), k_galerkin<T, NC><<<dim3(nblocks(nce, 128), 8 * NC), 128, 0, s>>>(fixedm, rho, kef, kec, ncx, ncy, ncz);
}
template <typename T, int NC>
void galerkin_child(const T* G, const T* rho, T* kec, int ncx, int ncy, int ncz, cudaStream_t s) {
  const i64 nce = (i64)ncx * ncy * ncz;
  note_launch(), k_galerkin_child<T, NC><<<dim3(nblocks(nce, 128), 64 * NC * NC), 128, 0, s>>>(G, rho, kec, ncx,
                                                                                             ncy, ncz);
}
template <typename T, int NC>
void diag_inv(const T* fixedm, const T* rho, const T* ke, T* dinv, int nx, int ny, int nz,
              cudaStream_t s) {
  const i64 nn = (i64)nx * ny * nz;
  note_launch(), k_diag_inv<T, NC><<<nblocks(nn), kB, 0, s>>>(fixedm, rho, ke, dinv, nx, ny, nz);
}
template <typename T, int NC>
void elem_lmax(const T* ke, i64 ne, unsigned int* out, cudaStream_t s) {
  note_launch(), k_elem_lmax<T, NC><<<nblocks(ne, 64), 64, 0, s>>>(ke, ne, out);
}
template <typename T>
void dense_solve(const T* Ainv, int n, const T* b, i64 bs, T* x, i64 xs, i64 nn, int nc, int nrhs,
                 const int* active, cudaStream_t s) {
  (void)nn;
  (void)nc;
  note_launch(), k_dense_solve<T><<<dim3(nblocks(n, 128), nrhs), 128, 0, s>>>(Ainv, n, b, bs, x, xs, active);
}

#define INST_NC(T, NC)                                                                              \
  template void cheb_init<T, NC>(const T*, i64, T*, i64, T*, i64, const T*, const T*, i64, int, const int*, \
                                 cudaStream_t);                                                     \
  template void axpy_view<T, NC>(T*, i64, const T*, i64, i64, int, const int*, cudaStream_t);        \
  template void restrict_fw<T, NC>(const T*, i64, T*, i64, int, int, int, int, const int*,          \
                                   cudaStream_t);                                                   \
  template void prolong_add<T, NC>(const T*, i64, T*, i64, int, int, int, int, const int*,          \
                                   cudaStream_t, const T*);                                         \
  template void galerkin<T, NC>(const T*, const T*, const T*, T*, int, int, int, cudaStream_t);     \
  template void galerkin_child<T, NC>(const T*, const T*, T*, int, int, int, cudaStream_t);         \
  template void restrict_init<T, NC>(const T*, i64, T*, T*, T*, i64, const T*, const T*, int, int, int, \
                                     int, const int*, cudaStream_t);                                \
  template void diag_inv<T, NC>(const T*, const T*, const T*, T*, int, int, int, cudaStream_t);     \
  template void elem_lmax<T, NC>(const T*, i64, unsigned int*, cudaStream_t);
INST_NC(float, 1)
INST_NC(float, 3)
INST_NC(double, 1)
INST_NC(double, 3)
template void dense_solve<float>(const float*, int, const float*, i64, float*, i64, i64, int, int,
                                 const int*, cudaStream_t);
template void dense_solve<double>(const double*, int, const double*, i64, double*, i64, i64, int,
                                  int, const int*, cudaStream_t);
#undef INST_NC

}  // namespace cell
