// Internal declarations shared by the library's CUDA translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>

namespace cell {

typedef long long i64;

// Record the failure that cell_last_error() reports to the calling thread.
void report_error(const char* what, cudaError_t e);

// Count of kernels launched by the library (cell_launch_count()).
extern std::atomic<long long> g_launches;
inline void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Leading dimension of the per-load Krylov scalars (Gram-Schmidt columns,
// partial sums); bounds the GMRES restart length.
constexpr int kNvMax = 64;

// Loads: F = K0 Zbar (32 x 9, row-major) for the right-hand sides.
struct RhsParams {
  double F[32 * 9];
};

// Sensitivity: the affine load fields Zbar (32 x 9, row-major) and the
// upstream weights G (9 x 9, row-major) of L = sum G_IJ H_IJ.
struct SensParams {
  double Z[32 * 9];
  double G[81];
};

// Element sensitivities in eigen-modes of the symmetrised upstream weights
// sym(G) = Q diag(lam) Q^T (modes with lam = 0 dropped): X^m = sum_I Q_Im W^I.
struct SensQ {
  double q[81];   // Q[I*9 + m]
  int R;          // number of modes kept
};
template <typename T>
struct SensModes {
  T ku[1024];     // upper triangle of K0 (row-major), off-diagonal entries doubled
  T zq[32 * 9];   // affine part of the modes at local dof a: (Zbar Q)[a*9 + m]
  T lam[9];
  int R;
};

// Energy difference of two solutions (FP64): the full K0, the affine part of
// the modes and the eigenvalues of sym(G).
struct SensPair {
  double k[1024];
  double zq[32 * 9];
  double lam[9];
  int R;
};

// Fixed element matrix passed by value as a kernel parameter: (8*NCM)^2
// entries, row-major over local dofs NCM*node + comp.  Kernel parameters live
// in the constant bank, so fully unrolled loops read the entries as FFMA/DFMA
// constant operands.
template <typename T, int NCM>
struct FixedMat {
  T k[64 * NCM * NCM];
};

enum ApplyMode {
  AM_LINEAR = 0,       // y = alpha*(A x) + beta*b            (b optional)
  AM_CHEB = 1,         // x = d_old(gathered):  sol += d_old; r -= A d_old;
                       //                       d_new = c1 d_old + c2 Dinv r
  AM_CHEB_LAST = 2,    // sol += d_old; r -= A d_old
  AM_RESID_CHEB0 = 3   // x = sol(gathered): r = b - A sol; d_new = c2 Dinv r
};

// Pointers of an operator application.  Every field vector is a set of nrhs
// component-planar blocks: value(rhs q, comp c, node n) = p[q*stride + c*nn + n].
template <typename T>
struct ApplyArgs {
  const T* x; i64 xs;      // gathered input
  T* y; i64 ys;            // LINEAR: output; CHEB modes: residual (in/out)
  const T* b; i64 bs;      // LINEAR: optional addend; RESID_CHEB0: right-hand side
  T* sol; i64 ss;          // CHEB modes: iterate (in/out)
  T* dout; i64 ds;         // CHEB / RESID_CHEB0: new search direction
  const T* dinv;           // [NC][nn] inverse diagonal
  const T* rho;            // per-element scale (fixed-matrix operators)
  const T* ke;             // per-element matrices, SoA: ke[entry*ne + e]
  const T* st;             // assembled 27-point block stencil, SoA: st[((q*NC+c)*NC+d)*nn + n]
  T alpha, beta, c1, c2;
  const T* cc;             // if set: device (c1, c2) pair used instead of c1, c2
  int nx, ny, nz;
  int sol_zero;            // CHEB modes: incoming sol is implicitly zero
  const int* active;       // per-rhs flag (nullptr = all active)
  int cslot1;              // FP32 fixed-matrix kernels: constant-bank slot + 1 (0 = use parameter)
  int nrhs;                // number of loads of the launch (set by the launchers)
};

// Constant-bank slots holding (K0, S0) in FP32 for the fixed-matrix kernels;
// returns slot + 1, or 0 if none is free.  Release with cslot_release.
int cslot_acquire(const float* K0f, const float* S0f);
void cslot_release(int slot1);

// ---- operator applies (apply.cu) -------------------------------------------
// Full nonsymmetric operator Ahat (4 -> 4 comps, potential rows negated).
template <typename T> void apply_full(const ApplyArgs<T>& a, const FixedMat<T, 4>& M, int mode,
                                      int nrhs, cudaStream_t s);
// Elastic block A (3 -> 3).
template <typename T> void apply_uu(const ApplyArgs<T>& a, const FixedMat<T, 4>& M, int mode,
                                    int nrhs, cudaStream_t s);
// Coupling block B (u -> phi rows of the symmetric form), LINEAR only.
template <typename T> void apply_pu(const ApplyArgs<T>& a, const FixedMat<T, 4>& M, int nrhs,
                                    cudaStream_t s);
// Local-Schur operator Sbar = sum rho_e S0 (1 -> 1).
template <typename T> void apply_ss(const ApplyArgs<T>& a, const FixedMat<T, 1>& M, int mode,
                                    int nrhs, cudaStream_t s);
// Per-element-matrix operator on a coarse level (NC = 1 or 3).
template <typename T, int NC> void apply_elem(const ApplyArgs<T>& a, int mode, int nrhs,
                                              cudaStream_t s);
// Assembled-stencil operator on a coarse level (NC = 1 or 3), a.st set; rg =
// loads per thread (1, 3 or 9; 0 = size heuristic), bitwise-neutral.
template <typename T, int NC> void apply_stencil(const ApplyArgs<T>& a, int mode, int nrhs,
                                                 cudaStream_t s, int rg = 0);
// Fastest rg for apply_stencil on this level (timed on a's buffers); 0 = default.
template <typename T, int NC> int stencil_autotune(const ApplyArgs<T>& a, int mode, int nrhs,
                                                   cudaStream_t s, float* best_us);
// Assemble the 27-point block stencil of a level from its element matrices.
template <typename T, int NC> void stencil_from_elem(const T* ke, T* st, int nx, int ny, int nz,
                                                     cudaStream_t s);

// FP64-grade residual r = b - Ahat x (r = Ahat x if b is null) in FP32 double-float arithmetic: x is
// given as FP32 pairs (x = xh + xl), K0 and rho likewise; products are
// error-free (FMA), sums use TwoSum.  kh/kl: high/low FP32 parts of K0 as row
// pairs, entry [(la * 2 + rp) * 32 + col] = (K0[4 la + 2 rp][col], K0[4 la + 2 rp + 1][col]).
struct DFMat {
  float2 kh[512];
  float2 kl[512];
};
void resid_df(const float* xh, const float* xl, i64 xs, const double* b, i64 bs, double* r, i64 rs,
              const float* rho_h, const float* rho_l, const DFMat& M, int nx, int ny, int nz,
              int nrhs, const int* active, cudaStream_t s);
// xh = fp32(x), xl = fp32(x - xh) for n values
void split_f64(const double* x, float* xh, float* xl, i64 n, cudaStream_t s);
// x64 += sc[q] * d; xh = fp32(x64), xl = fp32(x64 - xh)
template <typename T> void axpy_split(double* x, float* xh, float* xl, i64 xs, const T* d, i64 ds,
                                      i64 len, const double* sc, int nrhs, const int* active,
                                      cudaStream_t s);

// Tensor-core (tcgen05, 3xTF32) full-operator apply (apply_tc.cu); the grid
// must satisfy tc_shape_ok.  err counts bounded-wait expiries.  The tables
// (element matrix in the operand layout, hi and lo TF32 parts; gather
// indices) are built on the host once per material and grid.
struct TcTables {
  const float* b_full = nullptr;
  const unsigned short* g_full = nullptr;
};
bool tc_shape_ok(int nx, int ny, int nz);
void tc_prepare();
size_t tc_table_floats();
size_t tc_table_idx();
void tc_build_tables_host(const double* K0, float* b_full, unsigned short* g_full);
void apply_tc_full(const ApplyArgs<float>& a, const TcTables& T, int nrhs, int* err, cudaStream_t s);

// Tensor-core fine-level smoother applies, node-centric (apply_nc.cu,
// tcgen05 kind::tf32): NK_UU = elastic block A (3 -> 3) of one load per CTA,
// NK_SS4 = local-Schur operator on four loads per CTA.  B tables
// (nc_table_floats() floats per kind) come from nc_build_b; nc_prepare() once
// per device before launches or capture.  err counts expired bounded waits.
enum { NK_UU = 0, NK_SS4 = 1 };
bool nc_shape_ok(int nx, int ny, int nz);
void nc_prepare();
size_t nc_table_floats();
void nc_build_b(int kind, const double* K0, const double* S0, float* out);
// CTA tile: xt nodes along x (8, 16 or 32) by 16 rows, L z-planes per chunk;
// 0 = the default (widest tile, wave-count heuristic for L).
struct NcTile {
  int xt, L;
};
// Returns false (nothing launched) if the grid would exceed the launch limits.
bool apply_nc(int kind, const ApplyArgs<float>& a, const float* Btab, int mode, int nrhs, int* err,
              cudaStream_t s, NcTile tile);
// Times the tile candidates in the given mode on the caller's buffers (which
// it overwrites like that mode does) and returns the fastest; synchronises s.
// *best_us (if non-null) = its time per launch in microseconds.
NcTile nc_autotune(int kind, const ApplyArgs<float>& a, const float* Btab, int mode, int nrhs, int* err,
                   cudaStream_t s, float* best_us);

// ---- multigrid helpers (mg.cu) ----------------------------------------------
// r = b, d = c2 Dinv b with c2 read from device memory (*c2p)
template <typename T, int NC> void cheb_init(const T* b, i64 bs, T* r, i64 rs, T* d, i64 ds,
                                             const T* dinv, const T* c2p, i64 nn, int nrhs,
                                             const int* active, cudaStream_t s);
template <typename T, int NC> void axpy_view(T* x, i64 xs, const T* d, i64 ds, i64 nn, int nrhs,
                                             const int* active, cudaStream_t s);
template <typename T, int NC> void restrict_fw(const T* rf, i64 rs, T* bc, i64 bs, int nx, int ny,
                                               int nz, int nrhs, const int* active, cudaStream_t s);
// restrict_fw that also starts the coarse level's Chebyshev smoothing:
// bc = R rf, rc = bc, dc = (*c2p) Dinv bc (all with load stride cs)
template <typename T, int NC> void restrict_init(const T* rf, i64 rs, T* bc, T* rc, T* dc, i64 cs,
                                                 const T* dinv, const T* c2p, int nx, int ny, int nz,
                                                 int nrhs, const int* active, cudaStream_t s);
// level-1 coarse element matrices sum_c rho_c G_c (G: 8 child matrices, entry-major)
template <typename T, int NC> void galerkin_child(const T* G, const T* rho, T* kec, int ncx, int ncy,
                                                  int ncz, cudaStream_t s);
template <typename T, int NC> void prolong_add(const T* xc, i64 cs, T* xf, i64 fs, int nx, int ny,
                                               int nz, int nrhs, const int* active, cudaStream_t s,
                                               const T* dc = nullptr);
// Galerkin coarse element matrices.  Fine level given either as fixed matrix
// (device pointer to (8NC)^2 values) times rho, or as per-element SoA matrices.
template <typename T, int NC> void galerkin(const T* fixedm, const T* rho, const T* kef, T* kec,
                                            int ncx, int ncy, int ncz, cudaStream_t s);
template <typename T, int NC> void diag_inv(const T* fixedm, const T* rho, const T* ke, T* dinv,
                                            int nx, int ny, int nz, cudaStream_t s);
// max over elements of lambda_max(diag(K_e)^-1 K_e) (power iteration), as the
// float bits of a positive float in *out (atomicMax; *out must start at 0).
template <typename T, int NC> void elem_lmax(const T* ke, i64 ne, unsigned int* out, cudaStream_t s);
template <typename T> void dense_solve(const T* Ainv, int n, const T* b, i64 bs, T* x, i64 xs,
                                       i64 nn, int nc, int nrhs, const int* active, cudaStream_t s);

// ---- Krylov helpers (krylov.cu) ---------------------------------------------
// partial[(q*nblk + blk)*nvmax + i] = block-partial of <V_i, w> for rhs q.
template <typename T> void multidot(const T* V, i64 vstride, i64 rstride, int nv, const T* w,
                                    i64 wstride, i64 len, double* partial, int nblk, int nvmax,
                                    int nrhs, const int* active, cudaStream_t s);
// out[q*nvmax + i] (+)= sum over blocks of partial
void reduce_partials(const double* partial, int nblk, int nv, int nvmax, double* out, int accumulate,
                     int nrhs, const int* active, cudaStream_t s);
// w -= sum_i h[q*nvmax+i] V_i ; then (mode 1) partial dots <V_i,w> or (mode 2) partial |w|^2
template <typename T> void update(const T* V, i64 vstride, i64 rstride, int nv, const double* h,
                                  int nvmax, T* w, i64 wstride, i64 len, int mode, double* partial,
                                  int nblk, int nrhs, const int* active, cudaStream_t s);
// w -= sum_i h[q*nvmax+i] V_i fused with the next pass's partial dots <V_i, w>
// (partial[..*nvmax + i], i < nv) and |w|^2 (partial[..*nvmax + nv]); nv <= 63
template <typename T> void update_dots(const T* V, i64 vstride, i64 rstride, int nv, const double* h,
                                       int nvmax, T* w, i64 wstride, i64 len, double* partial,
                                       int nblk, int nrhs, const int* active, cudaStream_t s);
template <typename T> void scale_vec(T* w, i64 wstride, i64 len, const double* sc, int nrhs,
                                     cudaStream_t s);
template <typename T> void lincomb(const T* V, i64 vstride, i64 rstride, const double* y,
                                   const int* kcount, int nvmax, T* u, i64 ustride, i64 len,
                                   int nrhs, const int* active, cudaStream_t s);
void givens_step(double* H, double* cs, double* sn, double* g, const double* hcol,
                 const double* hnorm2, int j, int m, int* active, double* resid, const double* tolabs,
                 double* invscale, int* kcount, int nrhs, cudaStream_t s);
void backsolve(const double* H, const double* g, const int* kcount, int m, double* y, int nrhs,
               const int* mask, cudaStream_t s);
// reorth[q] = active[q] && |w_new|^2 < |w_old|^2 / 2 (|w_old|^2 in hcol[q][j+1])
void reorth_flag(const double* hcol, const double* hnorm2, int j, const int* active, int* reorth,
                 int nrhs, cudaStream_t s);
void start_cycle(const double* beta2, double* g, int m, int* active, const int* want, double* resid,
                 double* invscale, const double* tolabs, int* kcount, int nrhs, cudaStream_t s);
// v32[q] = (float)(r64[q] * sc[q])   or  x64[q] += sc[q] * d32[q]
void to_f32_scaled(const double* r, i64 rs, float* v, i64 vs, i64 len, const double* sc, int nrhs,
                   const int* active, cudaStream_t s);
template <typename T> void axpy_f64(double* x, i64 xs, const T* d, i64 ds, i64 len, const double* sc,
                                    int nrhs, const int* active, cudaStream_t s);
template <typename T> void fill(T* p, i64 n, T v, cudaStream_t s);

// ---- device-side control of a whole-solve graph (solvectl.cu) ---------------------
struct CtlParams {
  double tol;      // outer relative tolerance
  double inner;    // inner relative reduction of each cycle
  int mask;        // load mask
  int max_refine;  // refinement cap
  int max_iter;    // iteration cap per load
};
struct IterHandles {
  cudaGraphConditionalHandle h[kNvMax];   // IF condition of Arnoldi step j
  int m;
};
// ctl[0] = refinements started, ctl[1] = status, ctl[2] = Arnoldi steps executed
void refine_ctl(const double* bn2, const double* rn2, const double* bfloor, const CtlParams& P, int* want,
                double* tolabs, double* relres, const int* iters, int* ctl, cudaGraphConditionalHandle cond,
                cudaStream_t s);
void cycle_handles(const int* active, int* ran, const IterHandles& H, cudaStream_t s);
void next_step(const int* active, cudaGraphConditionalHandle next, cudaStream_t s);
void accum_iters(int* iters, const int* kcount, const int* ran, int* ctl, cudaStream_t s);
void ctl_reset(int* ctl, int* iters, cudaStream_t s);
// v[q] = r[q] * sc[q] (FP64, nrhs vectors of len values)
void copy_scale_f64(const double* r, double* v, i64 len, const double* sc, int nrhs, const int* active,
                    cudaStream_t s);

// ---- shape velocity (hilbert.cu) ----------------------------------------------
// Riesz representers in periodic H^1 (A = alpha^2 K + M, Chebyshev iteration
// with exact spectral bounds), projection of the objective representer off
// the constraint representers and the constraint correction; v (nn doubles).
// work: 4 (1 + ncons) nn doubles; dptrs_dev: device room for 1 + ncons
// pointers; partial / red as for reduce_partials; info (host, optional):
// ||P g_J||_H, Chebyshev iterations, mu_1..mu_ncons.
constexpr int kHilbertMaxCons = 8;
int hilbert_velocity(int nx, int ny, int nz, double alpha, const double* dJ, const double* const* dC,
                     const double* C, int ncons, double wJ, double wC, double* v, double* work,
                     const double** dptrs_dev, double* partial, int nblk, double* red, double* info,
                     cudaStream_t s);

// ---- cell-level kernels (cellk.cu) -------------------------------------------
// g_e = sum_IJ G_IJ (W1^I.K0 W1^J - W2^I.K0 W2^J) for two solution sets y1, y2
// of one grid and material (W = Zbar + y), as B(W1 + W2, W1 - W2); xwork holds
// 2 x 9 x 4 x nn doubles.
void energy_difference(const double* y1, const double* y2, const SensQ& Q, const SensPair& P, double* xwork,
                       double* g, int nx, int ny, int nz, cudaStream_t s);
template <typename Tin> void ersatz(const Tin* phi, int nx, int ny, int nz, double rho_void,
                                    double eta, float* rho32, double* rho64, double* drho,
                                    cudaStream_t s);
// out = phi - dt v |grad phi| (first-order Godunov upwind, periodic grid)
template <typename T> void hj_step(const T* phi, const T* v, int nx, int ny, int nz, double dt, T* out,
                                   cudaStream_t s);
// gn[node] = sum over the 8 elements around the node of ge[e] drho[e] / 8
template <typename T> void chain_phi(const double* ge, const double* drho, int nx, int ny, int nz, T* gn,
                                     cudaStream_t s);
template <typename Tin> void rho_copy(const Tin* in, i64 n, float* rho32, double* rho64,
                                      int* bad, cudaStream_t s);
void rhs9(const double* rho, const RhsParams& F, int mask, double* b, int nx, int ny, int nz,
          cudaStream_t s);
// per-(rhs, comp) sums -> out[q*4 + c]
void comp_sums(const double* x, i64 nn, int nrhs, double* partial, int nblk, double* out,
               cudaStream_t s);
void sub_means(double* x, i64 nn, int nrhs, const double* sums, cudaStream_t s);
// G_IJ (+)= sum_n sum_c sgn_c u^I_c v^J_c, sgn = -1 for the potential component
void gram9(const double* u, const double* v, i64 nn, double* partial, int nblk, double* out,
           cudaStream_t s);
// out[0] = sum of x[0..n) (or of the squares)  (device scalar)
void sum_reduce(const double* x, i64 n, double* partial, int nblk, double* out, cudaStream_t s,
                int squares = 0);
// g_e = (rho_e if times_rho) * sum_IJ G_IJ W_e^I . K0 W_e^J, W = Zbar + y_e,
// evaluated as sum_m lam_m X^m.K0 X^m; xwork holds Q.R x 8 x nn floats (T =
// float: FP32 pairs of the mode fields) or Q.R x 4 x nn doubles.
template <typename T> void sensitivity(const double* y, const double* rho, const SensQ& Q,
                                       const SensModes<T>& P, T* xwork, T* g, int nx, int ny,
                                       int nz, int times_rho, cudaStream_t s);

}  // namespace cell
