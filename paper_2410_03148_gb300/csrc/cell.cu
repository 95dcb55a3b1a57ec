// Solver orchestration and the C ABI (include/cell.h).
//
// Hot path per design: S1 set-up (material scaling, K0, S0, rho_e, multigrid
// hierarchies), S2 right-hand sides, S3-S6 FP64-restarted SCP-GMRES (inner
// Krylov cycles in FP32 or FP64), S7 null-space projection, S8 homogenised
// tensors, S9 element sensitivities.  Everything runs on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cell.h"
#include "hostmath.h"
#include "kernels.cuh"

using cell::i64;
using cell::kNvMax;

std::atomic<long long> cell::g_launches{0};

namespace {

thread_local std::string g_last_error;

void set_error(const char* what, cudaError_t e = cudaSuccess) {
  g_last_error = what;
  if (e != cudaSuccess) {
    g_last_error += ": ";
    g_last_error += cudaGetErrorString(e);
  }
}

}  // namespace

namespace cell {
void report_error(const char* what, cudaError_t e) { set_error(what, e); }
}  // namespace cell

namespace {

#define CK(call)                                     \
  do {                                               \
    cudaError_t _e = (call);                         \
    if (_e != cudaSuccess) {                         \
      set_error(#call, _e);                          \
      return _e == cudaErrorMemoryAllocation ? CELL_ENOMEM : CELL_ECUDA; \
    }                                                \
  } while (0)

#define CKS(call)                     \
  do {                                \
    int _s = (call);                  \
    if (_s != CELL_OK) return _s;     \
  } while (0)

// Owned device allocations of a handle.
struct Arena {
  std::vector<void*> ptrs;
  template <typename T>
  int alloc(T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
      set_error("cudaMalloc", e);
      return e == cudaErrorMemoryAllocation ? CELL_ENOMEM : CELL_ECUDA;
    }
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return CELL_OK;
  }
  void release() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

// Optional CUDA-event timing of kernel classes.  Outside graph capture the
// events come from a recycled pool; while a GMRES iteration is being captured
// into a CUDA graph, begin/end create events owned by that graph, which become
// event-record nodes and are read after every replay of the graph.
struct GraphMark {
  int cls;
  cudaEvent_t e0, e1;
};

struct Prof {
  bool on = false;
  unsigned mask = ~0u;  // kernel classes to time
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, int>> marks[CELL_PROF_CLASSES];  // (start, stop) per class
  long long units[CELL_PROF_CLASSES] = {0};
  double acc_ms[CELL_PROF_CLASSES] = {0};
  int acc_cnt[CELL_PROF_CLASSES] = {0};
  int cur_units = 9;   // loads processed by the launches being timed
  size_t used = 0;
  std::vector<GraphMark>* cap = nullptr;  // capture target (graph-owned events)
  cudaEvent_t get() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  int begin(cudaStream_t s, int cls) {
    if (!on || !((mask >> cls) & 1u)) return -1;
    if (cap) {
      // external records become event-record nodes that timestamp each replay
      GraphMark m{-1, nullptr, nullptr};
      cudaEventCreate(&m.e0);
      cudaEventRecordWithFlags(m.e0, s, cudaEventRecordExternal);
      cap->push_back(m);
      return (int)cap->size() - 1;
    }
    const int i = (int)used;
    cudaEventRecord(get(), s);
    return i;
  }
  void end(int cls, int i0, cudaStream_t s) {
    if (!on || i0 < 0) return;
    if (cap) {
      GraphMark& m = (*cap)[i0];
      m.cls = cls;
      cudaEventCreate(&m.e1);
      cudaEventRecordWithFlags(m.e1, s, cudaEventRecordExternal);
      return;
    }
    const int i1 = (int)used;
    cudaEventRecord(get(), s);
    marks[cls].push_back({i0, i1});
    units[cls] += cur_units;
  }
  // after a replay of a graph has completed
  void add_graph(const std::vector<GraphMark>& gm, int nunits) {
    for (const GraphMark& m : gm) {
      if (m.cls < 0) continue;
      float f = 0.f;
      if (cudaEventElapsedTime(&f, m.e0, m.e1) != cudaSuccess) {
        cudaGetLastError();  // timing is best effort; never fail a solve on it
        continue;
      }
      acc_ms[m.cls] += f;
      acc_cnt[m.cls] += 1;
      units[m.cls] += nunits;
    }
  }
  void collect(double* ms, int* cnt, long long* un) {
    for (int c = 0; c < CELL_PROF_CLASSES; ++c) {
      double t = acc_ms[c];
      for (auto& m : marks[c]) {
        float f = 0.f;
        if (cudaEventElapsedTime(&f, pool[m.first], pool[m.second]) != cudaSuccess) cudaGetLastError();
        t += f;
      }
      ms[c] = t;
      cnt[c] = (int)marks[c].size() + acc_cnt[c];
      un[c] = units[c];
      units[c] = 0;
      acc_ms[c] = 0;
      acc_cnt[c] = 0;
      marks[c].clear();
    }
    used = 0;
  }
  ~Prof() {
    for (auto e : pool) cudaEventDestroy(e);
  }
};

// One captured GMRES iteration (for a fixed Arnoldi index j).
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  std::vector<GraphMark> marks;
  long long nkernels = 0;  // kernels per replay (for cell_launch_count)
};

template <typename T>
struct Level {
  int nx = 0, ny = 0, nz = 0;
  i64 nn = 0;
  T* ke = nullptr;       // per-element Galerkin matrices (levels >= 1), SoA
  T* st = nullptr;       // assembled 27-point block stencil (levels >= 1), SoA
  T* dinv = nullptr;     // [NC][nn]
  double lmax = 1.0;
  T *b = nullptr, *x = nullptr, *r = nullptr, *d = nullptr, *d2 = nullptr;  // [9][NC][nn]
  T* cc = nullptr;       // Chebyshev coefficients on the device: (0, 1/theta), (c1_k, c2_k)
  int deg = 0;           // Chebyshev steps of this level
  int rg = 0;            // loads per thread of the stencil apply (0 = default; tuned at set-up)
  T* dense = nullptr;    // coarsest: regularised inverse (n x n, symmetric)
  int ndense = 0;
  bool coarsest = false;
};

template <typename T>
struct BlockMG {
  int nc = 0;
  std::vector<Level<T>> lv;
  T* fixedm = nullptr;   // device copy of the level-0 element block ((8nc)^2)
  T* childm = nullptr;   // the 8 child matrices P_c^T K P_c of level 1 (8 (8nc)^2)
  std::vector<double> fixed_host;
  std::vector<T> dense_host;   // staging of the coarsest inverse (kept alive for the async copy)
  std::vector<T> cc_host;      // staging of the Chebyshev coefficients of all levels
  T* cc_dev = nullptr;
  unsigned int* lbits = nullptr;  // per-level lambda_max bounds (float bits)
};

template <typename T>
struct Krylov {
  int m = 0;
  i64 len = 0;
  T* V = nullptr;        // (m+1) x 9 x len
  T* Z = nullptr;        // m x 9 x len: preconditioned directions z_j = P^-1 v_j (flexible GMRES)
  T* u = nullptr;        // 9 x len
  T* tphi = nullptr;     // 9 x nn (Schur block right-hand side)
  T* ru = nullptr;       // 9 x 3nn (extra elastic V-cycles)
  T* eu = nullptr;
  T* rp = nullptr;       // 9 x nn (extra Schur V-cycles)
  T* ep = nullptr;
  cell::FixedMat<T, 4> K0;
  cell::FixedMat<T, 1> S0;
  const T* rho = nullptr;
  BlockMG<T> mgu, mgp;
};

}  // namespace

struct cell_handle {
  cell_desc d{};
  int dev = 0;             // CUDA device current at set-up
  int nx = 0, ny = 0, nz = 0;
  i64 nn = 0;
  cudaStream_t st = nullptr;
  double C0 = 1, k0 = 1;
  double Cn[36], en[18], kn[9];
  double h[3];
  double K0[1024], S0[64], Z[288], F[288], H0e[81];
  Arena arena;
  float* rho32 = nullptr;
  double* rho64 = nullptr;
  double* drho = nullptr;   // level-set input: d rho_e / d phi_e (§2.6 smoothing)
  double* gtmp = nullptr;   // level-set input: element sensitivities before the chain
  double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr;
  // mixed path: x64 as FP32 pairs and rho's low part, for the double-float residual
  float *xh = nullptr, *xl = nullptr, *rho_l = nullptr, *rho_tmp = nullptr;
  int* bad = nullptr;
  const double** dptrs = nullptr;   // device pointer table of cell_hilbert_velocity
  int* tc_err = nullptr;   // tensor-core kernels: expired bounded waits
  bool tc_ok = false;      // grid tiles into tensor-core bricks
  bool nc_ok = false;      // grid suits the node-centric tensor-core smoothers
  float* ncb = nullptr;    // their B operands: [NK_UU | NK_SS4][nc_table_floats()]
  cell::NcTile nct[2] = {{0, 0}, {0, 0}};   // their CTA tiles (autotuned at set-up)
  float nct_us[2] = {0.f, 0.f};
  cell::TcTables tct;      // tensor-core operand tables (device)
  int cslot1 = 0;          // constant-bank slot of the FP32 element matrices (+1)
  cell::DFMat DF;
  double *partial = nullptr, *red = nullptr, *red2 = nullptr;
  int nblk = 0;
  // per-load magnitude of the element contributions, sqrt(sum rho_e^2) |K0 Zbar^I|:
  // right-hand sides or residuals below 1e-13 of it are rounding noise
  double bfloor[9];
  // Krylov-scalar state (FP64, device)
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *hcol = nullptr, *hnorm = nullptr;
  double *resid = nullptr, *invscale = nullptr, *tolabs = nullptr, *ybuf = nullptr, *beta2 = nullptr;
  double* ones = nullptr;
  int *active = nullptr, *kcount = nullptr, *want = nullptr, *ranmask = nullptr, *reorth = nullptr;
  Krylov<float> kf;
  Krylov<double> kd;
  bool solved = false;
  Prof prof;
  cell_stats last{};
  // CUDA graphs of the GMRES iterations (one per Arnoldi index), captured on
  // an internal stream at first use and replayed on the caller's stream
  std::vector<IterGraph> graphs;
  cudaStream_t cap_st = nullptr;
  // whole-solve graph (options.graphs >= 2): device-side control state and
  // the kernels per captured segment (for cell_launch_count)
  cudaGraphExec_t solve_exec = nullptr;
  int solve_prec = -1;
  long long seg_pro = 0, seg_cb = 0, seg_it = 0, seg_ce = 0, seg_epi = 0;
  double *bn2d = nullptr, *relres_d = nullptr, *bfloor_d = nullptr;
  int *ctl_d = nullptr, *iters_d = nullptr;
  struct GraphStats {
    int ctl[4];
    int iters[9];
    int tcerr;
    double relres[9];
  };
  GraphStats* gstat = nullptr;   // pinned host copy of the solve statistics
  std::chrono::steady_clock::time_point gt0;
  void free_graphs() {
    if (solve_exec) cudaGraphExecDestroy(solve_exec);
    solve_exec = nullptr;
    for (IterGraph& g : graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (GraphMark& m : g.marks) {
        if (m.e0) cudaEventDestroy(m.e0);
        if (m.e1) cudaEventDestroy(m.e1);
      }
    }
    graphs.clear();
    if (cap_st) cudaStreamDestroy(cap_st);
    cap_st = nullptr;
  }
};

namespace {

template <typename T> Krylov<T>& kry(cell_handle* h);
template <> Krylov<float>& kry<float>(cell_handle* h) { return h->kf; }

int tune_tiles(cell_handle* h);
template <typename T, int NC> void tune_stencils(cell_handle* h, BlockMG<T>& mg);
void tile_stats(const cell_handle* h, cell_stats& S);
template <> Krylov<double>& kry<double>(cell_handle* h) { return h->kd; }

template <typename T> const T* rho_of(cell_handle* h);
template <> const float* rho_of<float>(cell_handle* h) { return h->rho32; }
template <> const double* rho_of<double>(cell_handle* h) { return h->rho64; }

// ---------------------------------------------------------------------------
// multigrid hierarchy
// ---------------------------------------------------------------------------

template <typename T, int NC>
void level_apply(cell_handle* h, BlockMG<T>& mg, int l, int mode, const cell::ApplyArgs<T>& a0,
                 const int* mask) {
  cell::ApplyArgs<T> a = a0;
  Level<T>& L = mg.lv[l];
  a.nx = L.nx;
  a.ny = L.ny;
  a.nz = L.nz;
  a.dinv = L.dinv;
  a.active = mask;
  a.cslot1 = h->cslot1;
  Krylov<T>& K = kry<T>(h);
  const int pcls = l > 0 ? CELL_PROF_COARSE : (NC == 3 ? CELL_PROF_ELASTIC0 : CELL_PROF_SCHUR0);
  const int ip = h->prof.begin(h->st, pcls);
  if (l == 0) {
    a.rho = K.rho;
    if constexpr (sizeof(T) == 4) {
      const int kind = NC == 3 ? cell::NK_UU : cell::NK_SS4;
      if (h->nc_ok && h->d.opt.tensor_cores >= 1 &&
          cell::apply_nc(kind, a, h->ncb + cell::nc_table_floats() * kind, mode, 9, h->tc_err, h->st,
                         h->nct[kind])) {
      } else if constexpr (NC == 3) {
        cell::apply_uu<T>(a, K.K0, mode, 9, h->st);
      } else {
        cell::apply_ss<T>(a, K.S0, mode, 9, h->st);
      }
    } else if constexpr (NC == 3) {
      cell::apply_uu<T>(a, K.K0, mode, 9, h->st);
    } else {
      cell::apply_ss<T>(a, K.S0, mode, 9, h->st);
    }
  } else {
    a.st = L.st;
    cell::apply_stencil<T, NC>(a, mode, 9, h->st, L.rg);
  }
  h->prof.end(pcls, ip, h->st);
}

// Dense assembly of a level's operator on the host (coarsest level only).
template <typename T, int NC>
int assemble_dense(cell_handle* h, BlockMG<T>& mg, int l, std::vector<double>& A) {
  Level<T>& L = mg.lv[l];
  const int R = 8 * NC;
  const i64 nn = L.nn;
  const int n = (int)(NC * nn);
  A.assign((size_t)n * n, 0.0);
  std::vector<T> ke;
  std::vector<double> rho;
  if (l == 0) {
    rho.resize(nn);
    CK(cudaMemcpyAsync(rho.data(), h->rho64, nn * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  } else {
    ke.resize((size_t)R * R * nn);
    CK(cudaMemcpyAsync(ke.data(), L.ke, ke.size() * sizeof(T), cudaMemcpyDeviceToHost, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  for (i64 e = 0; e < nn; ++e) {
    const int i = (int)(e % L.nx), j = (int)((e / L.nx) % L.ny), k = (int)(e / ((i64)L.nx * L.ny));
    i64 node[8];
    for (int a = 0; a < 8; ++a)
      node[a] = (i + (a & 1)) % L.nx + (i64)L.nx * (((j + ((a >> 1) & 1)) % L.ny) + (i64)L.ny * ((k + (a >> 2)) % L.nz));
    for (int a = 0; a < 8; ++a)
      for (int c = 0; c < NC; ++c)
        for (int b = 0; b < 8; ++b)
          for (int dd = 0; dd < NC; ++dd) {
            const int entry = (a * NC + c) * R + b * NC + dd;
            const double v = l == 0 ? rho[e] * mg.fixed_host[entry] : (double)ke[(size_t)entry * nn + e];
            A[(size_t)(c * nn + node[a]) * n + dd * nn + node[b]] += v;
          }
  }
  return CELL_OK;
}

// Structure and allocations of a block's multigrid hierarchy (once per handle).
template <typename T, int NC>
int alloc_mg(cell_handle* h, BlockMG<T>& mg, const double* fixed_block) {
  const cell_options& o = h->d.opt;
  const int R = 8 * NC;
  mg.nc = NC;
  mg.fixed_host.assign(fixed_block, fixed_block + R * R);
  std::vector<T> fb(R * R);
  for (int i = 0; i < R * R; ++i) fb[i] = (T)fixed_block[i];
  CKS(h->arena.alloc(&mg.fixedm, R * R));
  CK(cudaMemcpyAsync(mg.fixedm, fb.data(), R * R * sizeof(T), cudaMemcpyHostToDevice, h->st));
  // G_c[(A, d), (B, e)] = sum_{a, b} w(c, a, A) w(c, b, B) K[(a, d), (b, e)]
  {
    std::vector<T> G((size_t)8 * R * R);
    for (int c = 0; c < 8; ++c)
      for (int A = 0; A < 8; ++A)
        for (int B = 0; B < 8; ++B)
          for (int d = 0; d < NC; ++d)
            for (int e = 0; e < NC; ++e) {
              double v = 0.0;
              for (int a = 0; a < 8; ++a) {
                const double wa = cellhost::child_weight(c, a, A);
                if (wa == 0.0) continue;
                for (int b = 0; b < 8; ++b) {
                  const double wb = cellhost::child_weight(c, b, B);
                  if (wb != 0.0) v += wa * wb * fixed_block[(a * NC + d) * R + b * NC + e];
                }
              }
              G[(size_t)c * R * R + (A * NC + d) * R + B * NC + e] = (T)v;
            }
    CKS(h->arena.alloc(&mg.childm, (size_t)8 * R * R));
    CK(cudaMemcpy(mg.childm, G.data(), G.size() * sizeof(T), cudaMemcpyHostToDevice));
  }
  mg.lv.clear();
  Level<T> L0;
  L0.nx = h->nx;
  L0.ny = h->ny;
  L0.nz = h->nz;
  L0.nn = h->nn;
  L0.lmax = cellhost::jacobi_lmax(fixed_block, R);
  mg.lv.push_back(L0);
  // coarsen while every size is even, the coarse grid keeps >= 2 nodes per
  // direction, and the level is still larger than the dense coarse target
  while (true) {
    Level<T>& P = mg.lv.back();
    const bool even = (P.nx % 2 == 0) && (P.ny % 2 == 0) && (P.nz % 2 == 0);
    const bool big = P.nn * NC > (i64)o.coarse_dofs;
    if (!(even && big && P.nx >= 4 && P.ny >= 4 && P.nz >= 4)) break;
    Level<T> C;
    C.nx = P.nx / 2;
    C.ny = P.ny / 2;
    C.nz = P.nz / 2;
    C.nn = (i64)C.nx * C.ny * C.nz;
    mg.lv.push_back(C);
  }
  const int nl = (int)mg.lv.size();
  CKS(h->arena.alloc(&mg.lbits, nl));
  for (int l = 0; l < nl; ++l) {
    Level<T>& L = mg.lv[l];
    CKS(h->arena.alloc(&L.dinv, NC * L.nn));
    if (l > 0) {
      CKS(h->arena.alloc(&L.ke, (size_t)R * R * L.nn));
      CKS(h->arena.alloc(&L.st, (size_t)27 * NC * NC * L.nn));
    }
    const size_t wn = (size_t)9 * NC * L.nn;
    if (l > 0) {
      CKS(h->arena.alloc(&L.b, wn));
      CKS(h->arena.alloc(&L.x, wn));
    }
    CKS(h->arena.alloc(&L.r, wn));
    CKS(h->arena.alloc(&L.d, wn));
    CKS(h->arena.alloc(&L.d2, wn));
  }
  Level<T>& Lc = mg.lv.back();
  Lc.coarsest = true;
  const i64 n = NC * Lc.nn;
  if (n <= 3000) {
    CKS(h->arena.alloc(&Lc.dense, (size_t)n * n));
    Lc.ndense = (int)n;
  }
  // Chebyshev coefficients: 2 (deg + 1) values per level, on the device so
  // that captured graphs stay valid when a new design changes them
  const int degc = std::max(8, 4 * o.cheb_degree);
  const int stride = 2 * (degc + 1);
  CKS(h->arena.alloc(&mg.cc_dev, (size_t)stride * nl));
  mg.cc_host.assign((size_t)stride * nl, T(0));
  for (int l = 0; l < nl; ++l) {
    Level<T>& L = mg.lv[l];
    L.cc = mg.cc_dev + (size_t)stride * l;
    L.deg = (L.coarsest && !L.dense) ? degc : o.cheb_degree;
  }
  return CELL_OK;
}

// Numerics of the hierarchy for the handle's current rho (every design):
// Galerkin coarse element matrices, stencils, Jacobi diagonals, Chebyshev
// bounds and the coarsest regularised inverse.
template <typename T, int NC>
int fill_mg(cell_handle* h, BlockMG<T>& mg) {
  const int nl = (int)mg.lv.size();
  CK(cudaMemsetAsync(mg.lbits, 0, nl * sizeof(unsigned), h->st));
  for (int l = 0; l < nl; ++l) {
    Level<T>& L = mg.lv[l];
    if (l > 0) {
      Level<T>& F = mg.lv[l - 1];
      if (l == 1) cell::galerkin_child<T, NC>(mg.childm, rho_of<T>(h), L.ke, L.nx, L.ny, L.nz, h->st);
      else cell::galerkin<T, NC>(nullptr, nullptr, F.ke, L.ke, L.nx, L.ny, L.nz, h->st);
      cell::diag_inv<T, NC>(nullptr, nullptr, L.ke, L.dinv, L.nx, L.ny, L.nz, h->st);
      cell::stencil_from_elem<T, NC>(L.ke, L.st, L.nx, L.ny, L.nz, h->st);
      cell::elem_lmax<T, NC>(L.ke, L.nn, mg.lbits + l, h->st);
    } else {
      cell::diag_inv<T, NC>(mg.fixedm, rho_of<T>(h), nullptr, L.dinv, L.nx, L.ny, L.nz, h->st);
    }
  }
  std::vector<unsigned> bits(nl, 0u);
  CK(cudaMemcpyAsync(bits.data(), mg.lbits, nl * sizeof(unsigned), cudaMemcpyDeviceToHost, h->st));
  Level<T>& Lc = mg.lv.back();
  if (Lc.dense) {
    const i64 n = Lc.ndense;
    std::vector<double> A;
    CKS((assemble_dense<T, NC>(h, mg, nl - 1, A)));  // synchronises the stream
    // regularise the null space (componentwise constants) and invert
    double tr = 0.0;
    for (i64 i = 0; i < n; ++i) tr += A[(size_t)i * n + i];
    const double alpha = tr / (double)n;
    for (int c = 0; c < NC; ++c)
      for (i64 p = 0; p < Lc.nn; ++p)
        for (i64 q = 0; q < Lc.nn; ++q) A[(size_t)(c * Lc.nn + p) * n + c * Lc.nn + q] += alpha / (double)Lc.nn;
    if (cellhost::spd_inverse(A.data(), (int)n) != 0) {
      set_error("coarsest multigrid level is not positive definite (rho must be > 0)");
      return CELL_EINVAL;
    }
    mg.dense_host.resize(A.size());
    for (size_t i = 0; i < A.size(); ++i) mg.dense_host[i] = (T)A[i];
    CK(cudaMemcpyAsync(Lc.dense, mg.dense_host.data(), mg.dense_host.size() * sizeof(T),
                       cudaMemcpyHostToDevice, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  for (int l = 1; l < nl; ++l) {
    float lf;
    std::memcpy(&lf, &bits[l], sizeof(float));
    mg.lv[l].lmax = lf > 0 ? (double)lf : 1.0;
  }
  const cell_options& o = h->d.opt;
  const size_t stride = mg.cc_host.size() / nl;
  for (int l = 0; l < nl; ++l) {
    const double hi = mg.lv[l].lmax * o.cheb_hi, lo = hi * o.cheb_lo;
    const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
    T* c = mg.cc_host.data() + stride * l;
    c[0] = T(0);
    c[1] = (T)(1.0 / theta);
    double rp = 1.0 / sigma;
    for (int k = 1; k < mg.lv[l].deg; ++k) {
      const double rk = 1.0 / (2.0 * sigma - rp);
      c[2 * k] = (T)(rk * rp);
      c[2 * k + 1] = (T)(2.0 * rk / delta);
      rp = rk;
    }
  }
  CK(cudaMemcpyAsync(mg.cc_dev, mg.cc_host.data(), mg.cc_host.size() * sizeof(T), cudaMemcpyHostToDevice,
                     h->st));
  return CELL_OK;
}

// x = V-cycle approximation of A_l^-1 b (zero initial guess).  Chebyshev
// coefficients are read from the level's device table (see fill_mg).
template <typename T, int NC>
void vcycle(cell_handle* h, BlockMG<T>& mg, int l, const T* b, i64 bs, T* x, i64 xs, const int* mask,
            bool started = false, const T** pending = nullptr) {
  Level<T>& L = mg.lv[l];
  const i64 ws = NC * L.nn;
  if (L.coarsest && L.dense) {
    cell::dense_solve<T>(L.dense, L.ndense, b, bs, x, xs, L.nn, NC, 9, mask, h->st);
    return;
  }
  const int deg = L.deg;
  cell::ApplyArgs<T> a{};
  // pre-smoothing from x = 0 (started: the restriction already wrote r, d)
  if (!started) cell::cheb_init<T, NC>(b, bs, L.r, ws, L.d, ws, L.dinv, L.cc + 1, L.nn, 9, mask, h->st);
  T* d = L.d;
  T* d2 = L.d2;
  int zero = 1;
  for (int k = 1; k < deg; ++k) {
    a = cell::ApplyArgs<T>{};
    a.x = d; a.xs = ws; a.y = L.r; a.ys = ws; a.sol = x; a.ss = xs; a.dout = d2; a.ds = ws;
    a.cc = L.cc + 2 * k; a.sol_zero = zero;
    level_apply<T, NC>(h, mg, l, cell::AM_CHEB, a, mask);
    std::swap(d, d2);
    zero = 0;
  }
  a = cell::ApplyArgs<T>{};
  a.x = d; a.xs = ws; a.y = L.r; a.ys = ws; a.sol = x; a.ss = xs; a.sol_zero = zero;
  level_apply<T, NC>(h, mg, l, cell::AM_CHEB_LAST, a, mask);
  if (L.coarsest) return;
  Level<T>& C = mg.lv[l + 1];
  const i64 cs = NC * C.nn;
  const T* dpend = nullptr;   // coarse level's last direction, folded into the prolongation
  if (C.coarsest && C.dense) {
    cell::restrict_fw<T, NC>(L.r, ws, C.b, cs, L.nx, L.ny, L.nz, 9, mask, h->st);
    vcycle<T, NC>(h, mg, l + 1, C.b, cs, C.x, cs, mask);
  } else {
    cell::restrict_init<T, NC>(L.r, ws, C.b, C.r, C.d, cs, C.dinv, C.cc + 1, L.nx, L.ny, L.nz, 9, mask, h->st);
    vcycle<T, NC>(h, mg, l + 1, C.b, cs, C.x, cs, mask, true, &dpend);
  }
  cell::prolong_add<T, NC>(C.x, cs, x, xs, L.nx, L.ny, L.nz, 9, mask, h->st, dpend);
  // post-smoothing
  a = cell::ApplyArgs<T>{};
  a.x = x; a.xs = xs; a.b = b; a.bs = bs; a.y = L.r; a.ys = ws; a.dout = L.d; a.ds = ws;
  a.cc = L.cc;
  level_apply<T, NC>(h, mg, l, cell::AM_RESID_CHEB0, a, mask);
  d = L.d;
  d2 = L.d2;
  for (int k = 1; k < deg; ++k) {
    a = cell::ApplyArgs<T>{};
    a.x = d; a.xs = ws; a.y = L.r; a.ys = ws; a.sol = x; a.ss = xs; a.dout = d2; a.ds = ws;
    a.cc = L.cc + 2 * k; a.sol_zero = 0;
    level_apply<T, NC>(h, mg, l, cell::AM_CHEB, a, mask);
    std::swap(d, d2);
  }
  if (pending) *pending = d;   // the caller adds it while prolongating x
  else cell::axpy_view<T, NC>(x, xs, d, ws, L.nn, 9, mask, h->st);
}

// k V-cycles by residual correction: x ~ A^-1 b.
template <typename T, int NC>
void block_solve(cell_handle* h, BlockMG<T>& mg, int cycles, const T* b, i64 bs, T* x, i64 xs,
                 T* rwork, T* ework, const int* mask) {
  vcycle<T, NC>(h, mg, 0, b, bs, x, xs, mask);
  const i64 ws = NC * h->nn;
  for (int c = 1; c < cycles; ++c) {
    cell::ApplyArgs<T> a{};
    a.x = x; a.xs = xs; a.y = rwork; a.ys = ws; a.b = b; a.bs = bs; a.alpha = T(-1); a.beta = T(1);
    level_apply<T, NC>(h, mg, 0, cell::AM_LINEAR, a, mask);
    vcycle<T, NC>(h, mg, 0, rwork, ws, ework, ws, mask);
    cell::axpy_view<T, NC>(x, xs, ework, ws, h->nn, 9, mask, h->st);
  }
}

// z = P_SCP^-1 v (§2.5.3): z_u ~ A^-1 v_u, z_phi ~ Sbar^-1 (v_phi + B z_u).
template <typename T>
void precond(cell_handle* h, const T* v, T* z, const int* mask) {
  Krylov<T>& K = kry<T>(h);
  const i64 nn = h->nn, len = K.len;
  block_solve<T, 3>(h, K.mgu, h->d.opt.vcycles_u, v, len, z, len, K.ru, K.eu, mask);
  if (h->d.opt.precond == CELL_PRECOND_DBP) {
    // P_DBP = diag(A, C) in the nonsymmetric form: z_phi ~ C^-1 v_phi
    block_solve<T, 1>(h, K.mgp, h->d.opt.vcycles_phi, v + 3 * nn, len, z + 3 * nn, len, K.rp, K.ep, mask);
    return;
  }
  cell::ApplyArgs<T> a{};
  a.x = z; a.xs = len; a.y = K.tphi; a.ys = nn; a.b = v + 3 * nn; a.bs = len;
  a.alpha = T(1); a.beta = T(1); a.rho = K.rho; a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
  a.active = mask;
  a.cslot1 = h->cslot1;
  const int ip = h->prof.begin(h->st, CELL_PROF_COUPLING);
  cell::apply_pu<T>(a, K.K0, 9, h->st);
  h->prof.end(CELL_PROF_COUPLING, ip, h->st);
  block_solve<T, 1>(h, K.mgp, h->d.opt.vcycles_phi, K.tphi, nn, z + 3 * nn, len, K.rp, K.ep, mask);
}

template <typename T>
void apply_full_T(cell_handle* h, const T* x, i64 xs, T* y, i64 ys, const T* b, i64 bs, T alpha,
                  T beta, const int* mask, int nrhs) {
  cell::ApplyArgs<T> a{};
  a.x = x; a.xs = xs; a.y = y; a.ys = ys; a.b = b; a.bs = bs; a.alpha = alpha; a.beta = beta;
  a.rho = rho_of<T>(h); a.nx = h->nx; a.ny = h->ny; a.nz = h->nz; a.active = mask;
  a.cslot1 = h->cslot1;
  const int pcls = sizeof(T) == 4 ? CELL_PROF_FULL32 : CELL_PROF_FULL64;
  const int ip = h->prof.begin(h->st, pcls);
  if constexpr (sizeof(T) == 4) {
    if (h->tc_ok && h->d.opt.tensor_cores >= 2) cell::apply_tc_full(a, h->tct, nrhs, h->tc_err, h->st);
    else cell::apply_full<T>(a, h->kf.K0, cell::AM_LINEAR, nrhs, h->st);
  } else {
    cell::apply_full<T>(a, h->kd.K0, cell::AM_LINEAR, nrhs, h->st);
  }
  h->prof.end(pcls, ip, h->st);
}

template <typename T>
int setup_krylov(cell_handle* h) {
  Krylov<T>& K = kry<T>(h);
  const cell_options& o = h->d.opt;
  K.m = o.restart;
  K.len = 4 * h->nn;
  K.rho = rho_of<T>(h);
  for (int i = 0; i < 1024; ++i) K.K0.k[i] = (T)h->K0[i];
  for (int i = 0; i < 64; ++i) K.S0.k[i] = (T)h->S0[i];
  CKS(h->arena.alloc(&K.V, (size_t)(K.m + 1) * 9 * K.len));
  CKS(h->arena.alloc(&K.Z, (size_t)K.m * 9 * K.len));
  CKS(h->arena.alloc(&K.u, (size_t)9 * K.len));
  CKS(h->arena.alloc(&K.tphi, (size_t)9 * h->nn));
  if (o.vcycles_u > 1) {
    CKS(h->arena.alloc(&K.ru, (size_t)27 * h->nn));
    CKS(h->arena.alloc(&K.eu, (size_t)27 * h->nn));
  }
  if (o.vcycles_phi > 1) {
    CKS(h->arena.alloc(&K.rp, (size_t)9 * h->nn));
    CKS(h->arena.alloc(&K.ep, (size_t)9 * h->nn));
  }
  // level-0 blocks of the preconditioner: A_e (24x24 u-block of K0), S0
  std::vector<double> Auu(576);
  for (int a = 0; a < 8; ++a)
    for (int c = 0; c < 3; ++c)
      for (int b = 0; b < 8; ++b)
        for (int d = 0; d < 3; ++d) Auu[(a * 3 + c) * 24 + b * 3 + d] = h->K0[(4 * a + c) * 32 + 4 * b + d];
  CKS((alloc_mg<T, 3>(h, K.mgu, Auu.data())));
  CKS((alloc_mg<T, 1>(h, K.mgp, h->S0)));
  return CELL_OK;
}

template <typename T>
int fill_krylov(cell_handle* h) {
  Krylov<T>& K = kry<T>(h);
  CKS((fill_mg<T, 3>(h, K.mgu)));
  CKS((fill_mg<T, 1>(h, K.mgp)));
  return CELL_OK;
}

// One Arnoldi step j of the batched GMRES (all kernels, no host sync):
// z = P^-1 v_j, w = Ahat z, Gram-Schmidt against v_0..v_j, Givens update,
// normalisation.  Launches go to h->st (the capture stream while captured).
template <typename T>
void iteration(cell_handle* h, int j) {
  Krylov<T>& K = kry<T>(h);
  const int m = K.m;
  const i64 len = K.len;
  const i64 vstride = 9 * len;
  cudaStream_t s = h->st;
  const int nblk = h->nblk;
  T* vj = K.V + (i64)j * vstride;
  T* w = K.V + (i64)(j + 1) * vstride;
  T* zj = K.Z + (i64)j * vstride;
  precond<T>(h, vj, zj, h->active);
  apply_full_T<T>(h, zj, len, w, len, nullptr, 0, T(1), T(0), h->active, 9);
  // Classical Gram-Schmidt with selective reorthogonalisation: one pass of
  // dots (w is V_{j+1}, so the same pass also gives |w|^2); one pass that
  // updates w and, from the same basis reads, forms the second pass's dots
  // and the new norm; a second update only for loads whose norm dropped
  // below 1/sqrt(2) of its value before the first (three basis passes).
  const int ipk = h->prof.begin(s, CELL_PROF_KRYLOV);
  cell::multidot<T>(K.V, vstride, len, j + 2, w, len, len, h->partial, nblk, kNvMax, 9, h->active, s);
  cell::reduce_partials(h->partial, nblk, j + 2, kNvMax, h->hcol, 0, 9, h->active, s);
  // first update fused with the second pass's dots and the new norm
  cell::update_dots<T>(K.V, vstride, len, j + 1, h->hcol, kNvMax, w, len, len, h->partial, nblk, 9, h->active, s);
  cell::reduce_partials(h->partial + (j + 1), nblk, 1, kNvMax, h->hnorm, 0, 9, h->active, s);
  cell::reorth_flag(h->hcol, h->hnorm, j, h->active, h->reorth, 9, s);
  cell::reduce_partials(h->partial, nblk, j + 1, kNvMax, h->ybuf, 0, 9, h->reorth, s);
  cell::update<T>(K.V, vstride, len, j + 1, h->ybuf, kNvMax, w, len, len, 2, h->partial, nblk, 9, h->reorth, s);
  cell::reduce_partials(h->partial, nblk, 1, kNvMax, h->hnorm, 0, 9, h->reorth, s);
  // hcol += second-pass coefficients (a one-block "reduction" of ybuf)
  cell::reduce_partials(h->ybuf, 1, j + 1, kNvMax, h->hcol, 1, 9, h->reorth, s);
  h->prof.end(CELL_PROF_KRYLOV, ipk, s);
  cell::givens_step(h->H, h->cs, h->sn, h->g, h->hcol, h->hnorm, j, m, h->active, h->resid,
                    h->tolabs, h->invscale, h->kcount, 9, s);
  cell::scale_vec<T>(w, len, len, h->invscale, 9, s);
}

// One restarted GMRES cycle (<= m iterations) on Ahat d = r64 for the loads
// in h->want, in precision T; on return x64 += d.
template <typename T>
int gmres_cycle(cell_handle* h, const double* tolabs_host, int* iters) {
  Krylov<T>& K = kry<T>(h);
  const int m = K.m;
  const i64 len = K.len;
  const i64 vstride = 9 * len;
  cudaStream_t s = h->st;
  const int nblk = h->nblk;
  // beta^2 = |r|^2
  cell::multidot<double>(h->r64, 0, len, 1, h->r64, len, len, h->partial, nblk, kNvMax, 9, h->want, s);
  cell::reduce_partials(h->partial, nblk, 1, kNvMax, h->beta2, 0, 9, h->want, s);
  CK(cudaMemcpyAsync(h->tolabs, tolabs_host, 9 * sizeof(double), cudaMemcpyHostToDevice, s));
  cell::start_cycle(h->beta2, h->g, m, h->active, h->want, h->resid, h->invscale, h->tolabs, h->kcount, 9, s);
  CK(cudaMemcpyAsync(h->ranmask, h->active, 9 * sizeof(int), cudaMemcpyDeviceToDevice, s));
  if constexpr (sizeof(T) == 4) {
    cell::to_f32_scaled(h->r64, len, reinterpret_cast<float*>(K.V), len, len, h->invscale, 9, h->ranmask, s);
  } else {
    CK(cudaMemcpyAsync(K.V, h->r64, 9 * len * sizeof(double), cudaMemcpyDeviceToDevice, s));
    cell::scale_vec<T>(K.V, len, len, h->invscale, 9, s);
  }
  int ran[9];
  CK(cudaMemcpyAsync(ran, h->ranmask, sizeof(ran), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  int nran = 0;
  for (int q = 0; q < 9; ++q) nran += ran[q] ? 1 : 0;
  if (!nran) return CELL_OK;
  h->prof.cur_units = nran;
  const bool graphs = h->d.opt.graphs != 0;
  if (graphs && h->graphs.empty()) {
    h->graphs.resize(m);
    CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
  }
  int j = 0;
  int nunits = nran;
  for (; j < m; ++j) {
    if (graphs) {
      IterGraph& G = h->graphs[j];
      if (!G.exec) {
        // capture this iteration once: launches go to the capture stream
        cudaStream_t user = h->st;
        h->st = h->cap_st;
        h->prof.cap = &G.marks;
        cudaGraph_t graph = nullptr;
        const long long n0 = cell::g_launches.load();
        cudaError_t e = cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          iteration<T>(h, j);
          e = cudaStreamEndCapture(h->cap_st, &graph);
        }
        // captured launches run at each replay, not now
        G.nkernels = cell::g_launches.load() - n0;
        cell::g_launches.fetch_sub(G.nkernels);
        h->prof.cap = nullptr;
        h->st = user;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
          set_error("CUDA graph capture of a GMRES iteration", e);
          return CELL_ECUDA;
        }
      }
      CK(cudaGraphLaunch(G.exec, s));
      cell::g_launches.fetch_add(G.nkernels);
    } else {
      iteration<T>(h, j);
    }
    int act[9];
    CK(cudaMemcpyAsync(act, h->active, sizeof(act), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (graphs && h->prof.on) h->prof.add_graph(h->graphs[j].marks, nunits);
    int nact = 0;
    for (int q = 0; q < 9; ++q) nact += act[q] ? 1 : 0;
    if (!nact) break;
    h->prof.cur_units = nact;
    nunits = nact;
  }
  h->prof.cur_units = nran;
  cell::backsolve(h->H, h->g, h->kcount, m, h->ybuf, 9, h->ranmask, s);

  // flexible GMRES: d = Z y with the stored preconditioned directions, so the
  // preconditioner may vary between iterations (reduced-precision smoothers)
  cell::lincomb<T>(K.Z, vstride, len, h->ybuf, h->kcount, kNvMax, K.u, len, len, 9, h->ranmask, s);
  if constexpr (sizeof(T) == 4)
    cell::axpy_split<T>(h->x64, h->xh, h->xl, len, K.u, len, len, h->ones, 9, h->ranmask, s);
  else
    cell::axpy_f64<T>(h->x64, len, K.u, len, len, h->ones, 9, h->ranmask, s);
  int kc[9];
  CK(cudaMemcpyAsync(kc, h->kcount, sizeof(kc), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int q = 0; q < 9; ++q)
    if (ran[q]) iters[q] += kc[q];
  CK(cudaGetLastError());
  return CELL_OK;
}

int check_options(const cell_options& o) {
  if (!(o.tol > 0.0) || !(o.tol < 1.0)) return CELL_EINVAL;
  if (o.restart < 1 || o.restart > kNvMax - 1) return CELL_EINVAL;
  if (o.max_iter < 1) return CELL_EINVAL;
  if (o.precision != CELL_FP64 && o.precision != CELL_MIXED_FP32) return CELL_EINVAL;
  if (o.precision == CELL_MIXED_FP32 && !(o.inner_tol > 0.0 && o.inner_tol < 1.0)) return CELL_EINVAL;
  if (o.max_refine < 1) return CELL_EINVAL;
  if (o.vcycles_u < 1 || o.vcycles_phi < 1 || o.cheb_degree < 1 || o.cheb_degree > 16) return CELL_EINVAL;
  if (!(o.cheb_lo > 0.0 && o.cheb_lo < 1.0) || !(o.cheb_hi > 0.0)) return CELL_EINVAL;
  if (!(o.schur_shift >= 0.0) || o.coarse_dofs < 1) return CELL_EINVAL;
  if ((o.load_mask & 0x1FF) == 0 || (o.load_mask & ~0x1FF)) return CELL_EINVAL;
  if (o.tensor_cores < 0 || o.tensor_cores > 2) return CELL_EINVAL;
  if (o.precond != CELL_PRECOND_SCP && o.precond != CELL_PRECOND_DBP) return CELL_EINVAL;
  if (o.graphs < 0 || o.graphs > 3) return CELL_EINVAL;
  return CELL_OK;
}

// Map a design (rho or level set, device pointer of the kind/dtype given at
// set-up) into the handle: rho_e on the device, its FP32 split, the rounding
// floor of the loads, and the multigrid numerics.  No allocation.
int load_design(cell_handle* h, const void* input) {
  const cell_desc* d = &h->d;
  const i64 nn = h->nn;
  CK(cudaMemsetAsync(h->bad, 0, sizeof(int), h->st));
  if (d->input_kind == CELL_INPUT_PHI) {
    const double eta = d->eta > 0 ? d->eta : 2.0 * std::max(h->h[0], std::max(h->h[1], h->h[2]));
    if (d->input_dtype == CELL_F32)
      cell::ersatz<float>(static_cast<const float*>(input), h->nx, h->ny, h->nz, d->rho_void, eta, h->rho32, h->rho64, h->drho, h->st);
    else
      cell::ersatz<double>(static_cast<const double*>(input), h->nx, h->ny, h->nz, d->rho_void, eta, h->rho32, h->rho64, h->drho, h->st);
  } else {
    if (d->input_dtype == CELL_F32)
      cell::rho_copy<float>(static_cast<const float*>(input), nn, h->rho32, h->rho64, h->bad, h->st);
    else
      cell::rho_copy<double>(static_cast<const double*>(input), nn, h->rho32, h->rho64, h->bad, h->st);
  }
  // rho_l = fp32(rho64 - rho32)
  cell::split_f64(h->rho64, h->rho_tmp, h->rho_l, nn, h->st);
  double srho2 = 0.0;
  int nbad = 0;
  cell::sum_reduce(h->rho64, nn, h->partial, h->nblk, h->red, h->st, 1);
  CK(cudaMemcpyAsync(&srho2, h->red, sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(&nbad, h->bad, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (nbad) {
    set_error("rho input has non-positive or non-finite values");
    return CELL_EINVAL;
  }
  for (int I = 0; I < 9; ++I) {
    double f2 = 0.0;
    for (int a = 0; a < 32; ++a) f2 += h->F[a * 9 + I] * h->F[a * 9 + I];
    h->bfloor[I] = 1e-13 * std::sqrt(srho2 * f2);
  }
  // the whole-solve graph reads the floors from device memory (h->bfloor
  // outlives the copy)
  CK(cudaMemcpyAsync(h->bfloor_d, h->bfloor, sizeof(h->bfloor), cudaMemcpyHostToDevice, h->st));
  if (d->opt.precision == CELL_MIXED_FP32) CKS(fill_krylov<float>(h));
  else CKS(fill_krylov<double>(h));
  h->solved = false;
  CK(cudaGetLastError());
  return CELL_OK;
}

int setup_impl(const cell_desc* d, cell_handle* h) {
  h->d = *d;
  h->d.input = nullptr;
  h->nx = d->nx;
  h->ny = d->ny;
  h->nz = d->nz;
  h->nn = (i64)d->nx * d->ny * d->nz;
  h->st = static_cast<cudaStream_t>(d->stream);
  CK(cudaGetDevice(&h->dev));
  h->prof.on = d->opt.profile != 0;
  h->prof.mask = d->opt.profile_mask ? (unsigned)d->opt.profile_mask : ~0u;
  cellhost::nondimensionalise(d->C, d->e, d->kappa, h->Cn, h->en, h->kn, &h->C0, &h->k0);
  h->h[0] = 1.0 / d->nx;
  h->h[1] = 1.0 / d->ny;
  h->h[2] = 1.0 / d->nz;
  cellhost::element_matrix(h->Cn, h->en, h->kn, h->h, h->K0);
  if (cellhost::local_schur(h->K0, d->opt.schur_shift, h->S0) != 0) {
    set_error("elastic element block is not positive definite (check C)");
    return CELL_EINVAL;
  }
  if (d->opt.precond == CELL_PRECOND_DBP) {
    // diagonal block preconditioner (§2.5.1): the potential block is the
    // dielectric block C_e itself (K0 = [[A, B^T], [B, -C]]), no coupling
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) h->S0[a * 8 + b] = -h->K0[(4 * a + 3) * 32 + 4 * b + 3];
  }
  cellhost::affine_loads(h->h, h->Z);
  for (int a = 0; a < 32; ++a)
    for (int I = 0; I < 9; ++I) {
      double s = 0.0;
      for (int b = 0; b < 32; ++b) s += h->K0[a * 32 + b] * h->Z[b * 9 + I];
      h->F[a * 9 + I] = s;
    }
  for (int I = 0; I < 9; ++I)
    for (int J = 0; J < 9; ++J) {
      double s = 0.0;
      for (int a = 0; a < 32; ++a) s += h->Z[a * 9 + I] * h->F[a * 9 + J];
      h->H0e[I * 9 + J] = s;
    }
  // the FP64 operator serves the refinement residual of the FP64 path
  std::memcpy(h->kd.K0.k, h->K0, sizeof(h->kd.K0.k));
  std::memcpy(h->kd.S0.k, h->S0, sizeof(h->kd.S0.k));
  for (int la = 0; la < 8; ++la)
    for (int rp = 0; rp < 2; ++rp)
      for (int col = 0; col < 32; ++col) {
        const double k0 = h->K0[(4 * la + 2 * rp) * 32 + col], k1 = h->K0[(4 * la + 2 * rp + 1) * 32 + col];
        const float h0 = (float)k0, h1 = (float)k1;
        h->DF.kh[(la * 2 + rp) * 32 + col] = make_float2(h0, h1);
        h->DF.kl[(la * 2 + rp) * 32 + col] = make_float2((float)(k0 - (double)h0), (float)(k1 - (double)h1));
      }
  // every device allocation of the handle happens here
  const i64 nn = h->nn;
  const i64 len = 4 * nn;
  Arena& A = h->arena;
  CKS(A.alloc(&h->rho32, nn));
  CKS(A.alloc(&h->rho64, nn));
  if (d->input_kind == CELL_INPUT_PHI) {
    CKS(A.alloc(&h->drho, nn));
    CKS(A.alloc(&h->gtmp, nn));
  }
  CKS(A.alloc(&h->rho_l, nn));
  CKS(A.alloc(&h->rho_tmp, nn));
  CKS(A.alloc(&h->bad, 1));
  CKS(A.alloc(&h->dptrs, 1 + cell::kHilbertMaxCons));
  CKS(A.alloc(&h->bn2d, 9 * kNvMax));
  CKS(A.alloc(&h->relres_d, 9));
  CKS(A.alloc(&h->bfloor_d, 9));
  CKS(A.alloc(&h->ctl_d, 4));
  CKS(A.alloc(&h->iters_d, 9));
  CK(cudaMallocHost(reinterpret_cast<void**>(&h->gstat), sizeof(cell_handle::GraphStats)));
  CKS(A.alloc(&h->tc_err, 1));
  CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), h->st));
  h->tc_ok = cell::tc_shape_ok(h->nx, h->ny, h->nz);
  if (h->tc_ok) {
    cell::tc_prepare();
    std::vector<float> bf(cell::tc_table_floats());
    std::vector<unsigned short> gf(cell::tc_table_idx());
    cell::tc_build_tables_host(h->K0, bf.data(), gf.data());
    float* dbf;
    unsigned short* dgf;
    CKS(A.alloc(&dbf, bf.size()));
    CKS(A.alloc(&dgf, gf.size()));
    CK(cudaMemcpy(dbf, bf.data(), bf.size() * sizeof(float), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dgf, gf.data(), gf.size() * 2, cudaMemcpyHostToDevice));
    h->tct.b_full = dbf;
    h->tct.g_full = dgf;
  }
  h->nc_ok = cell::nc_shape_ok(h->nx, h->ny, h->nz);
  if (h->nc_ok) {
    cell::nc_prepare();
    const size_t nt = cell::nc_table_floats();
    std::vector<float> tb(2 * nt);
    cell::nc_build_b(cell::NK_UU, h->K0, h->S0, tb.data());
    cell::nc_build_b(cell::NK_SS4, h->K0, h->S0, tb.data() + nt);
    CKS(A.alloc(&h->ncb, tb.size()));
    CK(cudaMemcpy(h->ncb, tb.data(), tb.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  for (int i = 0; i < 1024; ++i) h->kf.K0.k[i] = (float)h->K0[i];
  h->kd.rho = h->rho64;
  CKS(A.alloc(&h->b64, 9 * len));
  CKS(A.alloc(&h->x64, 9 * len));
  CKS(A.alloc(&h->r64, 9 * len));
  CKS(A.alloc(&h->xh, 9 * len));
  CKS(A.alloc(&h->xl, 9 * len));
  // blocks per load of the reductions: ~8192 entries per block (32 per thread)
  h->nblk = (int)std::min<i64>(1024, std::max<i64>(1, (len + 8191) / 8192));
  CKS(A.alloc(&h->partial, (size_t)9 * 4 * h->nblk * kNvMax));
  CKS(A.alloc(&h->red, 9 * kNvMax));
  CKS(A.alloc(&h->red2, 9 * kNvMax));
  const int m = d->opt.restart;
  CKS(A.alloc(&h->H, (size_t)9 * (m + 1) * m));
  CKS(A.alloc(&h->cs, 9 * m));
  CKS(A.alloc(&h->sn, 9 * m));
  CKS(A.alloc(&h->g, 9 * (m + 1)));
  CKS(A.alloc(&h->hcol, 9 * kNvMax));
  CKS(A.alloc(&h->hnorm, 9 * kNvMax));
  CKS(A.alloc(&h->ybuf, 9 * kNvMax));
  CKS(A.alloc(&h->beta2, 9 * kNvMax));
  CKS(A.alloc(&h->resid, 9));
  CKS(A.alloc(&h->invscale, 9));
  CKS(A.alloc(&h->tolabs, 9));
  CKS(A.alloc(&h->ones, 9));
  {
    const double one9[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1};
    CK(cudaMemcpyAsync(h->ones, one9, sizeof(one9), cudaMemcpyHostToDevice, h->st));
  }
  CKS(A.alloc(&h->active, 9));
  CKS(A.alloc(&h->kcount, 9));
  CKS(A.alloc(&h->want, 9));
  CKS(A.alloc(&h->ranmask, 9));
  CKS(A.alloc(&h->reorth, 9));
  CK(cudaMemsetAsync(h->x64, 0, 9 * len * sizeof(double), h->st));
  if (d->opt.precision == CELL_MIXED_FP32) {
    float k0f[1024], s0f[64];
    for (int i = 0; i < 1024; ++i) k0f[i] = (float)h->K0[i];
    for (int i = 0; i < 64; ++i) s0f[i] = (float)h->S0[i];
    if (d->opt.const_bank) h->cslot1 = cell::cslot_acquire(k0f, s0f);
    CKS(setup_krylov<float>(h));
  } else {
    CKS(setup_krylov<double>(h));
  }
  CKS(load_design(h, d->input));
  if (h->nc_ok && d->opt.precision == CELL_MIXED_FP32 && d->opt.tensor_cores >= 1 && d->opt.autotune)
    CKS(tune_tiles(h));
  if (d->opt.precision == CELL_MIXED_FP32 && d->opt.autotune) {
    tune_stencils<float, 3>(h, h->kf.mgu);
    tune_stencils<float, 1>(h, h->kf.mgp);
  }
  CK(cudaStreamSynchronize(h->st));
  CK(cudaGetLastError());
  return CELL_OK;
}

// ---------------------------------------------------------------------------
// whole solve as one graph (options.graphs >= 2)
// ---------------------------------------------------------------------------

template <typename T>
cell::CtlParams ctl_params(const cell_handle* h) {
  const cell_options& o = h->d.opt;
  cell::CtlParams P;
  P.tol = o.tol;
  P.inner = sizeof(T) == 4 ? o.inner_tol : o.tol * 0.5;
  P.mask = o.load_mask;
  P.max_refine = o.max_refine;
  P.max_iter = o.max_iter;
  return P;
}

// Launches of one captured segment, into the graph being built (the calls
// enqueue on h->st, redirected to the capture stream while capturing).
// Returns the kernels the segment launched (not counted as launches now).
template <typename F>
cudaError_t capture_into(cell_handle* h, cudaGraph_t g, F&& body, long long* nk, bool keep_open = false) {
  cudaStream_t user = h->st;
  h->st = h->cap_st;
  const long long n0 = cell::g_launches.load();
  cudaError_t e = cudaStreamBeginCaptureToGraph(h->cap_st, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    e = body();
    if (!keep_open) {
      cudaGraph_t out = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(h->cap_st, &out);
      if (e == cudaSuccess) e = e2;
    }
  }
  *nk = cell::g_launches.load() - n0;
  cell::g_launches.fetch_sub(*nk);
  h->st = user;
  return e;
}

// Add a conditional node (IF / WHILE) at the current end of the capture on
// cap_st and continue the capture after it; *body receives its body graph.
cudaError_t add_conditional(cell_handle* h, cudaGraphConditionalHandle c, cudaGraphConditionalNodeType type,
                            cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(h->cap_st, &cs, nullptr, &g, &deps, &ed, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = c;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, ed, nd, &p);
  if (e != cudaSuccess) return e;
  *body = p.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(h->cap_st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Graph:  prologue (loads, zero iterate, |b|^2, r = b, |r|^2, control)
//         WHILE (refinement wanted) {
//           cycle start (|r|^2, start_cycle, first basis vector, IF conditions)
//           IF step 0 { Arnoldi step 0; condition of step 1 }  ...  IF step m-1 { ... }
//           cycle end (least squares, x += Z y, residual, |r|^2, control)
//         }
//         epilogue (null-space projection)
//
// The solve is added to `top` as an independent branch (its first nodes have
// no dependencies), so several handles' solves can share one graph.
template <typename T>
int add_solve_graph(cell_handle* h, cudaGraph_t top) {
  Krylov<T>& K = kry<T>(h);
  const int m = K.m;
  const i64 len = K.len;
  const int nblk = h->nblk;
  const cell::CtlParams P = ctl_params<T>(h);
  if (!h->cap_st) CK(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
  cudaGraphConditionalHandle wh;
  cudaError_t e = cudaGraphConditionalHandleCreate(&wh, top, 0, cudaGraphCondAssignDefault);
  cudaGraph_t wbody = nullptr;
  // top level: prologue, WHILE node, epilogue
  long long n_top = 0, n_epi = 0;
  if (e == cudaSuccess)
    e = capture_into(h, top, [&]() -> cudaError_t {
      cudaStream_t s = h->st;
      cell::RhsParams RP;
      std::memcpy(RP.F, h->F, sizeof(RP.F));
      cell::rhs9(h->rho64, RP, h->d.opt.load_mask, h->b64, h->nx, h->ny, h->nz, s);
      cudaMemsetAsync(h->x64, 0, 9 * len * sizeof(double), s);
      cudaMemsetAsync(h->xh, 0, 9 * len * sizeof(float), s);
      cudaMemsetAsync(h->xl, 0, 9 * len * sizeof(float), s);
      cell::multidot<double>(h->b64, 0, len, 1, h->b64, len, len, h->partial, nblk, kNvMax, 9, nullptr, s);
      cell::reduce_partials(h->partial, nblk, 1, kNvMax, h->bn2d, 0, 9, nullptr, s);
      cudaMemcpyAsync(h->r64, h->b64, 9 * len * sizeof(double), cudaMemcpyDeviceToDevice, s);
      cell::multidot<double>(h->r64, 0, len, 1, h->r64, len, len, h->partial, nblk, kNvMax, 9, nullptr, s);
      cell::reduce_partials(h->partial, nblk, 1, kNvMax, h->red, 0, 9, nullptr, s);
      cell::ctl_reset(h->ctl_d, h->iters_d, s);
      cell::refine_ctl(h->bn2d, h->red, h->bfloor_d, P, h->want, h->tolabs, h->relres_d, h->iters_d, h->ctl_d, wh, s);
      cudaError_t e1 = add_conditional(h, wh, cudaGraphCondTypeWhile, &wbody);
      if (e1 != cudaSuccess) return e1;
      const long long nb = cell::g_launches.load();
      cell::comp_sums(h->x64, h->nn, 9, h->partial, nblk, h->red2, s);
      cell::sub_means(h->x64, h->nn, 9, h->red2, s);
      n_epi = cell::g_launches.load() - nb;
      return cudaGetLastError();
    }, &n_top);
  // WHILE body: cycle start, the IF chain of Arnoldi steps, cycle end
  cell::IterHandles IH{};
  IH.m = m;
  for (int j = 0; j < m && e == cudaSuccess; ++j)
    e = cudaGraphConditionalHandleCreate(&IH.h[j], wbody, 0, cudaGraphCondAssignDefault);
  std::vector<cudaGraph_t> ifbody(m, nullptr);
  long long n_body = 0;
  if (e == cudaSuccess)
    e = capture_into(h, wbody, [&]() -> cudaError_t {
      cudaStream_t s = h->st;
      cell::multidot<double>(h->r64, 0, len, 1, h->r64, len, len, h->partial, nblk, kNvMax, 9, h->want, s);
      cell::reduce_partials(h->partial, nblk, 1, kNvMax, h->beta2, 0, 9, h->want, s);
      cell::start_cycle(h->beta2, h->g, m, h->active, h->want, h->resid, h->invscale, h->tolabs, h->kcount, 9, s);
      cell::cycle_handles(h->active, h->ranmask, IH, s);
      if constexpr (sizeof(T) == 4)
        cell::to_f32_scaled(h->r64, len, reinterpret_cast<float*>(K.V), len, len, h->invscale, 9, h->ranmask, s);
      else
        cell::copy_scale_f64(h->r64, reinterpret_cast<double*>(K.V), len, h->invscale, 9, h->ranmask, s);
      for (int j = 0; j < m; ++j) {
        cudaError_t e1 = add_conditional(h, IH.h[j], cudaGraphCondTypeIf, &ifbody[j]);
        if (e1 != cudaSuccess) return e1;
      }
      const long long nb = cell::g_launches.load();
      cell::backsolve(h->H, h->g, h->kcount, m, h->ybuf, 9, h->ranmask, s);
      cell::lincomb<T>(K.Z, 9 * len, len, h->ybuf, h->kcount, kNvMax, K.u, len, len, 9, h->ranmask, s);
      if constexpr (sizeof(T) == 4)
        cell::axpy_split<T>(h->x64, h->xh, h->xl, len, K.u, len, len, h->ones, 9, h->ranmask, s);
      else
        cell::axpy_f64<T>(h->x64, len, K.u, len, len, h->ones, 9, h->ranmask, s);
      cell::accum_iters(h->iters_d, h->kcount, h->ranmask, h->ctl_d, s);
      if constexpr (sizeof(T) == 4)
        cell::resid_df(h->xh, h->xl, len, h->b64, len, h->r64, len, h->rho32, h->rho_l, h->DF, h->nx, h->ny,
                       h->nz, 9, nullptr, s);
      else
        apply_full_T<double>(h, h->x64, len, h->r64, len, h->b64, len, -1.0, 1.0, nullptr, 9);
      cell::multidot<double>(h->r64, 0, len, 1, h->r64, len, len, h->partial, nblk, kNvMax, 9, nullptr, s);
      cell::reduce_partials(h->partial, nblk, 1, kNvMax, h->red, 0, 9, nullptr, s);
      cell::refine_ctl(h->bn2d, h->red, h->bfloor_d, P, h->want, h->tolabs, h->relres_d, h->iters_d, h->ctl_d, wh, s);
      h->seg_ce = cell::g_launches.load() - nb;
      return cudaGetLastError();
    }, &n_body);
  // every Arnoldi step sets the condition of the next one
  long long n_it = 0, n_it0 = 0;
  for (int j = 0; j < m && e == cudaSuccess; ++j) {
    e = capture_into(h, ifbody[j], [&]() -> cudaError_t {
      iteration<T>(h, j);
      if (j + 1 < m) cell::next_step(h->active, IH.h[j + 1], h->st);
      return cudaGetLastError();
    }, &n_it);
    if (j == 0) n_it0 = n_it;
  }
  if (e != cudaSuccess) {
    set_error("whole-solve CUDA graph (conditional nodes)", e);
    return CELL_ECUDA;
  }
  h->seg_epi = n_epi;
  h->seg_pro = n_top - n_epi;
  h->seg_cb = n_body - h->seg_ce;
  h->seg_it = n_it0;   // kernels per Arnoldi step (the last step of a cycle has one fewer)
  return CELL_OK;
}

template <typename T>
int build_solve_graph(cell_handle* h) {
  cudaGraph_t top = nullptr;
  CK(cudaGraphCreate(&top, 0));
  int rc = add_solve_graph<T>(h, top);
  if (rc == CELL_OK) {
    const cudaError_t e = cudaGraphInstantiate(&h->solve_exec, top, 0);
    if (e != cudaSuccess) {
      h->solve_exec = nullptr;
      set_error("whole-solve CUDA graph (conditional nodes)", e);
      rc = CELL_ECUDA;
    }
  }
  cudaGraphDestroy(top);
  if (rc == CELL_OK) h->solve_prec = sizeof(T) == 4 ? 1 : 0;
  return rc;
}

// Asynchronous copy of a graph solve's statistics to the pinned host block,
// ordered after the solve on stream s.
int copy_solve_stats(cell_handle* h, cudaStream_t s) {
  cell_handle::GraphStats* G = h->gstat;
  CK(cudaMemcpyAsync(G->ctl, h->ctl_d, sizeof(G->ctl), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(G->iters, h->iters_d, sizeof(G->iters), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(G->relres, h->relres_d, sizeof(G->relres), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&G->tcerr, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  return CELL_OK;
}

// Launch of a whole solve (graph built on first use) and the asynchronous
// copy of its statistics; solve_graph_finish waits for them.
template <typename T>
int solve_graph_launch(cell_handle* h) {
  h->gt0 = std::chrono::steady_clock::now();
  if (!h->solve_exec || h->solve_prec != (sizeof(T) == 4 ? 1 : 0)) CKS(build_solve_graph<T>(h));
  CK(cudaGraphLaunch(h->solve_exec, h->st));
  return copy_solve_stats(h, h->st);
}

template <typename T>
int solve_graph_finish(cell_handle* h, cell_stats* st) {
  cudaStream_t s = h->st;
  CK(cudaStreamSynchronize(s));
  const cell_handle::GraphStats& G = *h->gstat;
  cell::g_launches.fetch_add(h->seg_pro + h->seg_epi + (long long)G.ctl[0] * (h->seg_cb + h->seg_ce) +
                             (long long)G.ctl[2] * h->seg_it);
  cell_stats S{};
  int status = G.ctl[1];
  if (G.tcerr) {
    set_error("a tensor-core kernel's bounded wait expired");
    status = CELL_ETIMEOUT;
    CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
  }
  CK(cudaGetLastError());
  for (int q = 0; q < 9; ++q) {
    S.iters[q] = G.iters[q];
    S.rel_residual[q] = G.relres[q];
  }
  S.refinements = G.ctl[0];
  S.status = status;
  S.nlevels_u = (int)kry<T>(h).mgu.lv.size();
  S.nlevels_phi = (int)kry<T>(h).mgp.lv.size();
  tile_stats(h, S);
  S.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - h->gt0).count();
  h->solved = (status == CELL_OK);
  h->last = S;
  if (st) *st = S;
  return status;
}

template <typename T>
int solve_graph(cell_handle* h, cell_stats* st) {
  CKS(solve_graph_launch<T>(h));
  return solve_graph_finish<T>(h, st);
}

template <typename T>
int solve_impl(cell_handle* h, cell_stats* st) {
  const cell_options& o = h->d.opt;
  if (o.graphs >= 2 && !h->prof.on) return solve_graph<T>(h, st);
  cudaStream_t s = h->st;
  const i64 len = 4 * h->nn;
  const int nblk = h->nblk;
  cell_stats S{};
  auto t0 = std::chrono::steady_clock::now();
  cell::RhsParams RP;
  std::memcpy(RP.F, h->F, sizeof(RP.F));
  cell::rhs9(h->rho64, RP, o.load_mask, h->b64, h->nx, h->ny, h->nz, s);
  CK(cudaMemsetAsync(h->x64, 0, 9 * len * sizeof(double), s));
  CK(cudaMemsetAsync(h->xh, 0, 9 * len * sizeof(float), s));
  CK(cudaMemsetAsync(h->xl, 0, 9 * len * sizeof(float), s));
  double bn2[9], rn2[9];
  cell::multidot<double>(h->b64, 0, len, 1, h->b64, len, len, h->partial, nblk, kNvMax, 9, nullptr, s);
  cell::reduce_partials(h->partial, nblk, 1, kNvMax, h->red, 0, 9, nullptr, s);
  std::vector<double> tmp(9 * kNvMax);
  CK(cudaMemcpyAsync(tmp.data(), h->red, 9 * kNvMax * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->r64, h->b64, 9 * len * sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  for (int q = 0; q < 9; ++q) bn2[q] = tmp[q * kNvMax];
  int status = CELL_OK;
  int refine = 0;
  while (true) {
    cell::multidot<double>(h->r64, 0, len, 1, h->r64, len, len, h->partial, nblk, kNvMax, 9, nullptr, s);
    cell::reduce_partials(h->partial, nblk, 1, kNvMax, h->red, 0, 9, nullptr, s);
    CK(cudaMemcpyAsync(tmp.data(), h->red, 9 * kNvMax * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int want[9];
    double tolabs[9];
    bool any = false;
    int maxit = 0;
    for (int q = 0; q < 9; ++q) {
      rn2[q] = tmp[q * kNvMax];
      const double bn = std::sqrt(bn2[q]), rn = std::sqrt(rn2[q]);
      S.rel_residual[q] = bn > h->bfloor[q] ? rn / bn : 0.0;
      want[q] = ((o.load_mask >> q) & 1) && rn > std::max(o.tol * bn, h->bfloor[q]);
      any = any || want[q];
      maxit = std::max(maxit, S.iters[q]);
      const double inner = sizeof(T) == 4 ? o.inner_tol : o.tol * 0.5;
      tolabs[q] = std::max(inner * rn, 0.5 * o.tol * bn);
    }
    if (!any) break;
    if (refine >= o.max_refine || maxit >= o.max_iter) {
      status = CELL_ENOTCONV;
      break;
    }
    CK(cudaMemcpyAsync(h->want, want, sizeof(want), cudaMemcpyHostToDevice, s));
    CKS(gmres_cycle<T>(h, tolabs, S.iters));
    ++refine;
    // FP64-grade residual of the updated iterate: r = bhat - Ahat x
    h->prof.cur_units = 9;
    if constexpr (sizeof(T) == 4) {
      const int ip = h->prof.begin(s, CELL_PROF_FULL64);
      cell::resid_df(h->xh, h->xl, len, h->b64, len, h->r64, len, h->rho32, h->rho_l, h->DF,
                     h->nx, h->ny, h->nz, 9, nullptr, s);
      h->prof.end(CELL_PROF_FULL64, ip, s);
    } else {
      apply_full_T<double>(h, h->x64, len, h->r64, len, h->b64, len, -1.0, 1.0, nullptr, 9);
    }
  }
  // null-space projection (mean displacement and potential per load)
  cell::comp_sums(h->x64, h->nn, 9, h->partial, nblk, h->red2, s);
  cell::sub_means(h->x64, h->nn, 9, h->red2, s);
  int tcerr = 0;
  CK(cudaMemcpyAsync(&tcerr, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (tcerr) {
    set_error("a tensor-core kernel's bounded wait expired");
    status = CELL_ETIMEOUT;
    CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
  }
  CK(cudaGetLastError());
  auto t1 = std::chrono::steady_clock::now();
  S.solve_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  S.refinements = refine;
  S.status = status;
  S.nlevels_u = (int)kry<T>(h).mgu.lv.size();
  S.nlevels_phi = (int)kry<T>(h).mgp.lv.size();
  tile_stats(h, S);
  if (h->prof.on) h->prof.collect(S.class_ms, S.class_count, S.class_units);
  h->solved = (status == CELL_OK);
  h->last = S;
  if (st) *st = S;
  return status;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

namespace {
// Upstream gradients in SI units -> the nondimensional G of g_e = sum G_IJ
// W^I.K0 W^J (H = [[C^H, -e^H^T], [-e^H, -kappa^H]] in scaled units).
cell::SensParams sens_params(const cell_handle* h, const double dC[36], const double de[18],
                             const double dk[9]) {
  cell::SensParams P;
  std::memcpy(P.Z, h->Z, sizeof(P.Z));
  std::memset(P.G, 0, sizeof(P.G));
  const double se = std::sqrt(h->C0 * h->k0);
  for (int p = 0; p < 6; ++p)
    for (int q = 0; q < 6; ++q) P.G[p * 9 + q] = dC ? h->C0 * dC[p * 6 + q] : 0.0;
  for (int i = 0; i < 3; ++i)
    for (int p = 0; p < 6; ++p) {
      const double v = de ? -0.5 * se * de[i * 6 + p] : 0.0;
      P.G[(6 + i) * 9 + p] = v;
      P.G[p * 9 + 6 + i] = v;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) P.G[(6 + i) * 9 + 6 + j] = dk ? -h->k0 * dk[i * 3 + j] : 0.0;
  return P;
}

// sym(G) = Q diag(lam) Q^T (host, FP64 Jacobi): the mode tables of the
// sensitivity kernels.  Modes with |lam| <= 1e-15 max|lam| are dropped.
template <typename T>
void sens_modes(const cell_handle* h, const cell::SensParams& P, cell::SensQ* Q, cell::SensModes<T>* M) {
  double Gs[81], lam[9], V[81];
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) Gs[i * 9 + j] = 0.5 * (P.G[i * 9 + j] + P.G[j * 9 + i]);
  cellhost::sym_eig(Gs, 9, lam, V);
  double lmax = 0.0;
  for (int k = 0; k < 9; ++k) lmax = std::max(lmax, std::fabs(lam[k]));
  int R = 0;
  std::memset(Q, 0, sizeof(*Q));
  std::memset(M, 0, sizeof(*M));
  for (int k = 0; k < 9; ++k) {
    if (!(std::fabs(lam[k]) > 1e-15 * lmax)) continue;
    for (int I = 0; I < 9; ++I) Q->q[I * 9 + R] = V[I * 9 + k];
    M->lam[R] = (T)lam[k];
    for (int a = 0; a < 32; ++a) {
      double z = 0.0;
      for (int I = 0; I < 9; ++I) z += P.Z[a * 9 + I] * V[I * 9 + k];
      M->zq[a * 9 + R] = (T)z;
    }
    ++R;
  }
  Q->R = R;
  M->R = R;
  for (int a = 0; a < 32; ++a)
    for (int b = 0; b < 32; ++b)
      M->ku[a * 32 + b] = b == a ? (T)h->K0[a * 32 + a] : (b > a ? (T)(2.0 * h->K0[a * 32 + b]) : T(0));
}

// The mode fields (R x 8 x nn floats or R x 4 x nn doubles, R <= 9) go to the
// Krylov basis, which is free between solves: (m + 1) x 9 x 4nn values of the
// Krylov type (m >= 1) hold 9 x 4nn doubles.
template <typename T>
void run_sensitivity(cell_handle* h, const cell::SensParams& P, T* g) {
  cell::SensQ Q;
  cell::SensModes<T> M;
  sens_modes<T>(h, P, &Q, &M);
  void* work = h->d.opt.precision == CELL_MIXED_FP32 ? (void*)h->kf.V : (void*)h->kd.V;
  cell::sensitivity<T>(h->x64, h->rho64, Q, M, static_cast<T*>(work), g, h->nx, h->ny, h->nz, 0, h->st);
}
}  // namespace


namespace {

// Tile autotuning of the tensor-core smoothers (options.autotune): each
// block's Chebyshev step on the fine level is timed for every tile candidate
// on the handle's own scratch vectors (level-0 r, d, d2 and the Krylov basis,
// all rewritten by every solve before use) and the fastest tile is kept.  The
// tile changes launch geometry only, never a result.
int tune_tiles(cell_handle* h) {
  Krylov<float>& K = h->kf;
  for (int kind = 0; kind < 2; ++kind) {
    Level<float>& L0 = kind == cell::NK_UU ? K.mgu.lv[0] : K.mgp.lv[0];
    const i64 ws = (kind == cell::NK_UU ? 3 : 1) * h->nn;
    cell::ApplyArgs<float> a{};
    a.x = L0.d; a.xs = ws; a.y = L0.r; a.ys = ws; a.sol = K.V; a.ss = ws; a.dout = L0.d2; a.ds = ws;
    a.cc = L0.cc; a.sol_zero = 0;
    a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    a.dinv = L0.dinv; a.rho = K.rho; a.cslot1 = h->cslot1;
    h->nct[kind] = cell::nc_autotune(kind, a, h->ncb + cell::nc_table_floats() * kind, cell::AM_CHEB, 9,
                                     h->tc_err, h->st, &h->nct_us[kind]);
  }
  int err = 0;
  CK(cudaMemcpyAsync(&err, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (err) return CELL_ECUDA;   // a bounded wait expired: the tensor-core path is not usable
  return CELL_OK;
}

// Loads per thread of every coarse level's stencil apply, timed at set-up in
// the Chebyshev mode on the level's own scratch vectors (bitwise-neutral).
template <typename T, int NC>
void tune_stencils(cell_handle* h, BlockMG<T>& mg) {
  for (size_t l = 1; l < mg.lv.size(); ++l) {
    Level<T>& L = mg.lv[l];
    if (!L.st || L.dense) continue;
    const i64 ws = NC * L.nn;
    cell::ApplyArgs<T> a{};
    a.x = L.d; a.xs = ws; a.y = L.r; a.ys = ws; a.sol = L.x; a.ss = ws; a.dout = L.d2; a.ds = ws;
    a.dinv = L.dinv; a.cc = L.cc; a.st = L.st;
    a.nx = L.nx; a.ny = L.ny; a.nz = L.nz;
    L.rg = cell::stencil_autotune<T, NC>(a, cell::AM_CHEB, 9, h->st, nullptr);
  }
}

void tile_stats(const cell_handle* h, cell_stats& S) {
  const bool tc = h->nc_ok && h->d.opt.precision == CELL_MIXED_FP32 && h->d.opt.tensor_cores >= 1;
  for (int k = 0; k < 2; ++k) {
    S.tc_tile_xt[k] = tc ? h->nct[k].xt : 0;
    S.tc_tile_L[k] = tc ? h->nct[k].L : 0;
    S.tc_tile_us[k] = tc ? h->nct_us[k] : 0.0;
  }
  if (h->d.opt.precision == CELL_MIXED_FP32) {
    const auto& u = h->kf.mgu.lv;
    const auto& p = h->kf.mgp.lv;
    for (int l = 0; l < 8; ++l) {
      S.stencil_rg[0][l] = l < (int)u.size() ? u[l].rg : 0;
      S.stencil_rg[1][l] = l < (int)p.size() ? p[l].rg : 0;
    }
  }
}

// ---------------------------------------------------------------------------
// one graph for a batch of solves
// ---------------------------------------------------------------------------

// The whole-solve graphs of several handles (same device) as independent
// branches of one executable graph: a batch is one graph launch, and the
// solves run concurrently however their iteration counts differ (each
// branch's refinement loop and Arnoldi steps are its own conditional nodes).
// The executable graph of the last batch is kept and reused while the same
// handles, in the same order, are solved again; destroying one of them drops it.
struct BatchGraph {
  std::vector<cell_handle*> hs;
  std::vector<int> prec;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev = nullptr;
  int dev = -1;
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    if (ev) cudaEventDestroy(ev);
    exec = nullptr;
    ev = nullptr;
    hs.clear();
    prec.clear();
    dev = -1;
  }
};
std::mutex g_batch_mu;
BatchGraph g_batch;

int prec_of(const cell_handle* h) { return h->d.opt.precision == CELL_MIXED_FP32 ? 1 : 0; }

// Build (or reuse) the batch graph of hs[0..n) and launch it on hs[0]'s
// stream, ordered after the work already queued on every handle's stream;
// every handle's stream is ordered after the batch and its statistics copy.
int solve_batch_graph(cell_handle** hs, int n) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  BatchGraph& B = g_batch;
  bool same = B.exec && (int)B.hs.size() == n && B.dev == hs[0]->dev;
  for (int i = 0; same && i < n; ++i) same = B.hs[i] == hs[i] && B.prec[i] == prec_of(hs[i]);
  CK(cudaSetDevice(hs[0]->dev));
  const auto t0 = std::chrono::steady_clock::now();
  if (!same) {
    B.reset();
    cudaGraph_t top = nullptr;
    CK(cudaGraphCreate(&top, 0));
    int rc = CELL_OK;
    for (int i = 0; i < n && rc == CELL_OK; ++i)
      rc = prec_of(hs[i]) ? add_solve_graph<float>(hs[i], top) : add_solve_graph<double>(hs[i], top);
    if (rc == CELL_OK) {
      const cudaError_t e = cudaGraphInstantiate(&B.exec, top, 0);
      if (e != cudaSuccess) {
        B.exec = nullptr;
        set_error("batched whole-solve CUDA graph", e);
        rc = CELL_ECUDA;
      }
    }
    cudaGraphDestroy(top);
    if (rc == CELL_OK && cudaEventCreateWithFlags(&B.ev, cudaEventDisableTiming) != cudaSuccess) {
      set_error("cudaEventCreateWithFlags");
      rc = CELL_ECUDA;
    }
    if (rc != CELL_OK) {
      B.reset();
      return rc;
    }
    B.hs.assign(hs, hs + n);
    for (int i = 0; i < n; ++i) B.prec.push_back(prec_of(hs[i]));
    B.dev = hs[0]->dev;
  }
  cudaStream_t L = hs[0]->st;
  for (int i = 1; i < n; ++i) {
    CK(cudaEventRecord(B.ev, hs[i]->st));
    CK(cudaStreamWaitEvent(L, B.ev, 0));
  }
  for (int i = 0; i < n; ++i) hs[i]->gt0 = t0;
  CK(cudaGraphLaunch(B.exec, L));
  for (int i = 0; i < n; ++i) CKS(copy_solve_stats(hs[i], L));
  CK(cudaEventRecord(B.ev, L));
  for (int i = 1; i < n; ++i) CK(cudaStreamWaitEvent(hs[i]->st, B.ev, 0));
  return CELL_OK;
}

void forget_batch(const cell_handle* h) {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  for (const cell_handle* q : g_batch.hs)
    if (q == h) {
      g_batch.reset();
      return;
    }
}

}  // namespace

extern "C" {

void cell_default_options(cell_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-10;
  o->restart = 30;
  o->max_iter = 400;
  o->precision = CELL_MIXED_FP32;
  o->inner_tol = 1e-4;
  o->max_refine = 40;
  o->vcycles_u = 1;
  o->vcycles_phi = 1;
  o->cheb_degree = 3;
  o->cheb_lo = 0.03;
  o->cheb_hi = 1.0;
  o->schur_shift = 1e-10;
  o->coarse_dofs = 200;
  o->load_mask = 0x1FF;
  o->profile = 0;
  o->tensor_cores = 1;
  o->const_bank = 1;
  o->graphs = 2;
  o->profile_mask = 0;
  o->precond = CELL_PRECOND_SCP;
  o->autotune = 1;
}

int cell_setup(const cell_desc* d, cell_handle** out) {
  if (!d || !out) return CELL_EINVAL;
  *out = nullptr;
  if (d->nx < 2 || d->ny < 2 || d->nz < 2) return CELL_EINVAL;
  if ((double)d->nx * d->ny * d->nz > 4.0e8) return CELL_EINVAL;
  if (!d->input) return CELL_EINVAL;
  if (d->input_kind != CELL_INPUT_RHO && d->input_kind != CELL_INPUT_PHI) return CELL_EINVAL;
  if (d->input_dtype != CELL_F32 && d->input_dtype != CELL_F64) return CELL_EINVAL;
  if (d->input_kind == CELL_INPUT_PHI && !(d->rho_void > 0.0 && d->rho_void <= 1.0)) return CELL_EINVAL;
  for (int i = 0; i < 36; ++i) if (!std::isfinite(d->C[i])) return CELL_EINVAL;
  for (int i = 0; i < 18; ++i) if (!std::isfinite(d->e[i])) return CELL_EINVAL;
  for (int i = 0; i < 9; ++i) if (!std::isfinite(d->kappa[i])) return CELL_EINVAL;
  if (check_options(d->opt) != CELL_OK) return CELL_EINVAL;
  cell_handle* h = new cell_handle();
  const int s = setup_impl(d, h);
  if (s != CELL_OK) {
    cudaStreamSynchronize(h->st);
    h->arena.release();
    if (h->gstat) cudaFreeHost(h->gstat);
    delete h;
    return s;
  }
  *out = h;
  return CELL_OK;
}

int cell_update(cell_handle* h, const void* input) {
  if (!h || !input) return CELL_EINVAL;
  return load_design(h, input);
}

int cell_solve(cell_handle* h, cell_stats* st) {
  if (!h) return CELL_EINVAL;
  if (h->d.opt.precision == CELL_MIXED_FP32) return solve_impl<float>(h, st);
  return solve_impl<double>(h, st);
}

int cell_hj_step(const void* phi, const void* v, int nx, int ny, int nz, double dt, void* out, int dtype,
                 void* stream) {
  if (!phi || !v || !out || nx < 2 || ny < 2 || nz < 2 || !std::isfinite(dt)) return CELL_EINVAL;
  if (dtype != CELL_F32 && dtype != CELL_F64) return CELL_EINVAL;
  if (phi == out) return CELL_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == CELL_F64)
    cell::hj_step<double>(static_cast<const double*>(phi), static_cast<const double*>(v), nx, ny, nz, dt,
                          static_cast<double*>(out), s);
  else
    cell::hj_step<float>(static_cast<const float*>(phi), static_cast<const float*>(v), nx, ny, nz, dt,
                         static_cast<float*>(out), s);
  CK(cudaGetLastError());
  return CELL_OK;
}

int cell_solve_batch(cell_handle** hs, int n, cell_stats* st) {
  if (!hs || n < 0) return CELL_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return CELL_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return CELL_EINVAL;
  }
  // whole-solve graphs: with graphs == 2 on every handle of one device, all
  // solves are branches of one graph and the batch is one launch; with
  // graphs == 3 (or handles on several devices), every handle's solve graph is
  // launched on its own stream.  The host never waits between launches, so the
  // solves overlap on the GPU; the statistics are collected afterwards.
  bool all_graphs = true, one_graph = n > 1;
  for (int i = 0; i < n; ++i) {
    all_graphs = all_graphs && hs[i]->d.opt.graphs >= 2 && !hs[i]->prof.on;
    one_graph = one_graph && hs[i]->d.opt.graphs == 2 && hs[i]->dev == hs[0]->dev;
  }
  if (all_graphs) {
    std::vector<int> rc(n, CELL_OK);
    std::vector<std::string> errs(n);
    if (one_graph) {
      const int r = solve_batch_graph(hs, n);
      if (r != CELL_OK) return r;
    }
    for (int i = 0; i < n && !one_graph; ++i) {
      cell_handle* h = hs[i];
      if (cudaSetDevice(h->dev) != cudaSuccess) {
        rc[i] = CELL_ECUDA;
        continue;
      }
      rc[i] = h->d.opt.precision == CELL_MIXED_FP32 ? solve_graph_launch<float>(h) : solve_graph_launch<double>(h);
      if (rc[i] != CELL_OK) errs[i] = g_last_error;
    }
    for (int i = 0; i < n; ++i) {   // every launched solve is collected
      cell_handle* h = hs[i];
      if (rc[i] != CELL_OK) {
        if (st) st[i].status = rc[i];
        continue;
      }
      if (cudaSetDevice(h->dev) != cudaSuccess) {
        rc[i] = CELL_ECUDA;
        continue;
      }
      rc[i] = h->d.opt.precision == CELL_MIXED_FP32 ? solve_graph_finish<float>(h, st ? st + i : nullptr)
                                                    : solve_graph_finish<double>(h, st ? st + i : nullptr);
      if (rc[i] != CELL_OK) errs[i] = g_last_error;
    }
    for (int i = 0; i < n; ++i)
      if (rc[i] != CELL_OK) {
        g_last_error = errs[i];
        return rc[i];
      }
    return CELL_OK;
  }
  // otherwise one host worker per handle (at most kBatchThreads): each drives
  // its handle's solve on the handle's own stream and device
  constexpr int kBatchThreads = 16;
  std::vector<int> rc(n, CELL_OK);
  std::vector<std::string> errs(n);
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      if (cudaSetDevice(hs[i]->dev) != cudaSuccess) {
        rc[i] = CELL_ECUDA;
        errs[i] = "cudaSetDevice";
        continue;
      }
      rc[i] = cell_solve(hs[i], st ? st + i : nullptr);
      if (rc[i] != CELL_OK) errs[i] = g_last_error;
    }
  };
  const int nt = std::min(n, kBatchThreads);
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int t = 0; t < nt; ++t) th.emplace_back(worker);
  for (auto& t : th) t.join();
  for (int i = 0; i < n; ++i)
    if (rc[i] != CELL_OK) {
      g_last_error = errs[i];
      return rc[i];
    }
  return CELL_OK;
}

int cell_homogenise(cell_handle* h, double CH[36], double eH[18], double kH[9]) {
  if (!h || !CH || !eH || !kH) return CELL_EINVAL;
  if (!h->solved || h->d.opt.load_mask != 0x1FF) return CELL_ESTATE;
  cudaStream_t s = h->st;
  const int nblk = h->nblk;
  double G1[81], G2[81], srho;
  cell::sum_reduce(h->rho64, h->nn, h->partial, nblk, h->red, s);
  CK(cudaMemcpyAsync(&srho, h->red, sizeof(double), cudaMemcpyDeviceToHost, s));
  cell::gram9(h->b64, h->x64, h->nn, h->partial, nblk, h->red, s);
  CK(cudaMemcpyAsync(G1, h->red, sizeof(G1), cudaMemcpyDeviceToHost, s));
  cell::gram9(h->x64, h->r64, h->nn, h->partial, nblk, h->red2, s);
  CK(cudaMemcpyAsync(G2, h->red2, sizeof(G2), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // energy form: H = sum rho H0e - b.y - y.r   (H0e = Zbar^T K0 Zbar)
  double H[81];
  for (int i = 0; i < 81; ++i) H[i] = srho * h->H0e[i] - G1[i] - G2[i];
  for (int I = 0; I < 9; ++I)
    for (int J = I + 1; J < 9; ++J) {
      const double v = 0.5 * (H[I * 9 + J] + H[J * 9 + I]);
      H[I * 9 + J] = H[J * 9 + I] = v;
    }
  const double se = std::sqrt(h->C0 * h->k0);
  for (int p = 0; p < 6; ++p)
    for (int q = 0; q < 6; ++q) CH[p * 6 + q] = h->C0 * H[p * 9 + q];
  for (int i = 0; i < 3; ++i)
    for (int p = 0; p < 6; ++p) eH[i * 6 + p] = -se * H[(6 + i) * 9 + p];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) kH[i * 3 + j] = -h->k0 * H[(6 + i) * 9 + 6 + j];
  return CELL_OK;
}

int cell_sensitivity(cell_handle* h, const double dC[36], const double de[18], const double dk[9],
                     void* g, int dtype) {
  if (!h || !g || (dtype != CELL_F32 && dtype != CELL_F64)) return CELL_EINVAL;
  if (!h->solved) return CELL_ESTATE;
  const cell::SensParams P = sens_params(h, dC, de, dk);
  if (dtype == CELL_F32) run_sensitivity<float>(h, P, static_cast<float*>(g));
  else run_sensitivity<double>(h, P, static_cast<double*>(g));
  CK(cudaGetLastError());
  return CELL_OK;
}

int cell_hilbert_velocity(cell_handle* h, double alpha, const double* dJ, const double* const* dC,
                          const double* C, int ncons, double wJ, double wC, double* v, double* info) {
  if (!h || !dJ || !v || !(alpha > 0.0) || !std::isfinite(alpha)) return CELL_EINVAL;
  if (ncons < 0 || ncons > cell::kHilbertMaxCons || (ncons > 0 && (!dC || !C))) return CELL_EINVAL;
  for (int i = 0; i < ncons; ++i)
    if (!dC[i] || !std::isfinite(C[i])) return CELL_EINVAL;
  if (!std::isfinite(wJ) || !std::isfinite(wC)) return CELL_EINVAL;
  // workspace: 4 (1 + ncons) nn doubles of the Krylov basis ((m + 1) x 9 x 4 nn values)
  const bool mixed = h->d.opt.precision == CELL_MIXED_FP32;
  if ((mixed ? (h->d.opt.restart + 1) / 2 : h->d.opt.restart + 1) < 1) return CELL_EINVAL;
  double* work = mixed ? reinterpret_cast<double*>(h->kf.V) : h->kd.V;
  const int st = cell::hilbert_velocity(h->nx, h->ny, h->nz, alpha, dJ, dC, C, ncons, wJ, wC, v, work, h->dptrs,
                                        h->partial, h->nblk, h->red, info, h->st);
  if (st == CELL_ECUDA) set_error("cell_hilbert_velocity", cudaGetLastError());
  if (st == CELL_EINVAL) set_error("cell_hilbert_velocity: constraint sensitivities are linearly dependent");
  return st;
}

int cell_energy_difference(cell_handle* h, const cell_handle* ref, const double dC[36], const double de[18],
                           const double dk[9], double* g) {
  if (!h || !ref || !g || h == ref) return CELL_EINVAL;
  if (h->nx != ref->nx || h->ny != ref->ny || h->nz != ref->nz) return CELL_EINVAL;
  for (int i = 0; i < 1024; ++i)
    if (h->K0[i] != ref->K0[i]) return CELL_EINVAL;
  if (!h->solved || !ref->solved) return CELL_ESTATE;
  // workspace: 2 x 9 x 4 nn doubles of h's Krylov basis ((m + 1) x 9 x 4 nn values)
  const bool mixed = h->d.opt.precision == CELL_MIXED_FP32;
  if ((mixed ? (h->d.opt.restart + 1) / 2 : h->d.opt.restart + 1) < 2) return CELL_EINVAL;
  const cell::SensParams P = sens_params(h, dC, de, dk);
  cell::SensQ Q;
  cell::SensModes<double> M;
  sens_modes<double>(h, P, &Q, &M);
  cell::SensPair SP;
  std::memcpy(SP.k, h->K0, sizeof(SP.k));
  std::memcpy(SP.zq, M.zq, sizeof(SP.zq));
  std::memcpy(SP.lam, M.lam, sizeof(SP.lam));
  SP.R = M.R;
  double* work = mixed ? reinterpret_cast<double*>(h->kf.V) : h->kd.V;
  if (ref->st != h->st) {   // the reference's solution must be final on its own stream
    CK(cudaStreamSynchronize(ref->st));
  }
  cell::energy_difference(h->x64, ref->x64, Q, SP, work, g, h->nx, h->ny, h->nz, h->st);
  CK(cudaGetLastError());
  return CELL_OK;
}

int cell_sensitivity_phi(cell_handle* h, const double dC[36], const double de[18], const double dk[9],
                         void* g, int dtype) {
  if (!h || !g || (dtype != CELL_F32 && dtype != CELL_F64)) return CELL_EINVAL;
  if (h->d.input_kind != CELL_INPUT_PHI || !h->drho) return CELL_EINVAL;
  if (!h->solved) return CELL_ESTATE;
  const cell::SensParams P = sens_params(h, dC, de, dk);
  run_sensitivity<double>(h, P, h->gtmp);
  if (dtype == CELL_F32)
    cell::chain_phi<float>(h->gtmp, h->drho, h->nx, h->ny, h->nz, static_cast<float*>(g), h->st);
  else
    cell::chain_phi<double>(h->gtmp, h->drho, h->nx, h->ny, h->nz, static_cast<double*>(g), h->st);
  CK(cudaGetLastError());
  return CELL_OK;
}

namespace {
// 6x6 inverse by Gauss-Jordan with partial pivoting; false if singular.
bool inverse6(const double* C, double* Inv) {
  double S[36];
  std::memcpy(S, C, sizeof(S));
  for (int i = 0; i < 36; ++i) Inv[i] = 0.0;
  for (int i = 0; i < 6; ++i) Inv[i * 6 + i] = 1.0;
  for (int k = 0; k < 6; ++k) {
    int p = k;
    for (int i = k + 1; i < 6; ++i)
      if (std::fabs(S[i * 6 + k]) > std::fabs(S[p * 6 + k])) p = i;
    if (!(std::fabs(S[p * 6 + k]) > 0.0)) return false;
    for (int j = 0; j < 6; ++j) {
      std::swap(S[k * 6 + j], S[p * 6 + j]);
      std::swap(Inv[k * 6 + j], Inv[p * 6 + j]);
    }
    const double piv = S[k * 6 + k];
    for (int j = 0; j < 6; ++j) {
      S[k * 6 + j] /= piv;
      Inv[k * 6 + j] /= piv;
    }
    for (int i = 0; i < 6; ++i) {
      if (i == k) continue;
      const double f = S[i * 6 + k];
      for (int j = 0; j < 6; ++j) {
        S[i * 6 + j] -= f * S[k * 6 + j];
        Inv[i * 6 + j] -= f * Inv[k * 6 + j];
      }
    }
  }
  return true;
}
}  // namespace

int cell_figure(int which, const double C[36], const double e[18], double* value, double dC[36],
                double de[18]) {
  if (!C || !value) return CELL_EINVAL;
  if (which == CELL_FIG_DH && !e) return CELL_EINVAL;
  if (which < CELL_FIG_DH || which > CELL_FIG_CZZZZ) return CELL_EINVAL;
  if (de)
    for (int i = 0; i < 18; ++i) de[i] = 0.0;
  if (dC)
    for (int i = 0; i < 36; ++i) dC[i] = 0.0;
  if (which == CELL_FIG_BVOIGT) {  // C_iijj / 9: the normal-normal block of Voigt C
    double v = 0.0;
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q) {
        v += C[p * 6 + q];
        if (dC) dC[p * 6 + q] = 1.0 / 9.0;
      }
    *value = v / 9.0;
    return CELL_OK;
  }
  if (which == CELL_FIG_CZZZZ) {  // poling-direction stiffness C_33 (Voigt)
    *value = C[2 * 6 + 2];
    if (dC) dC[2 * 6 + 2] = 1.0;
    return CELL_OK;
  }
  double S[36];
  if (!inverse6(C, S)) return CELL_EINVAL;
  // m = (1,1,1,0,0,0); w = S m, wt = S^T m
  double w[6], wt[6];
  for (int i = 0; i < 6; ++i) {
    w[i] = S[i * 6 + 0] + S[i * 6 + 1] + S[i * 6 + 2];
    wt[i] = S[0 * 6 + i] + S[1 * 6 + i] + S[2 * 6 + i];
  }
  if (which == CELL_FIG_BREUSS) {  // 1 / S_iijj; d(m.S m) = -(S^T m)(S m)^T : dC
    const double sm = w[0] + w[1] + w[2];
    if (!(sm != 0.0)) return CELL_EINVAL;
    *value = 1.0 / sm;
    if (dC)
      for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) dC[i * 6 + j] = wt[i] * w[j] / (sm * sm);
    return CELL_OK;
  }
  // d_h = e_3 . S m, d = e S
  double se3[6];
  for (int i = 0; i < 6; ++i) {
    double t = 0.0;
    for (int j = 0; j < 6; ++j) t += S[j * 6 + i] * e[12 + j];
    se3[i] = t;   // (S^T e_3)_i
  }
  double v = 0.0;
  for (int p = 0; p < 6; ++p) v += e[12 + p] * w[p];
  *value = v;
  if (dC)
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) dC[i * 6 + j] = -se3[i] * w[j];
  if (de)
    for (int p = 0; p < 6; ++p) de[12 + p] = w[p];
  return CELL_OK;
}

int cell_dh(const double C[36], const double e[18], double* dh, double dC[36], double de[18]) {
  return cell_figure(CELL_FIG_DH, C, e, dh, dC, de);
}

int cell_get_solution(cell_handle* h, double* out) {
  if (!h || !out) return CELL_EINVAL;
  CK(cudaMemcpyAsync(out, h->x64, 9 * 4 * h->nn * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  return CELL_OK;
}

int cell_apply(cell_handle* h, const void* x, void* y, int nrhs, int dtype) {
  if (!h || !x || !y || nrhs < 1 || nrhs > 65535) return CELL_EINVAL;
  const i64 len = 4 * h->nn;
  if (dtype == CELL_F32) {
    cell::ApplyArgs<float> a{};
    a.x = static_cast<const float*>(x); a.xs = len; a.y = static_cast<float*>(y); a.ys = len;
    a.alpha = 1.f; a.rho = h->rho32; a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    a.cslot1 = h->cslot1;   // the kernels the solver runs
    cell::FixedMat<float, 4> M;
    for (int i = 0; i < 1024; ++i) M.k[i] = (float)h->K0[i];
    cell::apply_full<float>(a, M, cell::AM_LINEAR, nrhs, h->st);
  } else if (dtype == CELL_F64) {
    cell::ApplyArgs<double> a{};
    a.x = static_cast<const double*>(x); a.xs = len; a.y = static_cast<double*>(y); a.ys = len;
    a.alpha = 1.0; a.rho = h->rho64; a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    cell::FixedMat<double, 4> M;
    std::memcpy(M.k, h->K0, sizeof(M.k));
    cell::apply_full<double>(a, M, cell::AM_LINEAR, nrhs, h->st);
  } else if (dtype == CELL_F32_TC) {
    if (!h->tc_ok) return CELL_EINVAL;
    cell::ApplyArgs<float> a{};
    a.x = static_cast<const float*>(x); a.xs = len; a.y = static_cast<float*>(y); a.ys = len;
    a.alpha = 1.f; a.rho = h->rho32; a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    cell::apply_tc_full(a, h->tct, nrhs, h->tc_err, h->st);
  } else if (dtype == CELL_F64_DF) {
    if (nrhs > 9) return CELL_EINVAL;
    cell::split_f64(static_cast<const double*>(x), h->xh, h->xl, (i64)nrhs * len, h->st);
    cell::resid_df(h->xh, h->xl, len, nullptr, 0, static_cast<double*>(y), len, h->rho32, h->rho_l,
                   h->DF, h->nx, h->ny, h->nz, nrhs, nullptr, h->st);
  } else {
    return CELL_EINVAL;
  }
  CK(cudaGetLastError());
  return CELL_OK;
}

int cell_set_tile(cell_handle* h, int block, int xt, int L) {
  if (!h || (block != CELL_BLOCK_A && block != CELL_BLOCK_SBAR)) return CELL_EINVAL;
  if (!h->nc_ok || h->d.opt.precision != CELL_MIXED_FP32 || h->d.opt.tensor_cores < 1) return CELL_EINVAL;
  const int xmax = h->nx >= 32 ? 32 : ((h->nx + 7) / 8) * 8;
  const bool dflt = xt == 0 && L == 0;
  if (!dflt && (!(xt == 8 || xt == 16 || xt == 32) || xt > xmax || L < 1)) return CELL_EINVAL;
  const int kind = block == CELL_BLOCK_A ? cell::NK_UU : cell::NK_SS4;
  h->nct[kind] = cell::NcTile{xt, L};
  h->nct_us[kind] = 0.f;
  return CELL_OK;
}

int cell_set_stencil_rg(cell_handle* h, int block, int level, int rg) {
  if (!h || (block != CELL_BLOCK_A && block != CELL_BLOCK_SBAR)) return CELL_EINVAL;
  if (h->d.opt.precision != CELL_MIXED_FP32 || !(rg == 0 || rg == 1 || rg == 3 || rg == 9)) return CELL_EINVAL;
  auto& lv = block == CELL_BLOCK_A ? h->kf.mgu.lv : h->kf.mgp.lv;
  if (level < 1 || level >= (int)lv.size()) return CELL_EINVAL;
  lv[level].rg = rg;
  return CELL_OK;
}

int cell_apply_block(cell_handle* h, int block, const void* x, void* y, int nrhs, int dtype) {
  if (!h || !x || !y || nrhs < 1 || nrhs > 65535) return CELL_EINVAL;
  if (block != CELL_BLOCK_A && block != CELL_BLOCK_SBAR) return CELL_EINVAL;
  const int nc = block == CELL_BLOCK_A ? 3 : 1;
  const i64 len = nc * h->nn;
  if (dtype == CELL_F32 || dtype == CELL_F32_TC) {
    cell::ApplyArgs<float> a{};
    a.x = static_cast<const float*>(x); a.xs = len; a.y = static_cast<float*>(y); a.ys = len;
    a.alpha = 1.f; a.rho = h->rho32; a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    a.cslot1 = h->cslot1;   // the kernels the solver runs
    if (dtype == CELL_F32_TC) {
      if (!h->nc_ok) return CELL_EINVAL;
      const int kind = nc == 3 ? cell::NK_UU : cell::NK_SS4;
      if (!cell::apply_nc(kind, a, h->ncb + cell::nc_table_floats() * kind, cell::AM_LINEAR, nrhs,
                          h->tc_err, h->st, h->nct[kind]))
        return CELL_EINVAL;
    } else if (nc == 3) {
      cell::FixedMat<float, 4> M;
      for (int i = 0; i < 1024; ++i) M.k[i] = (float)h->K0[i];
      cell::apply_uu<float>(a, M, cell::AM_LINEAR, nrhs, h->st);
    } else {
      cell::FixedMat<float, 1> M;
      for (int i = 0; i < 64; ++i) M.k[i] = (float)h->S0[i];
      cell::apply_ss<float>(a, M, cell::AM_LINEAR, nrhs, h->st);
    }
  } else if (dtype == CELL_F64) {
    cell::ApplyArgs<double> a{};
    a.x = static_cast<const double*>(x); a.xs = len; a.y = static_cast<double*>(y); a.ys = len;
    a.alpha = 1.0; a.rho = h->rho64; a.nx = h->nx; a.ny = h->ny; a.nz = h->nz;
    if (nc == 3) {
      cell::FixedMat<double, 4> M;
      std::memcpy(M.k, h->K0, sizeof(M.k));
      cell::apply_uu<double>(a, M, cell::AM_LINEAR, nrhs, h->st);
    } else {
      cell::FixedMat<double, 1> M;
      std::memcpy(M.k, h->S0, sizeof(M.k));
      cell::apply_ss<double>(a, M, cell::AM_LINEAR, nrhs, h->st);
    }
  } else {
    return CELL_EINVAL;
  }
  CK(cudaGetLastError());
  return CELL_OK;
}

int cell_rhs(cell_handle* h, double* out) {
  if (!h || !out) return CELL_EINVAL;
  cell::RhsParams RP;
  std::memcpy(RP.F, h->F, sizeof(RP.F));
  cell::rhs9(h->rho64, RP, 0x1FF, out, h->nx, h->ny, h->nz, h->st);
  CK(cudaGetLastError());
  return CELL_OK;
}

int cell_get_rho(cell_handle* h, double* out) {
  if (!h || !out) return CELL_EINVAL;
  CK(cudaMemcpyAsync(out, h->rho64, h->nn * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  return CELL_OK;
}

int cell_element_matrices(const cell_desc* d, double K0[1024], double S0[64]) {
  if (!d || !K0 || !S0 || d->nx < 1 || d->ny < 1 || d->nz < 1) return CELL_EINVAL;
  double Cn[36], en[18], kn[9], C0, k0;
  cellhost::nondimensionalise(d->C, d->e, d->kappa, Cn, en, kn, &C0, &k0);
  const double hh[3] = {1.0 / d->nx, 1.0 / d->ny, 1.0 / d->nz};
  cellhost::element_matrix(Cn, en, kn, hh, K0);
  if (cellhost::local_schur(K0, d->opt.schur_shift, S0) != 0) return CELL_EINVAL;
  return CELL_OK;
}

void cell_destroy(cell_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  forget_batch(h);
  h->free_graphs();
  cell::cslot_release(h->cslot1);
  h->arena.release();
  if (h->gstat) cudaFreeHost(h->gstat);
  delete h;
}

const char* cell_status_str(int s) {
  switch (s) {
    case CELL_OK: return "ok";
    case CELL_EINVAL: return "invalid argument";
    case CELL_ENOMEM: return "out of device memory";
    case CELL_ENOTCONV: return "solver did not reach the tolerance";
    case CELL_ETIMEOUT: return "bounded device wait expired";
    case CELL_ECUDA: return "CUDA runtime error";
    case CELL_ESTATE: return "call out of order";
    default: return "unknown status";
  }
}

const char* cell_last_error(void) { return g_last_error.c_str(); }

long long cell_launch_count(void) { return cell::g_launches.load(); }

}  // extern "C"
