// Device-side control of a whole solve captured as one CUDA graph.
//
// The FP64 refinement loop of the mixed (or plain FP64) solve is a WHILE
// conditional node; each restarted GMRES cycle inside it is a chain of IF
// conditional nodes, one per Arnoldi index.  The decisions the host loop
// takes between launches (which loads still need work, the absolute inner
// tolerances, whether the refinement cap is reached, whether any load is
// still active after an Arnoldi step) are taken by the small kernels below,
// which set the conditions with cudaGraphSetConditional; the host launches
// the graph once per solve and reads the statistics once at the end.
#include "cell.h"
#include "kernels.cuh"

namespace cell {

namespace {

// Refinement control, one warp (lane q = load q).  Mirrors the host loop:
// relative residual per load, want = selected and above max(tol |b|, floor),
// inner absolute tolerance max(inner |r|, tol |b| / 2); stop (condition 0)
// with CELL_OK when no load wants work, with CELL_ENOTCONV at the refinement
// or iteration cap, else start one more cycle (condition 1, refine += 1).
__global__ void k_refine_ctl(const double* bn2, const double* rn2, const double* bfloor, CtlParams P,
                             int* want, double* tolabs, double* relres, const int* iters, int* ctl,
                             cudaGraphConditionalHandle cond) {
  const int q = threadIdx.x;
  bool w = false;
  int it = 0;
  if (q < 9) {
    const double bn = sqrt(fmax(bn2[q * kNvMax], 0.0)), rn = sqrt(fmax(rn2[q * kNvMax], 0.0));
    relres[q] = bn > bfloor[q] ? rn / bn : 0.0;
    w = ((P.mask >> q) & 1) && rn > fmax(P.tol * bn, bfloor[q]);
    want[q] = w ? 1 : 0;
    tolabs[q] = fmax(P.inner * rn, 0.5 * P.tol * bn);
    it = iters[q];
  }
  const unsigned anyw = __ballot_sync(0xffffffffu, w);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) it = max(it, __shfl_xor_sync(0xffffffffu, it, o));
  if (q == 0) {
    unsigned c = 0;
    if (!anyw) {
      ctl[1] = CELL_OK;
    } else if (ctl[0] >= P.max_refine || it >= P.max_iter) {
      ctl[1] = CELL_ENOTCONV;
    } else {
      c = 1;
      ctl[0] += 1;
    }
    cudaGraphSetConditional(cond, c);
  }
}

// Start of a cycle: ran = active, and the IF conditions of the Arnoldi steps
// (step 0 runs if any load is active, the others are set by their
// predecessors).
__global__ void k_cycle_handles(const int* active, int* ran, const IterHandles H) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int q = 0; q < 9; ++q) {
    ran[q] = active[q];
    any |= active[q];
  }
  cudaGraphSetConditional(H.h[0], any ? 1u : 0u);
  for (int j = 1; j < H.m; ++j) cudaGraphSetConditional(H.h[j], 0u);
}

__global__ void k_next_step(const int* active, cudaGraphConditionalHandle next) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int q = 0; q < 9; ++q) any |= active[q];
  cudaGraphSetConditional(next, any ? 1u : 0u);
}

// End of a cycle: iteration counts of the loads that ran, and the number of
// Arnoldi steps the graph executed (the largest count).
__global__ void k_accum_iters(int* iters, const int* kcount, const int* ran, int* ctl) {
  if (threadIdx.x != 0) return;
  int mx = 0;
  for (int q = 0; q < 9; ++q)
    if (ran[q]) {
      iters[q] += kcount[q];
      mx = max(mx, kcount[q]);
    }
  ctl[2] += mx;
}

__global__ void k_ctl_reset(int* ctl, int* iters) {
  const int q = threadIdx.x;
  if (q < 9) iters[q] = 0;
  if (q < 4) ctl[q] = 0;
}

__global__ void k_copy_scale(const double* __restrict__ r, double* __restrict__ v, i64 len,
                             const double* __restrict__ sc, const int* active) {
  const int q = blockIdx.y;
  if (active && !active[q]) return;
  const double f = sc[q];
  for (i64 k = (i64)blockIdx.x * blockDim.x + threadIdx.x; k < len; k += (i64)gridDim.x * blockDim.x)
    v[q * len + k] = r[q * len + k] * f;
}

}  // namespace

void refine_ctl(const double* bn2, const double* rn2, const double* bfloor, const CtlParams& P, int* want,
                double* tolabs, double* relres, const int* iters, int* ctl, cudaGraphConditionalHandle cond,
                cudaStream_t s) {
  note_launch(), k_refine_ctl<<<1, 32, 0, s>>>(bn2, rn2, bfloor, P, want, tolabs, relres, iters, ctl, cond);
}

void cycle_handles(const int* active, int* ran, const IterHandles& H, cudaStream_t s) {
  note_launch(), k_cycle_handles<<<1, 32, 0, s>>>(active, ran, H);
}

void next_step(const int* active, cudaGraphConditionalHandle next, cudaStream_t s) {
  note_launch(), k_next_step<<<1, 32, 0, s>>>(active, next);
}

void accum_iters(int* iters, const int* kcount, const int* ran, int* ctl, cudaStream_t s) {
  note_launch(), k_accum_iters<<<1, 32, 0, s>>>(iters, kcount, ran, ctl);
}

void ctl_reset(int* ctl, int* iters, cudaStream_t s) { note_launch(), k_ctl_reset<<<1, 32, 0, s>>>(ctl, iters); }

void copy_scale_f64(const double* r, double* v, i64 len, const double* sc, int nrhs, const int* active,
                    cudaStream_t s) {
  i64 b = (len + 255) / 256;
  if (b > 4096) b = 4096;
  note_launch(), k_copy_scale<<<dim3((unsigned)b, nrhs), 256, 0, s>>>(r, v, len, sc, active);
}

}  // namespace cell
