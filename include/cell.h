/*
 * cell.h -- C ABI of the GB300 periodic piezoelectric unit-cell library.
 *
 * The library solves the nine periodic cell problems of linear piezoelectric
 * homogenisation (Wegert, Roberts & Challis, arXiv 2410.03148, §2.2) on a
 * structured grid of Q1 hexahedra with 4 dofs per node (u1, u2, u3, phi) and
 * a per-element ersatz scale rho_e (§2.6), by approximate-Schur-complement
 * preconditioned GMRES (§2.5.3), and reduces the solutions to the homogenised
 * tensors C^H, e^H, kappa^H (Eqs. hom_C, hom_e, hom_kappa) and to element-wise
 * sensitivities.  All device work runs in the library's own sm_103a kernels on
 * the caller's CUDA stream.
 *
 * Conventions used throughout
 * ---------------------------
 * Grid.  The unit cell [0,1)^3 is split into nx*ny*nz boxes; nodes are
 *   periodic, so there are nx*ny*nz nodes and nx*ny*nz elements.  Node and
 *   element (i,j,k) both have flat index i + nx*(j + ny*k) (x fastest).
 *   Element (i,j,k) spans nodes (i+a, j+b, k+c) mod (nx,ny,nz), a,b,c in {0,1}.
 * Tensors.  IEEE Voigt order (11,22,33,23,13,12), row-major, SI units:
 *   C[6x6] in Pa, e[3x6] in C/m^2, kappa[3x3] in F/m.  Engineering shear.
 * Loads.  Load I = 0..5 is the unit macroscopic strain of Voigt component I,
 *   I = 6..8 the unit macroscopic electric field along x, y, z (§2.2).
 * Field vectors on device ("cell vectors").  A set of nrhs nodal fields is
 *   stored component-planar: value(load r, component c, node n) at offset
 *   (r*4 + c)*N + n with N = nx*ny*nz, c in {u1,u2,u3,phi}.
 * Units inside.  The system is solved in the nondimensional variables of
 *   §2.2 (C/C0, e/sqrt(C0 k0), kappa/k0 with C0 = max|C|, k0 = max|kappa|);
 *   vectors exchanged through cell_apply / cell_rhs / cell_get_solution are
 *   in those units.  Homogenised tensors are returned in SI units.
 * Ownership.  The caller owns every pointer it passes.  cell_setup copies
 *   the design (rho or phi) into library-owned device memory, so the caller's
 *   buffer may be freed or reused after it returns.  The library owns its
 *   workspaces (allocated in cell_setup, freed in cell_destroy).
 * Streams.  Every call enqueues its device work on the stream given in the
 *   descriptor (0 = legacy default stream).  Calls that return host results
 *   (cell_solve's stats, cell_homogenise) synchronise that stream.
 * Errors.  Every int-returning call returns a cell_status.  Invalid sizes,
 *   null pointers and unknown enums give CELL_EINVAL without touching the
 *   device.  CUDA failures give CELL_ECUDA; cell_last_error() describes the
 *   most recent failure of the calling thread.
 */
#ifndef PIEZO_CELL_H
#define PIEZO_CELL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum cell_status {
  CELL_OK = 0,
  CELL_EINVAL = 1,     /* invalid argument; nothing was done */
  CELL_ENOMEM = 2,     /* device allocation failed */
  CELL_ENOTCONV = 3,   /* solver stopped before reaching tol; stats filled */
  CELL_ETIMEOUT = 4,   /* a bounded device wait expired */
  CELL_ECUDA = 5,      /* a CUDA runtime call failed (see cell_last_error) */
  CELL_ESTATE = 6      /* call out of order (e.g. homogenise before solve) */
} cell_status;

typedef enum cell_precision {
  CELL_FP64 = 0,        /* every operator, smoother and Krylov vector in FP64 */
  CELL_MIXED_FP32 = 1   /* FP32 GMRES + multigrid inside FP64 iterative refinement */
} cell_precision;

typedef enum cell_input_kind {
  CELL_INPUT_RHO = 0,   /* input = per-element ersatz scale rho_e > 0 */
  CELL_INPUT_PHI = 1    /* input = nodal level-set values; rho from §2.6 smoothing */
} cell_input_kind;

typedef enum cell_dtype {
  CELL_F32 = 0,
  CELL_F64 = 1,
  CELL_F64_DF = 2,  /* FP64 data, arithmetic in FP32 pairs (cell_apply only) */
  CELL_F32_TC = 3   /* FP32 data, TF32 tensor-core element contraction (cell_apply,
                       cell_apply_block) */
} cell_dtype;

typedef enum cell_block {
  CELL_BLOCK_A = 0,     /* elastic block A of the coupled operator */
  CELL_BLOCK_SBAR = 1   /* element-wise Schur approximation Sbar */
} cell_block;

typedef struct cell_options {
  double tol;          /* stop when ||r_I||_2 <= tol * ||b_I||_2 for every load I
                          (true residual of the nondimensional system, FP64) */
  int restart;         /* GMRES restart length m (1..64) */
  int max_iter;        /* cap on GMRES iterations per load over the whole solve */
  int precision;       /* cell_precision */
  double inner_tol;    /* MIXED: relative residual reduction asked of each FP32
                          GMRES solve inside the FP64 refinement loop */
  int max_refine;      /* MIXED: cap on FP64 refinement steps */
  int vcycles_u;       /* V-cycles approximating A^-1 (elastic block) per application */
  int vcycles_phi;     /* V-cycles approximating Sbar^-1 (Schur block) per application */
  int cheb_degree;     /* Chebyshev-Jacobi smoothing steps per pre/post smoothing */
  double cheb_lo;      /* lower end of the Chebyshev interval, as a fraction of
                          the upper end */
  double cheb_hi;      /* multiplier applied to the element-wise lambda_max bound */
  double schur_shift;  /* diagonal shift added to A_e before inverting it in
                          Sbar = sum_e C_e + B_e A_e^-1 B_e^T (§2.5.3, 1e-10) */
  int coarse_dofs;     /* stop coarsening once a level has at most this many dofs */
  int load_mask;       /* bit I set = solve load I (default 0x1FF = all nine) */
  int profile;         /* nonzero: time kernel classes with CUDA events (cell_stats) */
  int tensor_cores;    /* MIXED: 0 = SIMT FP32 applies only; 1 (default) = fine-grid smoothing
                          applies of both preconditioner blocks (A and Sbar) on tcgen05
                          tensor cores: node-centric TF32 element contraction with FP32
                          accumulation, any grid size; 2 = also the Krylov operator Ahat
                          (3xTF32 split, FP32-accurate), used where nx % 16 == 0,
                          ny % 4 == 0, nz % 2 == 0. */
  int const_bank;      /* MIXED: nonzero (default) = FP32 element matrices in one of 4
                          library-wide __constant__ slots (shared by handles with equal
                          matrices), falling back to kernel parameters if all are taken */
  int graphs;          /* 0 = direct launches, the host deciding after every GMRES
                          iteration; 1 = each GMRES iteration captured once per handle
                          into a CUDA graph (on an internal stream) and replayed on the
                          caller's stream; 2 (default) = the whole solve captured once per
                          handle into one graph whose refinement loop (a WHILE node) and
                          Arnoldi steps (IF nodes) are controlled by device kernels, so a
                          solve is one launch and one synchronisation; cell_solve_batch
                          then puts all handles' solves into one graph (one launch per
                          batch); 3 = as 2, but cell_solve_batch launches each handle's
                          graph separately on its own stream.  With profile set, 2 and 3
                          behave as 1 (event timings need the host loop).  The first
                          solve of a handle pays the capture. */
  int profile_mask;    /* with profile set: bit c (cell_prof_class) = time class c;
                          0 = every class */
  int precond;         /* CELL_PRECOND_SCP (default, §2.5.3) or CELL_PRECOND_DBP (§2.5.1) */
  int autotune;        /* MIXED with tensor_cores >= 1: nonzero (default) = at cell_setup, time
                          the tensor-core smoothers' CTA tiles (x width 8/16/32 nodes, z-chunk
                          length) on this GPU and grid and keep the fastest per block (cell_stats
                          reports them); every tile gives bitwise the same result.  0 = widest
                          tile and a wave-count heuristic.  MIXED (any tensor_cores): nonzero also
                          times the coarse levels' stencil apply with 1, 3 and 9 loads per thread
                          and keeps the fastest per level (bitwise-neutral; cell_stats.stencil_rg). */
} cell_options;

typedef enum cell_precond {
  CELL_PRECOND_SCP = 0,  /* approximate Schur complement: P = [[A, 0], [-B, Sbar]] */
  CELL_PRECOND_DBP = 1   /* diagonal blocks: P = diag(A, -C) on the symmetric form, i.e.
                            diag(A, C) on the nonsymmetric one; the potential block's
                            multigrid (and cell_apply_block CELL_BLOCK_SBAR) then uses
                            C = sum_e rho_e C_e */
} cell_precond;

typedef struct cell_desc {
  int nx, ny, nz;      /* elements (= periodic nodes) per direction, each >= 2 */
  double C[36];        /* base stiffness, Pa */
  double e[18];        /* base piezoelectric coupling, C/m^2 */
  double kappa[9];     /* base permittivity, F/m */
  int input_kind;      /* cell_input_kind */
  int input_dtype;     /* cell_dtype of *input */
  const void* input;   /* DEVICE pointer, nx*ny*nz values, x fastest */
  double rho_void;     /* PHI input: void scale (paper: small ersatz value, default 1e-3) */
  double eta;          /* PHI input: smoothing half-width in phi units; <= 0 selects
                          2*max(1/nx,1/ny,1/nz) ("within two elements", §2.6) */
  cell_options opt;
  void* stream;        /* cudaStream_t */
} cell_desc;

/* Kernel classes timed with CUDA events when cell_options.profile is set. */
typedef enum cell_prof_class {
  CELL_PROF_FULL32 = 0,    /* full operator Ahat, FP32 (GMRES) */
  CELL_PROF_FULL64 = 1,    /* full operator Ahat, FP64 (refinement residual) */
  CELL_PROF_ELASTIC0 = 2,  /* elastic block A on the fine grid (smoothing, residuals) */
  CELL_PROF_SCHUR0 = 3,    /* local-Schur block Sbar on the fine grid */
  CELL_PROF_COUPLING = 4,  /* coupling block B */
  CELL_PROF_COARSE = 5,    /* every operator apply on coarse multigrid levels */
  CELL_PROF_KRYLOV = 6,    /* Gram-Schmidt dot / update passes */
  CELL_PROF_CLASSES = 7
} cell_prof_class;

typedef struct cell_stats {
  int status;               /* cell_status of the solve */
  int iters[9];             /* GMRES iterations per load (all refinement steps) */
  int refinements;          /* FP64 restarts / refinement steps taken */
  int nlevels_u, nlevels_phi;
  double rel_residual[9];   /* final true relative residual per load (FP64) */
  double solve_ms;          /* host wall time of cell_solve */
  double class_ms[CELL_PROF_CLASSES];   /* profile: summed device time per class */
  int class_count[CELL_PROF_CLASSES];   /* profile: launches timed per class */
  long long class_units[CELL_PROF_CLASSES]; /* profile: sum over timed launches of the
                                           number of loads each launch processed */
  int tc_tile_xt[2], tc_tile_L[2];  /* tensor-core smoother tile in use per block ([0] elastic
                                       A, [1] Schur Sbar): x width in nodes and z-chunk length;
                                       0 = not tuned (default tile or SIMT path) */
  double tc_tile_us[2];             /* the tuned tile's time per 9-load Chebyshev launch, us */
  int stencil_rg[2][8];             /* MIXED: loads per thread of the coarse stencil apply per
                                       multigrid level ([0] elastic, [1] Schur; level 0 = fine
                                       grid, always 0); 0 = size default, 1/3/9 = tuned at set-up
                                       (options.autotune; bitwise-neutral) */
} cell_stats;

typedef struct cell_handle cell_handle;

/* Fill *opt with the defaults (tol 1e-10, restart 30, MIXED_FP32, ...). */
void cell_default_options(cell_options* opt);

/* Build everything that depends only on the design (S1 of the hot path):
 * nondimensionalise the material, form the 32x32 element matrix K0 by 2x2x2
 * Gauss integration and the 8x8 local Schur complement S0 (§2.5.3), map the
 * design to rho_e on the device (smoothed Heaviside of the element-mean level
 * set for PHI input), and build the multigrid hierarchies of both
 * preconditioner blocks (Galerkin coarse element matrices, Jacobi diagonals,
 * Chebyshev bounds, coarsest dense inverse).  On success *out receives a new
 * handle.  Errors: CELL_EINVAL for sizes < 2, NaN/non-positive tolerances,
 * unknown enums or null pointers; CELL_ENOMEM; CELL_ECUDA. */
int cell_setup(const cell_desc* d, cell_handle** out);

/* Replace the design of an existing handle (same grid, material, input kind
 * and dtype as at cell_setup; input is a DEVICE pointer of nx*ny*nz values)
 * and rebuild everything that depends on it (rho_e, multigrid numerics)
 * without allocating: the repeated S1 of an optimisation loop.  Invalidates
 * the previous solution.  CELL_EINVAL for null pointers or invalid rho. */
int cell_update(cell_handle* h, const void* input);

/* Solve the selected cell problems (§2.2) for the design of the handle:
 * assemble b = -sum_e rho_e P_e^T K0 Zbar_e (negated potential rows, the
 * nonsymmetric form of Eq. (sym-piezo)), run right-preconditioned SCP-GMRES
 * (§2.5.3, flexible variant: the preconditioned directions are stored, so
 * reduced-precision smoothers may vary between iterations), and project the null space (mean displacement and potential) out
 * of the solutions.  st may be NULL.  Returns CELL_ENOTCONV (with stats and a
 * usable best solution) if tol was not reached within max_iter/max_refine. */
int cell_solve(cell_handle* h, cell_stats* st);

/* cell_solve for n distinct handles (cells of any sizes and options).
 * If every handle runs whole-solve graphs with graphs = 2 (no profiling) on
 * one device, the n solves are built into ONE executable CUDA graph, each an
 * independent branch with its own device-controlled refinement loop and
 * Arnoldi steps, and the batch is a single graph launch on hs[0]'s stream
 * (ordered after the work queued on every handle's stream; every handle's
 * stream is ordered after the batch).  The graph of the last batch is kept
 * and relaunched while the same handles are passed in the same order; the
 * first call of a new list pays the capture.  With graphs = 3 on every handle
 * (or handles on several devices), the calling thread launches one graph per
 * handle on the handle's stream; otherwise up to 16 host threads drive one
 * handle each.  Results are bitwise those of cell_solve on each handle.
 * st: NULL or n stats (st[i].status holds handle i's result).  Returns
 * CELL_OK, or the status of the first handle (in list order) that failed;
 * CELL_EINVAL for a NULL list entry or a handle listed twice (nothing solved).
 * Not thread-safe for handles shared between concurrent calls. */
int cell_solve_batch(cell_handle** hs, int n, cell_stats* st);

/* Homogenised tensors of the last solve (Eqs. hom_C, hom_e, hom_kappa with
 * Vol(D) = 1), in SI units, written to host arrays CH[36], eH[18], kH[9].
 * Computed in FP64 in the energy form H_IJ = sum_e rho_e W_e^I.K0 W_e^J
 * (W = total nodal field), whose error is quadratic in the solve error.
 * Needs all nine loads; CELL_ESTATE before a successful solve. */
int cell_homogenise(cell_handle* h, double CH[36], double eH[18], double kH[9]);

/* Element-wise sensitivities of L = sum dC.C^H + de.e^H + dk.kappa^H with
 * respect to rho_e (the adjoint states are the cell solutions themselves, as
 * the energy form is stationary in the fluctuations).  dC[36], de[18], dk[9]
 * are host arrays (any may be NULL = zero).  g is a DEVICE array of nx*ny*nz
 * values of dtype (CELL_F32 or CELL_F64), element-indexed.  The per-element
 * quadratic forms are evaluated in the dtype given.  CELL_ESTATE before a
 * successful solve. */
int cell_sensitivity(cell_handle* h, const double dC[36], const double de[18],
                     const double dk[9], void* g, int dtype);

/* Element-wise change of the same weighted energy between the solutions of two
 * handles on one grid and material: g_e = sum_IJ G_IJ (W_h^I.K0 W_h^J -
 * W_ref^I.K0 W_ref^J), G from dC, de, dk as in cell_sensitivity (no rho_e
 * factor).  It is evaluated in FP64 as B(W_h + W_ref, W_h - W_ref) of the
 * symmetric form B (polarisation), so its rounding scales with the difference
 * of the two fields rather than with the energies: central differences of
 * the homogenised tensors between nearby designs (sum_e rho_e g_e, with the
 * changed rho of the perturbed element handled by the caller) keep their
 * digits at small steps.  g: DEVICE array of nx*ny*nz doubles, written on h's
 * stream (ref's stream is synchronised first if it differs).  CELL_EINVAL for
 * different grids or materials, ref == h, or a restart length too short for
 * the workspace; CELL_ESTATE unless both handles hold a solution. */
int cell_energy_difference(cell_handle* h, const cell_handle* ref, const double dC[36],
                           const double de[18], const double dk[9], double* g);

/* Shape sensitivity on the level set: dL/dphi_n at every node (device
 * buffer g of nx*ny*nz values, node = i + nx*(j + ny*k), dtype CELL_F32 or
 * CELL_F64) for the same L as cell_sensitivity.  With the ersatz map of §2.6,
 * rho_e = 1 - (1 - rho_void) H_eta(phi_e) and phi_e the mean of the element's
 * 8 nodal values, the chain rule gives dL/dphi_n = sum over the 8 elements
 * around n of (dL/drho_e) (drho_e/dphi_e) / 8 (element sensitivities in
 * FP64).  Only for handles set up with CELL_INPUT_PHI (else CELL_EINVAL);
 * CELL_ESTATE before a successful solve. */
int cell_sensitivity_phi(cell_handle* h, const double dC[36], const double de[18],
                         const double dk[9], void* g, int dtype);

/* One explicit time step of the level-set evolution phi_t + v |grad phi| = 0
 * (Eq. HJ, §2.1) on the periodic nx*ny*nz node grid of the unit cell
 * (spacing 1/nx, 1/ny, 1/nz): out = phi - dt (max(v,0) |grad phi|+ +
 * min(v,0) |grad phi|-) with first-order Godunov upwind gradients.  phi, v,
 * out: device arrays of nx*ny*nz values (node = i + nx*(j + ny*k)), dtype
 * CELL_F32 or CELL_F64; out must not alias phi.  Stable for
 * dt max|v| (nx + ny + nz) <= 1.  No handle needed; asynchronous on stream
 * (NULL = legacy default stream).  CELL_EINVAL for bad sizes or pointers. */
int cell_hj_step(const void* phi, const void* v, int nx, int ny, int nz, double dt, void* out, int dtype,
                 void* stream);

/* Shape velocity for Eq. HJ by Hilbertian extension-regularisation and
 * projection (§2.6: the paper uses the Hilbertian projection method for
 * constrained optimisation and gives no formulas; this is the library's
 * reading).  Inner product <u, v>_H = int alpha^2 grad u.grad v + u v on the
 * periodic unit cell, discretised with the Q1 node basis (A = alpha^2 K + M).
 * Inputs are nodal sensitivities (dual vectors, e.g. from
 * cell_sensitivity_phi): dJ of the objective and dC[i] of ncons <= 8
 * constraints with current values C[i].  With g = A^-1 d their Riesz
 * representers, theta_k an H-orthonormal basis of the constraint
 * representers (Gram-Schmidt, g_i = sum_k R_ki theta_k) and P g_J the
 * objective representer made H-orthogonal to them, the velocity is
 *   v = wJ P g_J / ||P g_J||_H + sum_k mu_k theta_k,   R^T mu = wC C,
 * so that a step phi -= dt v |grad phi| lowers J to first order and moves each
 * constraint by -dt wC C_i.  dJ, dC[i] (a HOST array of DEVICE pointers) and v
 * are DEVICE arrays of nx*ny*nz doubles (node = i + nx*(j + ny*k)); C is host.
 * info (host, may be NULL) receives ||P g_J||_H, the Chebyshev iterations used
 * and mu_1..mu_ncons.  Uses the handle's grid, stream and Krylov workspace (so
 * not concurrently with a solve of the same handle); synchronises the stream.
 * CELL_EINVAL for alpha <= 0, null pointers, ncons > 8 or linearly dependent
 * constraint sensitivities. */
int cell_hilbert_velocity(cell_handle* h, double alpha, const double* dJ, const double* const* dC,
                          const double* C, int ncons, double wJ, double wC, double* v, double* info);

/* Hydrostatic strain coefficient d_h = d31 + d32 + d33 with d = e S, S = C^-1
 * (§2.3), and its gradient with respect to every entry of C (dC[36]) and
 * e (de[18]).  Host-only helper; dC/de may be NULL.  CELL_EINVAL if C is
 * singular. */
int cell_dh(const double C[36], const double e[18], double* dh, double dC[36], double de[18]);

/* Figures of merit of §2.3 on homogenised tensors (SI, Voigt order, host
 * FP64) and their gradients with respect to every entry of C (dC[36]) and e
 * (de[18]); dC/de may be NULL, e may be NULL except for CELL_FIG_DH.
 *   CELL_FIG_DH     d_h = d_zxx + d_zyy + d_zzz, d = e S, S = C^-1 (= cell_dh)
 *   CELL_FIG_BVOIGT B_Voigt = C_iijj / 9
 *   CELL_FIG_BREUSS B_Reuss = 1 / S_iijj
 *   CELL_FIG_CZZZZ  C_zzzz (stiffness along the poling direction, C_33)
 * The gradients are the upstream dC/de of cell_sensitivity for these
 * objectives.  CELL_EINVAL for an unknown figure or a singular C. */
typedef enum cell_figure_kind {
  CELL_FIG_DH = 0,
  CELL_FIG_BVOIGT = 1,
  CELL_FIG_BREUSS = 2,
  CELL_FIG_CZZZZ = 3
} cell_figure_kind;
int cell_figure(int which, const double C[36], const double e[18], double* value, double dC[36],
                double de[18]);

/* Copy the solutions (total fluctuation fields, loads in order 0..8 whether or
 * not solved) as FP64 cell vectors into the DEVICE buffer out (9*4*N values). */
int cell_get_solution(cell_handle* h, double* out);

/* y = Ahat x for nrhs cell vectors (device pointers, dtype CELL_F32 or
 * CELL_F64): the assembled nonsymmetric operator of Eq. (sym-piezo) second
 * form, sum_e rho_e P_e^T K0 P_e x with the potential rows negated.
 * CELL_F64_DF: FP64 vectors (nrhs <= 9), evaluated with the FP32 double-float
 * kernel that the mixed solver uses for its FP64-grade residuals (error-free
 * FMA products, TwoSum accumulation); it overwrites the handle's internal
 * split-iterate buffers, so call it only between solves.
 * CELL_F32_TC: FP32 vectors through the tcgen05 tensor-core kernel (TF32
 * inputs, FP32 accumulation); CELL_EINVAL if the grid does not tile into
 * 16 x 4 x 2 node bricks. */
int cell_apply(cell_handle* h, const void* x, void* y, int nrhs, int dtype);

/* Preconditioner blocks of P_SCP (§2.5.3) on the finest grid: y = A x with
 * block CELL_BLOCK_A (the elastic block of Eq. (sym-piezo), sum_e rho_e A_e,
 * 3 components per node) or y = Sbar x with CELL_BLOCK_SBAR (sum_e rho_e S0,
 * S0 = C_e + B_e (A_e + shift I)^-1 B_e^T, 1 component).  x, y: device,
 * nrhs vectors of [comp][node] (3nn or nn values each), not aliased.
 * dtype CELL_F32 / CELL_F64: SIMT; CELL_F32_TC: the node-centric tensor-core
 * kernel used by the smoothers (TF32 inputs, FP32 accumulation; any grid
 * size).  Asynchronous on the handle's stream. */
int cell_apply_block(cell_handle* h, int block, const void* x, void* y, int nrhs, int dtype);

/* Set the CTA tile of the tensor-core smoother of one block (cell_block) for
 * the rest of the handle's life, replacing the one cell_setup tuned or chose:
 * xt = nodes along x per CTA (8, 16 or 32, at most nx rounded up to a multiple
 * of 8), L = z-planes per CTA chunk (>= 1; values above nz act as nz); xt = L
 * = 0 restores the default tile.  Results do not depend on the tile (each
 * node's tensor-core sequence and epilogue arithmetic are the same); it
 * changes launch geometry and speed only.  Takes effect for later launches; a solve graph
 * captured before the call keeps the tile it was captured with.  Errors:
 * CELL_EINVAL for a null handle, an unknown block, a tile outside those ranges,
 * or a handle without the tensor-core path (FP64 precision, tensor_cores = 0
 * or a grid it does not support). */
int cell_set_tile(cell_handle* h, int block, int xt, int L);

/* Set the loads per thread (rg = 1, 3 or 9; 0 = the size default) of the
 * assembled-stencil apply on multigrid level `level` (>= 1) of one block
 * (cell_block), replacing the value cell_setup tuned.  Results do not depend
 * on rg (every (node, load) runs the same operation sequence); it changes
 * launch geometry and speed only.  Takes effect for later launches; a solve
 * graph captured before the call keeps the value it was captured with.
 * Levels small enough for the four-lane stencil kernel ignore it.  Errors:
 * CELL_EINVAL for a null handle, an unknown block, a level outside
 * 1 .. levels-1, an rg not in {0, 1, 3, 9}, or FP64 precision. */
int cell_set_stencil_rg(cell_handle* h, int block, int level, int rg);

/* The nine right-hand sides bhat = S_phi (-sum_e rho_e P_e^T K0 Zbar_e^I) as
 * FP64 cell vectors into the DEVICE buffer out (9*4*N values). */
int cell_rhs(cell_handle* h, double* out);

/* The per-element scale rho_e the handle uses, FP64, into DEVICE out (N values). */
int cell_get_rho(cell_handle* h, double* out);

/* Host: the nondimensional 32x32 element matrix K0 (row-major, local dof
 * 4*n + c, local node n = a + 2b + 4c at corner (a,b,c)) and the 8x8 local
 * Schur complement S0 for the material and grid of d (d->input unused). */
int cell_element_matrices(const cell_desc* d, double K0[1024], double S0[64]);

/* Homogenised tensors like cell_homogenise, but from fields the caller passes
 * and without allocating any device memory (the paper has no counterpart).
 * It serves callers that cannot allocate when they need the tensors: a
 * framework whose caching allocator owns the device-memory budget and forbids
 * allocation outside its pools, or a real-time loop that must not stall on
 * the driver's allocator (cudaMalloc may synchronise the device).
 * d gives the grid, material and stream (d->input and d->opt are unused).
 * rho: N element scales; bhat, y, rhat: 9 FP64 cell vectors each (9*4*N
 * values): the right-hand sides as from cell_rhs, the solutions as from
 * cell_get_solution, and the residuals bhat - Ahat y; all DEVICE pointers on
 * the current device, which must also own d->stream (else CELL_EINVAL).
 * Block partial sums live in one fixed device array inside the library
 * (83,195 doubles = 665,560 bytes, held on every GPU that loads it until the
 * process exits), shared by all calls: calls that overlap on the GPU race and
 * must be ordered (e.g. issued on one stream).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress).  The call copies
 * its three reductions to the host and synchronises d->stream before it
 * returns.  CELL_EINVAL for null pointers, sizes < 2, or more than 4,194,304
 * nodes; CELL_ECUDA if a launch or copy fails. */
int cell_homogenise_noalloc(const cell_desc* d, const double* rho, const double* bhat,
                            const double* y, const double* rhat, double CH[36], double eH[18],
                            double kH[9]);

/* Number of kernels this library has launched in the calling process so far
 * (all handles, all threads); lets a caller count the launches of a region. */
long long cell_launch_count(void);

void cell_destroy(cell_handle* h);
const char* cell_status_str(int status);
const char* cell_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PIEZO_CELL_H */
