// Host-side FP64 set-up math of the cell library: material scaling, the Q1
// element matrix, the affine macroscopic loads, the local Schur complement,
// multigrid transfer weights and small dense linear algebra.
#pragma once

namespace cellhost {

// §2.2: C0 = max|C|, k0 = max|kappa|; C/C0, e/sqrt(C0 k0), kappa/k0.
void nondimensionalise(const double C[36], const double e[18], const double kap[9],
                       double Cn[36], double en[18], double kn[9], double* C0, double* k0);

// 32x32 element matrix of the coupled bilinear form over a box with sides
// h[0..2]; rows/cols are local dofs 4*node + comp (comp 3 = potential).
// Blocks: [[A_e, B_e^T], [B_e, -C_e]] interleaved per node (Eq. sym-piezo).
void element_matrix(const double Cn[36], const double en[18], const double kn[9],
                    const double h[3], double K[1024]);

// 32x9 nodal values of the nine affine macroscopic fields in element-local
// coordinates (u = eps^(p) x for p < 6, phi = -x_j for load 6 + j).
void affine_loads(const double h[3], double Z[32 * 9]);

// 8x8 S0 = C_e + B_e (A_e + shift I)^-1 B_e^T from the element matrix (§2.5.3).
int local_schur(const double K[1024], double shift, double S[64]);

// Upper bound of lambda_max(diag(M)^-1 M) for a symmetric n x n matrix.
double jacobi_lmax(const double* M, int n);

// In-place inverse of a symmetric positive definite n x n matrix (Cholesky).
// Returns 0 on success, -1 if the matrix is not positive definite.
int spd_inverse(double* A, int n);

// Eigen-decomposition of a symmetric n x n matrix A (row-major, n <= 16) by
// cyclic Jacobi rotations: A = Q diag(lam) Q^T, column k of Q (Q[i*n + k])
// the eigenvector of lam[k].  A is not modified.
void sym_eig(const double* A, int n, double* lam, double* Q);

// Trilinear prolongation weight of coarse corner B for the fine local node a
// of child element c (all in 0..7, corner index = x + 2y + 4z).
double child_weight(int c, int a, int B);

}  // namespace cellhost
