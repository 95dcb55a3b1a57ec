// Host-side FP64 set-up math (see hostmath.h).
#include "hostmath.h"

#include <cmath>
#include <cstring>
#include <vector>

namespace cellhost {

void nondimensionalise(const double C[36], const double e[18], const double kap[9],
                       double Cn[36], double en[18], double kn[9], double* C0, double* k0) {
  double c0 = 0.0, q0 = 0.0;
  for (int i = 0; i < 36; ++i) c0 = std::fmax(c0, std::fabs(C[i]));
  for (int i = 0; i < 9; ++i) q0 = std::fmax(q0, std::fabs(kap[i]));
  const double se = std::sqrt(c0 * q0);
  for (int i = 0; i < 36; ++i) Cn[i] = C[i] / c0;
  for (int i = 0; i < 18; ++i) en[i] = e[i] / se;
  for (int i = 0; i < 9; ++i) kn[i] = kap[i] / q0;
  *C0 = c0;
  *k0 = q0;
}

// Material matrix over (engineering Voigt strain, grad phi):
// D = [[C, e^T], [e, -kappa]]; see the bilinear form of §2.2.
static void material_matrix(const double Cn[36], const double en[18], const double kn[9],
                            double D[81]) {
  std::memset(D, 0, sizeof(double) * 81);
  for (int p = 0; p < 6; ++p)
    for (int q = 0; q < 6; ++q) D[p * 9 + q] = Cn[p * 6 + q];
  for (int i = 0; i < 3; ++i)
    for (int p = 0; p < 6; ++p) {
      D[(6 + i) * 9 + p] = en[i * 6 + p];
      D[p * 9 + 6 + i] = en[i * 6 + p];
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D[(6 + i) * 9 + 6 + j] = -kn[i * 3 + j];
}

void element_matrix(const double Cn[36], const double en[18], const double kn[9],
                    const double h[3], double K[1024]) {
  double D[81];
  material_matrix(Cn, en, kn, D);
  std::memset(K, 0, sizeof(double) * 1024);
  const double g = 0.5 / std::sqrt(3.0);
  const double pts[2] = {0.5 - g, 0.5 + g};
  const double w = h[0] * h[1] * h[2] / 8.0;
  for (int qz = 0; qz < 2; ++qz)
    for (int qy = 0; qy < 2; ++qy)
      for (int qx = 0; qx < 2; ++qx) {
        const double xi[3] = {pts[qx], pts[qy], pts[qz]};
        // physical gradients of the 8 trilinear shape functions
        double dN[8][3];
        for (int n = 0; n < 8; ++n) {
          const int c[3] = {n & 1, (n >> 1) & 1, (n >> 2) & 1};
          double f[3], d[3];
          for (int k = 0; k < 3; ++k) {
            f[k] = c[k] ? xi[k] : 1.0 - xi[k];
            d[k] = c[k] ? 1.0 : -1.0;
          }
          dN[n][0] = d[0] * f[1] * f[2] / h[0];
          dN[n][1] = f[0] * d[1] * f[2] / h[1];
          dN[n][2] = f[0] * f[1] * d[2] / h[2];
        }
        // B: 9 x 32 (rows: e11 e22 e33 g23 g13 g12 phi_x phi_y phi_z)
        double B[9][32];
        std::memset(B, 0, sizeof(B));
        for (int n = 0; n < 8; ++n) {
          const int o = 4 * n;
          B[0][o + 0] = dN[n][0];
          B[1][o + 1] = dN[n][1];
          B[2][o + 2] = dN[n][2];
          B[3][o + 1] = dN[n][2];
          B[3][o + 2] = dN[n][1];
          B[4][o + 0] = dN[n][2];
          B[4][o + 2] = dN[n][0];
          B[5][o + 0] = dN[n][1];
          B[5][o + 1] = dN[n][0];
          B[6][o + 3] = dN[n][0];
          B[7][o + 3] = dN[n][1];
          B[8][o + 3] = dN[n][2];
        }
        double DB[9][32];
        for (int p = 0; p < 9; ++p)
          for (int a = 0; a < 32; ++a) {
            double s = 0.0;
            for (int q = 0; q < 9; ++q) s += D[p * 9 + q] * B[q][a];
            DB[p][a] = s;
          }
        for (int a = 0; a < 32; ++a)
          for (int b = 0; b < 32; ++b) {
            double s = 0.0;
            for (int p = 0; p < 9; ++p) s += B[p][a] * DB[p][b];
            K[a * 32 + b] += w * s;
          }
      }
  // exact symmetry (the sums above are symmetric up to rounding order)
  for (int a = 0; a < 32; ++a)
    for (int b = a + 1; b < 32; ++b) {
      const double s = 0.5 * (K[a * 32 + b] + K[b * 32 + a]);
      K[a * 32 + b] = K[b * 32 + a] = s;
    }
}

void affine_loads(const double h[3], double Z[32 * 9]) {
  // unit strains of §2.2 in Voigt order 11,22,33,23,13,12
  static const int kl[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  std::memset(Z, 0, sizeof(double) * 32 * 9);
  for (int n = 0; n < 8; ++n) {
    const double x[3] = {(n & 1) * h[0], ((n >> 1) & 1) * h[1], ((n >> 2) & 1) * h[2]};
    for (int p = 0; p < 6; ++p) {
      double E[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      E[kl[p][0]][kl[p][1]] += 0.5;
      E[kl[p][1]][kl[p][0]] += 0.5;
      for (int i = 0; i < 3; ++i)
        Z[(4 * n + i) * 9 + p] = E[i][0] * x[0] + E[i][1] * x[1] + E[i][2] * x[2];
    }
    for (int j = 0; j < 3; ++j) Z[(4 * n + 3) * 9 + 6 + j] = -x[j];
  }
}

// Solve the symmetric positive definite system M X = R (n x n, nr columns,
// row-major) by Cholesky; M is overwritten.
static int chol_solve(double* M, int n, double* R, int nr) {
  for (int j = 0; j < n; ++j) {
    double s = M[j * n + j];
    for (int k = 0; k < j; ++k) s -= M[j * n + k] * M[j * n + k];
    if (!(s > 0.0)) return -1;
    const double d = std::sqrt(s);
    M[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = M[i * n + j];
      for (int k = 0; k < j; ++k) t -= M[i * n + k] * M[j * n + k];
      M[i * n + j] = t / d;
    }
  }
  for (int c = 0; c < nr; ++c) {
    for (int i = 0; i < n; ++i) {
      double t = R[i * nr + c];
      for (int k = 0; k < i; ++k) t -= M[i * n + k] * R[k * nr + c];
      R[i * nr + c] = t / M[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double t = R[i * nr + c];
      for (int k = i + 1; k < n; ++k) t -= M[k * n + i] * R[k * nr + c];
      R[i * nr + c] = t / M[i * n + i];
    }
  }
  return 0;
}

int local_schur(const double K[1024], double shift, double S[64]) {
  // A_e (24x24, u dofs), B_e (8x24: potential rows, u columns), C_e = -K_pp
  double A[24 * 24], Bt[24 * 8];
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int b = 0; b < 8; ++b)
        for (int j = 0; j < 3; ++j) A[(3 * a + i) * 24 + 3 * b + j] = K[(4 * a + i) * 32 + 4 * b + j];
  for (int i = 0; i < 24; ++i) A[i * 24 + i] += shift;
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i)
      for (int b = 0; b < 8; ++b) Bt[(3 * a + i) * 8 + b] = K[(4 * b + 3) * 32 + 4 * a + i];
  double X[24 * 8];
  std::memcpy(X, Bt, sizeof(X));
  if (chol_solve(A, 24, X, 8) != 0) return -1;
  for (int p = 0; p < 8; ++p)
    for (int q = 0; q < 8; ++q) {
      double s = -K[(4 * p + 3) * 32 + 4 * q + 3];
      for (int k = 0; k < 24; ++k) s += Bt[k * 8 + p] * X[k * 8 + q];
      S[p * 8 + q] = s;
    }
  for (int p = 0; p < 8; ++p)
    for (int q = p + 1; q < 8; ++q) {
      const double s = 0.5 * (S[p * 8 + q] + S[q * 8 + p]);
      S[p * 8 + q] = S[q * 8 + p] = s;
    }
  return 0;
}

double jacobi_lmax(const double* M, int n) {
  // lambda_max of diag^-1/2 M diag^-1/2 by the cyclic Jacobi eigenvalue method
  std::vector<double> A(n * n);
  std::vector<double> s(n);
  for (int i = 0; i < n; ++i) s[i] = M[i * n + i] > 0 ? 1.0 / std::sqrt(M[i * n + i]) : 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = s[i] * M[i * n + j] * s[j];
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    if (off < 1e-30) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - sn * akq;
          A[k * n + q] = sn * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - sn * aqk;
          A[q * n + k] = sn * apk + c * aqk;
        }
      }
  }
  double lm = 0.0;
  for (int i = 0; i < n; ++i) lm = std::fmax(lm, A[i * n + i]);
  return lm;
}

void sym_eig(const double* A, int n, double* lam, double* Q) {
  double M[256];
  for (int i = 0; i < n * n; ++i) M[i] = A[i];
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) Q[i * n + k] = i == k ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        tot += M[i * n + j] * M[i * n + j];
        if (i != j) off += M[i * n + j] * M[i * n + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = M[p * n + q];
        if (apq == 0.0) continue;
        // rotation angle that zeroes M[p][q]: tan(2t) = 2 apq / (aqq - app)
        const double th = (M[q * n + q] - M[p * n + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {   // columns p, q of M
          const double mkp = M[k * n + p], mkq = M[k * n + q];
          M[k * n + p] = c * mkp - s * mkq;
          M[k * n + q] = s * mkp + c * mkq;
        }
        for (int k = 0; k < n; ++k) {   // rows p, q of M
          const double mpk = M[p * n + k], mqk = M[q * n + k];
          M[p * n + k] = c * mpk - s * mqk;
          M[q * n + k] = s * mpk + c * mqk;
        }
        for (int k = 0; k < n; ++k) {   // accumulate Q <- Q J
          const double qkp = Q[k * n + p], qkq = Q[k * n + q];
          Q[k * n + p] = c * qkp - s * qkq;
          Q[k * n + q] = s * qkp + c * qkq;
        }
      }
  }
  for (int k = 0; k < n; ++k) lam[k] = M[k * n + k];
}

int spd_inverse(double* A, int n) {
  std::vector<double> I(n * n, 0.0);
  for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
  if (chol_solve(A, n, I.data(), n) != 0) return -1;
  std::memcpy(A, I.data(), sizeof(double) * n * n);
  return 0;
}

double child_weight(int c, int a, int B) {
  double w = 1.0;
  for (int d = 0; d < 3; ++d) {
    const int p2 = ((c >> d) & 1) + ((a >> d) & 1);  // fine position * 2 in {0,1,2}
    const int Bd = (B >> d) & 1;
    if (p2 == 1) w *= 0.5;
    else if ((p2 == 0 && Bd == 1) || (p2 == 2 && Bd == 0)) return 0.0;
  }
  return w;
}

}  // namespace cellhost
