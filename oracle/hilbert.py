"""Hilbertian extension-regularisation and projection of the shape velocity
(§2.6), FP64.

Test infrastructure (see oracle/__init__.py).

The paper names the Hilbertian projection method (a null-space method: the
normal velocity of Eq. HJ combines the orthogonal projection of the objective
sensitivity with a weighted sum of orthogonal basis functions of the
constraint sensitivities) but prints no formulas.  Reading used here:

* The velocity space is periodic H^1 on the unit cell with
  <u, v>_H = int alpha^2 grad u . grad v + u v dx, discretised with the Q1
  node basis: <u, v>_H = u^T A v, A = alpha^2 K + M (Q1 stiffness and mass
  matrices, periodic assembly).
* A nodal sensitivity d_n = dJ/dphi_n is a dual vector; its Riesz
  representer (the extension-regularisation of the sensitivity) is
  g = A^-1 d.
* With constraint sensitivities dC_i and constraint values C_i: g_J = A^-1 dJ,
  g_i = A^-1 dC_i; theta_1..theta_N an H-orthonormal basis of span{g_i} by
  Gram-Schmidt, g_i = sum_{k <= i} R_ki theta_k; the projected objective
  direction P g_J = g_J - sum_k <g_J, theta_k>_H theta_k; mu solving
  R^T mu = w_C C; and the velocity
      v = w_J P g_J / ||P g_J||_H + sum_k mu_k theta_k.
* One step of Eq. HJ moves phi by -dt v |grad phi| (|grad phi| = 1 for a
  signed distance), so to first order dJ = -dt <g_J, v>_H
  = -dt w_J ||P g_J||_H <= 0 (descent) and dC_i = -dt <g_i, v>_H = -dt w_C C_i
  (each constraint moves toward zero by the fraction w_C dt).

Arrays are (nz, ny, nx) on the unit cell, node (i, j, k) at (i/nx, j/ny, k/nz),
node index i + nx (j + ny k).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_CORNERS = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]


def element_matrices(h):
    """(K_e, M_e): 8x8 Q1 stiffness int grad N_a . grad N_b and mass
    int N_a N_b on a box with sides h = (hx, hy, hz), by 2x2x2 Gauss
    quadrature (exact: the integrands are at most quadratic per axis)."""
    g = 0.5 / np.sqrt(3.0)
    pts = (0.5 - g, 0.5 + g)
    vol = h[0] * h[1] * h[2]
    K = np.zeros((8, 8))
    M = np.zeros((8, 8))
    for qz in pts:
        for qy in pts:
            for qx in pts:
                xi = (qx, qy, qz)
                N = np.zeros(8)
                dN = np.zeros((8, 3))
                for n, (a, b, c) in enumerate(_CORNERS):
                    f = [xi[d] if s else 1.0 - xi[d] for d, s in enumerate((a, b, c))]
                    s = [1.0 if t else -1.0 for t in (a, b, c)]
                    N[n] = f[0] * f[1] * f[2]
                    dN[n] = (s[0] * f[1] * f[2] / h[0], f[0] * s[1] * f[2] / h[1], f[0] * f[1] * s[2] / h[2])
                w = vol / 8.0
                K += w * dN @ dN.T
                M += w * np.outer(N, N)
    return K, M


def helmholtz_matrix(shape, alpha):
    """Sparse A = alpha^2 K + M on the periodic node grid of shape (nz, ny, nx)."""
    nz, ny, nx = shape
    h = (1.0 / nx, 1.0 / ny, 1.0 / nz)
    Ke, Me = element_matrices(h)
    Ae = alpha * alpha * Ke + Me
    rows, cols, vals = [], [], []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                nodes = [((i + a) % nx) + nx * (((j + b) % ny) + ny * ((k + c) % nz)) for (a, b, c) in _CORNERS]
                for p in range(8):
                    for q in range(8):
                        rows.append(nodes[p])
                        cols.append(nodes[q])
                        vals.append(Ae[p, q])
    n = nx * ny * nz
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def symbol(shape, alpha, kvec):
    """Eigenvalue of A for the periodic Fourier mode exp(2 pi i k . x) on the
    node grid: the Q1 matrices are tensor products of the 1D stiffness
    (2 - 2 cos t)/h and mass h (4 + 2 cos t)/6, t = 2 pi k_d / n_d."""
    nz, ny, nx = shape
    s, m = [], []
    for kd, nd in zip(kvec, (nx, ny, nz)):
        t = 2.0 * np.pi * kd / nd
        hd = 1.0 / nd
        s.append((2.0 - 2.0 * np.cos(t)) / hd)
        m.append(hd * (4.0 + 2.0 * np.cos(t)) / 6.0)
    stiff = s[0] * m[1] * m[2] + m[0] * s[1] * m[2] + m[0] * m[1] * s[2]
    return alpha * alpha * stiff + m[0] * m[1] * m[2]


def riesz(shape, alpha, d):
    """g = A^-1 d (d a dual vector of nodal values, shape (nz, ny, nx))."""
    A = helmholtz_matrix(shape, alpha)
    return spla.spsolve(A.tocsc(), np.asarray(d, dtype=float).ravel()).reshape(shape)


def h_inner(shape, alpha, u, v):
    A = helmholtz_matrix(shape, alpha)
    return float(np.asarray(u, dtype=float).ravel() @ (A @ np.asarray(v, dtype=float).ravel()))


def velocity(shape, alpha, dJ, dCs=(), Cs=(), wJ=1.0, wC=1.0):
    """The projected, regularised velocity v of the reading above, and
    (||P g_J||_H, mu, R)."""
    A = helmholtz_matrix(shape, alpha).tocsc()
    lu = spla.splu(A)
    ip = lambda u, v: float(u @ (A @ v))
    gJ = lu.solve(np.asarray(dJ, dtype=float).ravel())
    thetas = []
    N = len(dCs)
    R = np.zeros((N, N))
    for i, dc in enumerate(dCs):
        w = lu.solve(np.asarray(dc, dtype=float).ravel())
        for k, th in enumerate(thetas):       # classical Gram-Schmidt, then normalise
            R[k, i] = ip(th, w)
        for k, th in enumerate(thetas):
            w = w - R[k, i] * th
        R[i, i] = np.sqrt(ip(w, w))
        thetas.append(w / R[i, i])
    P = gJ.copy()
    for th in thetas:
        P = P - ip(gJ, th) * th
    nP = np.sqrt(max(ip(P, P), 0.0))
    mu = np.linalg.solve(R.T, wC * np.asarray(Cs, dtype=float)) if N else np.zeros(0)
    v = (wJ * P / nP) if nP > 0 else np.zeros_like(P)
    for k, th in enumerate(thetas):
        v = v + mu[k] * th
    return v.reshape(shape), (nP, mu, R)
