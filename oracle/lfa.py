"""Two-grid local Fourier analysis of the anisotropic grid (Appendix A.1 of the paper).

TEST INFRASTRUCTURE ONLY (part of the oracle): the closed forms the paper derives for the
constant-coefficient infinite grid with weight 1 along x and eps along y, coarsened 2:1 in x.
Each function states the equation it evaluates.

  Eq. (Lsymbol)   L(theta) = 4 sin^2(theta_x/2) + 4 eps sin^2(theta_y/2)
  smoother        S(theta) = 1 - L(theta) / M(theta),  M = (2 + 2 eps) - e^{-i theta_x} - eps e^{-i theta_y}
                  (forward Gauss-Seidel: M is the already-updated, lower-triangular part of L)
  Eq. (Psymbols)  caliber-1 P = (cos(theta_x/2), i sin(theta_x/2)), caliber-2 P = (c, s),
                  c = cos^2(theta_x/2), s = sin^2(theta_x/2)
  Eq. (tgsymbol)  T = S^nu [I - P (P* L P)^{-1} P* L] on the pair (theta, theta*),
                  theta* = (theta_x + pi, theta_y)
  Eq. (rhotrace)  rho(T) = |S(theta)^nu (1 - beta) + S(theta*)^nu beta|,
                  beta = |P_1|^2 l_1 / (|P_1|^2 l_1 + |P_2|^2 l_2)

Two independent evaluations are provided: the trace formula (rho_trace) and the spectral radius
of the explicitly assembled 2 x 2 matrix T (rho_matrix); the tests compare them.
"""
from __future__ import annotations

import numpy as np


def l_symbol(tx, ty, eps):
    """Eq. (Lsymbol): symbol of the 5-point anisotropic Laplacian."""
    return 4.0 * np.sin(tx / 2) ** 2 + 4.0 * eps * np.sin(ty / 2) ** 2


def m_symbol(tx, ty, eps):
    """Symbol of the lower-triangular part (diagonal plus already-updated west and south
    neighbours) of the Laplacian, the Gauss-Seidel preconditioner."""
    return (2.0 + 2.0 * eps) - np.exp(-1j * tx) - eps * np.exp(-1j * ty)


def s_symbol(tx, ty, eps):
    """Forward Gauss-Seidel error symbol S = 1 - L / M."""
    return 1.0 - l_symbol(tx, ty, eps) / m_symbol(tx, ty, eps)


def p_symbol(tx, caliber: int):
    """Eq. (Psymbols): interpolation symbol (smooth component, harmonic component)."""
    if caliber == 1:
        return np.cos(tx / 2) + 0j, 1j * np.sin(tx / 2)
    c, s = np.cos(tx / 2) ** 2, np.sin(tx / 2) ** 2
    return c + 0j, s + 0j


def beta(tx, ty, eps, caliber: int):
    """Fraction of the interpolant's L-energy on the smooth harmonic (Eq. rhotrace)."""
    p1, p2 = p_symbol(tx, caliber)
    l1, l2 = l_symbol(tx, ty, eps), l_symbol(tx + np.pi, ty, eps)
    a, b = np.abs(p1) ** 2 * l1, np.abs(p2) ** 2 * l2
    return a / (a + b)


def rho_trace(tx, ty, eps, caliber: int, nu: int = 3):
    """Eq. (rhotrace): spectral radius of the two-grid symbol through its trace."""
    bt = beta(tx, ty, eps, caliber)
    return np.abs(s_symbol(tx, ty, eps) ** nu * (1 - bt) + s_symbol(tx + np.pi, ty, eps) ** nu * bt)


def t_matrix(tx, ty, eps, caliber: int, nu: int = 3) -> np.ndarray:
    """Eq. (tgsymbol): the 2 x 2 two-grid operator on (theta, theta*) assembled explicitly."""
    p1, p2 = p_symbol(tx, caliber)
    P = np.array([[p1], [p2]])
    Lh = np.diag([l_symbol(tx, ty, eps), l_symbol(tx + np.pi, ty, eps)]).astype(complex)
    Sh = np.diag([s_symbol(tx, ty, eps), s_symbol(tx + np.pi, ty, eps)])
    Ph = P.conj().T
    cgc = np.eye(2) - P @ np.linalg.inv(Ph @ Lh @ P) @ Ph @ Lh
    return np.linalg.matrix_power(Sh, nu) @ cgc


def rho_matrix(tx, ty, eps, caliber: int, nu: int = 3) -> float:
    return float(np.max(np.abs(np.linalg.eigvals(t_matrix(tx, ty, eps, caliber, nu)))))


def sup_rho(eps, caliber: int, nu: int = 3, N: int = 256) -> float:
    """Supremum of rho over theta_x in (-pi/2, pi/2], theta_y in (-pi, pi], on an N x 2N grid of
    cell-centred frequencies (the constant mode theta = 0, where L vanishes, is not on it)."""
    tx = -np.pi / 2 + (np.arange(N) + 0.5) * (np.pi / N)
    ty = -np.pi + (np.arange(2 * N) + 0.5) * (np.pi / N)
    TX, TY = np.meshgrid(tx, ty, indexing="ij")
    return float(np.max(rho_trace(TX, TY, eps, caliber, nu)))
