"""Orr-Sommerfeld eigenvalues -- TEST INFRASTRUCTURE ONLY (part of the oracle).

Sec. 4.1 of the paper: a normal mode Psi = psi(z) exp(i alpha (x - c t)) of
the streamfunction of a 2-D perturbation of plane Poiseuille flow satisfies

    i alpha (U - c)(D^2 - alpha^2) psi - i alpha U'' psi = (1/Re)(D^2 - alpha^2)^2 psi,

with psi = psi' = 0 on both walls (the reading of the garbled boundary
condition of the paper), and grows like exp(lambda t), lambda = -i alpha c.

Here the channel is written in half-height units: eta = z - 1 in [-1, 1],
U = 1 - eta^2 (centreline velocity 1), Re = U_cl delta / nu.  The paper's
units (height 1, friction velocity) convert by Re_cl = Re_*^2 / 8,
alpha_half = alpha_paper / 2 and lambda_half = lambda_paper * 2 / Re_*.

Method: Chebyshev collocation on the Gauss-Lobatto points.  The clamped
condition is built into the fourth-derivative matrix by writing
psi = (1 - eta^2) q with q(+-1) = 0, for which
psi'''' = (1 - eta^2) q'''' - 8 eta q''' - 12 q''.
The generalized eigenproblem  A psi = lambda B psi  with
    B = D2 - alpha^2,
    A = (1/Re)(D4 - 2 alpha^2 D2 + alpha^4) - i alpha U (D2 - alpha^2) + i alpha U''
is solved densely with scipy.
"""
import numpy as np
import scipy.linalg


def cheb(N):
    """Chebyshev points x_j = cos(pi j / N) and the first-derivative matrix."""
    j = np.arange(N + 1)
    x = np.cos(np.pi * j / N)
    c = np.ones(N + 1)
    c[0] = c[-1] = 2.0
    c *= (-1.0) ** j
    X = np.tile(x, (N + 1, 1)).T
    dX = X - X.T
    D = np.outer(c, 1.0 / c) / (dX + np.eye(N + 1))
    D -= np.diag(D.sum(axis=1))
    return x, D


def os_spectrum(Re, alpha, N=120):
    """All finite eigenvalues lambda (growth rate = real part) and the
    interior-node eigenvectors psi, sorted by decreasing real part."""
    x, D = cheb(N)
    D2f = D @ D
    D3f = D2f @ D
    D4f = D3f @ D
    s = np.zeros(N + 1)
    s[1:-1] = 1.0 / (1.0 - x[1:-1] ** 2)
    D4 = (np.diag(1 - x**2) @ D4f - 8 * np.diag(x) @ D3f - 12 * D2f) @ np.diag(s)
    D4 = D4[1:-1, 1:-1]
    D2 = D2f[1:-1, 1:-1]
    I = np.eye(N - 1)
    xi = x[1:-1]
    U = 1 - xi**2
    Upp = -2.0 * np.ones_like(xi)
    a2 = alpha * alpha
    B = D2 - a2 * I
    A = (D4 - 2 * a2 * D2 + a2 * a2 * I) / Re - 1j * alpha * np.diag(U) @ B + 1j * alpha * np.diag(Upp)
    lam, vec = scipy.linalg.eig(A, B)
    ok = np.isfinite(lam) & (np.abs(lam) < 1e6)
    lam, vec = lam[ok], vec[:, ok]
    order = np.argsort(-lam.real)
    return lam[order], vec[:, order], xi


def least_stable(Re, alpha, N=120):
    """lambda of the least-stable mode (half-height, centreline units)."""
    lam, _, _ = os_spectrum(Re, alpha, N)
    return complex(lam[0])


def paper_to_half_height(Re_star, alpha_paper, lam_paper):
    """Convert the paper's units (height 1, friction velocity) to ours."""
    return Re_star**2 / 8.0, alpha_paper / 2.0, lam_paper * 2.0 / Re_star
