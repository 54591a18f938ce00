"""Oracle: Lanczos basis and the Krylov time step (Appendix A), complex128.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module.

Steps, in the order of Appendix A:

1. Lanczos (Algorithm "Lanczos"): v_0 = psi / ||psi||; for k = 0, 1, ...:
   x = H v_k; alpha_k = <v_k|x>; remove from x its components on the basis; the
   norm of the remainder is b_{k+1}; if b_{k+1} > 0 (above a breakdown tolerance)
   v_{k+1} = remainder / b_{k+1}.  The listing removes only the components on the
   last two vectors; Appendix A names explicit orthonormalisation against all
   previous vectors as the remedy for the loss of orthogonality, and this oracle
   uses it: classical Gram-Schmidt against every basis vector, applied twice.
   The basis has m vectors (v_0 .. v_{m-1}); T_m = V H V^dagger is tridiagonal
   with diagonal alpha_0..alpha_{m-1} and off-diagonal b_1..b_{m-1}.
2. Breakdown: if b_{k+1} <= tol * max(1, max|alpha| + max|b|) the basis stops at
   k+1 vectors (the subspace is invariant; the step is then exact).
3. Krylov step (Appendix A): psi(t+dt) ~ V^dagger exp(-i sigma dt T) V psi(t)
   with V psi = ||psi|| e_1.  exp(-i sigma dt T) e_1 is formed from the
   eigendecomposition of the small symmetric T (numpy.linalg.eigh).
   sigma = +1 propagates forward (U_j), sigma = -1 backward (U_j^dagger).

The a-posteriori error indicator returned with each step is
||psi|| * b_m * |[exp(-i sigma dt T_m) e_1]_{m-1}| (the residual term of the
Lanczos relation H V^dagger = V^dagger T + b_m v_m e_{m-1}^T), 0 after a breakdown.
"""
from __future__ import annotations

import numpy as np

DEFAULT_BREAKDOWN_TOL = 1e-12


def lanczos(apply_H, psi: np.ndarray, m: int, tol: float = DEFAULT_BREAKDOWN_TOL):
    """Krylov basis of (H, psi) with full CGS2 re-orthogonalisation.

    Returns (V [meff, D], alpha [meff], beta [meff-1], beta_m, norm_psi, broke).
    ``beta_m`` is the norm of the residual after the last vector (0 after breakdown).
    """
    nrm = float(np.linalg.norm(psi))
    D = psi.shape[0]
    if nrm == 0.0:
        return np.zeros((0, D), dtype=np.complex128), np.zeros(0), np.zeros(0), 0.0, 0.0, False
    V = np.zeros((m, D), dtype=np.complex128)
    V[0] = psi / nrm
    alpha: list[float] = []
    beta: list[float] = []
    beta_m = 0.0
    broke = False
    meff = m
    for k in range(m):
        x = apply_H(V[k])
        alpha.append(float(np.vdot(V[k], x).real))
        r = x
        for _ in range(2):  # classical Gram-Schmidt, twice: coeff_i = <v_i|r>
            coeff = (V[: k + 1] @ r.conj()).conj()
            r = r - coeff @ V[: k + 1]
        b = float(np.linalg.norm(r))
        if k == m - 1:
            beta_m = b
            break
        scale = max(1.0, max(abs(a) for a in alpha) + (max(beta) if beta else 0.0))
        if b <= tol * scale:
            meff = k + 1
            broke = True
            beta_m = 0.0
            break
        beta.append(b)
        V[k + 1] = r / b
    return V[:meff], np.array(alpha), np.array(beta), beta_m, nrm, broke


def tridiag(alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    n = alpha.shape[0]
    T = np.diag(alpha.astype(np.float64))
    for k in range(n - 1):
        T[k, k + 1] = beta[k]
        T[k + 1, k] = beta[k]
    return T


def expm_e1(alpha: np.ndarray, beta: np.ndarray, dt: float, sigma: int) -> np.ndarray:
    """exp(-i sigma dt T) e_1 for the symmetric tridiagonal T(alpha, beta), via eigh."""
    T = tridiag(alpha, beta)
    theta, Q = np.linalg.eigh(T)
    return Q @ (np.exp(-1j * sigma * dt * theta) * Q[0, :])


def krylov_step(apply_H, psi: np.ndarray, dt: float, m: int, sigma: int = 1,
                tol: float = DEFAULT_BREAKDOWN_TOL):
    """One Krylov time step psi -> V^dagger exp(-i sigma dt T_m) V psi.

    Returns (psi_new, info) with info = dict(alpha, beta, beta_m, err_est, broke, meff).
    """
    V, alpha, beta, beta_m, nrm, broke = lanczos(apply_H, psi, m, tol)
    if nrm == 0.0:
        return np.zeros_like(psi), dict(alpha=alpha, beta=beta, beta_m=0.0, err_est=0.0, broke=False, meff=0)
    c = expm_e1(alpha, beta, dt, sigma)
    psi_new = nrm * (c @ V)
    err = nrm * beta_m * abs(c[-1]) if not broke else 0.0
    return psi_new, dict(alpha=alpha, beta=beta, beta_m=beta_m, err_est=err, broke=broke, meff=V.shape[0])
