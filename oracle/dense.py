"""Oracle: dense propagators and the exact gradient (small chains, complex128).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module.

App. B, the paragraphs after Eq. gradp: U_j = Q diag(exp(-i lambda dt)) Q^dagger
from the eigendecomposition of H_j, and the eigendecomposition gives the exact
derivative of U_j with respect to the slice control.  The printed block for [F]_{jk}
is garbled; this oracle uses the textbook divided-difference (Daleckii-Krein)
form of that derivative:

    dU_j/du_j = Q ( Gamma o (Q^T Hc Q) ) Q^T,
    Gamma_ab  = (e^{-i l_a dt} - e^{-i l_b dt}) / (l_a - l_b),   Gamma_aa = -i dt e^{-i l_a dt}

(H_j is real symmetric here, so Q is real), evaluated in the equivalent form
Gamma_ab = -i dt e^{-i (l_a+l_b) dt / 2} sinc((l_a - l_b) dt / 2), which has no
0/0 for (near-)degenerate eigenvalues.  Then, with lambda_j = U_{j+1}^dag..U_N^dag f,
dbeta/du_j = <lambda_j| dU_j |psi_{j-1}> and dF/du_j = 2 Re(conj(beta) dbeta/du_j)
(App. B, the expression for grad I).
"""
from __future__ import annotations

import numpy as np

from .chain import Chain


def slice_eig(chain: Chain, uj: float):
    H = chain.dense_H(uj)
    if not np.allclose(H.imag, 0.0):
        raise ValueError("dense oracle expects a real symmetric Hamiltonian")
    lam, Q = np.linalg.eigh(H.real)
    return lam, Q


def propagator(lam: np.ndarray, Q: np.ndarray, dt: float) -> np.ndarray:
    return (Q * np.exp(-1j * dt * lam)) @ Q.T


def exact_forward(chain: Chain, u: np.ndarray, dt: float, psi0: np.ndarray):
    """psi_0..psi_N with the exact slice propagators."""
    psis = [np.asarray(psi0, dtype=np.complex128)]
    for uj in u:
        lam, Q = slice_eig(chain, float(uj))
        psis.append(propagator(lam, Q, dt) @ psis[-1])
    return psis


def exact_fidelity(chain: Chain, u: np.ndarray, dt: float, psi0: np.ndarray, target: np.ndarray) -> float:
    psis = exact_forward(chain, u, dt, psi0)
    return abs(np.vdot(target, psis[-1])) ** 2


def exact_gradient(chain: Chain, u: np.ndarray, dt: float, psi0: np.ndarray, target: np.ndarray):
    """(F, dF/du) with exact propagator derivatives (divided differences)."""
    u = np.asarray(u, dtype=np.float64)
    N = u.shape[0]
    eig = [slice_eig(chain, float(uj)) for uj in u]
    Us = [propagator(lam, Q, dt) for lam, Q in eig]
    psis = [np.asarray(psi0, dtype=np.complex128)]
    for U in Us:
        psis.append(U @ psis[-1])
    target = np.asarray(target, dtype=np.complex128)
    beta = np.vdot(target, psis[N])
    Hc = chain.dense_Hc().real
    lams = [None] * (N + 1)
    lams[N] = target
    for j in range(N, 0, -1):
        lams[j - 1] = Us[j - 1].conj().T @ lams[j]
    grad = np.zeros(N)
    for j in range(1, N + 1):
        lam, Q = eig[j - 1]
        diff = lam[:, None] - lam[None, :]
        mean = 0.5 * (lam[:, None] + lam[None, :])
        gamma = -1j * dt * np.exp(-1j * dt * mean) * np.sinc(diff * dt / (2.0 * np.pi))
        dU = Q @ (gamma * (Q.T @ Hc @ Q)) @ Q.T
        dbeta = np.vdot(lams[j], dU @ psis[j - 1])
        grad[j - 1] = 2.0 * float((np.conj(beta) * dbeta).real)
    return abs(beta) ** 2, grad
