"""Oracle: K-GRAPE fidelity and gradient for a piecewise-constant pulse (complex128).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module.

The steps follow Algorithm "Basic GRAPE" (Sec. 2, its steps 3-7) with the Krylov
propagator of Appendix A:

* PWC control (Eq. PWC): slice j = 1..N has constant control u_{j-1} (0-based
  array), H_j = H0 + u_{j-1} Hc (Eq. htot), U_j = exp(-i dt H_j) (App. B).
* forward: psi_0 = initial state, psi_j = U_j psi_{j-1} (Krylov step, sigma=+1).
* overlap (Eq. objective): beta = <f|psi_N>, F = |beta|^2 = 1 - I.
* backward: chi_N = beta f (Alg. step 5); chi_{j-1} = U_j^dagger chi_j (Krylov
  step, sigma=-1).  The definition chi_j = beta U_{j+1}^dagger ... U_N^dagger |f>
  (below Eq. gradI) fixes the index: chi_{j-1} is U_j^dagger applied to chi_j.
* overlaps: G_j = 2 dt Im <chi_j| Hc |psi_j>, j = 0..N.  With Eq. gradI,
  dI/du_{j-1} ~ -G_j, so dF/du_{j-1} ~ +G_j: the zeroth-order gradient places Hc
  at the end of slice j (App. B, the discussion of Eq. dId1).
* centred gradient (App. B, last paragraph): the natural gradient is evaluated at
  the middle of the slice instead of its end; read as the trapezoid rule over
  slice j, dF/du_{j-1} ~ (G_{j-1} + G_j) / 2.  Its error is O(dt^3) per component
  against O(dt^2) for the zeroth order, as App. B states.
* exact gradient (App. B, Eqs. natu_integr and natgrad): dF/du_{j-1} is the average
  over slice j of G(t) = 2 dt Im <chi(t)|Hc|psi(t)>, where inside the slice
  psi(t_{j-1} + s) = exp(-i s H_j) psi_{j-1} and chi(t_{j-1} + s) = exp(+i (dt - s) H_j) chi_j.
  App. B suggests integrating it numerically from the slice's Krylov bases; here with
  the 4-point Gauss-Lobatto rule: nodes s = 0, (1 -+ 1/sqrt 5) dt / 2, dt, weights
  1/12, 5/12, 5/12, 1/12 (exact for polynomials of degree 5).  The end nodes are
  G_{j-1} and G_j; the interior states are Krylov steps of psi_{j-1} and chi_j over
  the partial lengths.
* Taylor hierarchy (App. B, Eq. gradp): the slice average of the control operator,
  Hbar_c = (1/dt) int_0^dt e^{-i tau H_j} Hc e^{+i tau H_j} dtau, expanded in the Liouvillian
  L = [H_j, .]: Hbar_c^[P] = sum_{p<=P} (-i dt)^p / (p+1)! L^p Hc, and
  dF/du_{j-1} ~ 2 dt Im <chi_j| Hbar_c^[P] |psi_j>.  P = 0 is the zeroth-order gradient.
  (L^p Hc) x is formed by its recursive definition, (L^p Hc) x = H (L^{p-1} Hc) x -
  (L^{p-1} Hc) H x.  Grad modes "taylor1" .. "taylor6".

Returned gradients are of the fidelity F (= -dI/du).
"""
from __future__ import annotations

import numpy as np

from .chain import Chain
from .krylov import DEFAULT_BREAKDOWN_TOL, krylov_step

GRAD_MODES = ("none", "centered", "zeroth", "exact", "taylor1", "taylor2", "taylor3", "taylor4", "taylor5", "taylor6")


def forward(chain: Chain, u: np.ndarray, dt: float, m: int, psi0: np.ndarray,
            tol: float = DEFAULT_BREAKDOWN_TOL):
    """psi_0..psi_N and per-slice step info (forward sweep, Alg. step 4)."""
    psis = [np.asarray(psi0, dtype=np.complex128)]
    infos = []
    for j in range(1, len(u) + 1):
        uj = float(u[j - 1])
        nxt, info = krylov_step(lambda v, uj=uj: chain.apply_H(uj, v), psis[-1], dt, m, +1, tol)
        psis.append(nxt)
        infos.append(info)
    return psis, infos


def overlaps_G(chain: Chain, dt: float, chi: np.ndarray, psi: np.ndarray) -> float:
    """G = 2 dt Im <chi| Hc |psi>  (Eq. gradI with the sign of F)."""
    return 2.0 * dt * float(np.vdot(chi, chain.apply_Hc(psi)).imag)


def evaluate(chain: Chain, u: np.ndarray, dt: float, m: int, psi0: np.ndarray,
             target: np.ndarray, grad_mode: str = "centered",
             tol: float = DEFAULT_BREAKDOWN_TOL):
    """Fidelity F = |<f|psi_N>|^2 and its gradient with respect to u (length N).

    Returns (F, grad or None, diag) where diag holds beta, psi_N, G[0..N],
    the forward/backward Krylov error indicators and breakdown counts.
    """
    if grad_mode not in GRAD_MODES:
        raise ValueError(f"grad_mode must be one of {GRAD_MODES}")
    u = np.asarray(u, dtype=np.float64)
    N = u.shape[0]
    psis, finfo = forward(chain, u, dt, m, psi0, tol)
    target = np.asarray(target, dtype=np.complex128)
    beta = complex(np.vdot(target, psis[N]))
    F = abs(beta) ** 2
    diag = dict(beta=beta, psi_N=psis[N],
                err_fwd=max((i["err_est"] for i in finfo), default=0.0),
                breakdowns_fwd=sum(int(i["broke"]) for i in finfo),
                norm_drift=float(np.linalg.norm(psis[N]) - np.linalg.norm(psi0)))
    if grad_mode == "none":
        return F, None, diag
    G = np.zeros(N + 1)
    chi = beta * target
    G[N] = overlaps_G(chain, dt, chi, psis[N])
    berr = 0.0
    bbrk = 0
    for j in range(N, 0, -1):
        uj = float(u[j - 1])
        chi, info = krylov_step(lambda v, uj=uj: chain.apply_H(uj, v), chi, dt, m, -1, tol)
        berr = max(berr, info["err_est"])
        bbrk += int(info["broke"])
        G[j - 1] = overlaps_G(chain, dt, chi, psis[j - 1])
    diag.update(G=G, chi_0=chi, err_bwd=berr, breakdowns_bwd=bbrk)
    if grad_mode == "zeroth":
        grad = G[1:].copy()
    elif grad_mode.startswith("taylor"):
        grad = taylor_gradient(chain, u, dt, m, psis, beta * target, int(grad_mode[6:]), tol)
    elif grad_mode == "exact":
        Gi = lobatto_interior(chain, u, dt, m, psis, beta * target, tol)
        diag.update(G_interior=Gi)
        grad = (G[:-1] + G[1:]) / 12.0 + 5.0 * (Gi[:, 0] + Gi[:, 1]) / 12.0
    else:
        grad = 0.5 * (G[:-1] + G[1:])
    return F, grad, diag


def lobatto_nodes(dt: float):
    """Interior Gauss-Lobatto nodes of [0, dt] (4-point rule): (1 -+ 1/sqrt(5)) dt / 2."""
    s1 = 0.5 * dt * (1.0 - 1.0 / np.sqrt(5.0))
    return s1, dt - s1


def lobatto_interior(chain: Chain, u: np.ndarray, dt: float, m: int, psis, chi_N: np.ndarray,
                     tol: float = DEFAULT_BREAKDOWN_TOL) -> np.ndarray:
    """G at the two interior nodes of every slice: Gi[j-1, a] = G(t_{j-1} + s_a), j = 1..N.

    chi_j is propagated back slice by slice as in ``evaluate``; within slice j the states
    at t_{j-1} + s are Krylov steps of psi_{j-1} (length s, forward) and of chi_j (length
    dt - s, backward).
    """
    N = len(u)
    nodes = lobatto_nodes(dt)
    Gi = np.zeros((N, 2))
    chi = np.asarray(chi_N, dtype=np.complex128)
    for j in range(N, 0, -1):
        uj = float(u[j - 1])
        Hj = lambda v, uj=uj: chain.apply_H(uj, v)
        for a, s in enumerate(nodes):
            psi_s, _ = krylov_step(Hj, psis[j - 1], s, m, +1, tol)
            chi_s, _ = krylov_step(Hj, chi, dt - s, m, -1, tol)
            Gi[j - 1, a] = overlaps_G(chain, dt, chi_s, psi_s)
        chi, _ = krylov_step(Hj, chi, dt, m, -1, tol)
    return Gi


def liouvillian_power_hc(apply_H, apply_Hc, p: int, x: np.ndarray) -> np.ndarray:
    """(L^p Hc) x with L = [H, .], by the definition L^p Hc = H (L^{p-1} Hc) - (L^{p-1} Hc) H."""
    if p == 0:
        return apply_Hc(x)
    return apply_H(liouvillian_power_hc(apply_H, apply_Hc, p - 1, x)) - \
        liouvillian_power_hc(apply_H, apply_Hc, p - 1, apply_H(x))


def taylor_gradient(chain: Chain, u: np.ndarray, dt: float, m: int, psis, chi_N: np.ndarray, P: int,
                    tol: float = DEFAULT_BREAKDOWN_TOL) -> np.ndarray:
    """dF/du_{j-1} ~ 2 dt Im <chi_j| Hbar_c^[P] |psi_j>, j = 1..N (App. B, Eq. gradp).

    chi_j is propagated back slice by slice as in ``evaluate``; H = H_j inside slice j.
    """
    from math import factorial

    N = len(u)
    grad = np.zeros(N)
    chi = np.asarray(chi_N, dtype=np.complex128)
    for j in range(N, 0, -1):
        uj = float(u[j - 1])
        Hj = lambda v, uj=uj: chain.apply_H(uj, v)
        acc = 0j
        for p in range(P + 1):
            acc += (-1j * dt) ** p / factorial(p + 1) * np.vdot(chi, liouvillian_power_hc(Hj, chain.apply_Hc, p, psis[j]))
        grad[j - 1] = 2.0 * dt * acc.imag
        chi, _ = krylov_step(Hj, chi, dt, m, -1, tol)
    return grad


def segment_forward_backward(chain: Chain, u: np.ndarray, dt: float, m: int,
                             psi0: np.ndarray, chi_end: np.ndarray,
                             tol: float = DEFAULT_BREAKDOWN_TOL):
    """Forward over the given slices from psi0, then backward from chi_end.

    Same work per slice as ``evaluate`` (one Krylov step each way plus one overlap);
    used to time the oracle on a bounded sample of a long pulse.
    Returns (psi_end, G[0..len(u)]).
    """
    psis, _ = forward(chain, u, dt, m, psi0, tol)
    n = len(u)
    G = np.zeros(n + 1)
    chi = np.asarray(chi_end, dtype=np.complex128)
    G[n] = overlaps_G(chain, dt, chi, psis[n])
    for j in range(n, 0, -1):
        uj = float(u[j - 1])
        chi, _ = krylov_step(lambda v, uj=uj: chain.apply_H(uj, v), chi, dt, m, -1, tol)
        G[j - 1] = overlaps_G(chain, dt, chi, psis[j - 1])
    return psis[n], G
