"""Outer K-GRAPE loop: L-BFGS over the pulse with a Wolfe line search (Sec. 2).

Sec. 2 feeds the gradient to L-BFGS: the search direction p = -B^{-1} grad I comes from a
limited-memory BFGS approximation B of the Hessian, and the step along p is chosen by
backtracking until Wolfe's conditions hold.  The objective is the infidelity I = 1 - F of
Eq. objective; Sec. 3.2 stops at I <= I_target (1e-2) or when I changes by less than
Delta I_min = 10 EPS between iterations.

The loop is host logic: every evaluation of F and dF/du is one call of the library
(``PulseObjective``); nothing here touches the state vectors.
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np

FidelityAndGradient = Callable[[np.ndarray], "tuple[float, np.ndarray]"]


@dataclasses.dataclass
class LbfgsResult:
    u: np.ndarray            # best pulse found
    F: float                 # its fidelity
    iterations: int          # accepted L-BFGS steps
    evaluations: int         # calls of the objective
    history: list            # infidelity after every accepted step (first entry: the start)
    reason: str              # "target", "stalled", "max_iter" or "line_search"


def _two_loop(g: np.ndarray, S: list, Y: list) -> np.ndarray:
    """-H g with the L-BFGS inverse-Hessian approximation H from the pairs (s_i, y_i)."""
    q = g.copy()
    alphas = []
    for s, y in zip(reversed(S), reversed(Y)):
        rho = 1.0 / float(y @ s)
        a = rho * float(s @ q)
        alphas.append((a, rho, s, y))
        q -= a * y
    if S:
        gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1])
        q *= gamma
    for a, rho, s, y in reversed(alphas):
        b = rho * float(y @ q)
        q += (a - b) * s
    return -q


def lbfgs_maximize_fidelity(fun: FidelityAndGradient, u0: np.ndarray, *, target_infidelity: float = 1e-2,
                            min_change: float = 10 * np.finfo(np.float64).eps, max_iter: int = 500,
                            memory: int = 10, c1: float = 1e-4, c2: float = 0.9,
                            max_trials: int = 40) -> LbfgsResult:
    """Maximise F(u) (minimise I = 1 - F) from u0; ``fun(u)`` returns (F, dF/du).

    Line search: from the unit step (first iteration: a step of length 1 along the steepest
    descent direction), halve until the sufficient-decrease (Armijo) condition
    I(u + a p) <= I(u) + c1 a <grad I, p> holds; if that first point already satisfies it
    but violates the curvature condition <grad I(u + a p), p> >= c2 <grad I, p>, double the
    step while both the decrease holds and the curvature fails.  A pair (s, y) enters the
    memory only when s.y > 0, which keeps the approximation positive definite.
    """
    u = np.asarray(u0, dtype=np.float64).copy()
    F, dF = fun(u)
    nev = 1
    I, g = 1.0 - F, -np.asarray(dF, dtype=np.float64)
    hist = [I]
    S: list = []
    Y: list = []
    reason = "max_iter"
    it = 0
    while it < max_iter:
        if I <= target_infidelity:
            reason = "target"
            break
        p = _two_loop(g, S, Y)
        gp = float(g @ p)
        if not gp < 0.0:  # not a descent direction: restart from steepest descent
            S.clear()
            Y.clear()
            p = -g
            gp = float(g @ p)
        a = 1.0 if S else 1.0 / max(np.linalg.norm(p), 1e-300)
        accepted = None
        trials = 0
        expanding = False
        while trials < max_trials:
            un = u + a * p
            Fn, dFn = fun(un)
            nev += 1
            trials += 1
            In, gn = 1.0 - Fn, -np.asarray(dFn, dtype=np.float64)
            armijo = In <= I + c1 * a * gp
            curvature = float(gn @ p) >= c2 * gp
            if armijo and (curvature or trials == max_trials):
                accepted = (un, In, gn, a)
                break
            if armijo and not curvature and (trials == 1 or expanding):
                accepted = (un, In, gn, a)  # keep the best acceptable point while expanding
                expanding = True
                a *= 2.0
                continue
            if expanding:  # the expansion overshot: keep the last point that decreased I enough
                break
            a *= 0.5
        if accepted is None:
            reason = "line_search"
            break
        un, In, gn, a = accepted
        s, y = un - u, gn - g
        if float(s @ y) > 1e-300:
            S.append(s)
            Y.append(y)
            if len(S) > memory:
                S.pop(0)
                Y.pop(0)
        change = I - In
        u, I, g = un, In, gn
        it += 1
        hist.append(I)
        if abs(change) < min_change:
            reason = "stalled"
            break
    if I <= target_infidelity:
        reason = "target"
    return LbfgsResult(u=u, F=1.0 - I, iterations=it, evaluations=nev, history=hist, reason=reason)


class PulseObjective:
    """F and dF/du of a pulse through a ``KGrape`` engine, or a ``KGrapeSector`` engine created
    for one pulse (one library evaluation per call).

    The initial and target states stay on the device; each call copies the N controls in,
    runs one evaluation and reads F and the gradient back.
    """

    def __init__(self, engine, psi0, target):
        import torch

        batch = getattr(engine, "B", None)
        if batch not in (None, 1):
            raise ValueError("PulseObjective drives one pulse: create the subspace engine with B = 1")
        self.engine = engine
        self.psi0 = psi0
        self.target = target
        shape = (engine.opts.N,) if batch is None else (1, engine.opts.N)
        self.u = torch.empty(shape, dtype=torch.float64, device=psi0.device)

    def __call__(self, u: np.ndarray):
        import torch

        self.u.copy_(torch.as_tensor(u, dtype=torch.float64).reshape(self.u.shape))
        fid, grad = self.engine.evaluate(self.u, self.psi0, self.target)
        self.engine.sync()
        return float(fid.reshape(-1)[0].item()), grad.reshape(-1).cpu().numpy().copy()
