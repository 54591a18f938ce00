"""Seeded synthetic inputs for the K-GRAPE hot path.

This module only draws random numbers and lays out basis states; it holds none of
the method's arithmetic (no Hamiltonian, no propagation, no gradient).  Both the
CUDA path and the CPU oracle are fed from here, so that the two always see
identical inputs.

Conventions (fixed here, documented in the C header as well):

* basis index i in [0, 2**L); site k (1-based) <-> bit k-1 of i; bit value 0 means
  spin up (S^z = +1/2), following the spin-up-is-zero encoding of Sec. 3.1;
* the Neel string |0101...> lists sites 1..L from left to right, so site 1 is up,
  site 2 down, ... and its index is sum_{k even} 2**(k-1)  (L=8 -> 170);
* controls u_j ~ U(-1, 1) as in Sec. 3.2 ("random fields ... uniform in [-1, 1]");
* targets are Gaussian complex vectors normalised to 1 in float64.

Random-draw order for one instance with generator ``rng``: first the N controls,
then the real parts of the target, then the imaginary parts.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_BASE = 2010035980


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic K-GRAPE workload (an open XXZ chain driven by Sx on site 1)."""

    name: str
    L: int
    N: int
    dt: float
    m: int
    delta: float
    J: float = 1.0
    seed: int = SEED_BASE
    ckpt: int = 0  # keep every ckpt-th psi_j and recompute the rest in the backward sweep (0: keep all)

    @property
    def D(self) -> int:
        return 1 << self.L

    @property
    def Jxy(self) -> float:
        # H0 = J * sum (SxSx + SySy + Delta SzSz): flip-flop coupling J, Ising J*Delta.
        return self.J

    @property
    def Jz(self) -> float:
        return self.J * self.delta


# The five workloads of the hot path.  Index k (1-based) picks seed SEED_BASE + k.
WORKLOADS = {
    "xxz_L8_N64_m12": Workload("xxz_L8_N64_m12", L=8, N=64, dt=0.1, m=12, delta=0.5, seed=SEED_BASE + 1),
    "xxz_L16_N200_m20": Workload("xxz_L16_N200_m20", L=16, N=200, dt=0.05, m=20, delta=1.0, seed=SEED_BASE + 2),
    "xxz_L20_N400_m20": Workload("xxz_L20_N400_m20", L=20, N=400, dt=0.05, m=20, delta=0.5, seed=SEED_BASE + 3),
    "xxz_L24_N400_m24_ckpt20": Workload("xxz_L24_N400_m24_ckpt20", L=24, N=400, dt=0.05, m=24, delta=0.5,
                                        seed=SEED_BASE + 5, ckpt=20),
}

# Batched workload: 256 pulses, L_i ~ U{10..16}, Delta_i ~ U(0, 2), N=200, dt=0.05, m=16.
BATCH_SEED = SEED_BASE + 4
BATCH_SIZE = 256
BATCH_N = 200
BATCH_DT = 0.05
BATCH_M = 16


def neel_index(L: int) -> int:
    """Index of the Neel basis state |0101...> (site 1 up, site 2 down, ...)."""
    return sum(1 << (k - 1) for k in range(2, L + 1, 2))


def neel_state(L: int) -> np.ndarray:
    psi = np.zeros(1 << L, dtype=np.complex128)
    psi[neel_index(L)] = 1.0
    return psi


def draw_controls(rng: np.random.Generator, N: int) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, N).astype(np.float64)


def draw_target(rng: np.random.Generator, D: int) -> np.ndarray:
    re = rng.standard_normal(D)
    im = rng.standard_normal(D)
    f = re + 1j * im
    return (f / np.linalg.norm(f)).astype(np.complex128)


def instance(w: Workload, N: int | None = None, seed: int | None = None):
    """Controls, initial state and target for workload ``w``.

    ``N`` may shorten the pulse (the controls are then the first N draws of a
    fresh generator, and the target is drawn after them), e.g. for oracle-sized
    segments of a large chain.  Returns (u[N] float64, psi0[D] complex128,
    target[D] complex128).
    """
    n = w.N if N is None else N
    rng = np.random.default_rng(w.seed if seed is None else seed)
    u = draw_controls(rng, n)
    target = draw_target(rng, w.D)
    return u, neel_state(w.L), target


def batch_instances(B: int = BATCH_SIZE, N: int = BATCH_N, seed: int = BATCH_SEED,
                    L_min: int = 10, L_max: int = 16):
    """Independent pulses of the batched workload.

    Instance i draws from default_rng([seed, i]), in order: L_i ~ U{L_min..L_max},
    Delta_i ~ U(0, 2), the N controls, then the target.  Returns a list of dicts
    with keys L, delta, u, psi0, target.
    """
    out = []
    for i in range(B):
        rng = np.random.default_rng([seed, i])
        L = int(rng.integers(L_min, L_max + 1))
        delta = float(rng.uniform(0.0, 2.0))
        u = draw_controls(rng, N)
        target = draw_target(rng, 1 << L)
        out.append(dict(L=L, delta=delta, u=u, psi0=neel_state(L), target=target))
    return out


def fd_indices(w: Workload, count: int = 16) -> list[int]:
    """Seeded slice indices for central finite-difference checks of the gradient."""
    rng = np.random.default_rng([w.seed, 999])
    return sorted(int(i) for i in rng.choice(w.N, count, replace=False))


# ---------------------------------------------------------------- the paper's own workload
@dataclasses.dataclass(frozen=True)
class SectorWorkload:
    """Sec. 3.1-3.2: K excitations of an L-site XXZ chain, even parity, e_1 -> e_D.

    J = 1, alpha_z = 0.5 (Eq. H01), Hc = (J/2)(sigma^z_1 + sigma^z_L), dt = 0.5, m = 10 Krylov
    vectors, M = 4D controls drawn from U(-1, 1).  D (the subspace dimension) is not stored
    here: it comes from whoever builds the basis, and sets N = n_per_dim * D.
    """

    name: str
    L: int
    K: int
    parity: int = 1
    J: float = 1.0
    alpha_z: float = 0.5
    dt: float = 0.5
    m: int = 10
    n_per_dim: int = 4
    seed: int = SEED_BASE + 6


SECTOR_WORKLOADS = {
    "pe_L10_K4": SectorWorkload("pe_L10_K4", L=10, K=4),
    "pe_L14_K4": SectorWorkload("pe_L14_K4", L=14, K=4),
    "pe_L20_K4": SectorWorkload("pe_L20_K4", L=20, K=4),
}


def sector_instance(w: SectorWorkload, D: int, batch: int = 1, N: int | None = None):
    """Controls of `batch` independent pulses and the task e_1 -> e_D of a D-dimensional subspace.

    Pulse b draws its N (default n_per_dim * D) controls from default_rng([seed, b]).  Returns
    (u[batch, N] float64, psi0[D] complex128 = e_1, target[D] complex128 = e_D).
    """
    n = w.n_per_dim * D if N is None else N
    u = np.stack([draw_controls(np.random.default_rng([w.seed, b]), n) for b in range(batch)])
    psi0 = np.zeros(D, dtype=np.complex128)
    psi0[0] = 1.0
    target = np.zeros(D, dtype=np.complex128)
    target[D - 1] = 1.0
    return u, psi0, target
