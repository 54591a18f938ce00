"""Oracle: the XXZ chain in a parity-excitation (PE) subspace (Sec. 3.1), complex128.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module.

Sec. 3.1 splits the state space of the chain twice:

* H conserves the number of excitations, so it is block diagonal over the subspaces S_K
  spanned by the basis states with K excitations, of dimension D_K = C(L, K).  Here an
  excitation is a spin down, i.e. a set bit of the basis index (site k <-> bit k-1).
* H and the control (J/2)(sigma^z_1 + sigma^z_L) commute with the parity operator Pi, which
  mirrors the chain about its middle (site k <-> site L+1-k, i.e. bit k-1 <-> bit L-k), so
  each S_K splits again into an even and an odd PE subspace.

The reduced Hamiltonian is built the way Sec. 3.1 describes: (i) Pi written in S_K (a
permutation matrix), (ii) its eigenvectors, (iii) those of the wanted parity stacked as the
rows of a rectangular change of basis Q, (iv) H_red = Q H_K Q^T.  Pi is an involution that
permutes basis states, so its eigenvectors for the eigenvalue +1 are, for every orbit
{s, Pi s}, (|s> + |Pi s>)/sqrt 2 (or |s> when s is a palindrome), and for -1,
(|s> - |Pi s>)/sqrt 2 over the orbits of two states.  Sec. 3.1 orders the reduced basis by
the binary number of the bit sequences, ascending; the orbits are ordered here by the
smaller member, which is the same order whichever end of the chain the binary number starts
from (reversing the string maps an orbit onto itself).  parity = 0 keeps the whole S_K.

H_K is written out state by state with the matrix elements of Eq. H01 in the S-operator
normalisation of ``chain.py``: Jz/4 (parallel) or -Jz/4 (antiparallel) per bond on the
diagonal, Jxy/2 between |s> and |s xor (3 << b)> when bits b, b+1 differ.  The control is
Hc = hc_amp * sum_{s in mask} Sz_s (Sec. 3.1's (J/2)(sigma^z_1 + sigma^z_L) is hc_amp = J with
sites 1 and L).  ``SectorChain`` offers the interface of ``chain.Chain`` so the sweeps of
``grape.py`` run on it unchanged.
"""
from __future__ import annotations

from math import comb

import numpy as np
import scipy.sparse as sp


def k_sector_states(L: int, K: int) -> np.ndarray:
    """The basis states of S_K (K set bits among L), ascending."""
    if not (0 <= K <= L):
        raise ValueError("need 0 <= K <= L")
    idx = np.arange(1 << L, dtype=np.int64)
    pc = np.zeros_like(idx)
    for b in range(L):
        pc += (idx >> b) & 1
    out = idx[pc == K]
    assert out.shape[0] == comb(L, K)
    return out


def mirror(s, L: int):
    """Pi on basis indices: bit b <-> bit L-1-b (works on scalars and int arrays)."""
    s = np.asarray(s, dtype=np.int64)
    r = np.zeros_like(s)
    for b in range(L):
        r |= ((s >> b) & 1) << (L - 1 - b)
    return r


def parity_matrix(states: np.ndarray, L: int) -> sp.csr_matrix:
    """Step (i): Pi restricted to S_K (a permutation matrix on the sector basis)."""
    pos = {int(s): i for i, s in enumerate(states)}
    cols = np.arange(states.shape[0])
    rows = np.array([pos[int(t)] for t in mirror(states, L)], dtype=np.int64)
    return sp.csr_matrix((np.ones(states.shape[0]), (rows, cols)), shape=(states.shape[0],) * 2)


def pe_change_of_basis(states: np.ndarray, L: int, parity: int):
    """Steps (ii)-(iii): Q (rows = Pi eigenvectors of eigenvalue `parity`, orbit order) and the
    representative (smallest) state of each row.  parity 0: Q = identity."""
    n = states.shape[0]
    if parity == 0:
        return sp.identity(n, format="csr", dtype=np.float64), states.copy()
    if parity not in (1, -1):
        raise ValueError("parity must be 0, +1 or -1")
    pos = {int(s): i for i, s in enumerate(states)}
    mir = mirror(states, L)
    rows, cols, vals, reps = [], [], [], []
    for i, s in enumerate(states):  # ascending, so each orbit is met first at its smaller member
        t = int(mir[i])
        if t < int(s):
            continue
        r = len(reps)
        if t == int(s):
            if parity == 1:  # palindromes are even
                rows.append(r)
                cols.append(i)
                vals.append(1.0)
                reps.append(int(s))
            continue
        h = 1.0 / np.sqrt(2.0)
        rows += [r, r]
        cols += [i, pos[t]]
        vals += [h, parity * h]
        reps.append(int(s))
    Q = sp.csr_matrix((vals, (rows, cols)), shape=(len(reps), n))
    return Q, np.array(reps, dtype=np.int64)


def sector_H0(states: np.ndarray, L: int, Jxy: float, Jz: float) -> sp.csr_matrix:
    """H_K: the drift of Eq. H01 on S_K, element by element."""
    pos = {int(s): i for i, s in enumerate(states)}
    rows, cols, vals = [], [], []
    for i, s in enumerate(states):
        s = int(s)
        d = 0.0
        for b in range(L - 1):
            if ((s >> b) & 1) != ((s >> (b + 1)) & 1):
                d -= 0.25 * Jz
                rows.append(pos[s ^ (3 << b)])
                cols.append(i)
                vals.append(0.5 * Jxy)
            else:
                d += 0.25 * Jz
        rows.append(i)
        cols.append(i)
        vals.append(d)
    n = states.shape[0]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def sector_Hc(states: np.ndarray, L: int, hc_mask: int, hc_amp: float) -> sp.csr_matrix:
    """Hc = hc_amp * sum_{s in mask} Sz_s on S_K (diagonal; Sz = +1/2 for a clear bit)."""
    d = np.zeros(states.shape[0])
    for b in range(L):
        if (hc_mask >> b) & 1:
            d += np.where(((states >> b) & 1) == 0, 0.5, -0.5)
    return sp.diags(hc_amp * d, format="csr")


class SectorChain:
    """H(u) = H0 + u Hc on a PE subspace of the open XXZ chain (Sec. 3.1), as sparse matrices.

    Same interface as ``chain.Chain`` (D, apply_H0, apply_Hc, apply_H, dense_H, dense_Hc), so
    ``grape.evaluate`` propagates in the reduced basis.  ``embed`` maps a reduced vector to the
    2^L amplitudes of the full chain (Q^T, then the sector states' indices).
    """

    def __init__(self, L: int, K: int, parity: int, Jxy: float, Jz: float, hc_mask: int, hc_amp: float):
        if parity != 0 and mirror(hc_mask, L) != hc_mask:
            raise ValueError("a parity subspace needs a mirror-symmetric control mask")
        self.L, self.K, self.parity = int(L), int(K), int(parity)
        self.Jxy, self.Jz, self.hc_mask, self.hc_amp = float(Jxy), float(Jz), int(hc_mask), float(hc_amp)
        self.states = k_sector_states(L, K)
        self.P = parity_matrix(self.states, L)                                    # step (i)
        self.Q, self.reps = pe_change_of_basis(self.states, L, parity)            # steps (ii)-(iii)
        self.HK = sector_H0(self.states, L, Jxy, Jz)
        self.HcK = sector_Hc(self.states, L, hc_mask, hc_amp)
        self.H0 = (self.Q @ self.HK @ self.Q.T).tocsr()                            # step (iv)
        self.Hc = (self.Q @ self.HcK @ self.Q.T).tocsr()
        self.D = self.Q.shape[0]

    def apply_H0(self, v: np.ndarray) -> np.ndarray:
        return self.H0 @ v

    def apply_Hc(self, v: np.ndarray) -> np.ndarray:
        return self.Hc @ v

    def apply_H(self, u: float, v: np.ndarray) -> np.ndarray:
        return self.apply_H0(v) + float(u) * self.apply_Hc(v)

    def dense_H(self, u: float) -> np.ndarray:
        return (self.H0 + float(u) * self.Hc).toarray().astype(np.complex128)

    def dense_Hc(self) -> np.ndarray:
        return self.Hc.toarray().astype(np.complex128)

    def embed(self, v: np.ndarray) -> np.ndarray:
        full = np.zeros(1 << self.L, dtype=np.complex128)
        full[self.states] = self.Q.T @ np.asarray(v, dtype=np.complex128)
        return full


def paper_chain(L: int, K: int, parity: int = 1, J: float = 1.0, alpha_z: float = 0.5) -> SectorChain:
    """Sec. 3.1's setting: Eq. H01 with coupling J and anisotropy alpha_z, Hc = (J/2)(sigma^z_1 +
    sigma^z_L).  In the S-operator normalisation: Jxy = 2 J, Jz = 2 J alpha_z, Hc = J (Sz_1 + Sz_L)."""
    mask = 1 | (1 << (L - 1))
    return SectorChain(L, K, parity, 2.0 * J, 2.0 * J * alpha_z, mask, J)
