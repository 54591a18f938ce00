"""Oracle: open XXZ chain and its control operator, applied matrix-free (complex128).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module.

Model (Sec. 3.1, Eq. H01 and Eq. htot, under the normalisation of the workloads):

    H0 = sum_{b=0}^{L-2} [ Jxy (Sx_b Sx_{b+1} + Sy_b Sy_{b+1}) + Jz Sz_b Sz_{b+1} ]
    H(u) = H0 + u Hc

with spin operators S = sigma / 2.  Eq. H01 writes the drift with Pauli matrices and
a prefactor J/2; since sigma.sigma = 4 S.S it is the same operator with Jxy = 2 J and
Jz = 2 J alpha_z in the paper's symbols, so both normalisations are covered by (Jxy, Jz).

Basis: index i, site k (1-based) <-> bit k-1, bit 0 = spin up (Sz = +1/2).
On that basis (written out, no library):

    (Sx_b Sx_{b+1} + Sy_b Sy_{b+1}) |i> = 1/2 |i xor (3 << b)>   if bits b, b+1 differ, else 0
    Sz_b Sz_{b+1} |i> = +1/4 |i> if bits b, b+1 agree, -1/4 |i> otherwise

Control operators Hc (the one the workloads use first):
    kind "sx": Hc = amp * Sx_s,   Sx_s |i> = 1/2 |i xor (1 << s)>   (s = site - 1)
    kind "sz": Hc = amp * sum_{s in mask} Sz_s  (diagonal; Sec. 3.1 uses
               (J/2)(sigma^z_1 + sigma^z_L) = J (Sz_1 + Sz_L), i.e. amp = J, sites 1, L)

The H*v here is a plain gather over index arrays, one bond at a time.
"""
from __future__ import annotations

import numpy as np


class Chain:
    """Matrix-free open XXZ chain H(u) = H0 + u Hc on 2**L amplitudes."""

    def __init__(self, L: int, Jxy: float, Jz: float, hc_kind: str = "sx", hc_site: int = 0,
                 hc_mask: int = 0, hc_amp: float = 1.0):
        if L < 1:
            raise ValueError("L must be >= 1")
        if hc_kind not in ("sx", "sz"):
            raise ValueError("hc_kind must be 'sx' or 'sz'")
        self.L = int(L)
        self.D = 1 << self.L
        self.Jxy = float(Jxy)
        self.Jz = float(Jz)
        self.hc_kind = hc_kind
        self.hc_site = int(hc_site)
        self.hc_mask = int(hc_mask)
        self.hc_amp = float(hc_amp)
        idx = np.arange(self.D, dtype=np.int64)
        self._idx = idx
        # Diagonal of H0: Jz/4 per parallel bond, -Jz/4 per antiparallel bond.
        diag = np.zeros(self.D, dtype=np.float64)
        self._hops = []  # (rows i with bits b, b+1 antiparallel, their partners i ^ (3 << b)) per bond
        for b in range(self.L - 1):
            bit_b = (idx >> b) & 1
            bit_b1 = (idx >> (b + 1)) & 1
            anti = bit_b != bit_b1
            diag += np.where(anti, -0.25 * self.Jz, 0.25 * self.Jz)
            rows = np.nonzero(anti)[0]
            self._hops.append((rows, rows ^ (3 << b)))
        self._diag0 = diag
        if hc_kind == "sx":
            if not 0 <= self.hc_site < self.L:
                raise ValueError("hc_site out of range")
            self._hc_partner = idx ^ (1 << self.hc_site)
            self._hc_diag = None
        else:
            d = np.zeros(self.D, dtype=np.float64)
            for s in range(self.L):
                if (self.hc_mask >> s) & 1:
                    d += np.where(((idx >> s) & 1) == 0, 0.5, -0.5)
            self._hc_diag = self.hc_amp * d
            self._hc_partner = None

    def _col(self, x: np.ndarray, v: np.ndarray) -> np.ndarray:
        return x if v.ndim == 1 else x[:, None]

    def apply_H0(self, v: np.ndarray) -> np.ndarray:
        """H0 v for v of shape (D,) or (D, k)."""
        out = self._col(self._diag0, v) * v
        for rows, partner in self._hops:
            out[rows] += 0.5 * self.Jxy * v[partner]
        return out

    def apply_Hc(self, v: np.ndarray) -> np.ndarray:
        """Hc v (the control operator, without the amplitude u)."""
        if self.hc_kind == "sx":
            return 0.5 * self.hc_amp * v[self._hc_partner]
        return self._col(self._hc_diag, v) * v

    def apply_H(self, u: float, v: np.ndarray) -> np.ndarray:
        """H(u) v = H0 v + u Hc v  (Eq. htot with a constant control u)."""
        return self.apply_H0(v) + float(u) * self.apply_Hc(v)

    def dense_H(self, u: float) -> np.ndarray:
        """Dense H(u), built column by column from the matrix-free product (small L)."""
        if self.L > 12:
            raise ValueError("dense H only for L <= 12")
        return self.apply_H(u, np.eye(self.D, dtype=np.complex128))

    def dense_Hc(self) -> np.ndarray:
        return self.apply_Hc(np.eye(self.D, dtype=np.complex128))
