"""Pins of the parity-excitation (PE) subspace oracle (Sec. 3.1) against what does not come from it:
counting formulas, a hand-reduced 3-site example, the full-chain oracle (itself pinned to
Kronecker products) restricted to the sector, the spectrum of the parity operator, and the full
chain's fidelity and gradient for the embedded states."""
from math import comb

import numpy as np
import pytest

import oracle
import oracle.sector as S
from paper_2010_03598_gb300 import workloads as W


def palindromes(L, K):
    # a mirror-symmetric string is fixed by its first floor(L/2) bits (and the middle one for odd L)
    h = L // 2
    if L % 2 == 0:
        return comb(h, K // 2) if K % 2 == 0 else 0
    return comb(h, K // 2)  # the middle bit is K mod 2


@pytest.mark.parametrize("L", [2, 3, 5, 8, 9, 12])
def test_dimensions_follow_the_counting_formulas(L):
    for K in range(L + 1):
        states = S.k_sector_states(L, K)
        assert states.shape[0] == comb(L, K)
        p = palindromes(L, K)
        even = S.pe_change_of_basis(states, L, +1)[0].shape[0]
        odd = S.pe_change_of_basis(states, L, -1)[0].shape[0]
        assert even == (comb(L, K) + p) // 2 and odd == (comb(L, K) - p) // 2


def test_orbit_order_of_a_small_chain():
    # L = 5, K = 2: orbits {3, 24}, {5, 20}, {6, 12}, {9, 18}, {10}, {17} (10 = 01010, 17 = 10001 palindromes)
    states = S.k_sector_states(5, 2)
    assert list(S.pe_change_of_basis(states, 5, +1)[1]) == [3, 5, 6, 9, 10, 17]
    assert list(S.pe_change_of_basis(states, 5, -1)[1]) == [3, 5, 6, 9]


def test_hand_reduced_three_site_chain():
    # L = 3, K = 1, even: e_1 = (|001> + |100>)/sqrt2, e_2 = |010>.  By hand: <e_1|H|e_1> = 0,
    # <e_2|H|e_1> = (Jxy/2 + Jxy/2)/sqrt2, <e_2|H|e_2> = -Jz/2; Hc = a (Sz_1 + Sz_3) = diag(0, a).
    Jxy, Jz, a = 0.7, 1.3, 0.9
    c = S.SectorChain(3, 1, +1, Jxy, Jz, 0b101, a)
    np.testing.assert_allclose(c.H0.toarray(), [[0.0, Jxy / np.sqrt(2)], [Jxy / np.sqrt(2), -Jz / 2]], atol=1e-15)
    np.testing.assert_allclose(c.Hc.toarray(), np.diag([0.0, a]), atol=1e-15)


@pytest.mark.parametrize("L,K", [(6, 2), (7, 3), (8, 4)])
def test_sector_block_is_the_full_chain_restricted(L, K):
    mask = 1 | (1 << (L - 1))
    full = oracle.Chain(L, 0.8, 1.7, hc_kind="sz", hc_mask=mask, hc_amp=0.6)
    c = S.SectorChain(L, K, 0, 0.8, 1.7, mask, 0.6)
    idx = c.states
    H = full.dense_H(0.0).real
    np.testing.assert_allclose(c.HK.toarray(), H[np.ix_(idx, idx)], atol=1e-14)
    np.testing.assert_allclose(c.HcK.toarray(), full.dense_Hc().real[np.ix_(idx, idx)], atol=1e-14)
    # S_K is invariant: nothing leaves the sector
    out = np.setdiff1d(np.arange(1 << L), idx)
    assert np.abs(H[np.ix_(out, idx)]).max() == 0.0


@pytest.mark.parametrize("L,K,parity", [(7, 3, 1), (8, 4, 1), (8, 4, -1), (9, 2, 1)])
def test_change_of_basis_is_the_parity_eigenbasis(L, K, parity):
    c = S.SectorChain(L, K, parity, 2.0, 1.0, 1 | (1 << (L - 1)), 1.0)
    Q, P = c.Q.toarray(), c.P.toarray()
    np.testing.assert_allclose(Q @ Q.T, np.eye(c.D), atol=1e-15)
    np.testing.assert_allclose(P @ Q.T, parity * Q.T, atol=1e-15)
    # as many rows as the eigenvalue's multiplicity in the spectrum of Pi (numpy's eigensolver)
    ev = np.linalg.eigvalsh(P)
    assert int(np.sum(np.abs(ev - parity) < 1e-9)) == c.D
    # the subspace is invariant under H_K and Hc: H_K Q^T = Q^T H_red
    HK = c.HK.toarray()
    np.testing.assert_allclose(HK @ Q.T, Q.T @ c.H0.toarray(), atol=1e-13)
    np.testing.assert_allclose(c.HcK.toarray() @ Q.T, Q.T @ c.Hc.toarray(), atol=1e-13)


@pytest.mark.parametrize("L,K,parity,grad", [(8, 3, 1, "centered"), (8, 4, -1, "zeroth"), (7, 2, 0, "exact"),
                                             (9, 4, 1, "centered")])
def test_fidelity_and_gradient_equal_the_full_chain(L, K, parity, grad):
    # The PE subspace is invariant, so propagating the embedded states in the full 2^L space gives the
    # same F and gradient (Lanczos from an embedded vector never leaves the subspace).
    c = S.paper_chain(L, K, parity)
    full = oracle.Chain(L, c.Jxy, c.Jz, hc_kind="sz", hc_mask=c.hc_mask, hc_amp=c.hc_amp)
    rng = np.random.default_rng(L * 100 + K)
    N, dt, m = 12, 0.5, 10
    u = rng.uniform(-1, 1, N)
    psi0 = np.zeros(c.D, complex)
    psi0[0] = 1
    f = rng.standard_normal(c.D) + 1j * rng.standard_normal(c.D)
    f /= np.linalg.norm(f)
    F, g, _ = oracle.evaluate(c, u, dt, m, psi0, f, grad)
    Ff, gf, _ = oracle.evaluate(full, u, dt, m, c.embed(psi0), c.embed(f), grad)
    assert abs(F - Ff) <= 1e-12
    np.testing.assert_allclose(g, gf, rtol=0, atol=1e-11 * np.abs(gf).max())


def test_krylov_error_at_the_papers_settings_is_far_below_the_target_infidelity():
    # Sec. 3.2 checks that Krylov and exact final states differ by orders of magnitude less than
    # I_target = 1e-2 at dt = 0.5, m = 10; the dense propagators of the reduced H are the exact side.
    w = W.SECTOR_WORKLOADS["pe_L10_K4"]
    c = S.paper_chain(w.L, w.K)
    u, psi0, f = W.sector_instance(w, c.D)
    F, _, d = oracle.evaluate(c, u[0], w.dt, w.m, psi0, f, "none")
    psi_exact = oracle.exact_forward(c, u[0], w.dt, psi0)[-1]
    # the final states' mutual infidelity, the measure Sec. 3.2 compares with I_target
    assert 1.0 - abs(np.vdot(psi_exact, d["psi_N"])) ** 2 < 1e-4
    assert abs(F - oracle.exact_fidelity(c, u[0], w.dt, psi0, f)) < 1e-4
