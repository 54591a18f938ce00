"""Pins for the CPU oracle: every check compares it with something that does not
come from the oracle (Kronecker-product Hamiltonians, closed forms at L=1 and L=2,
scipy's expm, invariants, finite differences, error orders stated in the paper)."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_2010_03598_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

# ---------------------------------------------------------------- Kronecker model
SX = np.array([[0, 0.5], [0.5, 0]], dtype=np.complex128)
SY = np.array([[0, -0.5j], [0.5j, 0]], dtype=np.complex128)
SZ = np.array([[0.5, 0], [0, -0.5]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)


def site_op(L, bit, op):
    """Operator ``op`` on bit ``bit`` of the basis index (np.kron: first factor = MSB)."""
    out = np.ones((1, 1), dtype=np.complex128)
    for b in range(L - 1, -1, -1):
        out = np.kron(out, op if b == bit else I2)
    return out


def kron_H(L, Jxy, Jz, u, hc_kind="sx", hc_site=0, hc_mask=0, hc_amp=1.0):
    D = 1 << L
    H = np.zeros((D, D), dtype=np.complex128)
    for b in range(L - 1):
        H += Jxy * (site_op(L, b, SX) @ site_op(L, b + 1, SX) + site_op(L, b, SY) @ site_op(L, b + 1, SY))
        H += Jz * site_op(L, b, SZ) @ site_op(L, b + 1, SZ)
    if hc_kind == "sx":
        H += u * hc_amp * site_op(L, hc_site, SX)
    else:
        for s in range(L):
            if (hc_mask >> s) & 1:
                H += u * hc_amp * site_op(L, s, SZ)
    return H


def rand_state(rng, D):
    v = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    return v / np.linalg.norm(v)


# ---------------------------------------------------------------- conventions
def test_neel_index_from_string():
    # "|0101...>": site 1 first, '0' = spin up = bit value 0, site k <-> bit k-1.
    for L in range(1, 13):
        s = "".join("0" if k % 2 == 1 else "1" for k in range(1, L + 1))
        idx = sum(int(ch) << (k) for k, ch in enumerate(s))
        assert W.neel_index(L) == idx
    assert W.neel_index(8) == 170


@pytest.mark.parametrize("L", [1, 2, 3, 5, 7])
@pytest.mark.parametrize("kind", ["sx", "sz"])
def test_hv_matches_kronecker(L, kind):
    rng = np.random.default_rng(L * 7 + (kind == "sz"))
    Jxy, Jz, u = rng.uniform(0.3, 1.7), rng.uniform(-1.2, 1.2), rng.uniform(-1, 1)
    site = int(rng.integers(0, L))
    mask = 1 | (1 << (L - 1))
    ch = oracle.Chain(L, Jxy, Jz, kind, hc_site=site, hc_mask=mask, hc_amp=0.8)
    H = kron_H(L, Jxy, Jz, u, kind, site, mask, 0.8)
    v = rand_state(rng, 1 << L)
    np.testing.assert_allclose(ch.apply_H(u, v), H @ v, atol=1e-13, rtol=0)
    np.testing.assert_allclose(ch.dense_H(u), H, atol=1e-13, rtol=0)
    assert np.allclose(H, H.conj().T)


def test_paper_normalisation_reading():
    # Eq. H01: (J/2) sum sigma.sigma with anisotropy alpha_z equals
    # Jxy=2J, Jz=2J*alpha_z on S operators (S = sigma/2, sigma.sigma = 4 S.S).
    L, Jp, az = 4, 1.0, 0.5
    D = 1 << L
    sx, sy, sz = 2 * SX, 2 * SY, 2 * SZ
    Hp = np.zeros((D, D), dtype=np.complex128)
    for b in range(L - 1):
        Hp += 0.5 * Jp * (site_op(L, b, sx) @ site_op(L, b + 1, sx) + site_op(L, b, sy) @ site_op(L, b + 1, sy)
                          + az * site_op(L, b, sz) @ site_op(L, b + 1, sz))
    ch = oracle.Chain(L, 2 * Jp, 2 * Jp * az)
    np.testing.assert_allclose(ch.dense_H(0.0), Hp, atol=1e-13)


def test_sz_conservation_of_drift():
    L = 6
    Stot = sum(site_op(L, b, SZ) for b in range(L))
    H0 = kron_H(L, 1.0, 0.5, 0.0)
    assert np.abs(H0 @ Stot - Stot @ H0).max() < 1e-13
    ch = oracle.Chain(L, 1.0, 0.5, "sz", hc_mask=1 | (1 << (L - 1)), hc_amp=1.0)
    H = ch.dense_H(0.7)
    assert np.abs(H @ Stot - Stot @ H).max() < 1e-13


# ---------------------------------------------------------------- Krylov step
@pytest.mark.parametrize("L,dt,m,tol", [(6, 0.1, 12, 1e-12), (8, 0.1, 12, 1e-12), (8, 0.05, 20, 1e-12),
                                        (7, 0.5, 10, 1e-8)])
def test_krylov_step_vs_expm(L, dt, m, tol):
    rng = np.random.default_rng(100 + L)
    u = rng.uniform(-1, 1)
    ch = oracle.Chain(L, 1.0, 0.5)
    v = rand_state(rng, 1 << L)
    H = kron_H(L, 1.0, 0.5, u)
    ref = scipy.linalg.expm(-1j * dt * H) @ v
    got, info = oracle.krylov_step(lambda x: ch.apply_H(u, x), v, dt, m, +1)
    err = np.linalg.norm(got - ref)
    assert err < tol
    back, _ = oracle.krylov_step(lambda x: ch.apply_H(u, x), v, dt, m, -1)
    refb = scipy.linalg.expm(+1j * dt * H) @ v
    assert np.linalg.norm(back - refb) < tol
    # the a-posteriori indicator is of the size of the true error (or below rounding)
    assert info["err_est"] < 1e3 * max(err, 1e-15)
    if err > 1e-13:
        assert info["err_est"] > 1e-3 * err


def test_krylov_error_order_in_dt():
    # App. A: error O(dt^N) for a basis of N vectors when dt < N^2 / W.
    L, m = 8, 4
    rng = np.random.default_rng(5)
    ch = oracle.Chain(L, 1.0, 0.5)
    v = rand_state(rng, 1 << L)
    H = kron_H(L, 1.0, 0.5, 0.3)
    errs = []
    dts = [0.08, 0.04, 0.02]
    for dt in dts:
        ref = scipy.linalg.expm(-1j * dt * H) @ v
        got, _ = oracle.krylov_step(lambda x: ch.apply_H(0.3, x), v, dt, m, +1)
        errs.append(np.linalg.norm(got - ref))
    slopes = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    for s in slopes:
        assert m - 0.3 < s < m + 0.3, slopes


def test_expm_e1_against_scipy():
    rng = np.random.default_rng(9)
    for n in (1, 2, 5, 12, 24, 32):
        a = rng.uniform(-3, 3, n)
        b = rng.uniform(0.1, 2, n - 1)
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        for sigma in (1, -1):
            ref = scipy.linalg.expm(-1j * sigma * 0.37 * T)[:, 0]
            np.testing.assert_allclose(oracle.expm_e1(a, b, 0.37, sigma), ref, atol=1e-14)


def test_breakdown_is_exact():
    # D = 4 < m: the Krylov space is invariant after <= 4 vectors; step equals expm.
    rng = np.random.default_rng(3)
    ch = oracle.Chain(2, 1.0, 0.5)
    v = rand_state(rng, 4)
    got, info = oracle.krylov_step(lambda x: ch.apply_H(0.4, x), v, 0.3, 12, +1)
    assert info["broke"] and info["meff"] <= 4
    ref = scipy.linalg.expm(-1j * 0.3 * kron_H(2, 1.0, 0.5, 0.4)) @ v
    assert np.linalg.norm(got - ref) < 1e-13


# ---------------------------------------------------------------- closed forms
def test_L1_closed_form_fidelity_and_gradients():
    # L=1: H0 = 0, H = u Sx; the slices commute, psi_N = cos(th)|0> - i sin(th)|1>,
    # th = (dt/2) sum u.  [H_j, Hc] = 0 makes every gradient mode exact:
    # dF/du_j = (dt/2) dF/dth.
    rng = np.random.default_rng(11)
    N, dt = 9, 0.13
    u = rng.uniform(-1, 1, N)
    f = rand_state(rng, 2)
    th = 0.5 * dt * u.sum()
    A = np.conj(f[0]) * np.cos(th) - 1j * np.conj(f[1]) * np.sin(th)
    dA = -np.conj(f[0]) * np.sin(th) - 1j * np.conj(f[1]) * np.cos(th)
    F_ref = abs(A) ** 2
    g_ref = 0.5 * dt * 2.0 * (np.conj(A) * dA).real
    ch = oracle.Chain(1, 1.0, 0.5)
    for mode in ("centered", "zeroth"):
        F, g, d = oracle.evaluate(ch, u, dt, 12, W.neel_state(1), f, mode)
        assert abs(F - F_ref) < 1e-14
        np.testing.assert_allclose(g, np.full(N, g_ref), atol=1e-14)
    np.testing.assert_allclose(d["psi_N"], [np.cos(th), -1j * np.sin(th)], atol=1e-14)


def _exp2(M, tau):
    p, c, q = M[0, 0], M[0, 1], M[1, 1]
    a, b = 0.5 * (p + q), 0.5 * (p - q)
    w = np.hypot(b, c)
    if w == 0:
        return np.exp(-1j * a * tau) * np.eye(2)
    K = np.array([[b, c], [c, -b]]) / w
    return np.exp(-1j * a * tau) * (np.cos(w * tau) * np.eye(2) - 1j * np.sin(w * tau) * K)


def test_L2_closed_form_forward():
    # L=2: H commutes with the global spin flip; on the even basis
    # {(|0>+|3>)/r2, (|1>+|2>)/r2} H = [[Jz/4, u/2], [u/2, Jxy/2 - Jz/4]], on the odd basis
    # {(|0>-|3>)/r2, (|1>-|2>)/r2} H = [[Jz/4, u/2], [u/2, -Jxy/2 - Jz/4]].
    rng = np.random.default_rng(12)
    Jxy, Jz, N, dt = 1.0, 0.5, 17, 0.21
    u = rng.uniform(-1, 1, N)
    f = rand_state(rng, 4)
    r2 = np.sqrt(2.0)
    # Neel "01" = site 2 down = index 2 = (e2 - o2)/r2.
    ev = np.array([0.0, 1.0 / r2], dtype=np.complex128)
    od = np.array([0.0, -1.0 / r2], dtype=np.complex128)
    for uj in u:
        ev = _exp2(np.array([[Jz / 4, uj / 2], [uj / 2, Jxy / 2 - Jz / 4]]), dt) @ ev
        od = _exp2(np.array([[Jz / 4, uj / 2], [uj / 2, -Jxy / 2 - Jz / 4]]), dt) @ od
    psi = np.zeros(4, dtype=np.complex128)
    psi[0] = (ev[0] + od[0]) / r2
    psi[3] = (ev[0] - od[0]) / r2
    psi[1] = (ev[1] + od[1]) / r2
    psi[2] = (ev[1] - od[1]) / r2
    ch = oracle.Chain(2, Jxy, Jz)
    F, _, d = oracle.evaluate(ch, u, dt, 12, W.neel_state(2), f, "none")
    np.testing.assert_allclose(d["psi_N"], psi, atol=1e-13)
    assert abs(F - abs(np.vdot(f, psi)) ** 2) < 1e-13


# ---------------------------------------------------------------- invariants
def test_norm_and_sector_conservation():
    w = W.WORKLOADS["xxz_L8_N64_m12"]
    ch = oracle.Chain(w.L, w.Jxy, w.Jz)
    u0 = np.zeros(20)
    psis, _ = oracle.forward(ch, u0, w.dt, w.m, W.neel_state(w.L))
    idx = np.arange(w.D)
    pop = np.array([bin(i).count("1") for i in idx])
    outside = pop != w.L // 2
    for p in psis:
        assert np.all(p[outside] == 0.0)  # bitwise: H0 maps the sector into itself
        assert abs(np.linalg.norm(p) - 1.0) < 1e-13
    u, psi0, f = W.instance(w, N=20)
    psis, _ = oracle.forward(ch, u, w.dt, w.m, psi0)
    for p in psis:
        assert abs(np.linalg.norm(p) - 1.0) < 1e-13


def test_target_equal_final_state_gives_unit_fidelity_zero_gradient():
    w = W.WORKLOADS["xxz_L8_N64_m12"]
    ch = oracle.Chain(w.L, w.Jxy, w.Jz)
    u, psi0, _ = W.instance(w, N=16)
    psis, _ = oracle.forward(ch, u, w.dt, w.m, psi0)
    F, g, d = oracle.evaluate(ch, u, w.dt, w.m, psi0, psis[-1], "centered")
    assert abs(F - 1.0) < 1e-13
    assert np.abs(g).max() < 1e-13
    # backward sweep returns to the initial state
    assert np.linalg.norm(d["chi_0"] - psi0) < 1e-12


def test_global_phase_of_target_is_irrelevant():
    w = W.WORKLOADS["xxz_L8_N64_m12"]
    ch = oracle.Chain(w.L, w.Jxy, w.Jz)
    u, psi0, f = W.instance(w, N=12)
    F1, g1, _ = oracle.evaluate(ch, u, w.dt, w.m, psi0, f)
    F2, g2, _ = oracle.evaluate(ch, u, w.dt, w.m, psi0, np.exp(0.77j) * f)
    assert abs(F1 - F2) < 1e-15
    np.testing.assert_allclose(g1, g2, atol=1e-16, rtol=1e-12)


# ---------------------------------------------------------------- gradients
def test_krylov_fidelity_equals_dense():
    w = W.WORKLOADS["xxz_L8_N64_m12"]
    ch = oracle.Chain(w.L, w.Jxy, w.Jz)
    u, psi0, f = W.instance(w)
    F, _, d = oracle.evaluate(ch, u, w.dt, w.m, psi0, f, "none")
    psis = oracle.exact_forward(ch, u, w.dt, psi0)
    assert np.linalg.norm(d["psi_N"] - psis[-1]) < 1e-12
    assert abs(F - abs(np.vdot(f, psis[-1])) ** 2) <= 1e-12 * F


@pytest.mark.parametrize("kind", ["sx", "sz"])
def test_exact_gradient_vs_central_fd(kind):
    rng = np.random.default_rng(21)
    L, N, dt = 4, 10, 0.3
    ch = oracle.Chain(L, 1.0, 0.5, kind, hc_site=1, hc_mask=1 | (1 << (L - 1)), hc_amp=1.0)
    u = rng.uniform(-1, 1, N)
    psi0 = rand_state(rng, 1 << L)
    f = rand_state(rng, 1 << L)
    F, g = oracle.exact_gradient(ch, u, dt, psi0, f)
    h = 1e-4
    fd = np.zeros(N)
    for j in range(N):
        up, um = u.copy(), u.copy()
        up[j] += h
        um[j] -= h
        fd[j] = (oracle.exact_fidelity(ch, up, dt, psi0, f) - oracle.exact_fidelity(ch, um, dt, psi0, f)) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(fd)


def _grad_errors(mode, Ns, L=4, T=2.0):
    rng = np.random.default_rng(33)
    ch = oracle.Chain(L, 1.0, 0.5)
    psi0 = W.neel_state(L)
    f = rand_state(rng, 1 << L)
    errs = []
    for N in Ns:
        dt = T / N
        t = (np.arange(N) + 0.5) * dt
        u = 0.7 * np.sin(np.pi * t / T) + 0.4 * np.cos(3 * np.pi * t / T)
        _, g_ex = oracle.exact_gradient(ch, u, dt, psi0, f)
        _, g, _ = oracle.evaluate(ch, u, dt, 14, psi0, f, mode)
        errs.append(np.abs(g - g_ex).max())
    return errs


def test_zeroth_order_gradient_error_is_order_dt2():
    errs = _grad_errors("zeroth", [16, 32, 64])
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.4 < r < 4.6 for r in ratios), ratios


def test_centred_gradient_error_is_order_dt3():
    # App. B: the centred zeroth-order gradient has error O(dt^3) instead of O(dt^2).
    errs = _grad_errors("centered", [16, 32, 64])
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(6.8 < r < 9.2 for r in ratios), ratios


def test_centred_gradient_uses_both_slice_ends():
    # A plausible off-by-one (pairing G_j with G_{j+1}) breaks the O(dt^3) order;
    # the trapezoid pairing (G_{j-1}, G_j) is the one that matches the exact gradient best.
    rng = np.random.default_rng(44)
    L, N, dt = 4, 24, 0.1
    ch = oracle.Chain(L, 1.0, 0.5)
    u = rng.uniform(-1, 1, N)
    psi0 = W.neel_state(L)
    f = rand_state(rng, 1 << L)
    _, g_ex = oracle.exact_gradient(ch, u, dt, psi0, f)
    _, g_c, d = oracle.evaluate(ch, u, dt, 14, psi0, f, "centered")
    G = d["G"]
    shifted = 0.5 * (G[1:] + np.append(G[2:], G[-1]))
    assert np.abs(g_c - g_ex).max() < 0.5 * np.abs(shifted - g_ex).max()


def test_lobatto_gradient_error_is_order_dt7():
    # Eqs. natu_integr / natgrad integrated with the 4-point Gauss-Lobatto rule (degree 5):
    # the per-component error falls by 2^7 when dt halves.
    errs = _grad_errors("exact", [4, 8, 16])
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(90.0 < r < 170.0 for r in ratios), (errs, ratios)


@pytest.mark.parametrize("L", [4, 5, 6])
def test_lobatto_gradient_matches_the_dense_derivative(L):
    # Against the exact propagator derivative (divided differences of the slice eigensystem,
    # an independent route): agreement far beyond the trapezoid rule's, which pairs the same
    # end nodes -- a wrong interior node pairing (chi at s with psi at dt - s) or wrong weights
    # would leave an O(dt) or O(dt^3) error instead.
    rng = np.random.default_rng(10 + L)
    N, dt = 6, 0.2
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    ch = oracle.Chain(L, 1.0, 0.5)
    _, g_ex = oracle.exact_gradient(ch, u, dt, psi0, f)
    _, g_l, d = oracle.evaluate(ch, u, dt, 16, psi0, f, "exact")
    _, g_c, _ = oracle.evaluate(ch, u, dt, 16, psi0, f, "centered")
    err_l = np.linalg.norm(g_l - g_ex) / np.linalg.norm(g_ex)
    err_c = np.linalg.norm(g_c - g_ex) / np.linalg.norm(g_ex)
    assert err_l <= 1e-8 and err_l <= 1e-4 * err_c, (err_l, err_c)
    assert d["G_interior"].shape == (N, 2)


@pytest.mark.parametrize("mode,Ns,lo,hi", [("taylor1", [16, 32, 64], 6.8, 9.2),    # O(dt^3)
                                           ("taylor2", [8, 16, 32], 13.5, 18.5),   # O(dt^4)
                                           ("taylor3", [8, 16, 32], 26.0, 36.0)])  # O(dt^5)
def test_taylor_hierarchy_error_orders(mode, Ns, lo, hi):
    # App. B, Eq. gradp: each level p of Hbar_c^[P] adds one order in dt to the slice average of
    # the control operator, so the gradient error falls as dt^(P+2).
    errs = _grad_errors(mode, Ns)
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(lo < r < hi for r in ratios), (errs, ratios)


def test_taylor_level_zero_is_the_zeroth_order_gradient():
    from oracle.grape import taylor_gradient
    rng = np.random.default_rng(4)
    L, N, dt = 4, 10, 0.1
    ch = oracle.Chain(L, 1.0, 0.5)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    F, g0, d = oracle.evaluate(ch, u, dt, 14, psi0, f, "zeroth")
    psis, _ = oracle.forward(ch, u, dt, 14, psi0)
    gt = taylor_gradient(ch, u, dt, 14, psis, d["beta"] * f, 0)
    np.testing.assert_allclose(gt, g0, rtol=0, atol=1e-14)


def test_taylor_hierarchy_converges_to_the_dense_derivative():
    # Hbar_c^[P] is a convergent series: at P = 6 and dt = 0.1 the gradient equals the exact
    # propagator derivative (divided differences, an independent route) to ~1e-9.
    rng = np.random.default_rng(12)
    L, N, dt = 5, 6, 0.1
    ch = oracle.Chain(L, 1.0, 0.5)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    _, g_ex = oracle.exact_gradient(ch, u, dt, psi0, f)
    _, g6, _ = oracle.evaluate(ch, u, dt, 16, psi0, f, "taylor6")
    assert np.linalg.norm(g6 - g_ex) / np.linalg.norm(g_ex) < 1e-9
