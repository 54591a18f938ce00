"""GPU parity: the CUDA path (through the C ABI) against the complex128 oracle.

Tolerances (relative; gradients normwise, since single components can be ~0):
  complex128 path:            |dF|/F <= 1e-10, ||dg||/||g|| <= 1e-10
  complex64 + FP64 recurrences: |dF|/F <= 1e-5,  ||dg||/||g|| <= 1e-4
"""
import dataclasses
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2010_03598_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = {"c128": (1e-10, 1e-10), "c64": (1e-5, 1e-4)}


def api():
    from paper_2010_03598_gb300 import api as A
    return A


def golden(stem):
    with open(os.path.join(GOLDEN, stem + ".json")) as fh:
        return json.load(fh)


def to_dev(u, psi0, f):
    dev = torch.device("cuda", 0)
    return (torch.tensor(u, dtype=torch.float64, device=dev), torch.tensor(psi0, dtype=torch.complex128, device=dev),
            torch.tensor(f, dtype=torch.complex128, device=dev))


def run_gpu(chain, opts, u, psi0, f):
    A = api()
    eng = A.KGrape(chain, opts)
    ut, pt, ft = to_dev(u, psi0, f)
    fid, grad = eng.evaluate(ut, pt, ft)
    rep = eng.sync()
    F = float(fid.item())
    g = grad.cpu().numpy().copy() if opts.grad != "none" else None
    eng.close()
    return F, g, rep


def rel(a, b):
    return abs(a - b) / abs(b)


def nrel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def check(prec, F, g, F_ref, g_ref):
    tf, tg = TOL[prec]
    assert rel(F, F_ref) <= tf, (F, F_ref, rel(F, F_ref))
    if g_ref is not None:
        assert nrel(g, g_ref) <= tg, nrel(g, g_ref)


# ------------------------------------------------------------------ L=8, N=64, m=12
@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("mode", ["centered", "zeroth"])
def test_L8_workload_vs_oracle(prec, mode):
    w = W.WORKLOADS["xxz_L8_N64_m12"]
    gd = golden("oracle_xxz_L8_N64_m12")
    u, psi0, f = W.instance(w)
    A = api()
    F, g, rep = run_gpu(A.ChainSpec(w.L, w.Jxy, w.Jz), A.Options(w.N, w.dt, w.m, prec=prec, grad=mode), u, psi0, f)
    check(prec, F, g, gd[f"F_{mode}"], gd[f"grad_{mode}"])
    assert rep["status"] == 0
    assert abs(rep["norm_final"] - 1.0) < (1e-12 if prec == "c128" else 1e-5)


# ------------------------------------------------------------------ tiny and ragged shapes
@pytest.mark.parametrize("L,N,m", [(1, 3, 12), (2, 5, 12), (2, 1, 1), (3, 4, 2), (5, 7, 32), (4, 1, 6)])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_small_shapes_and_breakdown(L, N, m, prec):
    rng = np.random.default_rng(1000 + 10 * L + N)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    ch = oracle.Chain(L, 1.0, 0.5)
    F_ref, g_ref, _ = oracle.evaluate(ch, u, 0.1, m, psi0, f, "centered")
    A = api()
    F, g, rep = run_gpu(A.ChainSpec(L, 1.0, 0.5), A.Options(N, 0.1, m, prec=prec), u, psi0, f)
    check(prec, F, g, F_ref, g_ref)


@pytest.mark.parametrize("tile_bits,ctas", [(6, 1), (6, 3), (6, 16), (4, 7), (10, 1), (5, 0)])
def test_multi_cta_tilings_vs_oracle(tile_bits, ctas):
    # 2^10 amplitudes cut into 2^tile_bits tiles, dealt round robin to `ctas` CTAs
    # (ragged when the tile count is not a multiple of the CTA count).
    L, N, m = 10, 9, 10
    rng = np.random.default_rng(77)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    ch = oracle.Chain(L, 1.0, 0.7)
    F_ref, g_ref, _ = oracle.evaluate(ch, u, 0.07, m, psi0, f, "centered")
    A = api()
    for prec in ("c128", "c64"):
        F, g, rep = run_gpu(A.ChainSpec(L, 1.0, 0.7), A.Options(N, 0.07, m, prec=prec, tile_bits=tile_bits,
                                                                  ctas=ctas), u, psi0, f)
        check(prec, F, g, F_ref, g_ref)


@pytest.mark.parametrize("L,ctas,hc", [(14, 1, ("sx", 0)), (15, 3, ("sx", 13)), (16, 5, ("sz", None)),
                                        (15, 2, ("sx", 5))])
def test_streaming_complex64_tiles_vs_oracle(L, ctas, hc):
    # 4096-amplitude tiles, more than two per CTA (ragged: 4 pairs of tiles on 3 CTAs, 8 on 5):
    # the complex64 streaming loop, with the Sx control inside a tile, above the tile bits, and
    # the paper's Sz edge control.
    N, m, dt = 5, 12, 0.05
    rng = np.random.default_rng(300 + L + ctas)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    kind, site = hc
    if kind == "sx":
        ch = oracle.Chain(L, 1.0, 0.6, "sx", hc_site=site, hc_amp=0.8)
        spec = dict(hc_kind="sx", hc_site=site, hc_amp=0.8)
    else:
        mask = 1 | (1 << (L - 1))
        ch = oracle.Chain(L, 1.0, 0.6, "sz", hc_mask=mask, hc_amp=1.0)
        spec = dict(hc_kind="sz", hc_mask=mask, hc_amp=1.0)
    F_ref, g_ref, _ = oracle.evaluate(ch, u, dt, m, psi0, f, "centered")
    A = api()
    F, g, rep = run_gpu(A.ChainSpec(L, 1.0, 0.6, **spec), A.Options(N, dt, m, prec="c64", tile_bits=12, ctas=ctas),
                        u, psi0, f)
    assert rep["tile_bits"] == 12 and 2 * rep["ctas"] < (1 << (L - 12))  # streaming, not resident
    check("c64", F, g, F_ref, g_ref)


@pytest.mark.parametrize("L,m,dt,tile_bits,ctas", [(7, 32, 1.0, 0, 0), (10, 24, 0.5, 6, 5), (14, 16, 0.2, 12, 1)])
def test_full_reorthogonalisation_vs_oracle(L, m, dt, tile_bits, ctas):
    # KG_FLAG_FULL_REORTH: Gram-Schmidt twice against the whole basis every step, the oracle's
    # own arrangement (Appendix A's remedy).  Long bases over large slices (m = 32 on 128
    # amplitudes with dt = 1) are where plain three-term Lanczos loses orthogonality.
    N = 4
    rng = np.random.default_rng(400 + L)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    ch = oracle.Chain(L, 1.0, 0.5)
    F_ref, g_ref, _ = oracle.evaluate(ch, u, dt, m, psi0, f, "centered")
    A = api()
    for prec in ("c128", "c64"):
        F, g, rep = run_gpu(A.ChainSpec(L, 1.0, 0.5),
                            A.Options(N, dt, m, prec=prec, tile_bits=tile_bits, ctas=ctas, reorth=True), u, psi0, f)
        check(prec, F, g, F_ref, g_ref)
        assert rep["breakdowns"] == 0


@pytest.mark.parametrize("L,N,m,dt,tile_bits,ctas", [(8, 24, 12, 0.1, 0, 0), (10, 6, 12, 0.3, 6, 3),
                                                      (14, 5, 16, 0.05, 12, 1), (16, 6, 20, 0.05, 0, 0)])
def test_exact_gradient_vs_oracle(L, N, m, dt, tile_bits, ctas):
    # KG_GRAD_EXACT (App. B, Eqs. natu_integr / natgrad by Gauss-Lobatto quadrature): generic
    # (L=8, L=10 on ragged tiles), complex64 streaming (L=14 on one CTA) and resident (L=16).
    rng = np.random.default_rng(500 + L)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    ch = oracle.Chain(L, 1.0, 0.5)
    F_ref, g_ref, _ = oracle.evaluate(ch, u, dt, m, psi0, f, "exact")
    A = api()
    for prec in ("c128", "c64"):
        F, g, rep = run_gpu(A.ChainSpec(L, 1.0, 0.5),
                            A.Options(N, dt, m, prec=prec, grad="exact", tile_bits=tile_bits, ctas=ctas), u, psi0, f)
        check(prec, F, g, F_ref, g_ref)
        assert rep["breakdowns"] == 0


def test_exact_gradient_matches_the_dense_derivative():
    # Against the exact propagator derivative of the dense oracle (an independent route):
    # the quadrature leaves O(dt^7) per component, far below the trapezoid rule's O(dt^3).
    L, N, dt, m = 6, 8, 0.2, 16
    rng = np.random.default_rng(61)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    _, g_ex = oracle.exact_gradient(oracle.Chain(L, 1.0, 0.5), u, dt, psi0, f)
    A = api()
    _, g, _ = run_gpu(A.ChainSpec(L, 1.0, 0.5), A.Options(N, dt, m, prec="c128", grad="exact"), u, psi0, f)
    _, gc, _ = run_gpu(A.ChainSpec(L, 1.0, 0.5), A.Options(N, dt, m, prec="c128", grad="centered"), u, psi0, f)
    assert nrel(g, g_ex) <= 1e-8 and nrel(g, g_ex) <= 1e-4 * nrel(gc, g_ex)


@pytest.mark.parametrize("site", [0, 4, 8])
def test_sx_control_on_other_sites(site):
    L, N, m = 9, 6, 12
    rng = np.random.default_rng(5 + site)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    ch = oracle.Chain(L, 1.0, 0.5, "sx", hc_site=site, hc_amp=0.9)
    F_ref, g_ref, _ = oracle.evaluate(ch, u, 0.1, m, psi0, f, "zeroth")
    A = api()
    F, g, _ = run_gpu(A.ChainSpec(L, 1.0, 0.5, "sx", hc_site=site, hc_amp=0.9),
                      A.Options(N, 0.1, m, prec="c128", grad="zeroth", tile_bits=5), u, psi0, f)
    check("c128", F, g, F_ref, g_ref)


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_near_invariant_subspace_in_every_slice(prec):
    # psi0 = |0...0> (an eigenstate of H0 and of the Sz edge control) plus 1 % of a random state:
    # b_1^2 = ||H v_0||^2 - alpha_0^2 cancels to ~1e-4 of ||H v_0||^2 in every slice, so b_1 is
    # formed from ||W_1 - alpha_0 v_0||^2 explicitly before step 1 goes on (complex64 resident
    # loop: 2^14 amplitudes in 4096-amplitude tiles, two per CTA).
    L, N, m, dt = 14, 6, 12, 0.05
    D = 1 << L
    mask = 1 | (1 << (L - 1))
    rng = np.random.default_rng(41)
    u = rng.uniform(-1, 1, N)
    r = (rng.standard_normal(D) + 1j * rng.standard_normal(D)) / np.sqrt(2 * D)
    psi0 = 0.01 * r
    psi0[0] += 1.0
    psi0 /= np.linalg.norm(psi0)
    f = 0.5 * r  # a target with a share of the same random state: the gradient is O(1 %)
    f[0] += 1.0
    f /= np.linalg.norm(f)
    ch = oracle.Chain(L, 1.0, 0.6, "sz", hc_mask=mask, hc_amp=1.0)
    W1 = ch.apply_H(u[0], psi0)
    a0 = np.vdot(psi0, W1).real
    assert (np.vdot(W1, W1).real - a0 * a0) / np.vdot(W1, W1).real < 1e-3  # the identity for b_1^2 cancels
    F_ref, g_ref, _ = oracle.evaluate(ch, u, dt, m, psi0, f, "centered")
    A = api()
    tb = 12 if prec == "c64" else 0
    F, g, rep = run_gpu(A.ChainSpec(L, 1.0, 0.6, "sz", hc_mask=mask, hc_amp=1.0),
                        A.Options(N, dt, m, prec=prec, tile_bits=tb), u, psi0, f)
    # G_j = 2 dt Im <chi_j|Hc|psi_j> is ~2e-4 here, the imaginary part of an overlap of modulus
    # ~0.8: complex64 rounding of that overlap (~1e-7 of it) is ~1e-4 of G, so the complex64
    # gradient is held to 1e-3 (a wrong step-1 basis vector moves G by O(1) of itself).
    tf, tg = TOL[prec]
    assert rel(F, F_ref) <= tf, (F, F_ref)
    assert nrel(g, g_ref) <= (1e-3 if prec == "c64" else tg), nrel(g, g_ref)
    assert rep["status"] == 0 and rep["breakdowns"] == 0
    if prec == "c64":
        assert rep["tile_bits"] == 12 and rep["threads"] == 544  # 16 worker warps and the control warp


def test_paper_control_sz_edges():
    # Sec. 3.1's control Hc = (J/2)(sigma^z_1 + sigma^z_L) = J (Sz_1 + Sz_L)
    L, N, m = 9, 12, 10
    mask = 1 | (1 << (L - 1))
    rng = np.random.default_rng(8)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    ch = oracle.Chain(L, 2.0, 1.0, "sz", hc_mask=mask, hc_amp=1.0)
    F_ref, g_ref, _ = oracle.evaluate(ch, u, 0.5, m, psi0, f, "centered")
    A = api()
    for prec in ("c128", "c64"):
        F, g, _ = run_gpu(A.ChainSpec(L, 2.0, 1.0, "sz", hc_mask=mask, hc_amp=1.0),
                          A.Options(N, 0.5, m, prec=prec, tile_bits=6), u, psi0, f)
        check(prec, F, g, F_ref, g_ref)


@pytest.mark.parametrize("C", [1, 4, 7, 23, 40])
def test_checkpointing_is_bitwise_equal(C):
    # psi_j recomputed from checkpoints must reproduce the stored trajectory exactly.
    L, N, m = 10, 23, 8
    rng = np.random.default_rng(3)
    u = rng.uniform(-1, 1, N)
    f = W.draw_target(rng, 1 << L)
    psi0 = W.neel_state(L)
    A = api()
    for prec in ("c128", "c64"):
        F0, g0, _ = run_gpu(A.ChainSpec(L), A.Options(N, 0.05, m, prec=prec, tile_bits=6, ctas=5), u, psi0, f)
        F1, g1, _ = run_gpu(A.ChainSpec(L), A.Options(N, 0.05, m, prec=prec, tile_bits=6, ctas=5, ckpt_every=C),
                            u, psi0, f)
        assert F0 == F1
        assert np.array_equal(g0, g1)
    ch = oracle.Chain(L, 1.0, 0.5)
    F_ref, g_ref, _ = oracle.evaluate(ch, u, 0.05, m, psi0, f, "centered")
    check("c64", F1, g1, F_ref, g_ref)


# ------------------------------------------------------------------ L=16, N=200, m=20
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_L16_workload_vs_oracle(prec):
    w = W.WORKLOADS["xxz_L16_N200_m20"]
    gd = golden("oracle_xxz_L16_N200_m20")
    u, psi0, f = W.instance(w)
    A = api()
    F, g, rep = run_gpu(A.ChainSpec(w.L, w.Jxy, w.Jz), A.Options(w.N, w.dt, w.m, prec=prec), u, psi0, f)
    check(prec, F, g, gd["F_centered"], gd["grad_centered"])


# ------------------------------------------------------------------ L=20 (the benchmarked chain)
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_L20_short_pulse_vs_oracle(prec):
    # Full chain size and the benchmark's launch configuration; N=2 keeps the oracle to seconds.
    w = W.WORKLOADS["xxz_L20_N400_m20"]
    gd = golden("oracle_xxz_L20_N2_m20")
    u, psi0, f = W.instance(w, N=2)
    A = api()
    for mode in ("centered", "zeroth"):
        F, g, rep = run_gpu(A.ChainSpec(w.L, w.Jxy, w.Jz), A.Options(2, w.dt, w.m, prec=prec, grad=mode), u, psi0, f)
        check(prec, F, g, gd[f"F_{mode}"], gd[f"grad_{mode}"])


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_L20_full_pulse_vs_oracle(prec):
    # The benchmarked configuration in full (N = 400 slices, the benchmark's launch configuration)
    # against the complex128 oracle, element by element; the complex64 result is also
    # deterministic (bitwise equal in a second run).
    w = W.WORKLOADS["xxz_L20_N400_m20"]
    gd = golden("oracle_xxz_L20_N400_m20")
    u, psi0, f = W.instance(w)
    A = api()
    ch = A.ChainSpec(w.L, w.Jxy, w.Jz)
    F, g, rep = run_gpu(ch, A.Options(w.N, w.dt, w.m, prec=prec), u, psi0, f)
    check(prec, F, g, gd["F_centered"], gd["grad_centered"])
    if prec == "c64":
        F2, g2, _ = run_gpu(ch, A.Options(w.N, w.dt, w.m, prec=prec), u, psi0, f)
        assert F == F2 and np.array_equal(g, g2)
        assert abs(rep["norm_final"] - gd["norm_final"]) < 1e-5
    else:
        assert abs(rep["norm_final"] - gd["norm_final"]) < 1e-12
        assert rep["krylov_err_max"] < 1e-12


# ------------------------------------------------------------------ API surface
def test_autograd_function_returns_the_adjoint_gradient():
    w = W.WORKLOADS["xxz_L8_N64_m12"]
    u, psi0, f = W.instance(w)
    A = api()
    eng = A.KGrape(A.ChainSpec(w.L, w.Jxy, w.Jz), A.Options(w.N, w.dt, w.m, prec="c128"))
    ut, pt, ft = to_dev(u, psi0, f)
    ut.requires_grad_(True)
    F = A.fidelity(ut, eng, pt, ft)
    (2.0 * F).sum().backward()
    gd = golden("oracle_xxz_L8_N64_m12")
    assert nrel(ut.grad.cpu().numpy() / 2.0, gd["grad_centered"]) <= 1e-10
    eng.close()


def test_host_buffer_entry_point_matches_device_entry_point():
    w = W.WORKLOADS["xxz_L8_N64_m12"]
    u, psi0, f = W.instance(w)
    A = api()
    eng = A.KGrape(A.ChainSpec(w.L, w.Jxy, w.Jz), A.Options(w.N, w.dt, w.m, prec="c64", host_staging=True))
    uh = torch.tensor(u).pin_memory()
    ph = torch.tensor(psi0).pin_memory()
    fh = torch.tensor(f).pin_memory()
    Fh, gh = eng.evaluate_host(uh, ph, fh)
    ut, pt, ft = to_dev(u, psi0, f)
    Fd, gd_ = eng.evaluate(ut, pt, ft)
    eng.sync()
    assert float(Fh.item()) == float(Fd.item())
    assert np.array_equal(gh.numpy(), gd_.cpu().numpy())
    eng.close()


def test_nonfinite_control_is_reported():
    A = api()
    from paper_2010_03598_gb300 import _abi
    u = np.zeros(4)
    u[1] = np.nan
    eng = A.KGrape(A.ChainSpec(8), A.Options(4, 0.1, 8, prec="c128"))
    ut, pt, ft = to_dev(u, W.neel_state(8), W.draw_target(np.random.default_rng(0), 256))
    eng.evaluate(ut, pt, ft)
    with pytest.raises(_abi.KGrapeError) as ei:
        eng.sync()
    assert ei.value.status == _abi.KG_ERR_NONFINITE
    # the context stays usable
    u[1] = 0.3
    ut.copy_(torch.tensor(u))
    eng.evaluate(ut, pt, ft)
    eng.sync()
    eng.close()


def test_member_that_never_arrives_times_out_cleanly():
    # Fault injected on the host: CTA 0 skips its first barrier arrival; every wait is
    # bounded, so the launch ends with KG_ERR_TIMEOUT and the context stays usable.
    A = api()
    from paper_2010_03598_gb300 import _abi
    L = 10
    eng = A.KGrape(A.ChainSpec(L), A.Options(3, 0.1, 6, prec="c64", tile_bits=6, ctas=4))
    rng = np.random.default_rng(1)
    ut, pt, ft = to_dev(rng.uniform(-1, 1, 3), W.neel_state(L), W.draw_target(rng, 1 << L))
    try:
        A.set_wait_limit_ns(50_000_000)
        _abi.check(_abi.lib().kg_debug_set_fault(1), "kg_debug_set_fault")
        eng.evaluate(ut, pt, ft)
        with pytest.raises(_abi.KGrapeError) as ei:
            eng.sync()
        assert ei.value.status == _abi.KG_ERR_TIMEOUT
    finally:
        A.set_wait_limit_ns(2_000_000_000)
        _abi.lib().kg_debug_set_fault(0)
    eng.evaluate(ut, pt, ft)
    assert eng.sync()["status"] == 0
    eng.close()


def test_member_that_skips_a_lanczos_step_arrival_times_out_cleanly():
    # The same fault at the first Lanczos step's barrier of the resident complex64 loop (2^14
    # amplitudes, 4096-amplitude tiles, two CTAs): CTA 0's control warp does not arrive, every
    # control warp's wait runs out or sees the abort, answers its workers at both named barriers,
    # and the launch ends with KG_ERR_TIMEOUT; the next launch on the same engine is clean.
    A = api()
    from paper_2010_03598_gb300 import _abi
    L = 14
    eng = A.KGrape(A.ChainSpec(L), A.Options(3, 0.1, 8, prec="c64", tile_bits=12))
    rng = np.random.default_rng(2)
    ut, pt, ft = to_dev(rng.uniform(-1, 1, 3), W.neel_state(L), W.draw_target(rng, 1 << L))
    try:
        A.set_wait_limit_ns(50_000_000)
        _abi.check(_abi.lib().kg_debug_set_fault(2), "kg_debug_set_fault")
        eng.evaluate(ut, pt, ft)
        with pytest.raises(_abi.KGrapeError) as ei:
            eng.sync()
        assert ei.value.status == _abi.KG_ERR_TIMEOUT
    finally:
        A.set_wait_limit_ns(2_000_000_000)
        _abi.lib().kg_debug_set_fault(0)
    eng.evaluate(ut, pt, ft)
    rep = eng.sync()
    assert rep["status"] == 0 and rep["threads"] == 544 and rep["ctas"] == 2
    eng.close()


# ------------------------------------------------------------------ adjoint vs finite differences
def test_L20_adjoint_gradient_vs_central_finite_differences():
    # Central FD of F (FP64 path, step 1e-4) at 16 seeded slice indices.  The centred gradient
    # is an approximation with error O(dt^3) per component (App. B): measured 1.9e-4 relative at
    # dt = 0.05; the zeroth-order gradient, O(dt^2), is 50x further off, so 1e-3 discriminates.
    # The complex64 autograd gradient must match the FP64 path's gradient (1e-4).
    w = W.WORKLOADS["xxz_L20_N400_m20"]
    u, psi0, f = W.instance(w)
    idx = W.fd_indices(w)
    A = api()
    chain = A.ChainSpec(w.L, w.Jxy, w.Jz)
    ut, pt, ft = to_dev(u, psi0, f)
    e128 = A.KGrape(chain, A.Options(w.N, w.dt, w.m, prec="c128"))
    e128.evaluate(ut, pt, ft)
    e128.sync()
    g128 = e128.grad[: w.N].cpu().numpy().copy()
    h = 1e-4
    fd = []
    for j in idx:
        vals = []
        for s in (1.0, -1.0):
            uu = u.copy()
            uu[j] += s * h
            ut.copy_(torch.tensor(uu))
            e128.evaluate(ut, pt, ft)
            e128.sync()
            vals.append(float(e128.fid.item()))
        fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    e128.close()
    assert nrel(g128[idx], fd) <= 1e-3, nrel(g128[idx], fd)
    # complex64 adjoint through torch.autograd
    ut.copy_(torch.tensor(u))
    e64 = A.KGrape(chain, A.Options(w.N, w.dt, w.m, prec="c64"))
    ut.requires_grad_(True)
    F = A.fidelity(ut, e64, pt, ft)
    F.sum().backward()
    g64 = ut.grad.cpu().numpy()
    assert nrel(g64, g128) <= 1e-4
    assert nrel(g64[idx], fd) <= 1e-3
    e64.close()


# ------------------------------------------------------------------ autotuned schedule
def test_tuned_single_problem_schedule_gives_the_default_evaluation(tmp_path):
    # The tuner times tile sizes x CTAs; whichever it keeps, the evaluation is the same to rounding
    # (different tilings sum in another order), and the same schedule twice is bitwise equal.
    from paper_2010_03598_gb300 import tune
    A = api()
    w = W.WORKLOADS["xxz_L16_N200_m20"]
    u, psi0, f = W.instance(w, N=12)
    chain = A.ChainSpec(w.L, w.Jxy, w.Jz)
    opts = A.Options(12, w.dt, w.m, prec="c64")
    ut, pt, ft = to_dev(u, psi0, f)
    best = tune.tune_single(chain, opts, ut, pt, ft, cache_path=str(tmp_path / "tune.json"), repeats=1)
    assert sum(t["ms"] is not None for t in best["trials"]) >= 3
    F0, g0, _ = run_gpu(chain, opts, u, psi0, f)
    tuned = dataclasses.replace(opts, tile_bits=best["tile_bits"], ctas=best["ctas"])
    F1, g1, _ = run_gpu(chain, tuned, u, psi0, f)
    F2, g2, _ = run_gpu(chain, tuned, u, psi0, f)
    check("c64", F1, g1, F0, g0)
    assert F1 == F2 and np.array_equal(g1, g2)


# ------------------------------------------------------------------ automatic checkpoint interval
def test_automatic_checkpoint_interval_matches_the_explicit_one():
    # A budget one byte short of the full trajectory makes KG_CKPT_AUTO checkpoint every
    # ceil(sqrt(36)) = 6 slices: bitwise the same evaluation as asking for 6, and reported.
    L, N, m = 14, 36, 12
    A = api()
    chain = A.ChainSpec(L, 1.0, 0.5)
    rng = np.random.default_rng(36)
    u = rng.uniform(-1, 1, N)
    psi0, f = W.neel_state(L), W.draw_target(rng, 1 << L)
    full = A.workspace_bytes(chain, A.Options(N, 0.05, m, prec="c64", ckpt_every=0))
    Fa, ga, repa = run_gpu(chain, A.Options(N, 0.05, m, prec="c64", ckpt_every=-1, mem_budget=full - 1), u, psi0, f)
    Fe, ge, repe = run_gpu(chain, A.Options(N, 0.05, m, prec="c64", ckpt_every=6), u, psi0, f)
    assert repa["ckpt_every"] == 6 and repe["ckpt_every"] == 6
    assert Fa == Fe and np.array_equal(ga, ge)
    Ff, gf, repf = run_gpu(chain, A.Options(N, 0.05, m, prec="c64", ckpt_every=-1, mem_budget=full), u, psi0, f)
    assert repf["ckpt_every"] == 0
    check("c64", Fa, ga, Ff, gf)


# ------------------------------------------------------------------ L=24 with checkpoints
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_L24_checkpointed_backward_sweep_vs_oracle(prec):
    # The L = 24 chain (m = 24) on a 12-slice pulse: psi_j kept every 5 slices and recomputed in the
    # backward sweep, against the complex128 oracle element by element; in complex64 the
    # checkpointed run is also bitwise equal to the one that keeps every psi_j.
    w = W.WORKLOADS["xxz_L24_N400_m24_ckpt20"]
    gd = golden("oracle_xxz_L24_N12_m24")
    A = api()
    chain = A.ChainSpec(w.L, w.Jxy, w.Jz)
    u, psi0, f = W.instance(w, N=12)
    F1, g1, rep1 = run_gpu(chain, A.Options(12, w.dt, w.m, prec=prec, ckpt_every=5), u, psi0, f)
    check(prec, F1, g1, gd["F_centered"], gd["grad_centered"])
    assert abs(rep1["norm_final"] - gd["norm_final"]) < (1e-5 if prec == "c64" else 1e-12)
    if prec == "c64":
        F0, g0, _ = run_gpu(chain, A.Options(12, w.dt, w.m, prec=prec, ckpt_every=0), u, psi0, f)
        assert F0 == F1 and np.array_equal(g0, g1)
