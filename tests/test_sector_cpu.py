"""Host side of the parity-excitation subspace entry points (no GPU): the basis and the kernel's
H0 tables against the oracle's Sec. 3.1 reduction (index work bit-exact), and argument checks."""
import ctypes

import numpy as np
import pytest

import oracle.sector as S
from paper_2010_03598_gb300 import _abi
from paper_2010_03598_gb300 import api as A

@pytest.fixture(autouse=True, scope="module")
def library():
    # the host entry points live in libkgrape.so: build it in-tree if this checkout has none yet
    import os
    from paper_2010_03598_gb300 import build as kbuild
    if not os.path.exists(_abi.LIB_PATH):
        kbuild.build()
    return _abi.lib()


CASES = [(10, 4, 1), (14, 4, 1), (20, 4, 1), (8, 3, -1), (9, 4, 0), (5, 2, 1), (3, 1, 1), (12, 6, 1), (12, 6, -1),
         (2, 1, 1), (2, 1, -1), (6, 0, 1), (7, 7, 1), (17, 4, 1)]


@pytest.mark.parametrize("L,K,parity", CASES)
def test_basis_states_equal_the_oracles(L, K, parity):
    spec = A.SectorSpec(L, K, parity)
    st = A.sector_states(spec).astype(np.int64)
    reps = S.pe_change_of_basis(S.k_sector_states(L, K), L, parity)[1]
    assert A.sector_dim(spec) == reps.shape[0]
    np.testing.assert_array_equal(st, reps)


@pytest.mark.parametrize("L,K,parity", [c for c in CASES if c[0] <= 17])
def test_kernel_tables_reproduce_the_reduced_hamiltonian(L, K, parity):
    Jxy, Jz = 0.7, 1.3
    spec = A.SectorSpec(L, K, parity, Jxy=Jxy, Jz=Jz)
    c = S.SectorChain(L, K, parity, Jxy, Jz, 1 | (1 << (L - 1)), 1.0)
    rng = np.random.default_rng(L * 10 + K)
    v = rng.standard_normal(c.D) + 1j * rng.standard_normal(c.D)
    np.testing.assert_allclose(A.sector_apply_h0(spec, v), c.apply_H0(v), rtol=0, atol=1e-13 * np.abs(v).sum())


def _status(fn, *args):
    return fn(*args)


@pytest.mark.parametrize("kw,status", [
    (dict(L=1, K=0), _abi.KG_ERR_INVALID_ARG),
    (dict(L=6, K=7), _abi.KG_ERR_INVALID_ARG),
    (dict(L=6, K=2, parity=2), _abi.KG_ERR_INVALID_ARG),
    (dict(L=6, K=2, hc_mask=0b000011), _abi.KG_ERR_INVALID_ARG),  # not mirror-symmetric
    (dict(L=6, K=2, hc_mask=1 << 6), _abi.KG_ERR_INVALID_ARG),    # a site beyond L
    (dict(L=22, K=11), _abi.KG_ERR_UNSUPPORTED),                  # too large for one CTA
])
def test_sector_argument_checks(kw, status):
    spec = A.SectorSpec(**kw)
    D = ctypes.c_int32(0)
    assert _abi.lib().kg_sector_dim(ctypes.byref(spec.to_c()), ctypes.byref(D)) == status


def test_asymmetric_mask_is_fine_without_parity():
    assert A.sector_dim(A.SectorSpec(6, 2, 0, hc_mask=0b000011)) == 15


@pytest.mark.parametrize("opts_kw,status", [
    (dict(grad="exact"), _abi.KG_OK),
    (dict(grad="taylor1"), _abi.KG_OK),
    (dict(grad="taylor2"), _abi.KG_OK),
    (dict(ckpt_every=4), _abi.KG_ERR_UNSUPPORTED),
    (dict(tile_bits=6), _abi.KG_ERR_INVALID_ARG),
    (dict(host_staging=True), _abi.KG_ERR_INVALID_ARG),
    (dict(phase_timing=True), _abi.KG_OK),
    (dict(m=33), _abi.KG_ERR_INVALID_ARG),
    (dict(prec="ff"), _abi.KG_OK),
    (dict(prec="ff", grad="zeroth"), _abi.KG_OK),
    (dict(prec="ff", grad="none"), _abi.KG_OK),
    (dict(prec="ff", grad="exact"), _abi.KG_ERR_UNSUPPORTED),
    (dict(prec="ff", grad="taylor2"), _abi.KG_ERR_UNSUPPORTED),
])
def test_sector_option_checks(opts_kw, status):
    spec = A.SectorSpec(10, 4, 1)
    base = dict(N=16, dt=0.5, m=10)
    base.update(opts_kw)
    o = A.Options(**base)
    n = ctypes.c_size_t(0)
    assert _abi.lib().kg_sector_workspace_bytes(ctypes.byref(spec.to_c()), ctypes.byref(o.to_c()), 4,
                                                ctypes.byref(n)) == status


def test_sector_workspace_holds_a_trajectory_per_pulse():
    spec = A.SectorSpec(10, 4, 1)
    o = A.Options(N=440, dt=0.5, m=10, prec="c64")
    one, four = A.sector_workspace_bytes(spec, o, 1), A.sector_workspace_bytes(spec, o, 4)
    D = 110
    assert one >= (440 + 1 + 10) * D * 8
    assert four - one >= 3 * (440 + 1 + 10) * D * 8
    o128 = A.Options(N=440, dt=0.5, m=10, prec="c128")
    assert A.sector_workspace_bytes(spec, o128, 1) >= (440 + 1 + 10) * D * 16
    off = A.Options(N=440, dt=0.5, m=10, prec="ff")  # float-float: 16 bytes per amplitude
    assert A.sector_workspace_bytes(spec, off, 1) == A.sector_workspace_bytes(spec, o128, 1)


def test_sector_create_rejects_a_small_workspace():
    spec = A.SectorSpec(10, 4, 1)
    o = A.Options(N=16, dt=0.5, m=10)
    h = ctypes.c_void_p(0)
    st = _abi.lib().kg_sector_create(ctypes.byref(h), ctypes.byref(spec.to_c()), ctypes.byref(o.to_c()), 1,
                                     ctypes.c_void_p(256), ctypes.c_size_t(1024), None)
    assert st == _abi.KG_ERR_WORKSPACE


@pytest.mark.parametrize("grad", ["taylor1", "taylor2"])
def test_full_chain_refuses_taylor_gradients(grad):
    ch = A.ChainSpec(8, 1.0, 0.5)
    o = A.Options(N=16, dt=0.05, m=10, grad=grad)
    n = ctypes.c_size_t(0)
    assert _abi.lib().kg_workspace_bytes(ctypes.byref(ch.to_c()), ctypes.byref(o.to_c()),
                                         ctypes.byref(n)) == _abi.KG_ERR_UNSUPPORTED


def test_exact_gradient_workspace_keeps_the_interior_states():
    spec = A.SectorSpec(10, 4, 1)
    c = A.Options(N=440, dt=0.5, m=10, prec="c64")
    e = A.Options(N=440, dt=0.5, m=10, prec="c64", grad="exact")
    assert A.sector_workspace_bytes(spec, e, 1) - A.sector_workspace_bytes(spec, c, 1) >= 2 * 440 * 110 * 8


@pytest.mark.parametrize("L", [2, 3, 4, 5, 6, 7, 8, 9])
def test_every_small_subspace_matches_the_oracle(L):
    # every excitation number and parity of the short chains: the basis bit for bit, the kernel's
    # H0 tables against Q H_K Q^T (with an asymmetric-in-Jz coupling so that no term hides)
    rng = np.random.default_rng(L)
    for K in range(L + 1):
        for parity in (1, -1, 0):
            states = S.k_sector_states(L, K)
            reps = S.pe_change_of_basis(states, L, parity)[1]
            if reps.shape[0] == 0:
                continue  # e.g. the odd subspace of a sector of palindromes only
            spec = A.SectorSpec(L, K, parity, Jxy=0.9, Jz=1.7)
            assert A.sector_dim(spec) == reps.shape[0]
            np.testing.assert_array_equal(A.sector_states(spec).astype(np.int64), reps)
            c = S.SectorChain(L, K, parity, 0.9, 1.7, 1 | (1 << (L - 1)), 1.0)
            v = rng.standard_normal(c.D) + 1j * rng.standard_normal(c.D)
            np.testing.assert_allclose(A.sector_apply_h0(spec, v), c.apply_H0(v), rtol=0, atol=1e-13 * np.abs(v).sum())


def test_empty_subspace_is_reported_and_refused():
    # K = 0 on two sites: the only state |00> is a palindrome, so the odd subspace is empty
    spec = A.SectorSpec(2, 0, -1)
    assert A.sector_dim(spec) == 0
    o = A.Options(N=4, dt=0.5, m=4)
    h = ctypes.c_void_p(0)
    st = _abi.lib().kg_sector_create(ctypes.byref(h), ctypes.byref(spec.to_c()), ctypes.byref(o.to_c()), 1,
                                     ctypes.c_void_p(256), ctypes.c_size_t(1 << 20), None)
    assert st == _abi.KG_ERR_INVALID_ARG


def test_large_sectors_are_refused_without_enumerating_them():
    import time
    t0 = time.perf_counter()
    D = ctypes.c_int32(0)
    st = _abi.lib().kg_sector_dim(ctypes.byref(A.SectorSpec(30, 15, 1).to_c()), ctypes.byref(D))
    assert st == _abi.KG_ERR_UNSUPPORTED and time.perf_counter() - t0 < 0.5
    assert "dimension" in _abi.lib().kg_last_error().decode()


def test_closed_form_limit_keeps_odd_subspaces_near_the_limit():
    # L = 14, K = 7: C = 3432, no palindromes (odd K, even L): D = 1716 either parity -- accepted;
    # L = 16, K = 8: C = 12870, 70 palindromes: even 6470, odd 6400 -- refused
    assert A.sector_dim(A.SectorSpec(14, 7, -1)) == 1716
    D = ctypes.c_int32(0)
    for par in (1, -1):
        assert _abi.lib().kg_sector_dim(ctypes.byref(A.SectorSpec(16, 8, par).to_c()),
                                        ctypes.byref(D)) == _abi.KG_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", ["c64", "c128", "ff"])
@pytest.mark.parametrize("L,K", [(14, 4), (20, 4)])
def test_block_shapes_the_library_accepts_are_the_tuners_candidates(prec, L, K):
    # kg_sector_workspace_bytes answers KG_ERR_INVALID_ARG for a block that cannot cover D; the
    # autotuner must offer exactly the shapes it accepts (float-float takes the complex128 shapes)
    import dataclasses

    from paper_2010_03598_gb300 import tune
    D = A.sector_dim(A.SectorSpec(L, K, 1))
    ok = set()
    for nt in (0, 128, 256, 512):
        spec = dataclasses.replace(A.SectorSpec(L, K, 1), block_threads=nt)
        o = A.Options(N=16, dt=0.5, m=10, prec=prec)
        n = ctypes.c_size_t(0)
        st = _abi.lib().kg_sector_workspace_bytes(ctypes.byref(spec.to_c()), ctypes.byref(o.to_c()), 4,
                                                  ctypes.byref(n))
        assert st in (_abi.KG_OK, _abi.KG_ERR_INVALID_ARG)
        if st == _abi.KG_OK:
            ok.add(nt)
    assert ok == {c["block_threads"] for c in tune.sector_candidates(D, prec, 152)}
