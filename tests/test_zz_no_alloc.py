"""The allocation-free entry point kg_evaluate_static.

Callers that cannot allocate device memory (an application that owns the whole device
memory budget, a plain C caller without a device allocator, a loop that must not pay for
cudaMalloc's synchronisation) evaluate through kg_evaluate_static, which runs the same
evaluation kernel on a fixed scratch array compiled into the library.  These tests call it
through the C ABI and check it against the handle-based kg_evaluate, twice in a row (the
scratch keeps the previous call's contents, so the second call checks that nothing stale
leaks in).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2010_03598_gb300 import _abi
from paper_2010_03598_gb300 import workloads as W

TOL = {"c128": (1e-10, 1e-10), "c64": (1e-5, 1e-4)}


def _static_call(chain, opts, u, psi0, f, fid, grad):
    st = _abi.lib().kg_evaluate_static(ctypes.byref(chain.to_c()), ctypes.byref(opts.to_c()), u.data_ptr(),
                                       psi0.data_ptr(), f.data_ptr(), fid.data_ptr(), grad.data_ptr(), None)
    _abi.check(st, "kg_evaluate_static")


def test_static_entry_point_rejects_a_workspace_above_its_limit():
    from paper_2010_03598_gb300 import api as A
    chain = A.ChainSpec(20)
    opts = A.Options(400, 0.05, 20, prec="c64")
    st = _abi.lib().kg_evaluate_static(ctypes.byref(chain.to_c()), ctypes.byref(opts.to_c()), None, None, None, None,
                                       None, None)
    assert st == _abi.KG_ERR_WORKSPACE
    assert b"static scratch" in _abi.lib().kg_last_error()


@pytest.mark.skipif(torch.cuda.is_available(), reason="needs a process without a CUDA device")
def test_static_entry_point_without_a_context_returns_an_error_and_launches_nothing():
    # No device, hence no context: the call must stop with a status before any launch.
    from paper_2010_03598_gb300 import api as A
    chain = A.ChainSpec(8)
    opts = A.Options(4, 0.1, 6, prec="c64")
    fake = 1 << 12  # aligned, never dereferenced: the call returns before any device work
    st = _abi.lib().kg_evaluate_static(ctypes.byref(chain.to_c()), ctypes.byref(opts.to_c()), fake, fake, fake, fake,
                                       fake, None)
    assert st == _abi.KG_ERR_CUDA


@pytest.mark.gpu
def test_static_entry_point_refuses_a_capturing_stream():
    # The call waits for its stream, which a capture forbids: it must refuse before any work and
    # leave the capture intact.
    from paper_2010_03598_gb300 import api as A
    L, N, m = 8, 4, 6
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(7)
    u = torch.tensor(rng.uniform(-1, 1, N), device=dev)
    psi0 = torch.tensor(W.neel_state(L), device=dev)
    f = torch.tensor(W.draw_target(rng, 1 << L), device=dev)
    fid = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.zeros(N, dtype=torch.float64, device=dev)
    chain, opts = A.ChainSpec(L), A.Options(N, 0.1, m, prec="c64")
    s = torch.cuda.Stream(device=dev)
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g.capture_begin()
        st = _abi.lib().kg_evaluate_static(ctypes.byref(chain.to_c()), ctypes.byref(opts.to_c()), u.data_ptr(),
                                           psi0.data_ptr(), f.data_ptr(), fid.data_ptr(), grad.data_ptr(),
                                           ctypes.c_void_p(s.cuda_stream))
        g.capture_end()
    assert st == _abi.KG_ERR_INVALID_ARG
    assert b"capture" in _abi.lib().kg_last_error()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_static_entry_point_matches_the_workspace_entry_point(prec):
    from paper_2010_03598_gb300 import api as A
    L, N, m = 12, 24, 12
    rng = np.random.default_rng(2024)
    dev = torch.device("cuda", 0)
    u = torch.tensor(rng.uniform(-1, 1, N), device=dev)
    psi0 = torch.tensor(W.neel_state(L), device=dev)
    f = torch.tensor(W.draw_target(rng, 1 << L), device=dev)
    chain = A.ChainSpec(L, 1.0, 0.5)
    opts = A.Options(N, 0.05, m, prec=prec)
    assert A.workspace_bytes(chain, opts) <= _abi.KG_STATIC_WORKSPACE_BYTES

    eng = A.KGrape(chain, opts, device=dev)
    fid_ref, grad_ref = eng.evaluate(u, psi0, f)
    eng.sync()
    F_ref = float(fid_ref.item())
    g_ref = grad_ref.cpu().numpy().copy()
    eng.close()

    tf, tg = TOL[prec]
    for _ in range(2):
        fid = torch.full((1,), -1.0, dtype=torch.float64, device=dev)
        grad = torch.full((N,), -1.0, dtype=torch.float64, device=dev)
        _static_call(chain, opts, u, psi0, f, fid, grad)
        F = float(fid.item())
        g = grad.cpu().numpy()
        assert abs(F - F_ref) <= tf * abs(F_ref)
        assert np.linalg.norm(g - g_ref) <= tg * np.linalg.norm(g_ref)
