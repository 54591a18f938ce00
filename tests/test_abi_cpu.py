"""C-ABI checks that need no GPU: the library loads, exports every function that
include/kgrape.h declares, and rejects bad arguments with the documented status codes."""
import ctypes
import os
import re

import pytest

from paper_2010_03598_gb300 import _abi
from paper_2010_03598_gb300 import build as kbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def header_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(kg_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_abi.LIB_PATH):
        kbuild.build()
    return _abi.lib()


def test_header_declares_functions():
    names = header_functions()
    assert "kg_evaluate" in names and "kg_create" in names and len(names) >= 9


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    assert sorted(_abi.SIGNATURES) == header_functions()


def test_version_and_error_string(lib):
    assert lib.kg_version() >= 100
    assert isinstance(lib.kg_last_error(), bytes)


def _chain(**kw):
    c = dict(L=8, hc_kind=_abi.KG_HC_SX_SITE, hc_site=0, reserved0=0, hc_site_mask=0, Jxy=1.0, Jz=0.5, hc_amp=1.0)
    c.update(kw)
    return _abi.KgChain(**c)


def _opts(**kw):
    o = dict(N=64, m=12, prec=_abi.KG_PREC_C128, grad=_abi.KG_GRAD_CENTERED, ckpt_every=0, tile_bits=0, ctas=0,
             flags=0, dt=0.1, breakdown_tol=0.0)
    o.update(kw)
    return _abi.KgOptions(**o)


def _ws(lib, chain, opts):
    n = ctypes.c_size_t(0)
    st = lib.kg_workspace_bytes(ctypes.byref(chain), ctypes.byref(opts), ctypes.byref(n))
    return st, n.value


def test_workspace_bytes_covers_the_vectors(lib):
    for prec, s in ((_abi.KG_PREC_C128, 16), (_abi.KG_PREC_C64_F64REC, 8)):
        for L, N, m, C in ((8, 64, 12, 0), (10, 23, 5, 4), (16, 200, 20, 0), (20, 400, 20, 20)):
            st, n = _ws(lib, _chain(L=L), _opts(N=N, m=m, prec=prec, ckpt_every=C))
            assert st == _abi.KG_OK
            D = 1 << L
            traj = (N + 1) if C == 0 else (N // C + 1 + (N % C != 0)) + (C + 1)
            vectors = (m - 1) + traj + 2 + 3  # basis, trajectory/checkpoints, co-state pair, W pair + X
            assert n >= vectors * D * s
            assert n < (vectors + 1) * D * s + (1 << 20)
    st, n1 = _ws(lib, _chain(L=12), _opts(flags=_abi.KG_FLAG_HOST_STAGING))
    st, n0 = _ws(lib, _chain(L=12), _opts())
    assert n1 - n0 >= 2 * 16 * 4096


def test_exact_gradient_workspace_and_limits(lib):
    # KG_GRAD_EXACT keeps psi at two interior nodes of every slice (2N more vectors, 2N doubles)
    N, L = 40, 12
    st0, n0 = _ws(lib, _chain(L=L), _opts(N=N, grad=_abi.KG_GRAD_CENTERED))
    st1, n1 = _ws(lib, _chain(L=L), _opts(N=N, grad=_abi.KG_GRAD_EXACT))
    assert st0 == st1 == _abi.KG_OK
    assert n1 - n0 >= 2 * N * (1 << L) * 8
    st, _ = _ws(lib, _chain(L=L), _opts(N=N, grad=_abi.KG_GRAD_EXACT, ckpt_every=5))
    assert st == _abi.KG_ERR_UNSUPPORTED


def test_full_reorthogonalisation_flag_is_accepted(lib):
    # the flag selects another Lanczos arrangement, not more memory: the same workspace
    st1, n1 = _ws(lib, _chain(L=12), _opts(flags=_abi.KG_FLAG_FULL_REORTH))
    st0, n0 = _ws(lib, _chain(L=12), _opts())
    assert st1 == st0 == _abi.KG_OK and n1 == n0


@pytest.mark.parametrize("chain_kw,opts_kw,status", [
    (dict(L=0), {}, _abi.KG_ERR_INVALID_ARG),
    (dict(L=31), {}, _abi.KG_ERR_UNSUPPORTED),
    (dict(hc_site=8), {}, _abi.KG_ERR_INVALID_ARG),
    (dict(hc_kind=_abi.KG_HC_SZ_SITES, hc_site_mask=1 << 8), {}, _abi.KG_ERR_INVALID_ARG),
    (dict(hc_kind=7), {}, _abi.KG_ERR_INVALID_ARG),
    (dict(Jz=float("nan")), {}, _abi.KG_ERR_INVALID_ARG),
    (dict(reserved0=1), {}, _abi.KG_ERR_INVALID_ARG),
    ({}, dict(N=0), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(m=0), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(m=33), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(dt=0.0), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(dt=float("inf")), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(prec=5), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(prec=_abi.KG_PREC_FF), _abi.KG_ERR_UNSUPPORTED),  # float-float vectors: subspaces only
    ({}, dict(grad=9), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(ckpt_every=-2), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(tile_bits=14), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(ctas=5000), _abi.KG_ERR_INVALID_ARG),
    ({}, dict(flags=8), _abi.KG_ERR_INVALID_ARG),
])
def test_invalid_arguments(lib, chain_kw, opts_kw, status):
    st, _ = _ws(lib, _chain(**chain_kw), _opts(**opts_kw))
    assert st == status
    assert len(lib.kg_last_error()) > 0


def test_create_rejects_bad_workspace(lib):
    h = ctypes.c_void_p(0)
    c, o = _chain(), _opts()
    assert lib.kg_create(ctypes.byref(h), ctypes.byref(c), ctypes.byref(o), None, 0, None) == _abi.KG_ERR_WORKSPACE
    assert lib.kg_create(ctypes.byref(h), ctypes.byref(c), ctypes.byref(o), ctypes.c_void_p(256 * 7 + 8), 1 << 30,
                         None) == _abi.KG_ERR_WORKSPACE
    assert lib.kg_create(ctypes.byref(h), ctypes.byref(c), ctypes.byref(o), ctypes.c_void_p(256 * 8), 16,
                         None) == _abi.KG_ERR_WORKSPACE
    assert h.value is None
    assert lib.kg_create(None, ctypes.byref(c), ctypes.byref(o), None, 0, None) == _abi.KG_ERR_INVALID_ARG


def test_null_handles(lib):
    assert lib.kg_evaluate(None, None, None, None, None, None) == _abi.KG_ERR_INVALID_ARG
    assert lib.kg_evaluate_host(None, None, None, None, None, None) == _abi.KG_ERR_INVALID_ARG
    assert lib.kg_sync(None, None) == _abi.KG_ERR_INVALID_ARG
    assert lib.kg_destroy(None) == _abi.KG_OK


def test_wait_limit_and_fault_hook_arguments(lib):
    assert lib.kg_set_wait_limit_ns(0) == _abi.KG_ERR_INVALID_ARG
    assert lib.kg_set_wait_limit_ns(2_000_000_000) == _abi.KG_OK
    assert lib.kg_debug_set_fault(3) == _abi.KG_ERR_INVALID_ARG
    assert lib.kg_debug_set_fault(-1) == _abi.KG_ERR_INVALID_ARG
    assert lib.kg_debug_set_fault(2) == _abi.KG_OK
    assert lib.kg_debug_set_fault(0) == _abi.KG_OK


def test_automatic_checkpoint_interval_follows_the_budget(lib):
    # KG_CKPT_AUTO keeps every psi_j when that workspace fits the budget, and otherwise checkpoints
    # every ceil(sqrt(N)) slices -- the interval that minimises the N/C + C vectors held.
    C64 = _abi.KG_PREC_C64_F64REC
    ch = _chain(L=24)
    full = _ws(lib, ch, _opts(N=400, m=24, prec=C64, ckpt_every=0))[1]
    c20 = _ws(lib, ch, _opts(N=400, m=24, prec=C64, ckpt_every=20))[1]
    assert c20 < full
    for budget, expect in ((full, full), (full - 1, c20), (1, c20)):
        st, n = _ws(lib, ch, _opts(N=400, m=24, prec=C64, ckpt_every=_abi.KG_CKPT_AUTO, mem_budget=budget))
        assert st == _abi.KG_OK and n == expect
    for N, C in ((390, 20), (401, 21), (10, 4)):
        want = _ws(lib, _chain(L=10), _opts(N=N, ckpt_every=C))[1]
        got = _ws(lib, _chain(L=10), _opts(N=N, ckpt_every=_abi.KG_CKPT_AUTO, mem_budget=1))[1]
        assert got == want, (N, C)
    # the exact gradient keeps every slice's interior states: no checkpoints whatever the budget
    ex = dict(N=40, grad=_abi.KG_GRAD_EXACT)
    st, n = _ws(lib, _chain(L=10), _opts(ckpt_every=_abi.KG_CKPT_AUTO, mem_budget=1, **ex))
    assert st == _abi.KG_OK and n == _ws(lib, _chain(L=10), _opts(ckpt_every=0, **ex))[1]
    # other negative intervals and negative budgets are refused
    assert _ws(lib, ch, _opts(ckpt_every=-2))[0] == _abi.KG_ERR_INVALID_ARG
    assert _ws(lib, ch, _opts(ckpt_every=_abi.KG_CKPT_AUTO, mem_budget=-5))[0] == _abi.KG_ERR_INVALID_ARG


def test_package_import_does_not_need_the_library():
    import importlib

    import paper_2010_03598_gb300.workloads as w
    importlib.reload(w)
    assert w.neel_index(4) == 10


def test_header_is_plain_c_and_a_c_program_links_against_the_library(lib, tmp_path):
    # The boundary is a C ABI: the header compiles as C99, and a C caller links against
    # libkgrape.so and calls the host-only entry points (no GPU needed for these).
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_2010_03598_gb300 import _abi
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "caller.c"
    src.write_text(r"""
#include <stdio.h>
#include "kgrape.h"
int main(void) {
  kg_sector s = {20, 4, 1, 0, (1ull << 0) | (1ull << 19), 2.0, 1.0, 1.0};
  int32_t D = 0;
  if (kg_sector_dim(&s, &D) != KG_OK) { printf("error %s\n", kg_last_error()); return 1; }
  kg_chain c = {8, KG_HC_SX_SITE, 0, 0, 0, 1.0, 0.5, 1.0};
  kg_options o = {64, 12, KG_PREC_C64_F64REC, KG_GRAD_CENTERED, 0, 0, 0, 0, 0.1, 0.0};
  size_t bytes = 0;
  if (kg_workspace_bytes(&c, &o, &bytes) != KG_OK) { printf("error %s\n", kg_last_error()); return 1; }
  o.m = 99;
  int bad = kg_workspace_bytes(&c, &o, &bytes);
  printf("%d %d %zu %d\n", kg_version(), D, bytes, bad);
  return 0;
}
""")
    exe = tmp_path / "caller"
    libdir = os.path.dirname(_abi.LIB_PATH)
    cmd = [gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-l:libkgrape.so", f"-Wl,-rpath,{libdir}"]
    cuda_lib = "/usr/local/cuda/lib64"
    if os.path.isdir(cuda_lib):
        cmd += [f"-Wl,-rpath,{cuda_lib}", f"-L{cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    version, D, nbytes, bad = out.stdout.split()
    assert int(D) == 2445 and int(nbytes) > 0 and int(bad) == _abi.KG_ERR_INVALID_ARG
