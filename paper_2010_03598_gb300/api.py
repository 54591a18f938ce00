"""Python binding of the K-GRAPE C ABI: one evaluation = one call into libkgrape.so.

PyTorch supplies device memory (the workspace and the input/output tensors) and the
CUDA stream; every step of the computation runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import _abi
from ._abi import check, lib

_PREC = {"c128": _abi.KG_PREC_C128, "c64": _abi.KG_PREC_C64_F64REC, "ff": _abi.KG_PREC_FF}
_GRAD = {"none": _abi.KG_GRAD_NONE, "centered": _abi.KG_GRAD_CENTERED, "zeroth": _abi.KG_GRAD_ZEROTH,
         "exact": _abi.KG_GRAD_EXACT, "taylor1": _abi.KG_GRAD_TAYLOR1, "taylor2": _abi.KG_GRAD_TAYLOR2}


@dataclasses.dataclass(frozen=True)
class ChainSpec:
    """Open XXZ chain H0 = sum Jxy (SxSx + SySy) + Jz SzSz with control Hc (Eq. H01, Eq. htot)."""

    L: int
    Jxy: float = 1.0
    Jz: float = 0.5
    hc_kind: str = "sx"      # "sx": hc_amp * Sx on site hc_site+1; "sz": hc_amp * sum_{s in mask} Sz_s
    hc_site: int = 0
    hc_mask: int = 0
    hc_amp: float = 1.0

    def to_c(self) -> _abi.KgChain:
        kind = {"sx": _abi.KG_HC_SX_SITE, "sz": _abi.KG_HC_SZ_SITES}[self.hc_kind]
        return _abi.KgChain(self.L, kind, self.hc_site, 0, self.hc_mask, self.Jxy, self.Jz, self.hc_amp)


@dataclasses.dataclass(frozen=True)
class Options:
    """Pulse (N slices of length dt), Krylov size m and execution options."""

    N: int
    dt: float
    m: int
    prec: str = "c64"         # "c64" (complex64 state, FP64 recurrences), "c128", or "ff" (float-float
                              # vectors; subspace engines only)
    grad: str = "centered"    # "none", "centered", "zeroth", "exact" (Gauss-Lobatto over each slice),
                              # "taylor1", "taylor2" (App. B's hierarchy; subspace engines only)
    ckpt_every: int = 0       # 0: keep every psi_j; C > 0: checkpoint every C slices; -1 (KG_CKPT_AUTO):
                              # every psi_j if the workspace fits mem_budget, else every ceil(sqrt(N))
    mem_budget: int = 0       # bytes for KG_CKPT_AUTO (0: 90 % of the device's free memory)
    tile_bits: int = 0
    ctas: int = 0
    host_staging: bool = False
    phase_timing: bool = False
    breakdown_tol: float = 0.0
    reorth: bool = False      # full Gram-Schmidt (twice) against the whole Krylov basis every step

    def to_c(self) -> _abi.KgOptions:
        flags = (_abi.KG_FLAG_HOST_STAGING if self.host_staging else 0) | \
            (_abi.KG_FLAG_PHASE_TIMING if self.phase_timing else 0) | \
            (_abi.KG_FLAG_FULL_REORTH if self.reorth else 0)
        return _abi.KgOptions(self.N, self.m, _PREC[self.prec], _GRAD[self.grad], self.ckpt_every, self.tile_bits,
                              self.ctas, flags, self.dt, self.breakdown_tol, self.mem_budget)


def workspace_bytes(chain: ChainSpec, opts: Options) -> int:
    n = ctypes.c_size_t(0)
    check(lib().kg_workspace_bytes(ctypes.byref(chain.to_c()), ctypes.byref(opts.to_c()), ctypes.byref(n)),
          "kg_workspace_bytes")
    return int(n.value)


def set_wait_limit_ns(ns: int) -> None:
    check(lib().kg_set_wait_limit_ns(int(ns)), "kg_set_wait_limit_ns")


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


class KGrape:
    """One K-GRAPE problem bound to a device workspace and a CUDA stream.

    ``evaluate`` enqueues one fidelity(+gradient) evaluation (asynchronous);
    ``evaluate_host`` does the same from host buffers and waits; ``sync`` waits and
    returns the device report.  Calls on one object must not overlap.
    """

    def __init__(self, chain: ChainSpec, opts: Options, device: int | torch.device | None = None,
                 stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("KGrape needs a CUDA device; there is no CPU fallback")
        self.chain, self.opts = chain, opts
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = workspace_bytes(chain, opts)
        # over-allocate by 256 bytes and align by hand (the ABI wants 256-byte alignment)
        self._ws_raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws_raw.data_ptr()
        self._ws_off = (-base) % 256
        self.workspace_bytes = nbytes
        h = ctypes.c_void_p(0)
        with torch.cuda.device(self.device):
            check(lib().kg_create(ctypes.byref(h), ctypes.byref(chain.to_c()), ctypes.byref(opts.to_c()),
                                  ctypes.c_void_p(base + self._ws_off), ctypes.c_size_t(nbytes),
                                  ctypes.c_void_p(self.stream.cuda_stream)), "kg_create")
        self._h = h
        self.D = 1 << chain.L
        self.fid = torch.zeros(1, dtype=torch.float64, device=self.device)
        self.grad = torch.zeros(max(opts.N, 1), dtype=torch.float64, device=self.device)

    def _check_inputs(self, u, psi0, target):
        N, D = self.opts.N, self.D
        if u.dtype != torch.float64 or u.numel() != N or not u.is_contiguous():
            raise ValueError(f"u must be a contiguous float64 tensor of {N} controls")
        for name, t in (("psi0", psi0), ("target", target)):
            if t.dtype != torch.complex128 or t.numel() != D or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous complex128 tensor of {D} amplitudes")

    def evaluate(self, u: torch.Tensor, psi0: torch.Tensor, target: torch.Tensor,
                 fid: torch.Tensor | None = None, grad: torch.Tensor | None = None):
        """Enqueue F and dF/du on the stream; returns (fid[1], grad[N]) device tensors."""
        self._check_inputs(u, psi0, target)
        for name, t in (("u", u), ("psi0", psi0), ("target", target)):
            if t.device != self.device:
                raise ValueError(f"{name} must be on {self.device}")
        fid = self.fid if fid is None else fid
        grad = self.grad if grad is None else grad
        with torch.cuda.device(self.device):
            check(lib().kg_evaluate(self._h, _ptr(u), _ptr(psi0), _ptr(target), _ptr(fid),
                                    _ptr(grad) if self.opts.grad != "none" else None), "kg_evaluate")
        return fid, grad[: self.opts.N]

    def evaluate_host(self, u: torch.Tensor, psi0: torch.Tensor, target: torch.Tensor,
                      fid: torch.Tensor | None = None, grad: torch.Tensor | None = None):
        """Evaluate from host (CPU, ideally pinned) tensors; waits; returns host (fid, grad)."""
        if not self.opts.host_staging:
            raise ValueError("create KGrape with Options(host_staging=True) to use evaluate_host")
        self._check_inputs(u, psi0, target)
        for name, t in (("u", u), ("psi0", psi0), ("target", target)):
            if t.device.type != "cpu":
                raise ValueError(f"{name} must be a host tensor")
        if fid is None:
            fid = torch.zeros(1, dtype=torch.float64)
        if grad is None:
            grad = torch.zeros(self.opts.N, dtype=torch.float64)
        with torch.cuda.device(self.device):
            check(lib().kg_evaluate_host(self._h, _ptr(u), _ptr(psi0), _ptr(target), _ptr(fid),
                                         _ptr(grad) if self.opts.grad != "none" else None), "kg_evaluate_host")
        return fid, grad

    def sync(self) -> dict:
        """Wait for the stream; raise on a device-side error; return the report."""
        rep = _abi.KgReport()
        with torch.cuda.device(self.device):
            check(lib().kg_sync(self._h, ctypes.byref(rep)), "kg_sync")
        out = {f: getattr(rep, f) for f, _ in rep._fields_}
        out["phase_cycles"] = list(rep.phase_cycles)
        return out

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().kg_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class KGrapeFidelity(torch.autograd.Function):
    """F(u) with the hand-written adjoint: forward runs the whole forward + co-state
    sweep in one library call (the backward sweep needs the stored forward states), and
    backward returns grad_output * dF/du."""

    @staticmethod
    def forward(ctx, u, engine: KGrape, psi0, target):
        if engine.opts.grad == "none":
            raise ValueError("KGrapeFidelity needs an engine created with a gradient mode")
        fid, grad = engine.evaluate(u.detach(), psi0, target)
        ctx.save_for_backward(grad.clone())
        return fid.clone()

    @staticmethod
    def backward(ctx, g_out):
        (grad,) = ctx.saved_tensors
        return g_out * grad, None, None, None


def fidelity(u: torch.Tensor, engine: KGrape, psi0: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    """Differentiable F(u) (shape [1]) through the K-GRAPE adjoint kernels."""
    return KGrapeFidelity.apply(u, engine, psi0, target)


class KGrapeBatch:
    """Many independent pulses evaluated by one cooperative launch (complex64 path).

    ``chains`` (one ChainSpec per problem) and shared ``opts``; ``u``, ``psi0``, ``target`` are
    lists of device tensors (kept referenced).  ``fid`` (B) and ``grads`` (B x N) are device
    outputs owned by this object.  ``launch()`` enqueues (capturable in a CUDA graph),
    ``sync()`` waits and raises on a device error.
    """

    def __init__(self, chains, opts: Options, u, psi0, target, device=None, stream=None, ctas: int = 0,
                 tiles_per_cta: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("KGrapeBatch needs a CUDA device; there is no CPU fallback")
        B = len(chains)
        if not (len(u) == len(psi0) == len(target) == B):
            raise ValueError("one u, psi0 and target per chain")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.chains, self.opts, self.B = list(chains), opts, B
        for i, (c, ut, pt, ft) in enumerate(zip(chains, u, psi0, target)):
            D = 1 << c.L
            if ut.dtype != torch.float64 or ut.numel() != opts.N or ut.device != self.device:
                raise ValueError(f"problem {i}: u must be {opts.N} float64 on {self.device}")
            for name, t in (("psi0", pt), ("target", ft)):
                if t.dtype != torch.complex128 or t.numel() != D or t.device != self.device:
                    raise ValueError(f"problem {i}: {name} must be {D} complex128 on {self.device}")
        self._keep = (list(u), list(psi0), list(target))
        carr = (_abi.KgChain * B)(*[c.to_c() for c in chains])
        copts = opts.to_c()
        n = ctypes.c_size_t(0)
        check(lib().kg_batch_workspace_bytes(B, carr, ctypes.byref(copts), ctypes.byref(n)), "kg_batch_workspace_bytes")
        self._ws_raw = torch.empty(n.value + 256, dtype=torch.uint8, device=self.device)
        base = self._ws_raw.data_ptr() + ((-self._ws_raw.data_ptr()) % 256)
        self.fid = torch.zeros(B, dtype=torch.float64, device=self.device)
        self.grads = torch.zeros(B, max(opts.N, 1), dtype=torch.float64, device=self.device)
        P = ctypes.c_void_p * B
        up = P(*[t.data_ptr() for t in u])
        pp = P(*[t.data_ptr() for t in psi0])
        fp = P(*[t.data_ptr() for t in target])
        gp = P(*[self.grads[i].data_ptr() for i in range(B)])
        sched = _abi.KgBatchSchedule(ctas, tiles_per_cta, 0, 0)
        h = ctypes.c_void_p(0)
        with torch.cuda.device(self.device):
            check(lib().kg_batch_create(ctypes.byref(h), B, carr, ctypes.byref(copts), ctypes.byref(sched), up, pp,
                                        fp, self.fid.data_ptr(), gp, ctypes.c_void_p(base), ctypes.c_size_t(n.value),
                                        ctypes.c_void_p(self.stream.cuda_stream)), "kg_batch_create")
        self._h = h
        self.workspace_bytes = int(n.value)

    def launch(self) -> None:
        check(lib().kg_batch_launch(self._h), "kg_batch_launch")

    def sync(self) -> int:
        c = ctypes.c_int32(0)
        with torch.cuda.device(self.device):
            check(lib().kg_batch_sync(self._h, ctypes.byref(c)), "kg_batch_sync")
        return int(c.value)

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().kg_batch_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- parity-excitation subspaces
@dataclasses.dataclass(frozen=True)
class SectorSpec:
    """K excitations of an L-site XXZ chain in one parity subspace (Sec. 3.1); Hc = hc_amp sum Sz over mask."""

    L: int
    K: int
    parity: int = 1           # +1 even, -1 odd, 0 the whole K-excitation sector
    Jxy: float = 2.0          # Sec. 3.1 with J = 1, alpha_z = 0.5: Jxy = 2 J, Jz = 2 J alpha_z
    Jz: float = 1.0
    hc_mask: int | None = None  # default: sites 1 and L
    hc_amp: float = 1.0       # Sec. 3.1: (J/2)(sigma^z_1 + sigma^z_L) = J (Sz_1 + Sz_L)
    block_threads: int = 0    # threads per CTA: 0 = chosen from D, or 128, 256, 512 (tune.py times them)

    def to_c(self) -> _abi.KgSector:
        mask = (1 | (1 << (self.L - 1))) if self.hc_mask is None else int(self.hc_mask)
        return _abi.KgSector(self.L, self.K, self.parity, int(self.block_threads), mask, self.Jxy, self.Jz,
                             self.hc_amp)


def sector_dim(spec: SectorSpec) -> int:
    D = ctypes.c_int32(0)
    check(lib().kg_sector_dim(ctypes.byref(spec.to_c()), ctypes.byref(D)), "kg_sector_dim")
    return int(D.value)


def sector_states(spec: SectorSpec):
    """The smaller member s_r of every basis vector's orbit, in basis order (numpy uint64)."""
    import numpy as np

    D = sector_dim(spec)
    out = np.zeros(D, dtype=np.uint64)
    check(lib().kg_sector_states(ctypes.byref(spec.to_c()), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), D),
          "kg_sector_states")
    return out


def sector_apply_h0(spec: SectorSpec, v):
    """H0 v on the host with the kernel's own tables (numpy complex128 in, out): a check, no GPU."""
    import numpy as np

    v = np.ascontiguousarray(v, dtype=np.complex128)
    w = np.zeros_like(v)
    check(lib().kg_sector_apply_h0(ctypes.byref(spec.to_c()), v.ctypes.data, w.ctypes.data, v.shape[0]),
          "kg_sector_apply_h0")
    return w


def sector_workspace_bytes(spec: SectorSpec, opts: Options, B: int) -> int:
    n = ctypes.c_size_t(0)
    check(lib().kg_sector_workspace_bytes(ctypes.byref(spec.to_c()), ctypes.byref(opts.to_c()), B, ctypes.byref(n)),
          "kg_sector_workspace_bytes")
    return int(n.value)


class KGrapeSector:
    """B pulses of one parity-excitation subspace problem, one CTA per pulse (one launch per call).

    ``evaluate(u[B, N], psi0[D], target[D])`` enqueues F and dF/du of every pulse and returns the
    device tensors (fid[B], grad[B, N]); ``sync()`` waits and returns the report.
    """

    def __init__(self, spec: SectorSpec, opts: Options, B: int = 1, device=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("KGrapeSector needs a CUDA device; there is no CPU fallback")
        self.spec, self.opts, self.B = spec, opts, int(B)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.D = sector_dim(spec)
        nbytes = sector_workspace_bytes(spec, opts, self.B)
        self._ws_raw = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws_raw.data_ptr() + ((-self._ws_raw.data_ptr()) % 256)
        self.workspace_bytes = nbytes
        h = ctypes.c_void_p(0)
        with torch.cuda.device(self.device):
            check(lib().kg_sector_create(ctypes.byref(h), ctypes.byref(spec.to_c()), ctypes.byref(opts.to_c()),
                                         self.B, ctypes.c_void_p(base), ctypes.c_size_t(nbytes),
                                         ctypes.c_void_p(self.stream.cuda_stream)), "kg_sector_create")
        self._h = h
        self.fid = torch.zeros(self.B, dtype=torch.float64, device=self.device)
        self.grad = torch.zeros(self.B, max(opts.N, 1), dtype=torch.float64, device=self.device)

    def evaluate(self, u: torch.Tensor, psi0: torch.Tensor, target: torch.Tensor):
        B, N, D = self.B, self.opts.N, self.D
        if u.dtype != torch.float64 or tuple(u.shape) != (B, N) or not u.is_contiguous() or u.device != self.device:
            raise ValueError(f"u must be a contiguous float64 tensor of shape ({B}, {N}) on {self.device}")
        for name, t in (("psi0", psi0), ("target", target)):
            if t.dtype != torch.complex128 or t.numel() != D or not t.is_contiguous() or t.device != self.device:
                raise ValueError(f"{name} must be a contiguous complex128 tensor of {D} amplitudes on {self.device}")
        with torch.cuda.device(self.device):
            check(lib().kg_sector_evaluate(self._h, _ptr(u), _ptr(psi0), _ptr(target), _ptr(self.fid),
                                           _ptr(self.grad) if self.opts.grad != "none" else None),
                  "kg_sector_evaluate")
        return self.fid, self.grad[:, :N]

    def sync(self) -> dict:
        rep = _abi.KgReport()
        with torch.cuda.device(self.device):
            check(lib().kg_sector_sync(self._h, ctypes.byref(rep)), "kg_sector_sync")
        out = {f: getattr(rep, f) for f, _ in rep._fields_}
        out["phase_cycles"] = list(rep.phase_cycles)
        return out

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().kg_sector_destroy(self._h)
            self._h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
