"""B300-native FFT--HSS preconditioned GMRES for the periodic tangent-plane LLG
saddle system (arXiv 2607.15290).

Thin Python binding of the C ABI in ``include/llg.h``: every function here
only checks shapes/dtypes, allocates output tensors (PyTorch is used for device
memory and streams) and forwards raw device pointers to the CUDA library.  All
arithmetic of the method runs in the library's kernels; if the library is
missing the calls raise, there is no CPU fallback.

Array conventions: ``m`` is (3, *grid_shape) and saddle vectors ``x = (v, r)``
are (4, *grid_shape), float64 CUDA tensors, grid_shape = (n1, n0) in 2D or
(n2, n1, n0) in 3D (x fastest), matching the node index j = i0 + n0 (i1 + n1 i2).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

from . import _abi
from ._abi import CHAIN_F32X2, CHAIN_FP64, EX_FD2, EX_SPECTRAL, GS_F32X2, GS_FP64, PLAN_CLUSTER, PLAN_FIVE, PC_FFTHSS, PC_HERMITIAN, PC_NONE, PREC_FP32_FLEX, PREC_FP64

__all__ = [
    "LLGError", "Params", "Opts", "Context", "EX_SPECTRAL", "EX_FD2", "PREC_FP64", "PREC_FP32_FLEX",
    "llg_saddle_apply", "llg_saddle_apply_f32x2", "llg_ffthss_apply", "llg_ffthss_apply_f32", "llg_precond_saddle_apply",
    "llg_gmres_solve", "llg_step_euler", "llg_step_midpoint", "llg_adjoint_step", "llg_energy", "Ensemble",
]


def parse_axis_shape(shape):
    """(kind, E, TW, CB) of an axis-pass shape in the autotuner's notation: register(E8,TW16),
    staged(TW32,CB16), paired(E8,TW16), tma(TW8), tma(E16,TW8)."""
    import re
    m = re.fullmatch(r"(register|staged|paired|tma)\((.*)\)", shape.strip())
    if not m:
        raise ValueError(f"unknown axis shape {shape!r}")
    kv = dict(re.findall(r"([A-Z]+)(\d+)", m.group(2)))
    if not kv.get("TW") or set(kv) - {"E", "TW", "CB"}:
        raise ValueError(f"unknown axis shape {shape!r}")
    kind = {"register": 0, "staged": 1, "paired": 3, "tma": 4}[m.group(1)]
    return kind, int(kv.get("E", 8)), int(kv["TW"]), int(kv.get("CB", 0))


class LLGError(RuntimeError):
    def __init__(self, status, msg, info=None):
        super().__init__(f"{_abi.STATUS.get(status, status)}: {msg}")
        self.status = status
        self.info = info


@dataclass
class Params:
    alpha: float = 0.2
    c_ex: float = 1.0
    k: float = 1e-2
    theta: float = 1.0
    lam: float = 0.5
    h_ext: tuple = (0.0, 0.0, 0.0)
    exchange: int = EX_SPECTRAL
    # optional per-node applied field added to h_ext: CUDA float64 tensor (3, *grid), passed
    # per step (sampled at t_{n+1} for Euler, t_{n+1/2} for the midpoint scheme)
    h_field: object = None
    # uniaxial anisotropy k_an (1 - (e_an.m)^2) and the periodic demagnetising field (Sec. 4.6)
    k_an: float = 0.0
    e_an: tuple = (0.0, 0.0, 1.0)
    demag: int = 0

    def c(self, ctx=None):
        p = _abi.Params()
        p.alpha, p.c_ex, p.k, p.theta, p.lam = self.alpha, self.c_ex, self.k, self.theta, self.lam
        for i in range(3):
            p.h_ext[i] = self.h_ext[i]
            p.e_an[i] = self.e_an[i]
        p.exchange = self.exchange
        p.k_an, p.demag = self.k_an, int(self.demag)
        p.h_field = None
        if self.h_field is not None:
            hf = self.h_field
            torch = _torch()
            if not (isinstance(hf, torch.Tensor) and hf.is_cuda and hf.dtype == torch.float64 and hf.is_contiguous()):
                raise TypeError("h_field must be a contiguous CUDA float64 tensor of 3 planes")
            if ctx is not None and hf.numel() != 3 * ctx.nodes:
                raise ValueError(f"h_field has {hf.numel()} values, the grid needs {3 * ctx.nodes}")
            p.h_field = hf.data_ptr()
        return p


@dataclass
class Opts:
    restart: int = 30
    max_iters: int = 3000
    rtol: float = 1e-10
    precision: int = PREC_FP64
    picard_max: int = 50
    picard_tol: float = 1e-10
    diagnostics: int = 0
    preconditioner: int = PC_FFTHSS
    gs_arith: int = GS_FP64
    chain_arith: int = CHAIN_FP64

    def c(self):
        o = _abi.Opts()
        o.restart, o.max_iters, o.rtol, o.precision = self.restart, self.max_iters, self.rtol, self.precision
        o.picard_max, o.picard_tol, o.diagnostics = self.picard_max, self.picard_tol, self.diagnostics
        o.preconditioner, o.gs_arith = self.preconditioner, self.gs_arith
        o.chain_arith = self.chain_arith
        return o


def _torch():
    import torch
    return torch


class Context:
    """Owns an ``llg_ctx`` for one periodic grid on the current CUDA device/stream."""

    def __init__(self, n, L=None, stream=None):
        torch = _torch()
        self.lib = _abi.lib()
        self.n = tuple(int(v) for v in n)
        self.L = tuple(float(v) for v in (L if L is not None else (1.0,) * len(self.n)))
        g = _abi.Grid()
        g.dim = len(self.n)
        for i in range(3):
            g.n[i] = self.n[i] if i < g.dim else 1
            g.L[i] = self.L[i] if i < g.dim else 1.0
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        st = self.lib.llg_create(C.byref(g), C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != 0:
            raise LLGError(st, "llg_create failed")
        self.h = h

    @property
    def shape(self):
        return tuple(reversed(self.n))

    @property
    def nodes(self):
        return int(self.lib.llg_nodes(self.h))

    def launches(self):
        return int(self.lib.llg_launch_count(self.h))

    def autotune(self, fp64=True, fp32=True):
        """Pick the fastest valid launch shape of every Fourier axis pass for this grid;
        returns the tuner's report (timings per candidate and the choices)."""
        buf = C.create_string_buffer(8192)
        mask = (1 if fp64 else 0) | (2 if fp32 else 0)
        self._check(self.lib.llg_autotune(self.h, mask, buf, len(buf)))
        return buf.value.decode()

    _SLOTS = {"y(2D)": 0, "y-forward": 1, "z": 2, "y-inverse": 3}

    def set_axis_shape(self, slot, shape, fp32=True):
        """Set one axis pass's launch shape by the tuner's name for it, e.g.
        set_axis_shape("z", "tma(TW8)") or set_axis_shape("y-forward", "register(E8,TW16)")."""
        kind, E, TW, CB = parse_axis_shape(shape)
        if slot not in self._SLOTS:
            raise ValueError(f"unknown axis-pass slot {slot!r}")
        self._check(self.lib.llg_set_axis_shape(self.h, int(fp32), self._SLOTS[slot], kind, E, TW, CB))

    def profile_begin(self, kernel_class):
        """Time every launch of one kernel class ('xfwd', 'axis', 'xinv', 'arnoldi') live."""
        self._check(self.lib.llg_profile_begin(self.h, _abi.KCLASS[kernel_class]))

    def profile_end(self):
        """Returns dict(ms, launches, bytes, flops) summed over the profiled launches."""
        ms, n, by, fl = C.c_double(), C.c_longlong(), C.c_double(), C.c_double()
        self._check(self.lib.llg_profile_end(self.h, C.byref(ms), C.byref(n), C.byref(by), C.byref(fl)))
        return {"ms": ms.value, "launches": n.value, "bytes": by.value, "flops": fl.value}

    def set_pass_plan(self, plan):
        """PLAN_FIVE (default) or PLAN_CLUSTER for this context's 3D FP32 round trips."""
        self._check(self.lib.llg_set_pass_plan(self.h, int(plan)))

    def krylov_orthogonality(self):
        """(max |I - V^T V|, vectors compared) for the basis of this context's last GMRES cycle."""
        md, nv = C.c_double(), C.c_int()
        self._check(self.lib.llg_krylov_orthogonality(self.h, C.byref(md), C.byref(nv)))
        return md.value, nv.value

    def probe_fma_rate(self, fp64=True):
        """Measured multiply-add rate of this device in TFLOP/s (FP64 or FP32)."""
        out = C.c_double()
        self._check(self.lib.llg_probe_fma_rate(self.h, int(fp64), C.byref(out)))
        return out.value

    def check_conversions(self, n_doubles=1 << 26):
        """Compare the integer-pipe float<->double conversions with the hardware ones on the
        device (all 2^32 floats, n_doubles hashed doubles); returns the two mismatch counts."""
        f, d = C.c_longlong(), C.c_longlong()
        self._check(self.lib.llg_check_conversions(self.h, int(n_doubles), C.byref(f), C.byref(d)))
        return f.value, d.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.llg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ marshalling helpers
    def _check(self, st, info=None):
        if st != 0:
            raise LLGError(st, self.lib.llg_last_error(self.h).decode(), info)

    def _arr(self, t, comps, dtype=None):
        torch = _torch()
        dtype = dtype or torch.float64
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
            raise ValueError(f"expected a contiguous {dtype} CUDA tensor")
        if tuple(t.shape) != (comps,) + self.shape:
            raise ValueError(f"expected shape {(comps,) + self.shape}, got {tuple(t.shape)}")
        return C.c_void_p(t.data_ptr())

    def empty(self, comps, dtype=None):
        torch = _torch()
        return torch.empty((comps,) + self.shape, dtype=dtype or torch.float64, device="cuda")


def llg_saddle_apply(ctx: Context, prm: Params, m, x, transpose=False, out=None):
    y = out if out is not None else ctx.empty(4)
    ctx._check(ctx.lib.llg_saddle_apply(ctx.h, C.byref(prm.c(ctx)), ctx._arr(m, 3), ctx._arr(x, 4), ctx._arr(y, 4),
                                        int(transpose)))
    return y


def llg_saddle_apply_f32x2(ctx: Context, prm: Params, m, x, transpose=False, out=None):
    """The saddle matvec with its Fourier chain in FP32-pair arithmetic (FP64 in and out)."""
    y = out if out is not None else ctx.empty(4)
    ctx._check(ctx.lib.llg_saddle_apply_f32x2(ctx.h, C.byref(prm.c(ctx)), ctx._arr(m, 3), ctx._arr(x, 4),
                                              ctx._arr(y, 4), int(transpose)))
    return y


def llg_ffthss_apply(ctx: Context, prm: Params, m, p, transpose=False, out=None):
    z = out if out is not None else ctx.empty(4)
    ctx._check(ctx.lib.llg_ffthss_apply(ctx.h, C.byref(prm.c(ctx)), ctx._arr(m, 3), ctx._arr(p, 4), ctx._arr(z, 4),
                                        int(transpose)))
    return z


def llg_ffthss_apply_f32(ctx: Context, prm: Params, m, p, transpose=False, out=None):
    torch = _torch()
    z = out if out is not None else ctx.empty(4, torch.float32)
    ctx._check(ctx.lib.llg_ffthss_apply_f32(ctx.h, C.byref(prm.c(ctx)), ctx._arr(m, 3, torch.float32),
                                            ctx._arr(p, 4, torch.float32), ctx._arr(z, 4, torch.float32),
                                            int(transpose)))
    return z


def llg_precond_saddle_apply(ctx: Context, prm: Params, m, x, out=None):
    z = out if out is not None else ctx.empty(4)
    ctx._check(ctx.lib.llg_precond_saddle_apply(ctx.h, C.byref(prm.c(ctx)), ctx._arr(m, 3), ctx._arr(x, 4),
                                                ctx._arr(z, 4)))
    return z


def llg_gmres_solve(ctx: Context, prm: Params, opts: Opts, m, b, x=None, raise_on_error=True):
    """Returns (x, info dict); x is the solution (the initial guess is zeros unless given)."""
    if x is None:
        x = ctx.empty(4)
        x.zero_()
    info = _abi.Info()
    st = ctx.lib.llg_gmres_solve(ctx.h, C.byref(prm.c(ctx)), C.byref(opts.c()), ctx._arr(m, 3), ctx._arr(b, 4),
                                 ctx._arr(x, 4), C.byref(info))
    if raise_on_error:
        ctx._check(st, info.as_dict())
    return x, info.as_dict()


def llg_step_euler(ctx: Context, prm: Params, opts: Opts, m, m_next=None, x_out=None, raise_on_error=True):
    m_next = m_next if m_next is not None else ctx.empty(3)
    x_out = x_out if x_out is not None else ctx.empty(4)
    info = _abi.Info()
    st = ctx.lib.llg_step_euler(ctx.h, C.byref(prm.c(ctx)), C.byref(opts.c()), ctx._arr(m, 3), ctx._arr(m_next, 3),
                                ctx._arr(x_out, 4), C.byref(info))
    if raise_on_error:
        ctx._check(st, info.as_dict())
    return m_next, x_out, info.as_dict()


def llg_step_midpoint(ctx: Context, prm: Params, opts: Opts, m, v_prev=None, m_next=None, x_out=None,
                      raise_on_error=True):
    m_next = m_next if m_next is not None else ctx.empty(3)
    x_out = x_out if x_out is not None else ctx.empty(4)
    vp = C.c_void_p(0) if v_prev is None else ctx._arr(v_prev, 3)
    info = _abi.Info()
    st = ctx.lib.llg_step_midpoint(ctx.h, C.byref(prm.c(ctx)), C.byref(opts.c()), ctx._arr(m, 3), vp,
                                   ctx._arr(m_next, 3), ctx._arr(x_out, 4), C.byref(info))
    if raise_on_error:
        ctx._check(st, info.as_dict())
    return m_next, x_out, info.as_dict()


def llg_adjoint_step(ctx: Context, prm: Params, opts: Opts, m_n, x, mbar_next, mbar_n=None):
    """Returns (mbar_n, dL/dalpha contribution, dL/dh contribution (3,), info)."""
    mbar_n = mbar_n if mbar_n is not None else ctx.empty(3)
    da = C.c_double(0.0)
    dh = (C.c_double * 3)(0.0, 0.0, 0.0)
    info = _abi.Info()
    st = ctx.lib.llg_adjoint_step(ctx.h, C.byref(prm.c(ctx)), C.byref(opts.c()), ctx._arr(m_n, 3), ctx._arr(x, 4),
                                  ctx._arr(mbar_next, 3), ctx._arr(mbar_n, 3), C.byref(da), dh, C.byref(info))
    ctx._check(st, info.as_dict())
    return mbar_n, da.value, [dh[0], dh[1], dh[2]], info.as_dict()


class Ensemble:
    """Independent 2D problems advanced together by projected-Euler steps in one persistent
    launch (llg_ensemble_*).  problems: list of dicts with keys n (n0, n1), L, params (Params),
    m (3, n1, n0) float64 CUDA tensor (updated in place) and x (4, n1, n0) output tensor."""

    def __init__(self, problems, opts: Opts, stream=None):
        torch = _torch()
        self.lib = _abi.lib()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (_abi.Problem * len(problems))()
        for q, p in zip(arr, problems):
            q.n[0], q.n[1] = p["n"]
            q.L[0], q.L[1] = p.get("L", (1.0, 1.0))
            q.prm = p["params"].c()
            for key, comps in (("m", 3), ("x", 4)):
                t = p[key]
                if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                        and tuple(t.shape) == (comps, p["n"][1], p["n"][0])):
                    raise ValueError(f"problem {key}: expected a contiguous float64 CUDA tensor of shape "
                                     f"{(comps, p['n'][1], p['n'][0])}")
            q.m = p["m"].data_ptr()
            q.x = p["x"].data_ptr()
        self.count = len(problems)
        h = C.c_void_p()
        st = self.lib.llg_ensemble_create(arr, len(problems), C.byref(opts.c()), C.c_void_p(self.stream.cuda_stream),
                                          C.byref(h))
        if st != 0:
            raise LLGError(st, "llg_ensemble_create failed")
        self.h = h

    def autotune(self):
        b = C.c_int()
        st = self.lib.llg_ensemble_autotune(self.h, C.byref(b))
        if st != 0:
            raise LLGError(st, self.lib.llg_ensemble_last_error(self.h).decode())
        return b.value

    def set_barrier_test(self, budget_cycles=0, hold_block=-1):
        """Diagnostics: shorten the grid barrier's wait limit (0: default) and make one block
        withhold its first arrival (-1: none); see llg_ensemble_set_barrier_test."""
        st = self.lib.llg_ensemble_set_barrier_test(self.h, int(budget_cycles), int(hold_block))
        if st != 0:
            raise LLGError(st, "llg_ensemble_set_barrier_test failed")

    def run(self, steps):
        """Returns (infos in caller order, used_graph)."""
        infos = (_abi.Info * self.count)()
        g = C.c_int()
        st = self.lib.llg_ensemble_run(self.h, steps, infos, C.byref(g))
        if st not in (0, 3):
            raise LLGError(st, self.lib.llg_ensemble_last_error(self.h).decode())
        return [i.as_dict() for i in infos], bool(g.value)

    def close(self):
        if getattr(self, "h", None):
            self.lib.llg_ensemble_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def llg_energy(ctx: Context, prm: Params, m):
    out = C.c_double(0.0)
    ctx._check(ctx.lib.llg_energy(ctx.h, C.byref(prm.c(ctx)), ctx._arr(m, 3), C.byref(out)))
    return out.value


def llg_lower_order_field(ctx: Context, prm: Params, m, out=None):
    """h_low(m): uniform + per-node applied field, anisotropy and demagnetising fields (3 planes)."""
    out = out if out is not None else ctx.empty(3)
    ctx._check(ctx.lib.llg_lower_order_field(ctx.h, C.byref(prm.c(ctx)), ctx._arr(m, 3), ctx._arr(out, 3)))
    return out
