"""Plain FP64 CPU oracle for the periodic tangent-plane LLG saddle solve.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only callers.  The product path (the
CUDA library and its binding) never imports this module.

The arithmetic lives in ``llg_oracle.c`` (plain C, FP64, built with
``-O2 -ffp-contract=off``); this module only marshals numpy arrays.
Fields are SoA planes: ``m`` has shape (3, *grid), ``x = (v1, v2, v3, r)``
has shape (4, *grid), with grid shape (n2, n1, n0) in C order so that the
node index is ``j = i0 + n0 * (i1 + n1 * i2)`` (x fastest).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "llg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

SPECTRAL, FD2 = 0, 1
DFT, FFT = 0, 1
PC_FFTHSS, PC_HERMITIAN, PC_NONE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "llg_oracle.h"))
    ):
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
             "-D_DEFAULT_SOURCE", _SRC, "-o", _LIB, "-lm"]
        )
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("L", C.c_double * 3)]


class _Params(C.Structure):
    _fields_ = [("alpha", C.c_double), ("c_ex", C.c_double), ("k", C.c_double),
                ("theta", C.c_double), ("lam", C.c_double), ("h", C.c_double * 3),
                ("exchange", C.c_int), ("k_an", C.c_double), ("e_an", C.c_double * 3),
                ("demag", C.c_int), ("h_field", C.POINTER(C.c_double))]


class _Opts(C.Structure):
    _fields_ = [("restart", C.c_int), ("max_iters", C.c_int), ("rtol", C.c_double),
                ("picard_max", C.c_int), ("picard_tol", C.c_double), ("use_dense", C.c_int),
                ("precond", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("picard_iters", C.c_int),
                ("converged", C.c_int), ("rel_res_true", C.c_double), ("rel_res_prec", C.c_double)]


@dataclass
class Grid:
    """Periodic grid: ``n`` points per axis (x first), cell lengths ``L``."""
    n: tuple
    L: tuple = None

    def __post_init__(self):
        self.n = tuple(int(v) for v in self.n)
        if self.L is None:
            self.L = tuple(1.0 for _ in self.n)
        self.L = tuple(float(v) for v in self.L)

    @property
    def dim(self):
        return len(self.n)

    @property
    def nodes(self):
        return int(np.prod(self.n))

    @property
    def shape(self):
        """numpy plane shape in C order (slowest axis first)."""
        return tuple(reversed(self.n))

    def c(self):
        g = _Grid()
        g.dim = self.dim
        for i in range(3):
            g.n[i] = self.n[i] if i < self.dim else 1
            g.L[i] = self.L[i] if i < self.dim else 1.0
        return g


@dataclass
class Params:
    alpha: float = 0.2
    c_ex: float = 1.0
    k: float = 1e-2
    theta: float = 1.0
    lam: float = 0.5
    h: tuple = (0.0, 0.0, 0.0)
    exchange: int = SPECTRAL
    k_an: float = 0.0
    e_an: tuple = (0.0, 0.0, 1.0)
    demag: int = 0
    h_field: object = None   # optional (3, *grid shape) nodal applied field, added to h

    def c(self):
        p = _Params()
        p.alpha, p.c_ex, p.k, p.theta, p.lam = self.alpha, self.c_ex, self.k, self.theta, self.lam
        for i in range(3):
            p.h[i] = self.h[i]
            p.e_an[i] = self.e_an[i]
        p.exchange, p.k_an, p.demag = self.exchange, self.k_an, self.demag
        if self.h_field is not None:
            hf = np.ascontiguousarray(np.asarray(self.h_field, dtype=np.float64))
            p._hf = hf   # keeps the array alive as long as the struct
            p.h_field = hf.ctypes.data_as(C.POINTER(C.c_double))
        return p


@dataclass
class Opts:
    restart: int = 30
    max_iters: int = 5000
    rtol: float = 1e-10
    picard_max: int = 50
    picard_tol: float = 1e-10
    use_dense: int = 0
    precond: int = 0          # PC_FFTHSS, PC_HERMITIAN or PC_NONE

    def c(self):
        o = _Opts()
        o.restart, o.max_iters, o.rtol = self.restart, self.max_iters, self.rtol
        o.picard_max, o.picard_tol, o.use_dense = self.picard_max, self.picard_tol, self.use_dense
        o.precond = self.precond
        return o


@dataclass
class Info:
    iters: int = 0
    restarts: int = 0
    picard_iters: int = 0
    converged: bool = False
    rel_res_true: float = 0.0
    rel_res_prec: float = 0.0
    extra: dict = field(default_factory=dict)


def _info(ci):
    return Info(ci.iters, ci.restarts, ci.picard_iters, bool(ci.converged), ci.rel_res_true,
                ci.rel_res_prec)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER
        d = P(C.c_double)
        L = _lib
        L.orc_set_transform.argtypes = [C.c_int]
        L.orc_symbol.argtypes = [P(_Grid), C.c_int, P(C.c_int)]
        L.orc_symbol.restype = C.c_double
        L.orc_wavenumber.argtypes = [C.c_int, C.c_int]
        L.orc_transform.argtypes = [P(_Grid), d, d, C.c_int]
        L.orc_neg_laplacian.argtypes = [P(_Grid), C.c_int, d, d]
        L.orc_hermitian_solve.argtypes = [P(_Grid), P(_Params), d, d]
        L.orc_nodal_solve.argtypes = [P(_Grid), P(_Params), d, d, d, C.c_int]
        L.orc_ffthss_apply.argtypes = [P(_Grid), P(_Params), d, d, d, C.c_int]
        L.orc_saddle_apply.argtypes = [P(_Grid), P(_Params), d, d, d, C.c_int]
        L.orc_saddle_dense.argtypes = [P(_Grid), P(_Params), d, d]
        L.orc_dense_solve.argtypes = [C.c_int, d, d, d]
        L.orc_gmres_solve.argtypes = [P(_Grid), P(_Params), P(_Opts), d, d, d, C.c_int,
                                      P(_Info), d, C.c_int]
        L.orc_h_low.argtypes = [P(_Grid), P(_Params), d, d]
        L.orc_energy.argtypes = [P(_Grid), P(_Params), d]
        L.orc_energy.restype = C.c_double
        L.orc_step_euler.argtypes = [P(_Grid), P(_Params), P(_Opts), d, d, d, P(_Info)]
        L.orc_step_midpoint.argtypes = [P(_Grid), P(_Params), P(_Opts), d, d, d, d, P(_Info)]
        L.orc_adjoint_midpoint.argtypes = [P(_Grid), P(_Params), P(_Opts), d, d, d, d, d, d,
                                           P(_Info)]
        L.orc_beta_N.argtypes = [P(_Grid), P(_Params)]
        L.orc_beta_N.restype = C.c_double
        for nm, na in (("orc_q_bar", 3), ("orc_lambda_bd", 2), ("orc_gamma_m", 3),
                       ("orc_theta2", 2), ("orc_kappa", 3)):
            f = getattr(L, nm)
            f.argtypes = [C.c_double] * na
            f.restype = C.c_double
        L.orc_iteration_bound.argtypes = [C.c_double] * 3
        L.orc_iteration_bound.restype = C.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_transform(mode):
    lib().orc_set_transform(mode)


def symbol(grid: Grid, kvec, exchange=SPECTRAL):
    kv = (C.c_int * 3)(*(list(kvec) + [0] * (3 - len(kvec))))
    return lib().orc_symbol(C.byref(grid.c()), exchange, kv)


def transform(grid: Grid, z, sign=-1):
    re = _f64(np.real(z), grid.shape).copy()
    im = _f64(np.imag(z), grid.shape).copy()
    lib().orc_transform(C.byref(grid.c()), _p(re), _p(im), sign)
    return re + 1j * im


def neg_laplacian(grid: Grid, u, exchange=SPECTRAL):
    u = _f64(u, grid.shape)
    w = np.empty_like(u)
    lib().orc_neg_laplacian(C.byref(grid.c()), exchange, _p(u), _p(w))
    return w


def hermitian_solve(grid: Grid, prm: Params, p):
    p = _f64(p, (4,) + grid.shape)
    w = np.empty_like(p)
    lib().orc_hermitian_solve(C.byref(grid.c()), C.byref(prm.c()), _p(p), _p(w))
    return w


def nodal_solve(grid: Grid, prm: Params, m, w, transpose=False):
    m = _f64(m, (3,) + grid.shape)
    w = _f64(w, (4,) + grid.shape)
    z = np.empty_like(w)
    lib().orc_nodal_solve(C.byref(grid.c()), C.byref(prm.c()), _p(m), _p(w), _p(z), int(transpose))
    return z


def ffthss_apply(grid: Grid, prm: Params, m, p, transpose=False):
    m = _f64(m, (3,) + grid.shape)
    p = _f64(p, (4,) + grid.shape)
    z = np.empty_like(p)
    lib().orc_ffthss_apply(C.byref(grid.c()), C.byref(prm.c()), _p(m), _p(p), _p(z), int(transpose))
    return z


def saddle_apply(grid: Grid, prm: Params, m, x, transpose=False):
    m = _f64(m, (3,) + grid.shape)
    x = _f64(x, (4,) + grid.shape)
    y = np.empty_like(x)
    lib().orc_saddle_apply(C.byref(grid.c()), C.byref(prm.c()), _p(m), _p(x), _p(y), int(transpose))
    return y


def saddle_dense(grid: Grid, prm: Params, m):
    m = _f64(m, (3,) + grid.shape)
    n = 4 * grid.nodes
    A = np.empty((n, n))
    lib().orc_saddle_dense(C.byref(grid.c()), C.byref(prm.c()), _p(m), _p(A))
    return A


def dense_solve(A, b):
    A = _f64(A)
    b = _f64(b).ravel()
    x = np.empty_like(b)
    rc = lib().orc_dense_solve(A.shape[0], _p(A), _p(b), _p(x))
    if rc != 0:
        raise np.linalg.LinAlgError("singular matrix in oracle dense solve")
    return x


def gmres_solve(grid: Grid, prm: Params, opts: Opts, m, b, x0=None, transpose=False, hist_len=0):
    m = _f64(m, (3,) + grid.shape)
    b = _f64(b, (4,) + grid.shape)
    x = np.zeros_like(b) if x0 is None else _f64(x0, b.shape).copy()
    ci = _Info()
    hist = np.zeros(max(hist_len, 1))
    lib().orc_gmres_solve(C.byref(grid.c()), C.byref(prm.c()), C.byref(opts.c()), _p(m), _p(b),
                          _p(x), int(transpose), C.byref(ci), _p(hist), hist_len)
    info = _info(ci)
    if hist_len:
        info.extra["hist"] = hist[: min(info.iters, hist_len)].copy()
    return x, info


def h_low(grid: Grid, prm: Params, m):
    m = _f64(m, (3,) + grid.shape)
    hl = np.empty_like(m)
    lib().orc_h_low(C.byref(grid.c()), C.byref(prm.c()), _p(m), _p(hl))
    return hl


def energy(grid: Grid, prm: Params, m):
    m = _f64(m, (3,) + grid.shape)
    return lib().orc_energy(C.byref(grid.c()), C.byref(prm.c()), _p(m))


def step_euler(grid: Grid, prm: Params, opts: Opts, m):
    m = _f64(m, (3,) + grid.shape)
    mn = np.empty_like(m)
    x = np.empty((4,) + grid.shape)
    ci = _Info()
    lib().orc_step_euler(C.byref(grid.c()), C.byref(prm.c()), C.byref(opts.c()), _p(m), _p(mn),
                         _p(x), C.byref(ci))
    return mn, x, _info(ci)


def step_midpoint(grid: Grid, prm: Params, opts: Opts, m, v_prev=None):
    m = _f64(m, (3,) + grid.shape)
    mn = np.empty_like(m)
    x = np.empty((4,) + grid.shape)
    ci = _Info()
    vp = None if v_prev is None else _f64(v_prev, (3,) + grid.shape)
    lib().orc_step_midpoint(C.byref(grid.c()), C.byref(prm.c()), C.byref(opts.c()), _p(m),
                            _p(vp) if vp is not None else None, _p(mn), _p(x), C.byref(ci))
    return mn, x, _info(ci)


def adjoint_midpoint(grid: Grid, prm: Params, opts: Opts, m_n, x, mbar_next):
    m_n = _f64(m_n, (3,) + grid.shape)
    x = _f64(x, (4,) + grid.shape)
    mb = _f64(mbar_next, (3,) + grid.shape)
    mbar_n = np.empty_like(mb)
    da = C.c_double(0.0)
    dh = (C.c_double * 3)(0.0, 0.0, 0.0)
    ci = _Info()
    rc = lib().orc_adjoint_midpoint(C.byref(grid.c()), C.byref(prm.c()), C.byref(opts.c()),
                                    _p(m_n), _p(x), _p(mb), _p(mbar_n), C.byref(da), dh,
                                    C.byref(ci))
    if rc == 2:
        raise ValueError("oracle adjoint covers a uniform applied field only")
    return mbar_n, da.value, np.array(dh[:]), _info(ci)


def beta_N(grid: Grid, prm: Params):
    return lib().orc_beta_N(C.byref(grid.c()), C.byref(prm.c()))


def q_bar(lam, alpha, beta):
    return lib().orc_q_bar(lam, alpha, beta)


def lambda_bd(alpha, beta):
    return lib().orc_lambda_bd(alpha, beta)


def gamma_m(lam, m_min, m_max):
    return lib().orc_gamma_m(lam, m_min, m_max)


def theta2(q, gamma):
    return lib().orc_theta2(q, gamma)


def kappa(lam, m_min, m_max):
    return lib().orc_kappa(lam, m_min, m_max)


def iteration_bound(kap, th, eps):
    return lib().orc_iteration_bound(kap, th, eps)


# ---------------------------------------------------------------- multi-step drivers (oracle only)

def run_midpoint(grid: Grid, prm: Params, opts: Opts, m0, nsteps):
    """Run ``nsteps`` midpoint steps; returns (trajectory of m, list of x, infos)."""
    ms = [_f64(m0, (3,) + grid.shape)]
    xs, infos = [], []
    vprev = None
    for _ in range(nsteps):
        mn, x, info = step_midpoint(grid, prm, opts, ms[-1], vprev)
        ms.append(mn)
        xs.append(x)
        infos.append(info)
        vprev = x[:3]
    return ms, xs, infos


def run_euler(grid: Grid, prm: Params, opts: Opts, m0, nsteps, transform=None):
    """Run ``nsteps`` projected Euler steps; returns (m after the last step, infos).  With
    ``transform`` set (DFT or FFT), that transform mode is selected first: this makes the call
    self-contained for a worker process, whose module state starts at the default."""
    if transform is not None:
        set_transform(transform)
    m = _f64(m0, (3,) + grid.shape)
    infos = []
    for _ in range(nsteps):
        m, _, info = step_euler(grid, prm, opts, m)
        infos.append(info)
    return m, infos


def midpoint_loss_grad(grid: Grid, prm: Params, opts: Opts, m0, m_target, nsteps):
    """L = 1/2 sum |m^N - m_target|^2 and its gradient w.r.t. (alpha, h, m0) by the
    step-by-step adjoint of the converged midpoint map."""
    ms, xs, _ = run_midpoint(grid, prm, opts, m0, nsteps)
    diff = ms[-1] - m_target
    loss = 0.5 * float(np.sum(diff * diff))
    mbar = diff.copy()
    dalpha, dh = 0.0, np.zeros(3)
    for n in reversed(range(nsteps)):
        mbar, da, dhh, _ = adjoint_midpoint(grid, prm, opts, ms[n], xs[n], mbar)
        dalpha += da
        dh += dhh
    return loss, dalpha, dh, mbar, ms[-1]
