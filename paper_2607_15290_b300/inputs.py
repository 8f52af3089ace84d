"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws and shapes input
fields (magnetisations, right-hand sides, saddle vectors).  Both the CUDA path
and the CPU oracle are fed from it.  Arrays are float64 SoA planes of shape
(components, *grid_shape) with grid_shape = (n2, n1, n0) in C order (x fastest).

Workload recipes (the smooth 2D/3D fields and the broadband |k|^-1.5 field
follow the benchmark configurations; the 3D energy test field is the paper's
Sec. 4.6 initial condition on (0, 2 pi)^3):
  * smooth2d     m = normalise((sin 2pi x cos 2pi y, cos 2pi x, 0.5 + 0.3 sin 2pi(x+y)) + 1e-3 N(0,1))
  * smooth3d     m = normalise((cos 2pi z sin 2pi x, sin 2pi z sin 2pi y, cos 2pi x) + 1e-3 N(0,1))
  * broadband    per component: random phases, amplitude |k|^-1.5 over all resolved integer
                 wavevectors k != 0, real part of the inverse transform, then per-node normalise
  * energy3d     (sin(x+z) cos(y+z), cos(x+z) cos(y+z), sin(y+z)) on (0, 2pi)^3 (unit length)
  * ensemble_mix the batched workload: 32 problems each of 128^2, 256^2, 512^2 with seeded
                 damping, time-step multiple and smooth/broadband field mix
"""
from __future__ import annotations

import numpy as np

SEED = 20260724


def coords(n, L=None):
    """Node coordinates x_j = j L / n per axis, as a list of broadcastable arrays
    in C order (returns [x, y] for 2D and [x, y, z] for 3D)."""
    n = tuple(n)
    if L is None:
        L = (1.0,) * len(n)
    axes = [np.arange(ni) * (Li / ni) for ni, Li in zip(n, L)]
    grids = np.meshgrid(*reversed(axes), indexing="ij")   # slowest axis first
    return list(reversed(grids))


def _normalise(m):
    nrm = np.sqrt(np.sum(m * m, axis=0, keepdims=True))
    if np.any(nrm < 1e-8):
        raise ValueError("degenerate node while normalising a synthetic field")
    return m / nrm


def smooth2d(n, seed=SEED, noise=1e-3, L=(1.0, 1.0)):
    x, y = coords(n, L)
    tp = 2 * np.pi
    m = np.stack([np.sin(tp * x) * np.cos(tp * y), np.cos(tp * x), 0.5 + 0.3 * np.sin(tp * (x + y))])
    rng = np.random.default_rng(seed)
    m = m + noise * rng.standard_normal(m.shape)
    return _normalise(m)


def smooth3d(n, seed=SEED, noise=1e-3, L=(1.0, 1.0, 1.0)):
    x, y, z = coords(n, L)
    tp = 2 * np.pi
    m = np.stack([np.cos(tp * z) * np.sin(tp * x), np.sin(tp * z) * np.sin(tp * y), np.cos(tp * x)])
    rng = np.random.default_rng(seed)
    m = m + noise * rng.standard_normal(m.shape)
    return _normalise(m)


def broadband(n, seed=SEED, slope=1.5):
    shape = tuple(reversed(tuple(n)))
    rng = np.random.default_rng(seed)
    kk = np.meshgrid(*[np.fft.fftfreq(s) * s for s in shape], indexing="ij")
    kmag = np.sqrt(sum(k * k for k in kk))
    amp = np.zeros(shape)
    amp[kmag > 0] = kmag[kmag > 0] ** (-slope)
    comps = []
    for _ in range(3):
        phase = rng.uniform(0.0, 2 * np.pi, size=shape)
        comps.append(np.real(np.fft.ifftn(amp * np.exp(1j * phase))))
    m = np.stack(comps)
    m = m / np.sqrt(np.mean(m * m))
    return _normalise(m)


def energy3d(n):
    L = (2 * np.pi,) * 3
    x, y, z = coords(n, L)
    return np.stack([np.sin(x + z) * np.cos(y + z), np.cos(x + z) * np.cos(y + z), np.sin(y + z)])


def random_unit(n, seed=SEED):
    shape = tuple(reversed(tuple(n)))
    rng = np.random.default_rng(seed)
    return _normalise(rng.standard_normal((3,) + shape))


def random_saddle_vector(n, seed=SEED, zero_r=False):
    shape = tuple(reversed(tuple(n)))
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((4,) + shape)
    if zero_r:
        x[3] = 0.0
    return x


def gaussian_rhs(n, seed):
    """Deterministic normalised Gaussian velocity right-hand side, zero multiplier part."""
    x = random_saddle_vector(n, seed, zero_r=True)
    return x / np.sqrt(np.sum(x * x))


def manufactured2d(n, t, alpha, c_ex=1.0):
    """Periodic manufactured solution of the temporal-convergence test (Sec. 4.2) on
    (0, 2 pi)^2: m_e(x, y, t) = (sin(t+x) cos(t+y), cos(t+x) cos(t+y), sin(t+y)), |m_e| = 1,
    and the forcing g added to the lower-order field that makes it an exact solution of the
    tangent-plane LLG equation alpha dm/dt + m x dm/dt = (1 + alpha^2) [h - (m.h) m] with
    h = c_ex Lap m + g:
        g = (alpha dm_e/dt + m_e x dm_e/dt) / (1 + alpha^2) - c_ex Lap m_e,
    i.e. h is the tangent field (alpha dm_e/dt + m_e x dm_e/dt) / (1 + alpha^2) itself.  Any g
    differing by a multiple of m_e also makes m_e exact; this one keeps the exchange field's
    normal part in g, which is the reading under which the scheme reproduces the paper's
    printed errors.  Closed forms: dm_e/dt = (cos(a+b), -sin(a+b), cos b),
    Lap m_e = (-2 m1, -2 m2, -m3) with a = t + x, b = t + y.  Returns (m_e, g), each of shape
    (3, n1, n0)."""
    x, y = coords(n, (2 * np.pi, 2 * np.pi))
    a, b = t + x, t + y
    m = np.stack([np.sin(a) * np.cos(b), np.cos(a) * np.cos(b), np.sin(b)])
    dm = np.stack([np.cos(a + b), -np.sin(a + b), np.cos(b)])
    lap = np.stack([-2 * m[0], -2 * m[1], -m[2]])
    mxdm = np.stack([m[1] * dm[2] - m[2] * dm[1], m[2] * dm[0] - m[0] * dm[2], m[0] * dm[1] - m[1] * dm[0]])
    g = (alpha * dm + mxdm) / (1 + alpha ** 2) - c_ex * lap
    return m, g


def ensemble_mix(seed=20260725, sizes=(128, 256, 512), per_size=32):
    """The batched ensemble workload: for each grid size, `per_size` independent 2D problems
    with alpha ~ U[0.01, 0.5], a time-step multiple c ~ U[2, 16] (the caller scales the
    explicit exchange limit by it) and the field normalise(w smooth2d + (1 - w) broadband),
    w ~ U[0, 1], both drawn with seed 1000 n + i.  Returns a list of (n, alpha, c, m0)."""
    rng = np.random.default_rng(seed)
    out = []
    for n in sizes:
        for i in range(per_size):
            alpha = float(rng.uniform(0.01, 0.5))
            c = float(rng.uniform(2.0, 16.0))
            w = float(rng.uniform(0.0, 1.0))
            s = 1000 * n + i
            f = w * smooth2d((n, n), seed=s) + (1 - w) * broadband((n, n), seed=s)
            out.append((n, alpha, c, _normalise(f)))
    return out
