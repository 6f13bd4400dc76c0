"""FP64 CPU oracle of the Langevin nanoparticle-aggregation step (arXiv 2501.04456).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline leg
of the benchmark import this package; the GPU library never does.  It shares
no code with the CUDA path: it loads ``liboracle.so`` built from ``oracle.c``
(plain C, double precision, OpenMP over independent rows only).

Functions take and return numpy arrays: positions are row-major ``(n, 3)``
float64, types int32.  Each wrapper names the paper passage of the C function
it calls; the C file states the formula.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAX_TYPES = 8
K_F = 1.593  # fractal prefactor for a compact hexagonal aggregate, Sec. 3.1


def build(force: bool = False) -> str:
    """Compile liboracle.so next to oracle.c (gcc, -ffp-contract=off, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = C.CDLL(_LIB)
            _declare(_lib)
        return _lib


class Params(C.Structure):
    """Mirror of the oracle's own ``or_params_t``."""
    _fields_ = [
        ("n_types", C.c_int32), ("rot_mode", C.c_int32), ("lj_on", C.c_int32),
        ("coul_on", C.c_int32), ("wall_on", C.c_int32), ("integrator", C.c_int32),
        ("seed", C.c_uint64),
        ("dt", C.c_double), ("kT", C.c_double), ("R0", C.c_double),
        ("k_evap", C.c_double), ("g", C.c_double), ("omega", C.c_double),
        ("bjerrum", C.c_double), ("lj_cut", C.c_double),
        ("sigma", C.c_double * MAX_TYPES), ("eps", C.c_double * MAX_TYPES),
        ("mass", C.c_double * MAX_TYPES), ("charge", C.c_double * MAX_TYPES),
        ("gamma", C.c_double * MAX_TYPES), ("k_wall", C.c_double * MAX_TYPES),
        ("eps_override", C.c_double * (MAX_TYPES * MAX_TYPES)),
        ("has_eps_override", C.c_int32), ("pad_", C.c_int32),
        ("v_kick", C.c_double), ("coul_cut", C.c_double),
    ]


_P = np.ctypeslib.ndpointer
_d = C.POINTER(C.c_double)


def _declare(lib):
    u32p = C.POINTER(C.c_uint32)
    i64p = C.POINTER(C.c_int64)
    i32p = C.POINTER(C.c_int32)
    lib.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.or_philox_blocks.argtypes = [C.c_uint64, u32p, C.c_int64, u32p]
    lib.or_normals.argtypes = [C.c_uint64, C.c_int64, C.c_uint32, C.c_int64, _d]
    lib.or_mix_tables.argtypes = [C.c_int, _d, _d, _d, C.c_double, _d, _d, _d]
    lib.or_pair_forces.argtypes = [C.c_int64, _d, i32p, C.c_int, _d, _d, _d, _d, _d,
                                   C.c_double, C.c_int, C.c_int, C.c_int64, i64p, _d]
    lib.or_radius.argtypes = [C.c_double, C.c_double, C.c_double]
    lib.or_radius.restype = C.c_double
    lib.or_external_forces.argtypes = [C.POINTER(Params), C.c_int64, _d, i32p,
                                       C.c_double, _d]
    lib.or_total_forces.argtypes = [C.POINTER(Params), C.c_int64, _d, i32p,
                                    C.c_double, _d]
    lib.or_run.argtypes = [C.POINTER(Params), C.c_int64, _d, _d, i32p, C.c_int64,
                           C.c_int64, _d]
    lib.or_pair_hist.argtypes = [C.c_int64, _d, C.c_double, C.c_int, i64p]
    lib.or_rdf.argtypes = [C.c_int64, _d, C.c_double, C.c_int, C.c_double, i64p, _d]
    lib.or_radial_hist.argtypes = [C.c_int64, _d, C.c_double, C.c_int, C.c_double,
                                   i64p, _d]
    lib.or_rg.argtypes = [C.c_int64, _d, C.c_double, C.c_double, _d, _d, _d]
    lib.or_surface_count.argtypes = [C.c_int64, _d, i32p, _d, C.c_double]
    lib.or_surface_count.restype = C.c_int64
    lib.or_boxcount.argtypes = [C.c_int64, _d, C.c_double, C.c_int, i64p]
    lib.or_boxcount_df.argtypes = [C.c_int64, _d, C.c_double, C.c_double, C.c_int,
                                   i64p, _d]
    lib.or_boxcount_df.restype = C.c_int
    lib.or_lsq_slope.argtypes = [C.c_int, _d, _d]
    lib.or_lsq_slope.restype = C.c_double


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# --------------------------------------------------------------------------
# Philox4x32-10 and normals


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block (Salmon et al., SC'11): 4 u32 from counter/key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib.or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def philox_blocks(seed: int, ctr, n_blocks: int):
    """Blocks with counter (ctr0+b, ctr1 (+carry), ctr2, ctr3); returns (n_blocks, 4) u32."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros((n_blocks, 4), np.uint32)
    lib.or_philox_blocks(C.c_uint64(seed), _ptr(c, C.c_uint32), n_blocks,
                         _ptr(out, C.c_uint32))
    return out


def normals(seed: int, step: int, purpose: int, n: int):
    """The (n, 3) standard normals of step `step` (Box-Muller on Philox)."""
    lib = _load()
    out = np.zeros((n, 3))
    lib.or_normals(C.c_uint64(seed), step, purpose, n, _ptr(out, C.c_double))
    return out


# --------------------------------------------------------------------------
# Forces


def mix_tables(sigma, eps, eps_override=None, lj_cut=2.5):
    """Type-pair tables (sigma_ab, eps_ab, rc_ab), Lorentz-Berthelot unless overridden."""
    lib = _load()
    sigma = _f64(sigma)
    eps = _f64(eps)
    T = len(sigma)
    s = np.zeros((T, T))
    e = np.zeros((T, T))
    r = np.zeros((T, T))
    ov = None if eps_override is None else _f64(eps_override, (T, T))
    lib.or_mix_tables(T, _ptr(sigma, C.c_double), _ptr(eps, C.c_double),
                      None if ov is None else _ptr(ov, C.c_double), lj_cut,
                      _ptr(s, C.c_double), _ptr(e, C.c_double), _ptr(r, C.c_double))
    return s, e, r


def pair_forces(x, types, sigma, eps, charge, bjerrum, lj_cut=2.5, lj=True,
                coulomb=True, eps_override=None, sel=None, coulomb_cut=0.0):
    """Pair forces of Sec. 2.2 step (ii) on rows `sel` (all rows if None); with
    coulomb_cut > 0 the Coulomb term is truncated at coulomb_cut * sigma_ab."""
    lib = _load()
    x = _f64(x, (-1, 3))
    types = _i32(types)
    n = x.shape[0]
    s, e, r = mix_tables(sigma, eps, eps_override, lj_cut)
    q = _f64(charge)
    if sel is None:
        n_sel, selp, sel_arr = n, None, None
    else:
        sel_arr = np.ascontiguousarray(sel, dtype=np.int64)
        n_sel, selp = len(sel_arr), _ptr(sel_arr, C.c_int64)
    F = np.zeros((n_sel, 3))
    rcc = np.ascontiguousarray(coulomb_cut * s) if coulomb_cut > 0 else None
    lib.or_pair_forces(n, _ptr(x, C.c_double), _ptr(types, C.c_int32), len(q),
                       _ptr(s, C.c_double), _ptr(e, C.c_double), _ptr(r, C.c_double),
                       None if rcc is None else _ptr(rcc, C.c_double),
                       _ptr(q, C.c_double), bjerrum, int(lj), int(coulomb), n_sel,
                       selp, _ptr(F, C.c_double))
    return F


def radius(R0, k_evap, t):
    """Droplet radius by the radius-square law, Sec. 2.1 / step (iii)."""
    return _load().or_radius(R0, k_evap, t)


def make_params(sc) -> Params:
    """Fill the oracle's parameter struct from a workloads.Scenario."""
    p = Params()
    T = len(sc.types)
    p.n_types = T
    p.rot_mode = sc.rot_mode
    p.lj_on = int(sc.lj_mode != 0)
    p.coul_on = int(sc.coulomb)
    p.wall_on = 0 if not sc.wall else (2 if getattr(sc, "wall_band", False) else 1)
    p.integrator = sc.integrator
    p.v_kick = float(getattr(sc, "v_kick", 0.0))
    p.coul_cut = float(getattr(sc, "coulomb_cut", 0.0))
    p.seed = sc.seed
    p.dt, p.kT, p.R0, p.k_evap = sc.dt, sc.kT, sc.R0, sc.k_evap
    p.g, p.omega, p.bjerrum, p.lj_cut = sc.g, sc.omega, sc.bjerrum, sc.lj_cut
    for a, t in enumerate(sc.types):
        p.sigma[a], p.eps[a], p.mass[a] = t.sigma, t.eps, t.mass
        p.charge[a], p.gamma[a], p.k_wall[a] = t.charge, t.gamma, t.k_wall
    if sc.eps_override is not None:
        ov = np.asarray(sc.eps_override, dtype=np.float64).reshape(T, T)
        p.has_eps_override = 1
        for a in range(T):
            for b in range(T):
                p.eps_override[a * T + b] = ov[a, b]
    return p


def external_forces(sc, x, types, t):
    """Wall, gravity and centrifugal forces of steps (iv)-(v) at time t."""
    lib = _load()
    x = _f64(x, (-1, 3))
    types = _i32(types)
    F = np.zeros_like(x)
    p = make_params(sc)
    lib.or_external_forces(C.byref(p), x.shape[0], _ptr(x, C.c_double),
                           _ptr(types, C.c_int32), t, _ptr(F, C.c_double))
    return F


def total_forces(sc, x, types, t):
    """Pair plus external forces at (x, t)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    types = _i32(types)
    F = np.zeros_like(x)
    p = make_params(sc)
    lib.or_total_forces(C.byref(p), x.shape[0], _ptr(x, C.c_double),
                        _ptr(types, C.c_int32), t, _ptr(F, C.c_double))
    return F


def run(sc, x, v, types, step0: int, n_steps: int):
    """Advance (x, v) by n_steps from step0 (BAOAB or overdamped, step (vi)).

    Returns (x, v, F) with F the total force at the final state."""
    lib = _load()
    x = _f64(x, (-1, 3)).copy()
    v = _f64(v, (-1, 3)).copy()
    types = _i32(types)
    F = np.zeros_like(x)
    p = make_params(sc)
    lib.or_run(C.byref(p), x.shape[0], _ptr(x, C.c_double), _ptr(v, C.c_double),
               _ptr(types, C.c_int32), step0, n_steps, _ptr(F, C.c_double))
    return x, v, F


# --------------------------------------------------------------------------
# Statistics (Sec. 3)


def pair_hist(x, r_max, n_bins):
    """Ordered-pair distance histogram (int64) over [0, r_max)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    c = np.zeros(n_bins, np.int64)
    lib.or_pair_hist(x.shape[0], _ptr(x, C.c_double), r_max, n_bins, _ptr(c, C.c_int64))
    return c


def rdf(x, r_max, n_bins, R):
    """RDF g(r) of Sec. 3.2 with V the droplet volume; returns (counts, g)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    c = np.zeros(n_bins, np.int64)
    g = np.zeros(n_bins)
    lib.or_rdf(x.shape[0], _ptr(x, C.c_double), r_max, n_bins, R,
               _ptr(c, C.c_int64), _ptr(g, C.c_double))
    return c, g


def radial_concentration(x, r_max, n_bins, R):
    """C_NPs(r) about the droplet centre (Sec. 3.2); returns (counts, C)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    c = np.zeros(n_bins, np.int64)
    Cc = np.zeros(n_bins)
    lib.or_radial_hist(x.shape[0], _ptr(x, C.c_double), r_max, n_bins, R,
                       _ptr(c, C.c_int64), _ptr(Cc, C.c_double))
    return c, Cc


def surface_count(x, types, sigma, R):
    """N_surf: NPs with | |x_i| - R | < sigma_i / 2 (Sec. 1, Sec. 2.2 step iv)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    t = _i32(types)
    s = _f64(sigma)
    return int(lib.or_surface_count(x.shape[0], _ptr(x, C.c_double), _ptr(t, C.c_int32),
                                    _ptr(s, C.c_double), R))


def _sin_minus_ucos(u):
    """sin u - u cos u, by its Taylor series sum_k (-1)^(k+1) 2k u^(2k+1)/(2k+1)!
    below u = 0.5 (where the two terms cancel), directly above."""
    u = np.asarray(u, np.float64)
    out = np.sin(u) - u * np.cos(u)
    small = u < 0.5
    if np.any(small):
        us = u[small]
        term_sum = np.zeros_like(us)
        fact = 1.0  # (2k+1)!
        for k in range(1, 13):
            fact *= (2 * k) * (2 * k + 1)
            term_sum += (-1) ** (k + 1) * 2 * k * us ** (2 * k + 1) / fact
        out[small] = term_sum
    return out


def scattering(g, r_max, n_surf, q):
    """Light scattered by the NPs, Sec. 3.3: I(q) = N_surf^2 * integral of
    exp(i q.r) g(r) d^3r = N_surf^2 4 pi integral g(r) r^2 sin(qr)/(qr) dr, with g
    constant on the bins of [0, r_max): each bin contributes
    g_b [G(q r_{b+1}) - G(q r_b)]/q^3, G(u) = sin u - u cos u (the antiderivative
    of u sin u), and g_b (r_{b+1}^3 - r_b^3)/3 at q = 0."""
    g = np.asarray(g, np.float64)
    q = np.asarray(q, np.float64)
    edges = np.arange(len(g) + 1) * (r_max / len(g))
    out = np.empty(len(q))
    for k, qq in enumerate(q):
        if qq > 0:
            G = _sin_minus_ucos(qq * edges)
            out[k] = 4 * np.pi * np.sum(g * np.diff(G)) / qq ** 3
        else:
            out[k] = 4 * np.pi * np.sum(g * np.diff(edges ** 3)) / 3
    return n_surf ** 2 * out


def rg(x, d_mean, k_f=K_F):
    """(R_g, D_f, r0) from Eqs. N, Rg, r0 of Sec. 3.1."""
    lib = _load()
    x = _f64(x, (-1, 3))
    Rg = C.c_double()
    Df = C.c_double()
    r0 = np.zeros(3)
    lib.or_rg(x.shape[0], _ptr(x, C.c_double), d_mean, k_f, C.byref(Rg), C.byref(Df),
              _ptr(r0, C.c_double))
    return Rg.value, Df.value, r0


def boxcount(x, d, n_scales):
    """N_box at eps_k = d 2^k, k < n_scales (int64)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    nb = np.zeros(n_scales, np.int64)
    lib.or_boxcount(x.shape[0], _ptr(x, C.c_double), d, n_scales, _ptr(nb, C.c_int64))
    return nb


def boxcount_df(x, d, Rg, max_scales=32):
    """Box-counting D_f; returns (D_f, N_box per scale)."""
    lib = _load()
    x = _f64(x, (-1, 3))
    nb = np.zeros(max_scales, np.int64)
    Df = C.c_double()
    ns = lib.or_boxcount_df(x.shape[0], _ptr(x, C.c_double), d, Rg, max_scales,
                            _ptr(nb, C.c_int64), C.byref(Df))
    return Df.value, nb[:ns]


def lsq_slope(xs, ys):
    lib = _load()
    xs = _f64(xs)
    ys = _f64(ys)
    return lib.or_lsq_slope(len(xs), _ptr(xs, C.c_double), _ptr(ys, C.c_double))
