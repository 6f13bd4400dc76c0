"""Python binding of libnpsim, the GB300 (sm_103a) Langevin-dynamics library for
nanoparticle aggregation in an evaporating droplet (arXiv 2501.04456).

Argument marshalling only: every function here has the name of the C entry point
it calls (include/npsim.h) and converts numpy arrays to the C layouts; all
computation runs in the library's CUDA kernels.  There is no CPU fallback: if
``libnpsim.so`` has not been built, every call raises ``RuntimeError``.

PyTorch is optional and used only for streams and device buffers: a ``stream``
argument may be a ``torch.cuda.Stream``, a raw ``cudaStream_t`` integer or None
(None = torch's current stream when torch sees a GPU, else the default stream).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnpsim.so")
MAX_TYPES = 8
MAX_SCALES = 32

NPSIM_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "CUDA", -3: "NONFINITE", -4: "TIMEOUT", -5: "OOM",
          -6: "IO", -7: "NO_DEVICE", -8: "ESCAPED"}


class NpsimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"npsim error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class npsim_type_t(C.Structure):
    _fields_ = [("sigma", C.c_double), ("eps", C.c_double), ("mass", C.c_double),
                ("charge", C.c_double), ("gamma", C.c_double), ("k_wall", C.c_double)]


class npsim_params_t(C.Structure):
    _fields_ = [("n_types", C.c_int32), ("rot_mode", C.c_int32), ("lj_mode", C.c_int32),
                ("coulomb", C.c_int32), ("wall", C.c_int32), ("integrator", C.c_int32),
                ("sum_neutral", C.c_int32), ("reserved_", C.c_int32),
                ("seed", C.c_uint64), ("dt", C.c_double), ("kT", C.c_double),
                ("R0", C.c_double), ("k_evap", C.c_double), ("g", C.c_double),
                ("omega", C.c_double), ("bjerrum", C.c_double), ("lj_cut", C.c_double),
                ("eps_override", C.POINTER(C.c_double)), ("v_kick", C.c_double),
                ("coulomb_cut", C.c_double)]


class npsim_droplet_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("types", C.POINTER(npsim_type_t)),
                ("params", npsim_params_t), ("x0", C.POINTER(C.c_double)),
                ("v0", C.POINTER(C.c_double)), ("type", C.POINTER(C.c_int32))]


class npsim_stats_cfg_t(C.Structure):
    _fields_ = [("r_max", C.c_double), ("n_bins", C.c_int32), ("radial_bins", C.c_int32),
                ("boxcount", C.c_int32), ("max_scales", C.c_int32)]


class npsim_stats_t(C.Structure):
    _fields_ = [("R", C.c_double), ("d_mean", C.c_double), ("Rg", C.c_double),
                ("Df_rg", C.c_double), ("Df_box", C.c_double), ("center", C.c_double * 3),
                ("n_scales", C.c_int32), ("pad_", C.c_int32),
                ("nbox", C.c_int64 * MAX_SCALES), ("n_surf", C.c_int64)]


_lock = threading.Lock()
_lib = None
_d = C.POINTER(C.c_double)
_i64 = C.POINTER(C.c_int64)
_i32 = C.POINTER(C.c_int32)
_u32 = C.POINTER(C.c_uint32)
_h = C.c_void_p


def lib():
    """The loaded libnpsim.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -m paper_2501_04456_gb300.build` (needs nvcc, sm_103a)")
            L = C.CDLL(LIB_PATH)
            L.npsim_last_error.restype = C.c_char_p
            L.npsim_device_info.argtypes = [_i32, _i32, _i32, _i32]
            L.npsim_create.argtypes = [C.POINTER(npsim_type_t), C.POINTER(npsim_params_t),
                                       C.c_int64, _d, _d, _i32, C.c_void_p,
                                       C.POINTER(_h)]
            L.npsim_destroy.argtypes = [_h]
            L.npsim_destroy.restype = None
            L.npsim_step.argtypes = [_h, C.c_int64]
            L.npsim_get_state.argtypes = [_h, _d, _d, _d, _i64]
            L.npsim_set_state.argtypes = [_h, _d, _d, C.c_int64]
            L.npsim_forces.argtypes = [_h, C.c_int, _d]
            L.npsim_positions_device.argtypes = [_h, C.c_void_p]
            L.npsim_stats.argtypes = [_h, C.POINTER(npsim_stats_cfg_t), _i64, _d, _i64, _d,
                                      C.POINTER(npsim_stats_t)]
            L.npsim_scattering.argtypes = [_d, C.c_int32, C.c_double, C.c_double, C.c_double,
                                           C.c_double, _d, C.c_int32, _d, _d]
            L.npsim_step_record.argtypes = [_h, C.c_int64, C.c_int64, C.POINTER(C.c_float),
                                            C.c_int64]
            L.npsim_save.argtypes = [_h, C.c_char_p]
            L.npsim_load.argtypes = [C.c_char_p, C.POINTER(npsim_type_t),
                                     C.POINTER(npsim_params_t), C.c_void_p, C.POINTER(_h)]
            L.npsim_philox.argtypes = [C.c_uint64, _u32, C.c_int64, _u32]
            L.npsim_normals.argtypes = [C.c_uint64, C.c_int64, C.c_int64, _d]
            L.npsim_allpairs_config.argtypes = [_h, _i32, _i32, _i32, _i32, _i32, _i32]
            L.npsim_allpairs_num_configs.argtypes = [_i32]
            L.npsim_allpairs_ranges.argtypes = [_h, _i32]
            L.npsim_coulomb_forces_noalloc.argtypes = [C.c_void_p, C.c_int64, C.c_double,
                                                       C.c_void_p, C.c_void_p]
            L.npsim_launches_per_step.argtypes = [_h, _i32]
            L.npsim_fma_peak.argtypes = [C.c_int, C.c_int64, C.c_void_p, _d,
                                         C.POINTER(C.c_float), _i32]
            L.npsim_cell_grid.argtypes = [_h, _i32, _i64]
            L.npsim_nbr_info.argtypes = [_h, _i32, _d, _i64]
            L.npsim_ens_create.argtypes = [C.POINTER(npsim_droplet_t), C.c_int32, C.c_void_p,
                                           C.POINTER(_h)]
            L.npsim_ens_step.argtypes = [_h, C.c_int64]
            L.npsim_ens_get_state.argtypes = [_h, C.c_int32, _d, _d, _d, _i64]
            L.npsim_ens_forces.argtypes = [_h, C.c_int32, _d]
            L.npsim_ens_config.argtypes = [_h, _i32, _i32, _i32, _i32, _i32]
            L.npsim_ens_stats.argtypes = [_h, C.c_int32, C.POINTER(npsim_stats_cfg_t), _i64,
                                          _d, _i64, _d, C.POINTER(npsim_stats_t)]
            L.npsim_ens_info.argtypes = [_h, _i64, _d]
            L.npsim_ens_work.argtypes = [_h, _i64, _i32]
            L.npsim_ens_destroy.argtypes = [_h]
            L.npsim_ens_destroy.restype = None
            _f = C.POINTER(C.c_float)
            L.npsim_surr_create.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                            C.c_int32, C.c_uint64, C.POINTER(_h)]
            L.npsim_surr_destroy.argtypes = [_h]
            L.npsim_surr_destroy.restype = None
            L.npsim_surr_set_norm.argtypes = [_h, _f, _f, _f, _f]
            L.npsim_surr_param_count.argtypes = [_h, _i64]
            L.npsim_surr_get_params.argtypes = [_h, C.c_int32, _f, _f]
            L.npsim_surr_set_params.argtypes = [_h, C.c_int32, _f]
            L.npsim_surr_grads.argtypes = [_h, C.c_int32, _f, _f, C.c_int32, _f, _f, _f]
            L.npsim_surr_train.argtypes = [_h, _f, _f, C.c_int32, C.c_int32, C.c_int32,
                                           C.c_float, C.c_float, C.c_uint64, _f]
            L.npsim_surr_predict.argtypes = [_h, _f, C.c_int32, _f, _f]
            L.npsim_gemm_bf16.argtypes = [C.POINTER(C.c_uint16), C.POINTER(C.c_uint16),
                                          C.c_int32, C.c_int32, C.c_int32, C.c_int32, _f]
            L.npsim_chunk_steps.argtypes = [_h, _i32]
            L.npsim_test_wait_cycles.argtypes = [C.c_int64]
            L.npsim_profile.argtypes = [_h, C.c_int]
            L.npsim_kernel_times.argtypes = [_h, _d, _i32]
            L.npsim_ens_profile.argtypes = [_h, C.c_int]
            L.npsim_ens_kernel_times.argtypes = [_h, _d, _i32]
            _lib = L
        return _lib


def npsim_last_error() -> str:
    return lib().npsim_last_error().decode()


def _check(rc):
    if rc != NPSIM_OK:
        raise NpsimError(rc, npsim_last_error())


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _aos(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1, 3)
    if n is not None and a.shape[0] != n:
        raise ValueError(f"expected {n} x 3 array, got {a.shape}")
    return a


# --------------------------------------------------------------------------
# Scenario marshalling (duck-typed: any object with the fields of the C structs)


def types_from(specs):
    arr = (npsim_type_t * MAX_TYPES)()
    for k, t in enumerate(specs):
        arr[k] = npsim_type_t(t.sigma, t.eps, t.mass, t.charge, t.gamma, t.k_wall)
    return arr


def params_from(sc):
    """npsim_params_t from a scenario object (n_types taken from sc.types)."""
    p = npsim_params_t()
    p.n_types = len(sc.types)
    p.rot_mode = sc.rot_mode
    p.lj_mode = sc.lj_mode
    ccut = float(getattr(sc, "coulomb_cut", 0.0))
    p.coulomb = 0 if not sc.coulomb else (2 if ccut > 0 else 1)
    p.coulomb_cut = ccut
    p.wall = 0 if not sc.wall else (2 if getattr(sc, "wall_band", False) else 1)
    p.integrator = sc.integrator
    p.v_kick = float(getattr(sc, "v_kick", 0.0))
    p.sum_neutral = int(bool(getattr(sc, "sum_neutral", False)))
    p.seed = sc.seed
    p.dt, p.kT, p.R0, p.k_evap = sc.dt, sc.kT, sc.R0, sc.k_evap
    p.g, p.omega, p.bjerrum, p.lj_cut = sc.g, sc.omega, sc.bjerrum, sc.lj_cut
    ov = getattr(sc, "eps_override", None)
    if ov is not None:
        ov = np.ascontiguousarray(ov, dtype=np.float64).ravel()
        p._keep = ov
        p.eps_override = _p(ov, C.c_double)
    return p


# --------------------------------------------------------------------------
# Entry points


def npsim_device_info():
    a, b, c, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().npsim_device_info(C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
    return {"sm_count": a.value, "clock_khz": b.value, "cc": (c.value, d.value)}


def npsim_create(types, params, x0, v0, type, stream=None):
    x0 = _aos(x0)
    n = x0.shape[0]
    v0 = None if v0 is None else _aos(v0, n)
    ty = np.ascontiguousarray(type, dtype=np.int32)
    if ty.shape != (n,):
        raise ValueError("type must have one entry per particle")
    h = _h()
    _check(lib().npsim_create(types, C.byref(params), n, _p(x0, C.c_double),
                              None if v0 is None else _p(v0, C.c_double),
                              _p(ty, C.c_int32), _stream_handle(stream), C.byref(h)))
    return h


def npsim_destroy(h):
    lib().npsim_destroy(h)


def npsim_step(h, n_steps):
    _check(lib().npsim_step(h, int(n_steps)))


def npsim_get_state(h, n, out=None):
    """Positions, velocities and forces (n x 3 float64 each) and the step.  out:
    optional (x, v, F) arrays to fill, e.g. views of page-locked host memory,
    which the device copies reach faster than pageable memory."""
    if out is None:
        x, v, F = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3))
    else:
        x, v, F = out
        for a in (x, v, F):
            if a.shape != (n, 3) or a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ValueError("out arrays must be C-contiguous float64 of shape (n, 3)")
    st = C.c_int64()
    _check(lib().npsim_get_state(h, _p(x, C.c_double), _p(v, C.c_double),
                                 _p(F, C.c_double), C.byref(st)))
    return x, v, F, st.value


def npsim_set_state(h, x, v=None, step=0):
    x = _aos(x)
    v = None if v is None else _aos(v, x.shape[0])
    _check(lib().npsim_set_state(h, _p(x, C.c_double),
                                 None if v is None else _p(v, C.c_double), int(step)))


def npsim_forces(h, n, what=0):
    F = np.empty((n, 3))
    _check(lib().npsim_forces(h, int(what), _p(F, C.c_double)))
    return F


def npsim_positions_device(h, dev_ptr):
    _check(lib().npsim_positions_device(h, C.c_void_p(int(dev_ptr))))


def _stats_call(fn, r_max, n_bins, radial_bins, boxcount, max_scales):
    """Marshal the statistics outputs of npsim_stats / npsim_ens_stats: fn(cfg,
    rdf_counts, rdf_g, radial_counts, radial_c, out) returns the status."""
    cfg = npsim_stats_cfg_t(r_max, n_bins, radial_bins, int(boxcount), max_scales)
    counts = np.zeros(max(n_bins, 1), np.int64)
    g = np.zeros(max(n_bins, 1))
    rc_ = np.zeros(max(radial_bins, 1), np.int64)
    rcc = np.zeros(max(radial_bins, 1))
    out = npsim_stats_t()
    _check(fn(C.byref(cfg), _p(counts, C.c_int64), _p(g, C.c_double),
              _p(rc_, C.c_int64) if radial_bins else None,
              _p(rcc, C.c_double) if radial_bins else None, C.byref(out)))
    ns = out.n_scales
    return {"R": out.R, "d_mean": out.d_mean, "Rg": out.Rg, "Df_rg": out.Df_rg,
            "Df_box": out.Df_box, "center": np.array(out.center[:]),
            "nbox": np.array(out.nbox[:ns], np.int64), "n_surf": int(out.n_surf),
            "rdf_counts": counts[:n_bins], "rdf_g": g[:n_bins],
            "radial_counts": rc_[:radial_bins], "radial_c": rcc[:radial_bins]}


def npsim_stats(h, r_max=10.0, n_bins=128, radial_bins=0, boxcount=True,
                max_scales=MAX_SCALES):
    return _stats_call(lambda *a: lib().npsim_stats(h, *a), r_max, n_bins, radial_bins,
                       boxcount, max_scales)


def npsim_scattering(g, r_max, n_surf, q, Rg=1.0, Df=3.0):
    """I(q) of the NPs from the RDF g (Sec. 3.3) and the fractal form
    N_surf^2 (q R_g)^(-D_f); returns (I, I_frac) for the wave numbers q."""
    g = np.ascontiguousarray(g, np.float64)
    q = np.ascontiguousarray(q, np.float64)
    I = np.zeros(len(q))
    If = np.zeros(len(q))
    _check(lib().npsim_scattering(_p(g, C.c_double), len(g), r_max, float(n_surf), Rg, Df,
                                  _p(q, C.c_double), len(q), _p(I, C.c_double),
                                  _p(If, C.c_double)))
    return I, If


def frame_buffer(n_frames, n):
    """A float32 (n_frames, n, 4) array for recorded frames, in page-locked memory
    when torch can provide it (the library registers any other array per call)."""
    shape = (max(n_frames, 1), n, 4)
    try:
        import torch
        return torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy()
    except Exception:  # no torch or no pinned memory: a plain array
        return np.zeros(shape, np.float32)


def npsim_step_record(h, n, n_steps, every, out=None):
    """Advance n_steps steps recording every every-th frame: float32 (n_frames, n, 4)
    of (x, y, z, charge), into out (from frame_buffer) or a new buffer."""
    nf = n_steps // every
    frames = frame_buffer(nf, n) if out is None else out
    if frames.dtype != np.float32 or not frames.flags.c_contiguous or \
            frames.shape[1:] != (n, 4) or frames.shape[0] < nf:
        raise ValueError("out must be a C-contiguous float32 (>= n_frames, n, 4) array")
    _check(lib().npsim_step_record(h, n_steps, every, _p(frames, C.c_float), nf))
    return frames[:nf]


def npsim_save(h, path):
    _check(lib().npsim_save(h, os.fsencode(path)))


def npsim_load(path, types=None, params=None, stream=None):
    h = _h()
    _check(lib().npsim_load(os.fsencode(path), types,
                            None if params is None else C.byref(params),
                            _stream_handle(stream), C.byref(h)))
    return h


def npsim_philox(seed, ctr, n_blocks):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros((n_blocks, 4), np.uint32)
    _check(lib().npsim_philox(C.c_uint64(seed), _p(c, C.c_uint32), n_blocks,
                              _p(out, C.c_uint32)))
    return out


def npsim_normals(seed, step, n):
    out = np.zeros((n, 3))
    _check(lib().npsim_normals(C.c_uint64(seed), int(step), int(n), _p(out, C.c_double)))
    return out


def npsim_allpairs_config(h):
    v = [C.c_int32() for _ in range(6)]
    _check(lib().npsim_allpairs_config(h, *[C.byref(x) for x in v]))
    keys = ("block", "i_per_thread", "j_tile", "grid", "index", "packed")
    out = {k: x.value for k, x in zip(keys, v)}
    r = C.c_int32()
    _check(lib().npsim_allpairs_ranges(h, C.byref(r)))
    out["ranges"] = r.value
    return out


def npsim_allpairs_num_configs():
    a = C.c_int32()
    _check(lib().npsim_allpairs_num_configs(C.byref(a)))
    return a.value


def npsim_coulomb_forces_noalloc(dev_xyzq, n, bjerrum, dev_F, stream=None):
    """Coulomb forces from a device float4 (x, y, z, q) buffer into a device n x 3
    float64 buffer, with no device allocation (pointers as integers)."""
    _check(lib().npsim_coulomb_forces_noalloc(C.c_void_p(int(dev_xyzq)), int(n),
                                              float(bjerrum), C.c_void_p(int(dev_F)),
                                              _stream_handle(stream)))


def npsim_fma_peak(packed=True, iters=1 << 16, stream=None):
    """FP32 FMA microbenchmark: (flops, ms, grid) of one timed launch."""
    fl = C.c_double()
    ms = C.c_float()
    g = C.c_int32()
    _check(lib().npsim_fma_peak(int(bool(packed)), int(iters), _stream_handle(stream),
                                C.byref(fl), C.byref(ms), C.byref(g)))
    return fl.value, ms.value, g.value


def npsim_launches_per_step(h):
    a = C.c_int32()
    _check(lib().npsim_launches_per_step(h, C.byref(a)))
    return a.value


def npsim_cell_grid(h):
    """(cells per axis, cells) of the LJ cell list; (0, 0) without one."""
    d, c = C.c_int32(), C.c_int64()
    _check(lib().npsim_cell_grid(h, C.byref(d), C.byref(c)))
    return d.value, c.value


def npsim_nbr_info(h):
    """(list capacity, mean list length at the last build, builds so far) of the
    cell-list LJ neighbour lists; zeros without a cell list."""
    c, m, b = C.c_int32(), C.c_double(), C.c_int64()
    _check(lib().npsim_nbr_info(h, C.byref(c), C.byref(m), C.byref(b)))
    return c.value, m.value, b.value


def npsim_chunk_steps(h):
    a = C.c_int32()
    _check(lib().npsim_chunk_steps(h, C.byref(a)))
    return a.value


def npsim_profile(h, enable=True):
    _check(lib().npsim_profile(h, int(bool(enable))))


KERNEL_GROUPS = ("allpairs", "cell_build", "cell_lj", "integrate")


def npsim_kernel_times(h):
    ms = np.zeros(4)
    k = C.c_int32()
    _check(lib().npsim_kernel_times(h, _p(ms, C.c_double), C.byref(k)))
    return dict(zip(KERNEL_GROUPS, ms.tolist())), k.value


class Sim:
    """Owning wrapper around one simulation handle."""

    def __init__(self, scenario, x0, v0, types, stream=None):
        self.n = int(np.asarray(x0).reshape(-1, 3).shape[0])
        self.scenario = scenario
        self._types = types_from(scenario.types)
        self._params = params_from(scenario)
        self.h = npsim_create(self._types, self._params, x0, v0, types, stream)

    @classmethod
    def _wrap(cls, h, n, scenario=None):
        s = cls.__new__(cls)
        s.h, s.n, s.scenario = h, n, scenario
        return s

    @classmethod
    def load(cls, path, n, scenario=None, stream=None):
        """Resume a simulation of n NPs from a checkpoint written by save()."""
        return cls._wrap(npsim_load(path, stream=stream), n, scenario)

    def step(self, n_steps=1):
        npsim_step(self.h, n_steps)

    def record(self, n_steps, every=1, out=None):
        """Advance n_steps, returning every every-th frame of the float32 positions."""
        return npsim_step_record(self.h, self.n, n_steps, every, out)

    def state(self):
        return npsim_get_state(self.h, self.n)

    def set_state(self, x, v=None, step=0):
        npsim_set_state(self.h, x, v, step)

    def forces(self, what=0):
        return npsim_forces(self.h, self.n, what)

    def stats(self, **kw):
        return npsim_stats(self.h, **kw)

    def save(self, path):
        npsim_save(self.h, path)

    def allpairs_config(self):
        return npsim_allpairs_config(self.h)

    def launches_per_step(self):
        return npsim_launches_per_step(self.h)

    def chunk_steps(self):
        return npsim_chunk_steps(self.h)

    def cell_grid(self):
        return npsim_cell_grid(self.h)

    def nbr_info(self):
        return npsim_nbr_info(self.h)

    def profile(self, enable=True):
        npsim_profile(self.h, enable)

    def kernel_times(self):
        return npsim_kernel_times(self.h)

    def close(self):
        if getattr(self, "h", None):
            npsim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# --------------------------------------------------------------------------
# Ensemble of droplets


def npsim_ens_create(droplets, stream=None):
    """droplets: sequence of (scenario, x0, v0, type).  Returns (handle, keepalive)."""
    arr = (npsim_droplet_t * len(droplets))()
    keep = []
    for k, (sc, x0, v0, ty) in enumerate(droplets):
        x0 = _aos(x0)
        n = x0.shape[0]
        v0 = None if v0 is None else _aos(v0, n)
        ty = np.ascontiguousarray(ty, dtype=np.int32)
        tys = types_from(sc.types)
        par = params_from(sc)
        keep += [x0, v0, ty, tys, par]
        arr[k].n = n
        arr[k].types = C.cast(tys, C.POINTER(npsim_type_t))
        arr[k].params = par
        arr[k].x0 = _p(x0, C.c_double)
        arr[k].v0 = None if v0 is None else _p(v0, C.c_double)
        arr[k].type = _p(ty, C.c_int32)
    h = _h()
    _check(lib().npsim_ens_create(arr, len(droplets), _stream_handle(stream), C.byref(h)))
    return h


def npsim_ens_step(h, n_steps):
    _check(lib().npsim_ens_step(h, int(n_steps)))


def npsim_ens_get_state(h, d, n):
    x = np.empty((n, 3))
    v = np.empty((n, 3))
    F = np.empty((n, 3))
    st = C.c_int64()
    _check(lib().npsim_ens_get_state(h, int(d), _p(x, C.c_double), _p(v, C.c_double),
                                     _p(F, C.c_double), C.byref(st)))
    return x, v, F, st.value


def npsim_ens_forces(h, d, n):
    F = np.empty((n, 3))
    _check(lib().npsim_ens_forces(h, int(d), _p(F, C.c_double)))
    return F


def npsim_ens_config(h):
    v = [C.c_int32() for _ in range(5)]
    _check(lib().npsim_ens_config(h, *[C.byref(x) for x in v]))
    return dict(zip(("block", "i_per_thread", "j_tile", "grid", "index"), [x.value for x in v]))


def npsim_ens_stats(h, d, r_max=10.0, n_bins=128, radial_bins=0, boxcount=True,
                    max_scales=MAX_SCALES):
    return _stats_call(lambda *a: lib().npsim_ens_stats(h, int(d), *a), r_max, n_bins,
                       radial_bins, boxcount, max_scales)


def npsim_ens_info(h):
    n = C.c_int64()
    p = C.c_double()
    _check(lib().npsim_ens_info(h, C.byref(n), C.byref(p)))
    return n.value, p.value


def npsim_ens_work(h):
    n = C.c_int64()
    t = C.c_int32()
    _check(lib().npsim_ens_work(h, C.byref(n), C.byref(t)))
    return n.value, t.value


def npsim_ens_destroy(h):
    lib().npsim_ens_destroy(h)


def npsim_ens_profile(h, enable=True):
    _check(lib().npsim_ens_profile(h, int(bool(enable))))


ENS_KERNEL_GROUPS = ("allpairs", "integrate")


def npsim_ens_kernel_times(h):
    ms = np.zeros(2)
    k = C.c_int32()
    _check(lib().npsim_ens_kernel_times(h, _p(ms, C.c_double), C.byref(k)))
    return dict(zip(ENS_KERNEL_GROUPS, ms.tolist())), k.value


class Ensemble:
    """Owning wrapper around an ensemble handle; droplets = [(scenario, x0, v0, type)]."""

    def __init__(self, droplets, stream=None):
        self.sizes = [int(np.asarray(d[1]).reshape(-1, 3).shape[0]) for d in droplets]
        self.h = npsim_ens_create(droplets, stream)

    def step(self, n_steps=1):
        npsim_ens_step(self.h, n_steps)

    def state(self, d):
        return npsim_ens_get_state(self.h, d, self.sizes[d])

    def forces(self, d):
        return npsim_ens_forces(self.h, d, self.sizes[d])

    def config(self):
        return npsim_ens_config(self.h)

    def stats(self, d, **kw):
        return npsim_ens_stats(self.h, d, **kw)

    def info(self):
        return npsim_ens_info(self.h)

    def work(self):
        return npsim_ens_work(self.h)

    def profile(self, enable=True):
        npsim_ens_profile(self.h, enable)

    def kernel_times(self):
        return npsim_ens_kernel_times(self.h)

    def close(self):
        if getattr(self, "h", None):
            npsim_ens_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# --------------------------------------------------------------------------
# Learned surrogate (deep ensemble of MLPs on the tcgen05 tensor cores)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


def npsim_gemm_bf16(A_bits, B_bits, n_tile=64):
    """C = A B^T on the tensor-core GEMM; A (M x K), B (N x K) uint16 BF16 bit patterns."""
    A = np.ascontiguousarray(A_bits, dtype=np.uint16)
    B = np.ascontiguousarray(B_bits, dtype=np.uint16)
    M, K = A.shape
    N = B.shape[0]
    Cm = np.zeros((M, N), np.float32)
    _check(lib().npsim_gemm_bf16(_p(A, C.c_uint16), _p(B, C.c_uint16), M, N, K, n_tile,
                                 _p(Cm, C.c_float)))
    return Cm


def npsim_test_wait_cycles(cycles):
    """Bound (SM cycles) of the GEMM kernel's main-loop waits; 0 = default."""
    _check(lib().npsim_test_wait_cycles(int(cycles)))


class Surrogate:
    """Deep ensemble of MLPs: n_in -> n_layers x n_hidden (SiLU) -> n_out."""

    def __init__(self, n_in=8, n_hidden=256, n_layers=4, n_out=65, n_nets=4, seed=0):
        self.n_in, self.n_out, self.n_nets = n_in, n_out, n_nets
        self.h = _h()
        _check(lib().npsim_surr_create(n_in, n_hidden, n_layers, n_out, n_nets,
                                       C.c_uint64(seed), C.byref(self.h)))
        c = C.c_int64()
        _check(lib().npsim_surr_param_count(self.h, C.byref(c)))
        self.n_params = c.value

    def set_norm(self, x_mean=None, x_std=None, y_mean=None, y_std=None):
        args = []
        keep = []
        for v, n in ((x_mean, self.n_in), (x_std, self.n_in), (y_mean, self.n_out),
                     (y_std, self.n_out)):
            if v is None:
                args.append(None)
            else:
                a = _f32(v).reshape(n)
                keep.append(a)
                args.append(_p(a, C.c_float))
        _check(lib().npsim_surr_set_norm(self.h, *args))

    def get_params(self, net=0):
        p = np.zeros(self.n_params, np.float32)
        g = np.zeros(self.n_params, np.float32)
        _check(lib().npsim_surr_get_params(self.h, net, _p(p, C.c_float), _p(g, C.c_float)))
        return p, g

    def set_params(self, net, flat):
        f = _f32(flat).reshape(self.n_params)
        _check(lib().npsim_surr_set_params(self.h, net, _p(f, C.c_float)))

    def grads(self, net, X, Y):
        X = _f32(X, (-1, self.n_in))
        Y = _f32(Y, (-1, self.n_out))
        B = X.shape[0]
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_float()
        yh = np.zeros((B, self.n_out), np.float32)
        _check(lib().npsim_surr_grads(self.h, net, _p(X, C.c_float), _p(Y, C.c_float), B,
                                      _p(g, C.c_float), C.byref(loss), _p(yh, C.c_float)))
        return g, loss.value, yh

    def train(self, X, Y, epochs=10, batch=512, lr=1e-3, wd=1e-4, seed=0):
        X = _f32(X, (-1, self.n_in))
        Y = _f32(Y, (-1, self.n_out))
        loss = C.c_float()
        _check(lib().npsim_surr_train(self.h, _p(X, C.c_float), _p(Y, C.c_float), X.shape[0],
                                      epochs, batch, lr, wd, C.c_uint64(seed), C.byref(loss)))
        return loss.value

    def predict(self, X):
        X = _f32(X, (-1, self.n_in))
        B = X.shape[0]
        m = np.zeros((B, self.n_out), np.float32)
        sp = np.zeros((B, self.n_out), np.float32)
        _check(lib().npsim_surr_predict(self.h, _p(X, C.c_float), B, _p(m, C.c_float),
                                        _p(sp, C.c_float)))
        return m, sp

    def close(self):
        if getattr(self, "h", None):
            lib().npsim_surr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
