"""ctypes binding of libgpeshell (include/gpe.h).

Argument marshalling only: every function below calls the C function of the
same name, converting Python objects (numpy arrays, torch tensors, ints) to
pointers and out-parameters to return values, and raising ``GpeError`` on a
non-zero status.  All arithmetic of the method runs in the CUDA library.

torch is used only as plumbing: device memory (``tensor.data_ptr()``) and
streams (``torch.cuda.current_stream().cuda_stream``).  The library must have
been built (``paper_2603_05447_gb300._build.build()``); importing the binding
without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

from . import _build

# ----------------------------------------------------------------- constants
GPE_OK = 0
GPE_ERR_ARG = -1
GPE_ERR_CUDA = -2
GPE_ERR_OOM = -3
GPE_ERR_NONFINITE = -4
GPE_ERR_UNSTABLE = -5
GPE_ERR_NOT_CONVERGED = -6
GPE_ERR_STATE = -7
ERROR_NAMES = {v: k for k, v in dict(
    GPE_ERR_ARG=-1, GPE_ERR_CUDA=-2, GPE_ERR_OOM=-3, GPE_ERR_NONFINITE=-4,
    GPE_ERR_UNSTABLE=-5, GPE_ERR_NOT_CONVERGED=-6, GPE_ERR_STATE=-7).items()}

GPE_MASK_CELL, GPE_MASK_BRICK = 0, 1
GPE_ORDER_ZMAJOR, GPE_ORDER_MORTON = 0, 1
GPE_SCHED_STAGED, GPE_SCHED_WAVE, GPE_SCHED_WAVE2, GPE_SCHED_PAIR = 0, 1, 2, 3
GPE_F64, GPE_F32 = 1, 2
GPE_POT_HARMONIC, GPE_POT_ELLIPSOID_SHELL = 1, 2
GPE_C128, GPE_C64, GPE_R64, GPE_R32 = 1, 2, 3, 4
GPE_LAYOUT_DENSE, GPE_LAYOUT_COMPACT = 0, 1
GPE_RK4, GPE_RKHE3, GPE_RKCK = 0, 1, 2
GPE_V_STATIC, GPE_V_BLEND = 0, 1
GPE_MAX_KNOTS = 16


# ----------------------------------------------------------------- structs
class gpe_box(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
                ("hx", C.c_double), ("hy", C.c_double), ("hz", C.c_double),
                ("x0", C.c_double), ("y0", C.c_double), ("z0", C.c_double)]


class gpe_grid_opts(C.Structure):
    _fields_ = [("bx", C.c_int32), ("by", C.c_int32), ("bz", C.c_int32),
                ("mask_mode", C.c_int32), ("order", C.c_int32), ("sched", C.c_int32),
                ("chunk", C.c_int32), ("stencil", C.c_int32)]


class gpe_potential(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("p", C.c_double * 8)]


class gpe_grid_info(C.Structure):
    _fields_ = [("n_active", C.c_int64), ("n_bricks", C.c_int64), ("n_stored", C.c_int64),
                ("n_packed", C.c_int64), ("bx", C.c_int32), ("by", C.c_int32), ("bz", C.c_int32), ("mask_mode", C.c_int32),
                ("order", C.c_int32), ("n_slots", C.c_int32), ("v_max", C.c_double),
                ("box", gpe_box)]


class gpe_imag_params(C.Structure):
    _fields_ = [("g", C.c_double), ("dt", C.c_double), ("N", C.c_double)]


class gpe_real_params(C.Structure):
    _fields_ = [("g", C.c_double), ("dt", C.c_double), ("integrator", C.c_int32),
                ("potential", C.c_int32), ("n_knots", C.c_int32), ("reserved", C.c_int32),
                ("T_ramp", C.c_double), ("knots", C.c_double * GPE_MAX_KNOTS)]


class gpe_obs(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("norm", "energy", "mu", "nonfinite", "e_kin", "e_pot", "e_int")]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class gpe_tune_result(C.Structure):
    _fields_ = [("bx", C.c_int32), ("by", C.c_int32), ("bz", C.c_int32), ("sched", C.c_int32),
                ("chunk", C.c_int32), ("reserved", C.c_int32), ("cell_steps_per_s", C.c_double),
                ("ms_per_step", C.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


GPE_TUNE_REAL, GPE_TUNE_IMAG = 0, 1


class gpe_ramp_pot(C.Structure):
    _fields_ = [("analytic", C.POINTER(gpe_potential)), ("V", C.c_void_p), ("V_dtype", C.c_int32),
                ("V_on_device", C.c_int32)]


class gpe_stage_params(C.Structure):
    _fields_ = [("g", C.c_double), ("N", C.c_double), ("dt", C.c_double), ("cut_factor", C.c_double),
                ("t_hold", C.c_double), ("integrator", C.c_int32), ("reserved", C.c_int32)]


class gpe_stage_report(C.Structure):
    _fields_ = [("mu_a", C.c_double), ("mu_b", C.c_double), ("cut", C.c_double), ("n_active", C.c_int64),
                ("steps", C.c_int64), ("dt", C.c_double), ("norm_kept", C.c_double), ("norm_end", C.c_double),
                ("regrid_s", C.c_double)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GpeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


# ----------------------------------------------------------------- library
_lib = None
_P = C.c_void_p
_SIGS = {
    "gpe_version": (C.c_int, []),
    "gpe_last_error": (C.c_int, [C.c_char_p, C.c_size_t]),
    "gpe_launch_count": (C.c_int, [C.POINTER(C.c_uint64)]),
    "gpe_fma_peak": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "gpe_grid_create_dense": (C.c_int, [C.POINTER(gpe_box), _P, C.c_int, C.c_int, C.c_double,
                                        C.POINTER(gpe_grid_opts), C.POINTER(_P), _P]),
    "gpe_grid_create_analytic": (C.c_int, [C.POINTER(gpe_box), C.POINTER(gpe_potential), C.c_double,
                                           C.POINTER(gpe_grid_opts), C.POINTER(_P), _P]),
    "gpe_grid_create_blend": (C.c_int, [C.POINTER(gpe_box), C.POINTER(gpe_potential), C.c_double,
                                        C.POINTER(gpe_potential), C.c_double, C.POINTER(gpe_grid_opts),
                                        C.POINTER(_P), _P]),
    "gpe_grid_create_blend_dense": (C.c_int, [C.POINTER(gpe_box), _P, _P, C.c_int, C.c_int, C.c_double,
                                              C.c_double, C.POINTER(gpe_grid_opts), C.POINTER(_P), _P]),
    "gpe_grid_set_potential": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_int, _P]),
    "gpe_grid_get_info": (C.c_int, [_P, C.POINTER(gpe_grid_info)]),
    "gpe_grid_bricks": (C.c_int, [_P, _P, _P]),
    "gpe_grid_mask": (C.c_int, [_P, _P]),
    "gpe_grid_potential": (C.c_int, [_P, C.c_int, _P]),
    "gpe_grid_destroy": (C.c_int, [_P]),
    "gpe_tf_mu_dense": (C.c_int, [C.POINTER(gpe_box), _P, C.c_int, C.c_int, C.c_double, C.c_double,
                                  C.POINTER(C.c_double), _P]),
    "gpe_tf_mu_analytic": (C.c_int, [C.POINTER(gpe_box), C.POINTER(gpe_potential), C.c_double, C.c_double,
                                     C.POINTER(C.c_double), _P]),
    "gpe_state_create": (C.c_int, [_P, C.c_int, C.POINTER(_P)]),
    "gpe_state_load": (C.c_int, [_P, _P, C.c_int, C.c_int, _P]),
    "gpe_state_store": (C.c_int, [_P, _P, C.c_int, C.c_int, _P]),
    "gpe_state_copy": (C.c_int, [_P, _P, _P]),
    "gpe_state_remap": (C.c_int, [_P, _P, _P]),
    "gpe_state_device_ptr": (C.c_int, [_P, C.POINTER(_P)]),
    "gpe_state_destroy": (C.c_int, [_P]),
    "gpe_step_imag": (C.c_int, [_P, C.POINTER(gpe_imag_params), C.c_int64, _P]),
    "gpe_step_real": (C.c_int, [_P, C.POINTER(gpe_real_params), C.c_int64, C.c_double, _P]),
    "gpe_observables": (C.c_int, [_P, C.c_double, C.c_double, C.POINTER(gpe_obs), _P]),
    "gpe_overlap": (C.c_int, [_P, _P, C.POINTER(C.c_double), _P]),
    "gpe_step_real_traced": (C.c_int, [_P, C.POINTER(gpe_real_params), C.c_int64, C.c_double, C.c_int64,
                                       C.POINTER(gpe_obs), C.POINTER(C.c_int64), _P]),
    "gpe_state_set_graph": (C.c_int, [_P, C.c_int]),
    "gpe_wait_selftest": (C.c_int, [C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "gpe_batch_create": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_P)]),
    "gpe_batch_ground_state": (C.c_int, [_P, C.POINTER(gpe_imag_params), C.c_double, C.c_int64, C.c_int64,
                                         C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(gpe_obs), _P]),
    "gpe_batch_destroy": (C.c_int, [_P]),
    "gpe_autotune": (C.c_int, [C.POINTER(gpe_box), C.POINTER(gpe_potential), C.c_double, C.c_int, C.c_int, C.c_int,
                               C.POINTER(gpe_tune_result), C.POINTER(gpe_tune_result), C.POINTER(C.c_int), _P]),
    "gpe_batch_autotune": (C.c_int, [C.POINTER(gpe_box), C.POINTER(gpe_potential), C.POINTER(C.c_double), C.c_int,
                                     C.c_int, C.c_int, C.POINTER(gpe_tune_result), C.POINTER(gpe_tune_result),
                                     C.POINTER(C.c_int), _P]),
    "gpe_ramp_forward": (C.c_int, [_P, C.POINTER(gpe_real_params), C.c_int64, C.c_double, C.c_int, C.POINTER(_P), _P]),
    "gpe_ramp_backward": (C.c_int, [_P, _P, C.POINTER(C.c_double), C.POINTER(C.c_double), _P]),
    "gpe_tape_destroy": (C.c_int, [_P]),
    "gpe_ramp_stages": (C.c_int, [_P, C.POINTER(gpe_ramp_pot), C.c_int, C.POINTER(C.c_double),
                                  C.POINTER(gpe_stage_params), C.POINTER(gpe_grid_opts), C.POINTER(_P),
                                  C.POINTER(_P), C.POINTER(gpe_stage_report), _P]),
    "gpe_overlap_noalloc": (C.c_int, [_P, _P, C.c_int64, C.c_int, C.c_double, C.POINTER(C.c_double), _P]),
    "gpe_ground_state": (C.c_int, [_P, C.POINTER(gpe_imag_params), C.c_double, C.c_int64, C.c_int64,
                                   C.POINTER(C.c_int64), C.POINTER(gpe_obs), _P]),
}


def library_path() -> str:
    return _build.LIB


def load() -> C.CDLL:
    """Load the built library (no build, no fallback: raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libgpeshell.so is not built ({path}); call __graft_entry__.build() "
                           "or paper_2603_05447_gb300._build.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def gpe_last_error() -> str:
    buf = C.create_string_buffer(1024)
    load().gpe_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


last_error = gpe_last_error


def _check(rc):
    if rc != GPE_OK:
        raise GpeError(rc, last_error())
    return rc


# ----------------------------------------------------------------- marshalling
def _torch():
    return sys.modules.get("torch")


def stream_handle(stream=None) -> int:
    """cudaStream_t as an int: an int passes through, a torch stream gives its
    handle, None gives torch's current stream (0 if torch is not loaded)."""
    if stream is None:
        t = _torch()
        if t is not None and t.cuda.is_available() and t.cuda.is_initialized():
            return int(t.cuda.current_stream().cuda_stream)
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def pointer(x):
    """(address, on_device) of a numpy array, torch tensor or raw device int."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    if isinstance(x, int):
        return x, 1
    t = _torch()
    if t is not None and isinstance(x, t.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), int(x.is_cuda)
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


def real_dtype_code(x) -> int:
    dt = str(getattr(x, "dtype", ""))
    if dt.endswith("float64"):
        return GPE_F64
    if dt.endswith("float32"):
        return GPE_F32
    raise TypeError(f"potential must be float64 or float32, got {dt}")


def make_box(nx, ny, nz, hx, hy=None, hz=None, x0=None, y0=None, z0=None) -> gpe_box:
    hy = hx if hy is None else hy
    hz = hx if hz is None else hz
    x0 = -(nx - 1) / 2 * hx if x0 is None else x0
    y0 = -(ny - 1) / 2 * hy if y0 is None else y0
    z0 = -(nz - 1) / 2 * hz if z0 is None else z0
    return gpe_box(nx, ny, nz, hx, hy, hz, x0, y0, z0)


def make_opts(brick=(8, 8, 8), mask_mode=GPE_MASK_CELL, order=GPE_ORDER_ZMAJOR, sched=GPE_SCHED_STAGED,
              chunk=0, stencil=7) -> gpe_grid_opts:
    o = gpe_grid_opts()
    o.bx, o.by, o.bz = brick
    o.mask_mode = mask_mode
    o.order = order
    o.sched = sched
    o.chunk = chunk
    o.stencil = stencil
    return o


def packed_layout(grid):
    """Host-side map of the compact layout: (packed index, brick, local cell)
    of every active cell, from the brick list and the mask, by the rule of
    include/gpe.h (each brick stores, in order, its 4-cell x-segments that
    hold an active cell)."""
    info = gpe_grid_get_info(grid)
    bits = gpe_grid_mask(grid)
    bc = info.bx * info.by * info.bz
    act = np.unpackbits(bits.view(np.uint8), bitorder="little").astype(bool).reshape(info.n_bricks, bc)
    seg = act.reshape(info.n_bricks, bc // 4, 4).any(axis=2)
    nseg = seg.sum(axis=1)
    off = 4 * np.concatenate([[0], np.cumsum(nseg)[:-1]]).astype(np.int64)
    seg_rank = np.cumsum(seg, axis=1) - 1
    b, l = np.nonzero(act)
    return off[b] + 4 * seg_rank[b, l // 4] + (l % 4), b, l


def packed_coords(grid):
    """(packed index, i, j, k) of every active cell."""
    info = gpe_grid_get_info(grid)
    org, _ = gpe_grid_bricks(grid)
    idx, b, l = packed_layout(grid)
    i = org[b, 0] + l % info.bx
    j = org[b, 1] + (l // info.bx) % info.by
    k = org[b, 2] + l // (info.bx * info.by)
    return idx, i, j, k


def make_potential(kind, *params) -> gpe_potential:
    p = gpe_potential()
    p.kind = kind
    for i, v in enumerate(params):
        p.p[i] = float(v)
    return p


def real_params(g, dt, potential=GPE_V_STATIC, knots=None, T_ramp=0.0, integrator=GPE_RK4) -> gpe_real_params:
    p = gpe_real_params()
    p.g, p.dt = float(g), float(dt)
    p.integrator = integrator
    p.potential = potential
    if knots is not None:
        knots = list(knots)
        p.n_knots = len(knots)
        for i, v in enumerate(knots):
            p.knots[i] = float(v)
    p.T_ramp = float(T_ramp)
    return p


# ----------------------------------------------------------------- C ABI, same names
def gpe_version() -> int:
    return load().gpe_version()


def gpe_launch_count() -> int:
    n = C.c_uint64()
    _check(load().gpe_launch_count(C.byref(n)))
    return n.value


def gpe_fma_peak(dtype, iters):
    """Measured CUDA-core FMA throughput (TFLOP/s, seconds) in FP64 (GPE_F64)
    or FP32 (GPE_F32)."""
    t, sec = C.c_double(), C.c_double()
    _check(load().gpe_fma_peak(int(dtype), int(iters), C.byref(t), C.byref(sec)))
    return t.value, sec.value


def gpe_grid_create_dense(box, V, V_cut, opts=None, stream=None):
    ptr, dev = pointer(V)
    out = _P()
    _check(load().gpe_grid_create_dense(C.byref(box), ptr, real_dtype_code(V), dev, float(V_cut),
                                        C.byref(opts) if opts else None, C.byref(out), stream_handle(stream)))
    return out.value


def gpe_grid_create_analytic(box, pot, V_cut, opts=None, stream=None):
    out = _P()
    _check(load().gpe_grid_create_analytic(C.byref(box), C.byref(pot), float(V_cut),
                                           C.byref(opts) if opts else None, C.byref(out), stream_handle(stream)))
    return out.value


def gpe_grid_create_blend(box, pot0, cut0, pot1, cut1, opts=None, stream=None):
    out = _P()
    _check(load().gpe_grid_create_blend(C.byref(box), C.byref(pot0), float(cut0), C.byref(pot1), float(cut1),
                                        C.byref(opts) if opts else None, C.byref(out), stream_handle(stream)))
    return out.value


def gpe_grid_create_blend_dense(box, V0, V1, cut0, cut1, opts=None, stream=None):
    p0, dev0 = pointer(V0)
    p1, dev1 = pointer(V1)
    if dev0 != dev1 or real_dtype_code(V0) != real_dtype_code(V1):
        raise GpeError(GPE_ERR_ARG, "V0 and V1 must share dtype and location")
    out = _P()
    _check(load().gpe_grid_create_blend_dense(C.byref(box), p0, p1, real_dtype_code(V0), dev0, float(cut0),
                                              float(cut1), C.byref(opts) if opts else None, C.byref(out),
                                              stream_handle(stream)))
    return out.value


def gpe_grid_set_potential(grid, slot, V, stream=None):
    ptr, dev = pointer(V)
    _check(load().gpe_grid_set_potential(grid, int(slot), ptr, real_dtype_code(V), dev, stream_handle(stream)))


def gpe_grid_get_info(grid) -> gpe_grid_info:
    info = gpe_grid_info()
    _check(load().gpe_grid_get_info(grid, C.byref(info)))
    return info


def gpe_grid_bricks(grid):
    info = gpe_grid_get_info(grid)
    org = np.empty((info.n_bricks, 3), dtype=np.int32)
    nbr = np.empty((info.n_bricks, 6), dtype=np.int32)
    _check(load().gpe_grid_bricks(grid, org.ctypes.data, nbr.ctypes.data))
    return org, nbr


def gpe_grid_mask(grid):
    info = gpe_grid_get_info(grid)
    bits = np.empty(info.n_stored // 32, dtype=np.uint32)
    _check(load().gpe_grid_mask(grid, bits.ctypes.data))
    return bits


def gpe_grid_potential(grid, slot=0):
    info = gpe_grid_get_info(grid)
    V = np.empty(info.n_packed, dtype=np.float64)
    _check(load().gpe_grid_potential(grid, int(slot), V.ctypes.data))
    return V


def gpe_grid_destroy(grid):
    _check(load().gpe_grid_destroy(grid))


def gpe_tf_mu_dense(box, V, g, N, stream=None) -> float:
    ptr, dev = pointer(V)
    mu = C.c_double()
    _check(load().gpe_tf_mu_dense(C.byref(box), ptr, real_dtype_code(V), dev, float(g), float(N), C.byref(mu),
                                  stream_handle(stream)))
    return mu.value


def gpe_tf_mu_analytic(box, pot, g, N, stream=None) -> float:
    mu = C.c_double()
    _check(load().gpe_tf_mu_analytic(C.byref(box), C.byref(pot), float(g), float(N), C.byref(mu),
                                     stream_handle(stream)))
    return mu.value


def gpe_state_create(grid, dtype):
    out = _P()
    _check(load().gpe_state_create(grid, int(dtype), C.byref(out)))
    return out.value


def gpe_state_load(state, psi, layout, stream=None):
    ptr, dev = pointer(psi)
    _check(load().gpe_state_load(state, ptr, int(layout), dev, stream_handle(stream)))


def gpe_state_store(state, psi, layout, stream=None):
    ptr, dev = pointer(psi)
    _check(load().gpe_state_store(state, ptr, int(layout), dev, stream_handle(stream)))


def gpe_state_copy(dst, src, stream=None):
    _check(load().gpe_state_copy(dst, src, stream_handle(stream)))


def gpe_state_remap(dst, src, stream=None):
    """Remap src onto dst's grid (same box): cells active in both keep src's
    value, the others of dst become 0 (Sec. V regrid between ramp stages)."""
    _check(load().gpe_state_remap(dst, src, stream_handle(stream)))


def gpe_state_device_ptr(state) -> int:
    out = _P()
    _check(load().gpe_state_device_ptr(state, C.byref(out)))
    return out.value


def gpe_state_destroy(state):
    _check(load().gpe_state_destroy(state))


def gpe_step_imag(state, params: gpe_imag_params, nsteps, stream=None):
    _check(load().gpe_step_imag(state, C.byref(params), int(nsteps), stream_handle(stream)))


def gpe_step_real(state, params: gpe_real_params, nsteps, t0=0.0, stream=None):
    _check(load().gpe_step_real(state, C.byref(params), int(nsteps), float(t0), stream_handle(stream)))


def gpe_observables(state, g, s_blend=0.0, stream=None, check=True) -> dict:
    o = gpe_obs()
    rc = load().gpe_observables(state, float(g), float(s_blend), C.byref(o), stream_handle(stream))
    if rc != GPE_OK and (check or rc != GPE_ERR_NONFINITE):
        raise GpeError(rc, last_error())
    return o.asdict()


def gpe_step_real_traced(state, params, nsteps, every, t0=0.0, stream=None, check=True) -> list:
    """gpe_step_real with the observables every `every` steps: a list of
    dicts (the trace up to a non-finite point when check is False)."""
    n_max = max(1, -(-int(nsteps) // int(every))) if every > 0 else 1
    log = (gpe_obs * n_max)()
    n = C.c_int64()
    rc = load().gpe_step_real_traced(state, C.byref(params), int(nsteps), float(t0), int(every), log,
                                     C.byref(n), stream_handle(stream))
    if rc != GPE_OK and (check or rc != GPE_ERR_NONFINITE):
        raise GpeError(rc, last_error())
    return [log[i].asdict() for i in range(n.value)]


def gpe_overlap(a, b, stream=None) -> complex:
    out = (C.c_double * 2)()
    _check(load().gpe_overlap(a, b, out, stream_handle(stream)))
    return complex(out[0], out[1])


def gpe_wait_selftest(limit_s):
    """Returns (timed_out, waited seconds)."""
    t = C.c_int()
    w = C.c_double()
    _check(load().gpe_wait_selftest(float(limit_s), C.byref(t), C.byref(w)))
    return bool(t.value), w.value


def gpe_state_set_graph(state, steps_per_graph):
    _check(load().gpe_state_set_graph(state, int(steps_per_graph)))


def gpe_batch_create(states):
    arr = (_P * len(states))(*states)
    out = _P()
    _check(load().gpe_batch_create(arr, len(states), C.byref(out)))
    return out.value


def gpe_batch_ground_state(batch, per_shell, tol_dmu, check_every, max_steps, stream=None, check=True):
    """Returns (rc, converged[n], steps[n], obs list of dicts)."""
    n = len(per_shell)
    params = (gpe_imag_params * n)(*per_shell)
    conv = (C.c_int32 * n)()
    steps = (C.c_int64 * n)()
    obs = (gpe_obs * n)()
    rc = load().gpe_batch_ground_state(batch, params, float(tol_dmu), int(check_every), int(max_steps), conv, steps,
                                       obs, stream_handle(stream))
    if check and rc != GPE_OK:
        raise GpeError(rc, last_error())
    return rc, list(conv), list(steps), [o.asdict() for o in obs]


def gpe_batch_destroy(batch):
    _check(load().gpe_batch_destroy(batch))


def gpe_autotune(box, pot, V_cut, dtype, mode, nsteps, timings=True, stream=None):
    best = gpe_tune_result()
    allr = (gpe_tune_result * 8)()
    n = C.c_int()
    _check(load().gpe_autotune(C.byref(box), C.byref(pot), float(V_cut), int(dtype), int(mode), int(nsteps),
                               C.byref(best), allr if timings else None, C.byref(n), stream_handle(stream)))
    return best.asdict(), [allr[i].asdict() for i in range(n.value)]


def gpe_batch_autotune(boxes, pots, V_cuts, dtype, nsteps, stream=None):
    """Brick shape for a batch of shells: (best, every timing) as dicts."""
    n = len(boxes)
    if not (len(pots) == len(V_cuts) == n):
        raise ValueError("boxes, pots and V_cuts must have the same length")
    bx = (gpe_box * n)(*boxes)
    px = (gpe_potential * n)(*pots)
    vc = (C.c_double * n)(*[float(v) for v in V_cuts])
    best = gpe_tune_result()
    allr = (gpe_tune_result * 3)()
    m = C.c_int()
    _check(load().gpe_batch_autotune(bx, px, vc, n, int(dtype), int(nsteps), C.byref(best), allr, C.byref(m),
                                     stream_handle(stream)))
    return best.asdict(), [allr[i].asdict() for i in range(m.value)]


def gpe_ramp_forward(state, params: gpe_real_params, nsteps, t0=0.0, K=64, stream=None):
    out = _P()
    _check(load().gpe_ramp_forward(state, C.byref(params), int(nsteps), float(t0), int(K), C.byref(out),
                                   stream_handle(stream)))
    return out.value


def gpe_ramp_backward(tape, target, n_knots, stream=None):
    """Returns (loss, gradient list of n_knots floats)."""
    grad = (C.c_double * GPE_MAX_KNOTS)()
    loss = C.c_double()
    _check(load().gpe_ramp_backward(tape, target, grad, C.byref(loss), stream_handle(stream)))
    return loss.value, list(grad)[:n_knots]


def gpe_tape_destroy(tape):
    _check(load().gpe_tape_destroy(tape))


def stage_params(g, N, dt, cut_factor=5.0, t_hold=0.0, integrator=GPE_RK4) -> gpe_stage_params:
    p = gpe_stage_params()
    p.g, p.N, p.dt, p.cut_factor, p.t_hold = float(g), float(N), float(dt), float(cut_factor), float(t_hold)
    p.integrator = integrator
    return p


def gpe_ramp_stages(psi0, pots, durations, params, opts=None, stream=None):
    """Multi-stage ramp (Sec. V) through ``pots`` (each a gpe_potential or a
    dense float64/float32 array, all of one kind); returns (grid, state,
    reports).  The caller destroys the state, then the grid."""
    n = len(pots)
    if len(durations) != max(n - 1, 0):
        raise ValueError(f"{n} potentials need {max(n - 1, 0)} stage durations, got {len(durations)}")
    arr = (gpe_ramp_pot * n)()
    keep = []
    for i, P in enumerate(pots):
        if isinstance(P, gpe_potential):
            keep.append(P)
            arr[i].analytic = C.pointer(P)
        else:
            ptr, dev = pointer(P)
            arr[i].V, arr[i].V_dtype, arr[i].V_on_device = ptr, real_dtype_code(P), dev
    dur = (C.c_double * max(n - 1, 1))(*[float(d) for d in durations])
    reports = (gpe_stage_report * (n + 1))()
    grid, state = _P(), _P()
    _check(load().gpe_ramp_stages(psi0, arr, n, dur, C.byref(params), C.byref(opts) if opts else None,
                                  C.byref(grid), C.byref(state), reports, stream_handle(stream)))
    n_rep = n - 1 + (1 if params.t_hold > 0 else 0)
    return grid.value, state.value, [reports[i].asdict() for i in range(n_rep)]


def gpe_overlap_noalloc(a, b, n, dtype, dV, stream=None) -> complex:
    """Overlap of two device arrays (pointers or CUDA tensors) without any
    device allocation (see include/gpe.h for the limit and sharing rules)."""
    pa, _ = pointer(a)
    pb, _ = pointer(b)
    out = (C.c_double * 2)()
    _check(load().gpe_overlap_noalloc(pa, pb, int(n), int(dtype), float(dV), out, stream_handle(stream)))
    return complex(out[0], out[1])


def gpe_ground_state(state, params: gpe_imag_params, tol_dmu, check_every, max_steps, stream=None):
    steps = C.c_int64()
    o = gpe_obs()
    _check(load().gpe_ground_state(state, C.byref(params), float(tol_dmu), int(check_every), int(max_steps),
                                   C.byref(steps), C.byref(o), stream_handle(stream)))
    return steps.value, o.asdict()
