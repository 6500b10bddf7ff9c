"""Python binding of libfd (include/fd.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: all propagation work runs in the CUDA kernels of
libfd.so.  Importing this module fails loudly if the library has not been
built; there is no CPU fallback.

Host arrays are numpy arrays (copied by the library); device arrays are torch
CUDA tensors, passed by pointer to the ``*_dev`` entry points (never owned).
Streams are ``torch.cuda.Stream`` objects or raw ``cudaStream_t`` integers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FD_LIBRARY selects another build of the same library (e.g. a tuning variant).
LIB_PATH = os.environ.get("FD_LIBRARY") or os.path.join(_HERE, "libfd.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libfd.so is not built ({LIB_PATH}); run `python -m paper_2311_05038_b300.build`")

_lib = ctypes.CDLL(LIB_PATH)

FD_OK, FD_EINVAL, FD_ECFL, FD_ERANGE, FD_ENOMEM, FD_EBUDGET, FD_ECUDA, FD_ETIMEOUT, FD_ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
STATUS_NAMES = {0: "FD_OK", -1: "FD_EINVAL", -2: "FD_ECFL", -3: "FD_ERANGE", -4: "FD_ENOMEM",
                -5: "FD_EBUDGET", -6: "FD_ECUDA", -7: "FD_ETIMEOUT", -8: "FD_ESTATE"}

# Every entry point declared in include/fd.h.
EXPORTS = [
    "fd_cfl_limit", "fd_stencil_weights", "fd_model_create", "fd_model_create_dev", "fd_model_destroy",
    "fd_set_velocity", "fd_set_velocity_dev", "fd_set_source", "fd_set_receivers", "fd_set_trace_buffer",
    "fd_reset", "fd_set_wavefield", "fd_step", "fd_run_shot", "fd_gather_traces", "fd_get_wavefield",
    "fd_synchronize", "fd_get_step", "fd_get_source_index", "fd_get_receiver_indices",
    "fd_get_damping_profile", "fd_kernel_launch_count", "fd_last_error",
    "fd_batch_create", "fd_batch_destroy", "fd_batch_set_tuning", "fd_batch_get_tuning", "fd_batch_step",
    "fd_batch_autotune", "fd_batch_step_noalloc", "fd_routine", "fd_step_unfused",
    "fd_get_wavefield_dev", "fd_set_wavefield_dev", "fd_inject_receivers", "fd_imaging",
    "fd_set_sponge_vmax", "fd_batch_set_fault", "fd_step_lp", "fd_imaging_product",
    "fd_adjoint_segment", "fd_gather_traces_async", "fd_debug_poison_padding", "fd_step_image",
    "fd_inject_receivers_image", "fd_step_lp_n", "fd_adjoint_backward", "fd_debug_stall_stage",
    "fd_set_stream", "fd_stream_create", "fd_stream_destroy", "fd_velocity_from_slowness",
    "fd_gradient_from_image", "fd_set_time_fusion",
]


class FDError(RuntimeError):
    """A libfd call returned a negative fd_status."""

    def __init__(self, status: int, func: str, msg: str):
        self.status = status
        super().__init__(f"{func}: {STATUS_NAMES.get(status, status)}: {msg}")


class fd_grid_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("dt", ctypes.c_double), ("sponge_width", ctypes.c_int),
                ("sponge_R", ctypes.c_double)]


class fd_batch_tuning(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int), ("steps_per_launch", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("group_mb", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp = ctypes.c_void_p
_i = ctypes.c_int
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)
_sz = ctypes.c_size_t

_SIGS = {
    "fd_cfl_limit": (ctypes.c_double, [_i]),
    "fd_stencil_weights": (_i, [_fp]),
    "fd_model_create": (_i, [ctypes.POINTER(fd_grid_desc), _vp, _vp, ctypes.POINTER(_vp)]),
    "fd_model_create_dev": (_i, [ctypes.POINTER(fd_grid_desc), _vp, _vp, ctypes.POINTER(_vp)]),
    "fd_model_destroy": (_i, [_vp]),
    "fd_set_velocity": (_i, [_vp, _vp]),
    "fd_set_velocity_dev": (_i, [_vp, _vp]),
    "fd_set_source": (_i, [_vp, _i, _i, _i, _vp, _i]),
    "fd_set_receivers": (_i, [_vp, _vp, _i]),
    "fd_set_trace_buffer": (_i, [_vp, _vp, _i]),
    "fd_reset": (_i, [_vp]),
    "fd_set_wavefield": (_i, [_vp, _vp, _vp, _i]),
    "fd_step": (_i, [_vp, _i]),
    "fd_run_shot": (_i, [_vp, _i, _vp]),
    "fd_gather_traces": (_i, [_vp, _vp, _sz]),
    "fd_gather_traces_async": (_i, [_vp, _vp, _sz]),
    "fd_debug_poison_padding": (_i, [_vp]),
    "fd_debug_stall_stage": (_i, [_vp, _i]),
    "fd_step_image": (_i, [_vp, _vp, _vp]),
    "fd_inject_receivers_image": (_i, [_vp, _vp, _vp, _vp]),
    "fd_step_lp_n": (_i, [_vp, _i, _vp]),
    "fd_adjoint_backward": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "fd_get_wavefield": (_i, [_vp, _vp, _vp, _sz]),
    "fd_synchronize": (_i, [_vp]),
    "fd_get_step": (_i, [_vp, _ip]),
    "fd_get_source_index": (_i, [_vp, _i64p]),
    "fd_get_receiver_indices": (_i, [_vp, _vp, _i]),
    "fd_get_damping_profile": (_i, [_vp, _i, _vp, _i]),
    "fd_kernel_launch_count": (ctypes.c_uint64, []),
    "fd_batch_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp)]),
    "fd_batch_destroy": (_i, [_vp]),
    "fd_batch_set_tuning": (_i, [_vp, ctypes.POINTER(fd_batch_tuning)]),
    "fd_batch_get_tuning": (_i, [_vp, ctypes.POINTER(fd_batch_tuning)]),
    "fd_batch_step": (_i, [_vp, _i, _ip]),
    "fd_batch_autotune": (_i, [_vp, _i, ctypes.POINTER(fd_batch_tuning)]),
    "fd_batch_step_noalloc": (_i, [ctypes.POINTER(_vp), _i, _i]),
    "fd_routine": (_i, [_vp, _i]),
    "fd_get_wavefield_dev": (_i, [_vp, _vp, _vp]),
    "fd_set_wavefield_dev": (_i, [_vp, _vp, _vp, _i]),
    "fd_inject_receivers": (_i, [_vp, _vp]),
    "fd_imaging": (_i, [_vp, _vp, _vp]),
    "fd_step_lp": (_i, [_vp, _vp]),
    "fd_imaging_product": (_i, [_vp, _vp, _vp]),
    "fd_adjoint_segment": (_i, [_vp, _vp, _i, _i, _vp, _vp, _vp]),
    "fd_set_sponge_vmax": (_i, [_vp, ctypes.c_double]),
    "fd_batch_set_fault": (_i, [_vp, _i]),
    "fd_step_unfused": (_i, [_vp, _i]),
    "fd_set_stream": (_i, [_vp, _vp]),
    "fd_stream_create": (_i, [_i, ctypes.POINTER(_vp), _ip]),
    "fd_stream_destroy": (_i, [_vp]),
    "fd_velocity_from_slowness": (_i, [_vp, _vp, _sz, _vp]),
    "fd_gradient_from_image": (_i, [_vp, _i, _vp, _vp, _sz, _vp]),
    "fd_set_time_fusion": (_i, [_vp, _i]),
    "fd_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _check(status: int, func: str):
    if status != FD_OK:
        raise FDError(status, func, _lib.fd_last_error().decode())


def _host_f32(a, n=None):
    arr = np.ascontiguousarray(a, dtype=np.float32)
    if n is not None and arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    return arr


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _dev_ptr(t) -> int:
    if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
        raise ValueError("device arrays must be contiguous torch CUDA tensors")
    return int(t.data_ptr())


# ------------------------------------------------------------------ entry points

def fd_cfl_limit(ndim: int) -> float:
    return float(_lib.fd_cfl_limit(int(ndim)))


def fd_stencil_weights() -> np.ndarray:
    out = np.zeros(4, np.float32)
    _check(_lib.fd_stencil_weights(out.ctypes.data_as(_fp)), "fd_stencil_weights")
    return out


def make_desc(ndim, nx, ny, nz, h, dt, sponge_width=0, sponge_R=1e-3) -> fd_grid_desc:
    return fd_grid_desc(int(ndim), int(nx), int(ny), int(nz), float(h), float(dt), int(sponge_width),
                        float(sponge_R))


def fd_model_create(desc: fd_grid_desc, v_host, stream=None) -> int:
    v = _host_f32(v_host, desc.nx * desc.ny * desc.nz)
    out = _vp()
    _check(_lib.fd_model_create(ctypes.byref(desc), v.ctypes.data, _stream_ptr(stream), ctypes.byref(out)),
           "fd_model_create")
    return out.value


def fd_model_create_dev(desc: fd_grid_desc, v_dev, stream=None) -> int:
    if v_dev.numel() != desc.nx * desc.ny * desc.nz:
        raise ValueError("velocity size does not match the grid")
    out = _vp()
    _check(_lib.fd_model_create_dev(ctypes.byref(desc), _dev_ptr(v_dev), _stream_ptr(stream),
                                    ctypes.byref(out)), "fd_model_create_dev")
    return out.value


def fd_model_destroy(m: int):
    _check(_lib.fd_model_destroy(m), "fd_model_destroy")


def fd_set_time_fusion(m: int, steps: int):
    _check(_lib.fd_set_time_fusion(m, int(steps)), "fd_set_time_fusion")


def fd_set_stream(m: int, stream):
    _check(_lib.fd_set_stream(m, _stream_ptr(stream)), "fd_set_stream")


def fd_stream_create(priority: int = 0):
    """(stream handle, device's greatest priority) of a new library-owned stream."""
    out = _vp()
    most = ctypes.c_int(0)
    _check(_lib.fd_stream_create(int(priority), ctypes.byref(out), ctypes.byref(most)), "fd_stream_create")
    return out.value, most.value


def fd_stream_destroy(stream: int):
    _check(_lib.fd_stream_destroy(stream), "fd_stream_destroy")


def fd_set_velocity(m: int, v_host, n=None):
    v = _host_f32(v_host, n)
    _check(_lib.fd_set_velocity(m, v.ctypes.data), "fd_set_velocity")


def fd_set_velocity_ptr(m: int, host_ptr: int):
    """fd_set_velocity from a raw host pointer (e.g. a pinned torch tensor)."""
    _check(_lib.fd_set_velocity(m, host_ptr), "fd_set_velocity")


def fd_set_velocity_dev(m: int, v_dev):
    _check(_lib.fd_set_velocity_dev(m, _dev_ptr(v_dev)), "fd_set_velocity_dev")


def fd_set_sponge_vmax(m: int, vmax: float):
    _check(_lib.fd_set_sponge_vmax(m, float(vmax)), "fd_set_sponge_vmax")


def fd_set_source(m: int, ix: int, iy: int, iz: int, wavelet=None):
    if wavelet is None:
        _check(_lib.fd_set_source(m, int(ix), int(iy), int(iz), None, 0), "fd_set_source")
        return
    w = _host_f32(wavelet)
    _check(_lib.fd_set_source(m, int(ix), int(iy), int(iz), w.ctypes.data, int(w.size)), "fd_set_source")


def fd_set_receivers(m: int, xyz):
    r = np.ascontiguousarray(np.asarray(xyz, dtype=np.int32).reshape(-1, 3))
    _check(_lib.fd_set_receivers(m, r.ctypes.data if len(r) else None, int(len(r))), "fd_set_receivers")


def fd_set_trace_buffer(m: int, traces_dev, nt_rows: int):
    ptr = None if traces_dev is None else _dev_ptr(traces_dev)
    _check(_lib.fd_set_trace_buffer(m, ptr, int(nt_rows)), "fd_set_trace_buffer")


def fd_reset(m: int):
    _check(_lib.fd_reset(m), "fd_reset")


def fd_set_wavefield(m: int, p_host, pold_host, n: int = 0):
    p = _host_f32(p_host)
    po = _host_f32(pold_host, p.size)
    _check(_lib.fd_set_wavefield(m, p.ctypes.data, po.ctypes.data, int(n)), "fd_set_wavefield")


def fd_step(m: int, nsteps: int):
    _check(_lib.fd_step(m, int(nsteps)), "fd_step")


def fd_run_shot(m: int, nt: int, traces_dev=None):
    ptr = None if traces_dev is None else _dev_ptr(traces_dev)
    _check(_lib.fd_run_shot(m, int(nt), ptr), "fd_run_shot")


def fd_gather_traces(m: int, out: np.ndarray):
    """Fill the float32 host array ``out`` ([rows, nrec]) with the recorded traces."""
    if out.dtype != np.float32 or not out.flags.c_contiguous:
        raise ValueError("out must be a contiguous float32 array")
    _check(_lib.fd_gather_traces(m, out.ctypes.data, out.size), "fd_gather_traces")
    return out


def fd_gather_traces_ptr(m: int, host_ptr: int, cap: int):
    """fd_gather_traces into a raw host pointer (e.g. a pinned torch tensor)."""
    _check(_lib.fd_gather_traces(m, host_ptr, int(cap)), "fd_gather_traces")


def fd_gather_traces_async_ptr(m: int, host_ptr: int, cap: int):
    """Enqueue the trace download into a raw (pinned) host pointer; no synchronisation."""
    _check(_lib.fd_gather_traces_async(m, host_ptr, int(cap)), "fd_gather_traces_async")


def fd_get_wavefield(m: int, shape, with_old: bool = False):
    n = int(np.prod(shape))
    p = np.empty(shape, np.float32)
    po = np.empty(shape, np.float32) if with_old else None
    _check(_lib.fd_get_wavefield(m, p.ctypes.data, None if po is None else po.ctypes.data, n),
           "fd_get_wavefield")
    return (p, po) if with_old else p


def fd_debug_stall_stage(m: int, stage: int):
    """Test hook: the first CTA of each 3D step launch never issues P stage `stage` (-1 clears)."""
    _check(_lib.fd_debug_stall_stage(m, int(stage)), "fd_debug_stall_stage")


def fd_debug_poison_padding(m: int):
    """Test hook: NaN into the row padding (columns nx .. px-1) of the device fields."""
    _check(_lib.fd_debug_poison_padding(m), "fd_debug_poison_padding")


def fd_synchronize(m: int):
    _check(_lib.fd_synchronize(m), "fd_synchronize")


def fd_get_step(m: int) -> int:
    n = ctypes.c_int()
    _check(_lib.fd_get_step(m, ctypes.byref(n)), "fd_get_step")
    return n.value


def fd_get_source_index(m: int) -> int:
    i = ctypes.c_int64()
    _check(_lib.fd_get_source_index(m, ctypes.byref(i)), "fd_get_source_index")
    return i.value


def fd_get_receiver_indices(m: int, nrec: int) -> np.ndarray:
    out = np.zeros(max(nrec, 1), np.int64)
    _check(_lib.fd_get_receiver_indices(m, out.ctypes.data, int(nrec)), "fd_get_receiver_indices")
    return out[:nrec]


def fd_get_damping_profile(m: int, axis: int, n: int) -> np.ndarray:
    out = np.zeros(n, np.float32)
    _check(_lib.fd_get_damping_profile(m, int(axis), out.ctypes.data, int(n)), "fd_get_damping_profile")
    return out


def fd_kernel_launch_count() -> int:
    return int(_lib.fd_kernel_launch_count())


def fd_last_error() -> str:
    return _lib.fd_last_error().decode()


def fd_batch_create(model_handles) -> int:
    arr = (_vp * len(model_handles))(*model_handles)
    out = _vp()
    _check(_lib.fd_batch_create(arr, len(model_handles), ctypes.byref(out)), "fd_batch_create")
    return out.value


def fd_batch_destroy(b: int):
    _check(_lib.fd_batch_destroy(b), "fd_batch_destroy")


def fd_batch_set_tuning(b: int, tile: int, steps_per_launch: int, ctas_per_sm: int = 0, group_mb: int = 0):
    t = fd_batch_tuning(int(tile), int(steps_per_launch), int(ctas_per_sm), int(group_mb))
    _check(_lib.fd_batch_set_tuning(b, ctypes.byref(t)), "fd_batch_set_tuning")


def fd_batch_get_tuning(b: int) -> dict:
    t = fd_batch_tuning()
    _check(_lib.fd_batch_get_tuning(b, ctypes.byref(t)), "fd_batch_get_tuning")
    return t.as_dict()


def fd_batch_step(b: int, nsteps: int, nsteps_each=None):
    arr = None
    if nsteps_each is not None:
        each = np.ascontiguousarray(nsteps_each, dtype=np.int32)
        arr = each.ctypes.data_as(_ip)
    _check(_lib.fd_batch_step(b, int(nsteps), arr), "fd_batch_step")


def fd_batch_set_fault(b: int, stalled_item: int):
    _check(_lib.fd_batch_set_fault(b, int(stalled_item)), "fd_batch_set_fault")


def fd_batch_autotune(b: int, trial_steps: int) -> dict:
    t = fd_batch_tuning()
    _check(_lib.fd_batch_autotune(b, int(trial_steps), ctypes.byref(t)), "fd_batch_autotune")
    return t.as_dict()


def fd_batch_step_noalloc(model_handles, nsteps: int):
    """Advance the given 2D models nsteps steps without allocating device memory."""
    arr = (_vp * len(model_handles))(*model_handles)
    _check(_lib.fd_batch_step_noalloc(arr, len(model_handles), int(nsteps)), "fd_batch_step_noalloc")


FD_ROUTINE_ADD_SOURCE, FD_ROUTINE_PZZ, FD_ROUTINE_PXX, FD_ROUTINE_PYY, FD_ROUTINE_TIME, FD_ROUTINE_SWAP = range(6)


def fd_routine(m: int, routine: int):
    _check(_lib.fd_routine(m, int(routine)), "fd_routine")


def fd_step_unfused(m: int, nsteps: int):
    _check(_lib.fd_step_unfused(m, int(nsteps)), "fd_step_unfused")


def fd_get_wavefield_dev(m: int, p_dev, pold_dev=None):
    _check(_lib.fd_get_wavefield_dev(m, _dev_ptr(p_dev), None if pold_dev is None else _dev_ptr(pold_dev)),
           "fd_get_wavefield_dev")


def fd_set_wavefield_dev(m: int, p_dev, pold_dev, n: int = 0):
    _check(_lib.fd_set_wavefield_dev(m, _dev_ptr(p_dev), _dev_ptr(pold_dev), int(n)), "fd_set_wavefield_dev")


def fd_inject_receivers(m: int, values_dev):
    _check(_lib.fd_inject_receivers(m, _dev_ptr(values_dev)), "fd_inject_receivers")


def fd_imaging(adj: int, p_dev, grad_dev):
    _check(_lib.fd_imaging(adj, _dev_ptr(p_dev), _dev_ptr(grad_dev)), "fd_imaging")


def fd_step_lp(m: int, lp_dev):
    """One step that also writes L'P of the consumed level to lp_dev (dense, grid-shaped)."""
    _check(_lib.fd_step_lp(m, _dev_ptr(lp_dev)), "fd_step_lp")


def fd_imaging_product(adj: int, lp_dev, grad_dev):
    """grad_dev += (adj's current level) * lp_dev, pointwise."""
    _check(_lib.fd_imaging_product(adj, _dev_ptr(lp_dev), _dev_ptr(grad_dev)), "fd_imaging_product")


def fd_step_image(m: int, lp_dev, grad_dev):
    """One step that also adds the new level times lp_dev to grad_dev (dense)."""
    _check(_lib.fd_step_image(m, _dev_ptr(lp_dev), _dev_ptr(grad_dev)), "fd_step_image")


def fd_inject_receivers_image(m: int, values_dev, lp_dev, grad_dev):
    """fd_inject_receivers, also adding each injected value times lp_dev to grad_dev."""
    _check(_lib.fd_inject_receivers_image(m, None if values_dev is None else _dev_ptr(values_dev),
                                          _dev_ptr(lp_dev), _dev_ptr(grad_dev)), "fd_inject_receivers_image")


def fd_velocity_from_slowness(m_dev, v_dev, stream=None):
    """v = m^(-1/2) elementwise (device tensors of equal size)."""
    if m_dev.numel() != v_dev.numel():
        raise ValueError("m and v differ in size")
    _check(_lib.fd_velocity_from_slowness(_dev_ptr(m_dev), _dev_ptr(v_dev), m_dev.numel(), _stream_ptr(stream)),
           "fd_velocity_from_slowness")


def fd_gradient_from_image(acc_dev, m_dev, grad_dev, stream=None):
    """grad = -(sum over the leading axis of acc) / m; acc shaped (k,) + m.shape or m.shape."""
    n = m_dev.numel()
    if acc_dev.numel() % n or grad_dev.numel() != n:
        raise ValueError("acc, m and grad sizes do not match")
    _check(_lib.fd_gradient_from_image(_dev_ptr(acc_dev), acc_dev.numel() // n, _dev_ptr(m_dev), _dev_ptr(grad_dev),
                                       n, _stream_ptr(stream)), "fd_gradient_from_image")


def fd_step_lp_n(m: int, nsteps: int, lp_buf):
    """nsteps steps, the j-th writing L'P of its consumed level to lp_buf[j]."""
    _check(_lib.fd_step_lp_n(m, int(nsteps), _dev_ptr(lp_buf)), "fd_step_lp_n")


def fd_adjoint_backward(adj: int, n0: int, n1: int, lp_buf, g_dev, grad_dev):
    """The adjoint back from n1 to n0 through stored L'P fields lp_buf[0 .. n1-n0-1]."""
    _check(_lib.fd_adjoint_backward(adj, int(n0), int(n1), _dev_ptr(lp_buf),
                                    None if g_dev is None else _dev_ptr(g_dev), _dev_ptr(grad_dev)),
           "fd_adjoint_backward")


def fd_adjoint_segment(fwd: int, adj: int, n0: int, n1: int, lp_buf, g_dev, grad_dev):
    """Recompute [n0, n1) with fd_step_lp into lp_buf, then run the adjoint back through it."""
    _check(_lib.fd_adjoint_segment(fwd, adj, int(n0), int(n1), _dev_ptr(lp_buf),
                                   None if g_dev is None else _dev_ptr(g_dev), _dev_ptr(grad_dev)),
           "fd_adjoint_segment")


# ------------------------------------------------------------------ convenience

class Model:
    """Owning handle of one fd_model (destroyed on close / garbage collection)."""

    def __init__(self, ndim, shape, h, dt, vel, sponge_width=0, sponge_R=1e-3, stream=None):
        if ndim == 2:
            nz, nx = shape
            ny = 1
        else:
            nz, ny, nx = shape
        self.shape = tuple(shape)
        self.desc = make_desc(ndim, nx, ny, nz, h, dt, sponge_width, sponge_R)
        self.nrec = 0
        self.handle = None
        if hasattr(vel, "is_cuda"):
            self.handle = fd_model_create_dev(self.desc, vel, stream)
        else:
            self.handle = fd_model_create(self.desc, vel, stream)

    @classmethod
    def from_shot(cls, shot, stream=None):
        m = cls(shot.ndim, shot.shape, shot.h, shot.dt, shot.vel, shot.sponge_width, shot.sponge_R, stream)
        m.set_source(shot.src, shot.wavelet)
        m.set_receivers(shot.receivers)
        return m

    def set_source(self, xyz, wavelet):
        fd_set_source(self.handle, xyz[0], xyz[1], xyz[2], wavelet)

    def set_receivers(self, xyz):
        r = np.asarray(xyz, dtype=np.int32).reshape(-1, 3)
        fd_set_receivers(self.handle, r)
        self.nrec = len(r)

    def run_shot(self, nt, traces_dev=None):
        fd_run_shot(self.handle, nt, traces_dev)

    def set_time_fusion(self, steps):
        fd_set_time_fusion(self.handle, steps)

    def step(self, n):
        fd_step(self.handle, n)

    def traces(self, rows):
        out = np.empty((rows, self.nrec), np.float32)
        return fd_gather_traces(self.handle, out)

    def wavefield(self, with_old=False):
        return fd_get_wavefield(self.handle, self.shape, with_old)

    def close(self):
        if self.handle:
            fd_model_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning handle of one fd_batch over existing Model objects (kept alive here)."""

    def __init__(self, models):
        self.models = list(models)
        self.handle = fd_batch_create([m.handle for m in self.models])

    def set_tuning(self, tile=0, steps_per_launch=2000, ctas_per_sm=0, group_mb=96):
        fd_batch_set_tuning(self.handle, tile, steps_per_launch, ctas_per_sm, group_mb)

    def tuning(self):
        return fd_batch_get_tuning(self.handle)

    def step(self, nsteps, nsteps_each=None):
        fd_batch_step(self.handle, nsteps, nsteps_each)

    def run_shots(self, nts):
        """Reset every shot, give shot i a library-owned trace buffer of nts[i] rows, run."""
        for m, nt in zip(self.models, nts):
            fd_reset(m.handle)
            fd_set_trace_buffer(m.handle, None, int(nt))
        fd_batch_step(self.handle, 0, np.asarray(nts, np.int32))

    def autotune(self, trial_steps=20):
        return fd_batch_autotune(self.handle, trial_steps)

    def close(self):
        if self.handle:
            fd_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
