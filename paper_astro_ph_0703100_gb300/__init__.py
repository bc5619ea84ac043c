"""Softened direct-summation gravity on GB300: Python binding of libcunbody.

Thin marshalling over the C ABI of ``include/cunbody.h``: every function
here has the name of the C entry point it calls, checks tensor dtypes,
shapes and devices, allocates outputs with PyTorch when none are given, and
passes raw pointers plus the current CUDA stream. All arithmetic runs in
the library's sm_103a kernels; there is no CPU or PyTorch fallback.

Particle records are float32 tensors of shape (n, 4) holding (x, y, z, m),
as in the appendix driver of the paper (JDIM = 4). ``eps2`` is the squared
softening length.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from ._lib import CunbodyError, STATUS, cn_tune, check, load

__all__ = [
    "CunbodyError",
    "STATUS",
    "VARIANT",
    "cn_force",
    "cn_force_ws",
    "cn_force_noalloc",
    "cn_force_eps_i",
    "cn_force_dd",
    "cn_force_dd_ws",
    "cn_workspace_bytes",
    "cn_force_symmetric",
    "BatchPlan",
    "cn_batch_plan_create",
    "cn_batch_plan_destroy",
    "cn_batch_plan_workspace_bytes",
    "cn_batch_plan_info",
    "cn_batch_plan_capture",
    "cn_batch_plan_launch",
    "cn_list_plan_create",
    "cn_list_plan_create_indexed",
    "cn_list_plan_capture",
    "cn_status_string",
    "cn_last_error_message",
    "cn_force_batched",
    "ListPlan",
    "cn_force_lists",
    "cn_force_adjoint",
    "cn_force_jerk",
    "cn_potential_energy",
    "cn_potential_energy_dd",
    "cn_force_host",
    "cn_force_host_f64",
    "cn_tune_get",
    "cn_tune_set",
    "cn_tune_save",
    "cn_tune_load",
    "cn_autotune",
    "cn_autotune_batched",
    "cn_get_device_status",
    "cn_set_wait_limit_ns",
    "cn_debug_timeout_probe",
    "cn_probe_peaks",
    "cn_version",
    "GravityForce",
    "gravity",
    "load",
]

VARIANT = {
    "f32": 0,
    "f32_pot": 1,
    "dd": 2,
    "dd_pot": 3,
    "adjoint": 4,
    "batched": 5,
    "batched_pot": 6,
    "jerk": 7,
    "jerk_pot": 8,
    "symmetric": 9,
    "f32_eps_i": 10,
    "f32_eps_i_pot": 11,
}


def _torch():
    import torch

    return torch


_current_stream = None  # () -> cudaStream_t of PyTorch's current stream on the current device
_current_device = None  # () -> index of the current CUDA device


def _stream_handle(stream):
    """The cudaStream_t of `stream`, as an int; None means PyTorch's current
    stream on the current device (read through torch's raw-stream query where
    it exists: torch.cuda.current_stream() builds a Stream object, ~3 us)."""
    global _current_stream
    if stream is not None:
        return int(stream.cuda_stream)
    if _current_stream is None:
        torch = _torch()
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        dev = getattr(torch._C, "_cuda_getDevice", None)
        if raw is not None and dev is not None:
            _current_stream = lambda: raw(dev())
        else:
            _current_stream = lambda: int(torch.cuda.current_stream().cuda_stream)
    return _current_stream()


def _ptr(t):
    return None if t is None else t.data_ptr()


def _device_index():
    """Index of the current CUDA device (the library launches there)."""
    global _current_device
    if _current_device is None:
        torch = _torch()
        dev = getattr(torch._C, "_cuda_getDevice", None)
        _current_device = dev if dev is not None else torch.cuda.current_device
    return _current_device()


def _on_current_device(t, name):
    if t.get_device() != _device_index():
        raise TypeError(f"{name} is on cuda:{t.get_device()}, but the current device is cuda:{_device_index()} "
                        "(the library launches on the current device; use torch.cuda.device(...))")


def _like(t, ref, name):
    """A further CUDA tensor of a call: contiguous and on the device of `ref`."""
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and t.device == ref.device):
        raise TypeError(f"{name} must be a contiguous CUDA tensor on {ref.device}")
    return t


def _records(t, name):
    torch = _torch()
    if not (isinstance(t, torch.Tensor) and t.dtype == torch.float32 and t.dim() == 2 and t.shape[1] == 4):
        raise TypeError(f"{name} must be a float32 tensor of shape (n, 4)")
    if not (t.is_cuda and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    _on_current_device(t, name)
    return t


def _out(t, shape, dtype, device, name):
    torch = _torch()
    if t is None:
        return torch.empty(shape, dtype=dtype, device=device)
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous() or t.device != device:
        raise TypeError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)} on {device}")
    return t


def _variant(name):
    return VARIANT[name] if isinstance(name, str) else int(name)


# ------------------------------------------------------------------ force

def _force(fn, double, pos_i, pos_mass_j, eps2, acc_out, pot_out, potential, stream, ws=None):
    torch = _torch()
    _records(pos_i, "pos_i")
    _records(pos_mass_j, "pos_mass_j")
    n_i, n_j = pos_i.shape[0], pos_mass_j.shape[0]
    dt = torch.float64 if double else torch.float32
    acc = _out(acc_out, (n_i, 3), dt, pos_i.device, "acc_out")
    pot = None
    if potential or pot_out is not None:
        pot = _out(pot_out, (n_i,), dt, pos_i.device, "pot_out")
    lib = load()
    if ws is None:
        st = getattr(lib, fn)(n_i, _ptr(pos_i), n_j, _ptr(pos_mass_j), float(eps2), _ptr(acc), _ptr(pot),
                              _stream_handle(stream))
    else:
        _like(ws, pos_i, "workspace")
        st = getattr(lib, fn)(n_i, _ptr(pos_i), n_j, _ptr(pos_mass_j), float(eps2), _ptr(acc), _ptr(pot),
                              _ptr(ws), ws.numel() * ws.element_size(), _stream_handle(stream))
    check(st, fn)
    return acc, pot


def cn_force(pos_i, pos_mass_j, eps2, acc_out=None, pot_out=None, potential=False, stream=None):
    """FP32 accelerations (n_i, 3) and, if requested, potentials (n_i,)."""
    return _force("cn_force", False, pos_i, pos_mass_j, eps2, acc_out, pot_out, potential, stream)


def cn_force_eps_i(pos_eps_i, pos_mass_j, acc_out=None, pot_out=None, potential=False, stream=None):
    """FP32 accelerations (and potentials) with each i-particle's softening
    eps2_i taken from the 4th slot of its record (x, y, z, eps2_i)."""
    torch = _torch()
    _records(pos_eps_i, "pos_eps_i")
    _records(pos_mass_j, "pos_mass_j")
    n_i, n_j = pos_eps_i.shape[0], pos_mass_j.shape[0]
    acc = _out(acc_out, (n_i, 3), torch.float32, pos_eps_i.device, "acc_out")
    pot = None
    if potential or pot_out is not None:
        pot = _out(pot_out, (n_i,), torch.float32, pos_eps_i.device, "pot_out")
    check(load().cn_force_eps_i(n_i, _ptr(pos_eps_i), n_j, _ptr(pos_mass_j), _ptr(acc), _ptr(pot),
                                _stream_handle(stream)), "cn_force_eps_i")
    return acc, pot


def cn_force_noalloc(pos_i, pos_mass_j, eps2, acc_out=None, pot_out=None, potential=False, stream=None):
    """cn_force with the library's fixed static device scratch: the library
    allocates no device memory in the call (outputs not given are PyTorch
    tensors); calls that overlap in time share the scratch and must not."""
    return _force("cn_force_noalloc", False, pos_i, pos_mass_j, eps2, acc_out, pot_out, potential, stream)


def cn_force_ws(pos_i, pos_mass_j, eps2, workspace, acc_out=None, pot_out=None, potential=False, stream=None):
    """cn_force with a caller-owned workspace tensor (uint8 CUDA, no initialisation needed)."""
    return _force("cn_force_ws", False, pos_i, pos_mass_j, eps2, acc_out, pot_out, potential, stream, workspace)


def cn_force_dd(pos_i, pos_mass_j, eps2, acc_out=None, pot_out=None, potential=False, stream=None):
    """Compensated form (FP32 pair term with its roundings recovered, (hi, lo)
    sums folded into FP64); FP64 outputs."""
    return _force("cn_force_dd", True, pos_i, pos_mass_j, eps2, acc_out, pot_out, potential, stream)


def cn_force_dd_ws(pos_i, pos_mass_j, eps2, workspace, acc_out=None, pot_out=None, potential=False, stream=None):
    return _force("cn_force_dd_ws", True, pos_i, pos_mass_j, eps2, acc_out, pot_out, potential, stream, workspace)


def cn_force_symmetric(pos_mass, eps2, acc_out=None, pot_out=None, potential=False, stream=None):
    """Accelerations (n, 3) and, if requested, potentials (n,) of all
    particles, each unordered pair evaluated once."""
    torch = _torch()
    _records(pos_mass, "pos_mass")
    n = pos_mass.shape[0]
    acc = _out(acc_out, (n, 3), torch.float32, pos_mass.device, "acc_out")
    pot = None
    if potential or pot_out is not None:
        pot = _out(pot_out, (n,), torch.float32, pos_mass.device, "pot_out")
    check(load().cn_force_symmetric(n, _ptr(pos_mass), float(eps2), _ptr(acc), _ptr(pot), _stream_handle(stream)),
          "cn_force_symmetric")
    return acc, pot


def cn_workspace_bytes(variant, n_i, n_j) -> int:
    return int(load().cn_workspace_bytes(_variant(variant), int(n_i), int(n_j)))


# ------------------------------------------------------------------ batched

class BatchPlan:
    """An ensemble of independent clusters (records offsets[c] .. offsets[c+1]-1, softening eps2[c])."""

    def __init__(self, offsets, eps2, tune=None, potential=False):
        self.offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.eps2 = np.ascontiguousarray(np.asarray(eps2, dtype=np.float32))
        n_clusters = self.offsets.shape[0] - 1
        if n_clusters < 0 or self.eps2.shape[0] != n_clusters:
            raise ValueError("offsets must have n_clusters + 1 entries and eps2 n_clusters")
        handle = ctypes.c_void_p()
        t = ctypes.byref(_tune_struct(tune)) if tune is not None else None
        lib = load()
        check(lib.cn_batch_plan_create(n_clusters, self.offsets.ctypes.data_as(ctypes.c_void_p),
                                       self.eps2.ctypes.data_as(ctypes.c_void_p), t, int(bool(potential)),
                                       ctypes.byref(handle)), "cn_batch_plan_create")
        self._h = handle
        self.potential = bool(potential)
        self.n_clusters = n_clusters
        n_total = ctypes.c_int64()
        pairs = ctypes.c_double()
        check(lib.cn_batch_plan_info(self._h, ctypes.byref(n_total), ctypes.byref(pairs)), "cn_batch_plan_info")
        self.n_total = int(n_total.value)
        self.pairs = float(pairs.value)
        self._keep = None

    @property
    def workspace_bytes(self) -> int:
        return int(load().cn_batch_plan_workspace_bytes(self._h))

    def new_workspace(self, device="cuda"):
        torch = _torch()
        return torch.zeros(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)

    def _args(self, pos_mass, acc_out, pot_out):
        torch = _torch()
        _records(pos_mass, "pos_mass")
        if pos_mass.shape[0] != self.n_total:
            raise ValueError("pos_mass length does not match the plan")
        acc = _out(acc_out, (self.n_total, 3), torch.float32, pos_mass.device, "acc_out")
        pot = None
        if self.potential or pot_out is not None:
            pot = _out(pot_out, (self.n_total,), torch.float32, pos_mass.device, "pot_out")
        return acc, pot

    def run(self, pos_mass, acc_out=None, pot_out=None, workspace=None, stream=None):
        return cn_force_batched(self, pos_mass, acc_out, pot_out, workspace, stream)

    def capture(self, pos_mass, acc_out, pot_out=None, workspace=None, stream=None):
        """Capture one batched launch into a CUDA graph held by the plan."""
        acc, pot = self._args(pos_mass, acc_out, pot_out)
        if workspace is None:
            workspace = self.new_workspace(pos_mass.device)
        _like(workspace, pos_mass, "workspace")
        self._keep = (pos_mass, acc, pot, workspace)
        check(load().cn_batch_plan_capture(self._h, _ptr(pos_mass), _ptr(acc), _ptr(pot), _ptr(workspace),
                                           workspace.numel() * workspace.element_size(), _stream_handle(stream)),
              "cn_batch_plan_capture")
        return acc, pot

    def launch(self, stream=None):
        check(load().cn_batch_plan_launch(self._h, _stream_handle(stream)), "cn_batch_plan_launch")

    def close(self):
        if getattr(self, "_h", None):
            load().cn_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cn_force_batched(plan: BatchPlan, pos_mass, acc_out=None, pot_out=None, workspace=None, stream=None):
    acc, pot = plan._args(pos_mass, acc_out, pot_out)
    nbytes = 0 if workspace is None else _like(workspace, pos_mass, "workspace").numel() * workspace.element_size()
    check(load().cn_force_batched(plan._h, _ptr(pos_mass), _ptr(acc), _ptr(pot), _ptr(workspace), nbytes,
                                  _stream_handle(stream)), "cn_force_batched")
    return acc, pot


class ListPlan:
    """Groups of i-particles, each against its own list of j records (Section 4.4).

    Group g: i-particles ``i_offsets[g]:i_offsets[g+1]`` of ``pos_i`` against
    records ``j_begin[g]:j_begin[g]+j_count[g]`` of ``pos_mass_j``, softening
    ``eps2[g]`` (a scalar applies to every group).

    With ``j_index`` (int32 list entries, each the index of a source record)
    the lists are index arrays: group g's records are
    ``pos_mass_j[j_index[e]]`` for the entries
    ``e = j_begin[g] .. j_begin[g]+j_count[g]-1``, gathered by the kernel;
    ``pos_mass_j`` is then the source array of ``n_src`` records (by default
    one past the largest index).
    """

    def __init__(self, i_offsets, j_begin, j_count, eps2, tune=None, potential=False, j_index=None, n_src=None):
        self.i_offsets = np.ascontiguousarray(np.asarray(i_offsets, dtype=np.int64))
        n_groups = self.i_offsets.shape[0] - 1
        self.j_begin = np.ascontiguousarray(np.asarray(j_begin, dtype=np.int64))
        self.j_count = np.ascontiguousarray(np.asarray(j_count, dtype=np.int64))
        e = np.asarray(eps2, dtype=np.float32)
        self.eps2 = np.ascontiguousarray(np.full(n_groups, e, dtype=np.float32) if e.ndim == 0 else e)
        if n_groups < 0 or self.j_begin.shape[0] != n_groups or self.j_count.shape[0] != n_groups or \
                self.eps2.shape[0] != n_groups:
            raise ValueError("i_offsets needs n_groups + 1 entries; j_begin, j_count and eps2 n_groups")
        handle = ctypes.c_void_p()
        t = ctypes.byref(_tune_struct(tune)) if tune is not None else None
        lib = load()
        vpd = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        self.j_index = None
        if j_index is None:
            check(lib.cn_list_plan_create(n_groups, vpd(self.i_offsets), vpd(self.j_begin), vpd(self.j_count),
                                          vpd(self.eps2), t, int(bool(potential)), ctypes.byref(handle)),
                  "cn_list_plan_create")
        else:
            idx = np.asarray(j_index)
            if idx.ndim != 1 or not np.issubdtype(idx.dtype, np.integer):
                raise ValueError("j_index must be a 1-d integer array")
            if idx.size and (idx.min() < np.iinfo(np.int32).min or idx.max() > np.iinfo(np.int32).max):
                raise ValueError("j_index entries must fit in 32 bits")
            self.j_index = np.ascontiguousarray(idx, dtype=np.int32)
            if n_src is None:
                n_src = int(self.j_index.max()) + 1 if self.j_index.size else 0
            check(lib.cn_list_plan_create_indexed(n_groups, vpd(self.i_offsets), vpd(self.j_begin),
                                                  vpd(self.j_count), vpd(self.eps2),
                                                  vpd(self.j_index) if self.j_index.size else None,
                                                  self.j_index.size, int(n_src), t, int(bool(potential)),
                                                  ctypes.byref(handle)),
                  "cn_list_plan_create_indexed")
        self._h = handle
        self.potential = bool(potential)
        self.n_groups = n_groups
        n_total = ctypes.c_int64()
        pairs = ctypes.c_double()
        check(lib.cn_batch_plan_info(self._h, ctypes.byref(n_total), ctypes.byref(pairs)), "cn_batch_plan_info")
        self.n_i = int(n_total.value)
        if self.j_index is not None:
            self.n_j = int(n_src)
        else:
            self.n_j = int(max((self.j_begin + self.j_count)[self.j_count > 0].max(initial=0), 0)) if n_groups else 0
        self.pairs = float(pairs.value)
        self._keep = None

    @property
    def workspace_bytes(self) -> int:
        return int(load().cn_batch_plan_workspace_bytes(self._h))

    def new_workspace(self, device="cuda"):
        torch = _torch()
        return torch.zeros(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)

    def _args(self, pos_i, pos_mass_j, acc_out, pot_out):
        torch = _torch()
        _records(pos_i, "pos_i")
        _records(pos_mass_j, "pos_mass_j")
        if pos_i.shape[0] != self.n_i or pos_mass_j.shape[0] < self.n_j:
            raise ValueError("pos_i must hold n_i records and pos_mass_j every listed record")
        acc = _out(acc_out, (self.n_i, 3), torch.float32, pos_i.device, "acc_out")
        pot = None
        if self.potential or pot_out is not None:
            pot = _out(pot_out, (self.n_i,), torch.float32, pos_i.device, "pot_out")
        return acc, pot

    def run(self, pos_i, pos_mass_j, acc_out=None, pot_out=None, workspace=None, stream=None):
        return cn_force_lists(self, pos_i, pos_mass_j, acc_out, pot_out, workspace, stream)

    def capture(self, pos_i, pos_mass_j, acc_out, pot_out=None, workspace=None, stream=None):
        acc, pot = self._args(pos_i, pos_mass_j, acc_out, pot_out)
        if workspace is None:
            workspace = self.new_workspace(pos_i.device)
        _like(workspace, pos_i, "workspace")
        self._keep = (pos_i, pos_mass_j, acc, pot, workspace)
        check(load().cn_list_plan_capture(self._h, _ptr(pos_i), _ptr(pos_mass_j), _ptr(acc), _ptr(pot),
                                          _ptr(workspace), workspace.numel() * workspace.element_size(),
                                          _stream_handle(stream)),
              "cn_list_plan_capture")
        return acc, pot

    def launch(self, stream=None):
        check(load().cn_batch_plan_launch(self._h, _stream_handle(stream)), "cn_batch_plan_launch")

    def close(self):
        if getattr(self, "_h", None):
            load().cn_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cn_force_lists(plan: ListPlan, pos_i, pos_mass_j, acc_out=None, pot_out=None, workspace=None, stream=None):
    acc, pot = plan._args(pos_i, pos_mass_j, acc_out, pot_out)
    nbytes = 0 if workspace is None else _like(workspace, pos_i, "workspace").numel() * workspace.element_size()
    check(load().cn_force_lists(plan._h, _ptr(pos_i), _ptr(pos_mass_j), _ptr(acc), _ptr(pot), _ptr(workspace),
                                nbytes, _stream_handle(stream)), "cn_force_lists")
    return acc, pot


# ------------------------------------------------------------------ adjoint, energy

# Functions with the names of the plan entry points of the C ABI (the plan
# objects above hold the handle and call them).
def cn_batch_plan_create(offsets, eps2, tune=None, potential=False) -> BatchPlan:
    return BatchPlan(offsets, eps2, tune=tune, potential=potential)


def cn_list_plan_create(i_offsets, j_begin, j_count, eps2, tune=None, potential=False) -> ListPlan:
    return ListPlan(i_offsets, j_begin, j_count, eps2, tune=tune, potential=potential)


def cn_list_plan_create_indexed(i_offsets, j_begin, j_count, eps2, j_index, n_src=None, tune=None,
                                potential=False) -> ListPlan:
    return ListPlan(i_offsets, j_begin, j_count, eps2, tune=tune, potential=potential, j_index=j_index, n_src=n_src)


def cn_batch_plan_destroy(plan) -> None:
    plan.close()


def cn_batch_plan_workspace_bytes(plan) -> int:
    return plan.workspace_bytes


def cn_batch_plan_info(plan):
    """(i-particles, pair count) of a cluster or list plan."""
    return (plan.n_total if isinstance(plan, BatchPlan) else plan.n_i), plan.pairs


def cn_batch_plan_capture(plan: BatchPlan, pos_mass, acc_out, pot_out=None, workspace=None, stream=None):
    return plan.capture(pos_mass, acc_out, pot_out=pot_out, workspace=workspace, stream=stream)


def cn_list_plan_capture(plan: ListPlan, pos_i, pos_mass_j, acc_out, pot_out=None, workspace=None, stream=None):
    return plan.capture(pos_i, pos_mass_j, acc_out, pot_out=pot_out, workspace=workspace, stream=stream)


def cn_batch_plan_launch(plan, stream=None) -> None:
    plan.launch(stream)


def cn_status_string(status: int) -> str:
    return load().cn_status_string(int(status)).decode()


def cn_last_error_message() -> str:
    return load().cn_last_error_message().decode()


def cn_force_adjoint(pos_mass, eps2, w, grad_pos=None, grad_mass=None, stream=None):
    """dL/dx (n, 3) and dL/dm (n,) for L = sum_i w_i . a_i with i set = j set."""
    torch = _torch()
    _records(pos_mass, "pos_mass")
    n = pos_mass.shape[0]
    if w.dtype != torch.float32 or tuple(w.shape) != (n, 3):
        raise TypeError("w must be a float32 tensor of shape (n, 3)")
    _like(w, pos_mass, "w")
    gp = _out(grad_pos, (n, 3), torch.float32, pos_mass.device, "grad_pos")
    gm = _out(grad_mass, (n,), torch.float32, pos_mass.device, "grad_mass")
    check(load().cn_force_adjoint(n, _ptr(pos_mass), float(eps2), _ptr(w), _ptr(gp), _ptr(gm),
                                  _stream_handle(stream)), "cn_force_adjoint")
    return gp, gm


def cn_force_jerk(pos_i, vel_i, pos_mass_j, vel_j, eps2, acc_out=None, jerk_out=None, pot_out=None,
                  potential=False, stream=None):
    """Acceleration, jerk (d a / dt) and optionally potential: the outputs of
    the appendix's force-jerk-potential pipeline. Velocities are (n, 4) float32."""
    torch = _torch()
    for t, name in ((pos_i, "pos_i"), (vel_i, "vel_i"), (pos_mass_j, "pos_mass_j"), (vel_j, "vel_j")):
        _records(t, name)
    n_i, n_j = pos_i.shape[0], pos_mass_j.shape[0]
    if vel_i.shape[0] != n_i or vel_j.shape[0] != n_j:
        raise ValueError("velocity records must match the position records")
    acc = _out(acc_out, (n_i, 3), torch.float32, pos_i.device, "acc_out")
    jerk = _out(jerk_out, (n_i, 3), torch.float32, pos_i.device, "jerk_out")
    pot = None
    if potential or pot_out is not None:
        pot = _out(pot_out, (n_i,), torch.float32, pos_i.device, "pot_out")
    check(load().cn_force_jerk(n_i, _ptr(pos_i), _ptr(vel_i), n_j, _ptr(pos_mass_j), _ptr(vel_j), float(eps2),
                               _ptr(acc), _ptr(jerk), _ptr(pot), _stream_handle(stream)), "cn_force_jerk")
    return acc, jerk, pot


def _energy(fn, pos_mass, pot, w_out, stream):
    torch = _torch()
    _records(pos_mass, "pos_mass")
    _like(pot, pos_mass, "pot")
    w = _out(w_out, (1,), torch.float64, pos_mass.device, "w_out")
    check(getattr(load(), fn)(pos_mass.shape[0], _ptr(pos_mass), _ptr(pot), _ptr(w), _stream_handle(stream)), fn)
    return w


def cn_potential_energy(pos_mass, pot, w_out=None, stream=None):
    """W = 1/2 sum m_i phi_i (FP64, one-element CUDA tensor) from FP32 potentials."""
    torch = _torch()
    if pot.dtype != torch.float32 or tuple(pot.shape) != (pos_mass.shape[0],):
        raise TypeError("pot must be float32 of length n")
    return _energy("cn_potential_energy", pos_mass, pot, w_out, stream)


def cn_potential_energy_dd(pos_mass, pot, w_out=None, stream=None):
    torch = _torch()
    if pot.dtype != torch.float64 or tuple(pot.shape) != (pos_mass.shape[0],):
        raise TypeError("pot must be float64 of length n")
    return _energy("cn_potential_energy_dd", pos_mass, pot, w_out, stream)


# ------------------------------------------------------------------ host-memory forms

def _host_records(a, name):
    torch = _torch()
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float32 or a.dim() != 2 or a.shape[1] != 4 or not a.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float32 CPU tensor of shape (n, 4)")
        return a, a.data_ptr()
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 4:
        raise TypeError(f"{name} must be float32 (n, 4)")
    return a, a.ctypes.data


def cn_force_host(pos_i, pos_mass_j, eps2, acc_out=None, pot_out=None, potential=False, stream=None):
    """cn_force on host arrays (numpy or pinned CPU tensors); returns host outputs."""
    torch = _torch()
    pi, pi_ptr = _host_records(pos_i, "pos_i")
    pj, pj_ptr = (pi, pi_ptr) if pos_mass_j is pos_i else _host_records(pos_mass_j, "pos_mass_j")
    n_i, n_j = pi.shape[0], pj.shape[0]
    if acc_out is None:
        acc_out = np.empty((n_i, 3), dtype=np.float32)
    if (potential or pot_out is not None) and pot_out is None:
        pot_out = np.empty(n_i, dtype=np.float32)

    def addr(a):
        if a is None:
            return None
        return ctypes.c_void_p(a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data)

    check(load().cn_force_host(n_i, ctypes.c_void_p(pi_ptr), n_j, ctypes.c_void_p(pj_ptr), float(eps2),
                               addr(acc_out), addr(pot_out), _stream_handle(stream)), "cn_force_host")
    return acc_out, pot_out


def cn_force_host_f64(xj, mj, xi, eps2):
    """The paper's library routine (Section 3.1): FP64 host arrays in, a[ni][3] FP64 out."""
    xj = np.ascontiguousarray(xj, dtype=np.float64)
    mj = np.ascontiguousarray(mj, dtype=np.float64)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    a = np.empty((xi.shape[0], 3), dtype=np.float64)
    check(load().cn_force_host_f64(xj.ctypes.data_as(ctypes.c_void_p), mj.ctypes.data_as(ctypes.c_void_p),
                                   xi.ctypes.data_as(ctypes.c_void_p), float(eps2),
                                   a.ctypes.data_as(ctypes.c_void_p), xi.shape[0], xj.shape[0]),
          "cn_force_host_f64")
    return a


# ------------------------------------------------------------------ tuning, status

def _tune_struct(t):
    if isinstance(t, cn_tune):
        return t
    s = cn_tune()
    for k, v in dict(t).items():
        setattr(s, k, int(v))
    return s


def cn_tune_get(variant, n_i, n_j) -> dict:
    t = cn_tune()
    check(load().cn_tune_get(_variant(variant), int(n_i), int(n_j), ctypes.byref(t)), "cn_tune_get")
    return t.as_dict()


def cn_tune_set(variant, n_i, n_j, tune) -> None:
    ref = None if tune is None else ctypes.byref(_tune_struct(tune))
    check(load().cn_tune_set(_variant(variant), int(n_i), int(n_j), ref), "cn_tune_set")


def cn_tune_save(path) -> None:
    """Writes the current device's tuning entries to `path` (JSON)."""
    check(load().cn_tune_save(os.fsencode(path)), "cn_tune_save")


def cn_tune_load(path) -> int:
    """Stores the entries of a tuning file written on this kind of device;
    returns how many were stored."""
    n = ctypes.c_int32(0)
    check(load().cn_tune_load(os.fsencode(path), ctypes.byref(n)), "cn_tune_load")
    return int(n.value)


def cn_autotune(variant, pos_i, pos_mass_j, eps2, reps=3, stream=None) -> dict:
    torch = _torch()
    v = _variant(variant)
    double = v in (2, 3)
    pot = v in (1, 3)
    n_i = pos_i.shape[0]
    dt = torch.float64 if double else torch.float32
    acc = torch.empty((n_i, 3), dtype=dt, device=pos_i.device)
    potb = torch.empty((n_i,), dtype=dt, device=pos_i.device) if pot else None
    t = cn_tune()
    check(load().cn_autotune(v, n_i, _ptr(pos_i), pos_mass_j.shape[0], _ptr(pos_mass_j), float(eps2), _ptr(acc),
                             _ptr(potb), int(reps), _stream_handle(stream), ctypes.byref(t)), "cn_autotune")
    return t.as_dict()


def cn_autotune_batched(offsets, eps2, pos_mass, potential=False, reps=3, stream=None) -> dict:
    torch = _torch()
    offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    eps2 = np.ascontiguousarray(np.asarray(eps2, dtype=np.float32))
    n = pos_mass.shape[0]
    acc = torch.empty((n, 3), dtype=torch.float32, device=pos_mass.device)
    pot = torch.empty((n,), dtype=torch.float32, device=pos_mass.device) if potential else None
    t = cn_tune()
    check(load().cn_autotune_batched(offsets.shape[0] - 1, offsets.ctypes.data_as(ctypes.c_void_p),
                                     eps2.ctypes.data_as(ctypes.c_void_p), _ptr(pos_mass), _ptr(acc), _ptr(pot),
                                     int(reps), _stream_handle(stream), ctypes.byref(t)), "cn_autotune_batched")
    return t.as_dict()


def cn_get_device_status(stream=None) -> int:
    """Synchronise and return the status code (0, or 4 = CN_ERR_TIMEOUT after a timed-out wait)."""
    return int(load().cn_get_device_status(_stream_handle(stream)))


def cn_set_wait_limit_ns(ns: int) -> None:
    check(load().cn_set_wait_limit_ns(int(ns)), "cn_set_wait_limit_ns")


def cn_debug_timeout_probe(stream=None) -> None:
    check(load().cn_debug_timeout_probe(_stream_handle(stream)), "cn_debug_timeout_probe")


def cn_probe_peaks(stream=None) -> dict:
    out = (ctypes.c_double * 5)()
    check(load().cn_probe_peaks(_stream_handle(stream), out), "cn_probe_peaks")
    return {"ffma_per_s": out[0], "mufu_rsqrt_per_s": out[1], "pair_mix_per_s": out[2], "sm_mhz": out[3],
            "sms": int(out[4])}


def cn_version() -> str:
    return load().cn_version().decode()


# ------------------------------------------------------------------ autograd

def _gravity_function():
    torch = _torch()

    class GravityForce(torch.autograd.Function):
        """a = Eq. 1 with i set = j set; backward is the hand-written adjoint kernel."""

        @staticmethod
        def forward(ctx, pos_mass, eps2):
            pm = pos_mass.detach().contiguous()
            acc, _ = cn_force(pm, pm, eps2)
            ctx.save_for_backward(pm)
            ctx.eps2 = float(eps2)
            return acc

        @staticmethod
        def backward(ctx, grad_acc):
            (pm,) = ctx.saved_tensors
            w = grad_acc.detach().to(torch.float32).contiguous()
            gp, gm = cn_force_adjoint(pm, ctx.eps2, w)
            return torch.cat([gp, gm[:, None]], dim=1), None

    return GravityForce


class _Lazy:
    def __init__(self):
        self._cls = None

    def __call__(self):
        if self._cls is None:
            self._cls = _gravity_function()
        return self._cls


_gravity_cls = _Lazy()


def __getattr__(name):
    if name == "GravityForce":
        return _gravity_cls()
    raise AttributeError(name)


def gravity(pos_mass, eps2):
    """Differentiable accelerations of all particles under each other's gravity."""
    return _gravity_cls().apply(pos_mass, eps2)
