"""ctypes binding of ``libdpa1.so`` (the C ABI of ``include/dpa1.h``).

Argument marshalling only: every stage of the energy / force / virial path
runs in the library's CUDA kernels.  Importing this module loads the library
and raises ``ImportError`` if it has not been built (there is no fallback).
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libdpa1.so")

DP_OK = 0
STATUS = {0: "DP_OK", -1: "DP_ERR_ARG", -2: "DP_ERR_IO", -3: "DP_ERR_BOX", -4: "DP_ERR_CAPACITY",
          -5: "DP_ERR_CUDA", -6: "DP_ERR_TIMEOUT", -7: "DP_ERR_NAN", -8: "DP_ERR_UNSUPPORTED"}
PRECISION = {"fp32": 0, "bf16": 1, "fp16x": 2, "bf16x": 3}

EXPORTS = ("dp_init", "dp_compute", "dp_compute_device", "dp_compute_local", "dp_compute_device_local", "dp_compute_batch", "dp_reserve", "dp_set_precision",
           "dp_get_status", "dp_nlist_device", "dp_stats", "dp_inspect_weights", "dp_debug_copy", "dp_debug_poison",
           "dp_set_profiling", "dp_stage_times", "dp_kernel_launches", "dp_nlist_noalloc", "dp_md_run", "dp_param_count", "dp_get_params",
           "dp_set_params", "dp_get_grad", "dp_zero_grad", "dp_train_frame", "dp_adam_step", "dp_last_error",
           "dp_free")


class DPError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdpa1.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    D = ctypes.POINTER(ctypes.c_double)
    I = ctypes.POINTER(ctypes.c_int)
    lib.dp_init.argtypes = [ctypes.POINTER(P), ctypes.c_char_p, ctypes.POINTER(ctypes.c_char_p), ctypes.c_int,
                            ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.dp_compute.argtypes = [P, ctypes.c_int, D, D, I, D, D, D, D]
    lib.dp_compute_device.argtypes = [P, ctypes.c_int, P, P, P, P, P, P, P, P]
    lib.dp_compute_local.argtypes = [P, ctypes.c_int, ctypes.c_int, D, D, I, D, D, D, D]
    lib.dp_compute_device_local.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P, P, P]
    lib.dp_compute_batch.argtypes = [P, ctypes.c_int, I, D, D, I, D, D, D]
    lib.dp_reserve.argtypes = [P, ctypes.c_int]
    lib.dp_set_precision.argtypes = [P, ctypes.c_int]
    lib.dp_get_status.argtypes = [P]
    lib.dp_nlist_device.argtypes = [P, ctypes.c_int, P, P, P, P, P]
    lib.dp_stats.argtypes = [P, I, ctypes.POINTER(ctypes.c_longlong)]
    lib.dp_inspect_weights.argtypes = [ctypes.c_char_p, I, D]
    lib.dp_debug_copy.argtypes = [P, ctypes.c_char_p, P, ctypes.c_size_t]
    lib.dp_debug_copy.restype = ctypes.c_longlong
    lib.dp_debug_poison.argtypes = [P]
    lib.dp_set_profiling.argtypes = [P, ctypes.c_int]
    lib.dp_stage_times.argtypes = [P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float), ctypes.c_int]
    F = ctypes.POINTER(ctypes.c_float)
    lib.dp_param_count.argtypes = [P]
    lib.dp_get_params.argtypes = [P, F, ctypes.c_int]
    lib.dp_set_params.argtypes = [P, F, ctypes.c_int]
    lib.dp_get_grad.argtypes = [P, F, ctypes.c_int]
    lib.dp_zero_grad.argtypes = [P, P]
    lib.dp_train_frame.argtypes = [P, ctypes.c_int, P, P, P, ctypes.c_double, P, ctypes.c_double, ctypes.c_double,
                                   P, P]
    lib.dp_adam_step.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, P]
    lib.dp_md_run.argtypes = [P, ctypes.c_int, P, P, P, P, P, ctypes.c_double, ctypes.c_int, P, P, P, P, ctypes.c_int,
                              P]
    lib.dp_nlist_noalloc.argtypes = [ctypes.c_int, P, P, ctypes.c_double, ctypes.c_int, P, P, P, P]
    lib.dp_kernel_launches.argtypes = []
    lib.dp_kernel_launches.restype = ctypes.c_longlong
    lib.dp_last_error.argtypes = []
    lib.dp_last_error.restype = ctypes.c_char_p
    lib.dp_free.argtypes = [P]
    lib.dp_free.restype = None
    for name in EXPORTS:
        if name not in ("dp_debug_copy", "dp_last_error", "dp_free", "dp_kernel_launches"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code: int) -> None:
    if code != DP_OK:
        raise DPError(code, load_library().dp_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def box9(box) -> np.ndarray:
    b = np.asarray(box, dtype=np.float64)
    if b.shape == (3,):
        b = np.diag(b)
    return np.ascontiguousarray(b.reshape(9))


def nlist_noalloc(coord, box, rcut: float, sel: int, nlist, nnei, status, stream=None) -> None:
    """``dp_nlist_noalloc`` on CUDA tensors the caller allocated: coord
    [N,3] float64, box [9] float64, nlist [N,128] int32, nnei [N] int32,
    status [1] int32 (device-side failure bits, read after the stream)."""
    import torch

    st = stream if stream is not None else torch.cuda.current_stream(coord.device).cuda_stream
    _check(load_library().dp_nlist_noalloc(int(coord.shape[0]), coord.data_ptr(), box.data_ptr(), float(rcut),
                                           int(sel), nlist.data_ptr(), nnei.data_ptr(), status.data_ptr(), st))


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load_library().dp_kernel_launches())


def inspect_weights(path: str) -> Tuple[np.ndarray, np.ndarray]:
    ints = np.zeros(16, dtype=np.int32)
    dbls = np.zeros(8, dtype=np.float64)
    _check(load_library().dp_inspect_weights(path.encode(), _iptr(ints), _dptr(dbls)))
    return ints, dbls


class DPA1:
    """One loaded DPA-1 model on one GPU (``dp_init`` .. ``dp_free``)."""

    def __init__(self, weights_path: str, precision: str = "fp32", device: int = 0,
                 type_map: Optional[Sequence[str]] = None, rcut: float = -1.0, rcut_smth: float = -1.0,
                 sel: int = -1):
        self.lib = load_library()
        h = ctypes.c_void_p()
        tm = None
        nt = 0
        if type_map is not None:
            nt = len(type_map)
            tm = (ctypes.c_char_p * nt)(*[t.encode() for t in type_map])
        _check(self.lib.dp_init(ctypes.byref(h), weights_path.encode(), tm, nt, rcut, rcut_smth, sel,
                                PRECISION[precision], device))
        self.h = h
        self.precision = precision
        self.device = device

    # -- host arrays ---------------------------------------------------------
    def compute(self, coord, box, atype, atom_energy: bool = False, nlocal: Optional[int] = None):
        """(E, F [N,3], W [3,3], e [N] or None) from host arrays (``dp_compute``;
        with ``nlocal``, ``dp_compute_local``: atoms [nlocal, N) are ghosts)."""
        c = np.ascontiguousarray(coord, dtype=np.float64).reshape(-1, 3)
        t = np.ascontiguousarray(atype, dtype=np.int32)
        b = box9(box)
        n = c.shape[0]
        e = np.zeros(1)
        f = np.zeros((n, 3))
        w = np.zeros(9)
        ae = np.zeros(n) if atom_energy else None
        aep = _dptr(ae) if ae is not None else None
        if nlocal is None:
            _check(self.lib.dp_compute(self.h, n, _dptr(c), _dptr(b), _iptr(t), _dptr(e), _dptr(f), _dptr(w), aep))
        else:
            _check(self.lib.dp_compute_local(self.h, n, int(nlocal), _dptr(c), _dptr(b), _iptr(t), _dptr(e), _dptr(f),
                                             _dptr(w), aep))
        return float(e[0]), f, w.reshape(3, 3), ae

    def compute_batch(self, frames):
        """frames: list of (coord, atype, box); returns lists of E, F, W."""
        offs = np.zeros(len(frames) + 1, dtype=np.int32)
        for i, (c, t, b) in enumerate(frames):
            offs[i + 1] = offs[i] + len(t)
        coord = np.ascontiguousarray(np.concatenate([np.asarray(c).reshape(-1, 3) for c, _, _ in frames]), np.float64)
        atype = np.ascontiguousarray(np.concatenate([np.asarray(t) for _, t, _ in frames]), np.int32)
        box = np.ascontiguousarray(np.concatenate([box9(b) for _, _, b in frames]))
        e = np.zeros(len(frames))
        f = np.zeros((int(offs[-1]), 3))
        w = np.zeros(9 * len(frames))
        _check(self.lib.dp_compute_batch(self.h, len(frames), _iptr(offs), _dptr(coord), _dptr(box), _iptr(atype),
                                         _dptr(e), _dptr(f), _dptr(w)))
        return e, [f[offs[i]:offs[i + 1]] for i in range(len(frames))], w.reshape(-1, 3, 3)

    # -- device arrays (torch tensors) ----------------------------------------
    def compute_device(self, coord, box, atype, energy, force, virial, atom_energy=None, stream=None, nlocal=None):
        """``dp_compute_device`` (``dp_compute_device_local`` with ``nlocal``) on
        CUDA tensors; no host synchronisation."""
        import torch

        st = stream if stream is not None else torch.cuda.current_stream(coord.device).cuda_stream
        n = int(coord.shape[0])
        ae = atom_energy.data_ptr() if atom_energy is not None else None
        if nlocal is None:
            _check(self.lib.dp_compute_device(self.h, n, coord.data_ptr(), box.data_ptr(), atype.data_ptr(),
                                              energy.data_ptr(), force.data_ptr(), virial.data_ptr(), ae, st))
        else:
            _check(self.lib.dp_compute_device_local(self.h, n, int(nlocal), coord.data_ptr(), box.data_ptr(),
                                                    atype.data_ptr(), energy.data_ptr(), force.data_ptr(),
                                                    virial.data_ptr(), ae, st))

    def nlist_device(self, coord, box, stream=None):
        import torch

        n = int(coord.shape[0])
        nl = torch.empty((n, 128), dtype=torch.int32, device=coord.device)
        nn = torch.empty((n,), dtype=torch.int32, device=coord.device)
        st = stream if stream is not None else torch.cuda.current_stream(coord.device).cuda_stream
        _check(self.lib.dp_nlist_device(self.h, n, coord.data_ptr(), box.data_ptr(), nl.data_ptr(), nn.data_ptr(), st))
        return nl, nn

    def reserve(self, max_atoms: int) -> None:
        _check(self.lib.dp_reserve(self.h, int(max_atoms)))

    def set_precision(self, precision: str) -> None:
        _check(self.lib.dp_set_precision(self.h, PRECISION[precision]))
        self.precision = precision

    def status(self) -> None:
        _check(self.lib.dp_get_status(self.h))

    def stats(self) -> Tuple[int, int]:
        mx = ctypes.c_int()
        tr = ctypes.c_longlong()
        _check(self.lib.dp_stats(self.h, ctypes.byref(mx), ctypes.byref(tr)))
        return mx.value, tr.value

    def debug(self, name: str, shape, dtype=np.float32) -> np.ndarray:
        out = np.zeros(shape, dtype=dtype)
        r = self.lib.dp_debug_copy(self.h, name.encode(), out.ctypes.data, out.nbytes)
        if r < 0:
            _check(int(r))
        return out

    def debug_poison(self) -> None:
        """Fill the model's workspace with NaN / -1 bit patterns (dp_debug_poison)."""
        _check(self.lib.dp_debug_poison(self.h))

    # -- training (models without attention, FP32) ----------------------------
    def param_count(self) -> int:
        n = self.lib.dp_param_count(self.h)
        if n < 0:
            _check(n)
        return n

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count(), dtype=np.float32)
        _check(self.lib.dp_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(out)))
        return out

    def set_params(self, theta) -> None:
        t = np.ascontiguousarray(theta, dtype=np.float32)
        _check(self.lib.dp_set_params(self.h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(t)))

    def get_grad(self) -> np.ndarray:
        out = np.zeros(self.param_count(), dtype=np.float32)
        _check(self.lib.dp_get_grad(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(out)))
        return out

    def zero_grad(self, stream=None) -> None:
        _check(self.lib.dp_zero_grad(self.h, stream))

    def train_frame(self, coord, box, atype, e_ref: float, force_ref, loss, pe=1.0, pf=1.0, stream=None):
        """``dp_train_frame`` on CUDA tensors; ``loss`` is a float64 [3] tensor."""
        import torch

        st = stream if stream is not None else torch.cuda.current_stream(coord.device).cuda_stream
        _check(self.lib.dp_train_frame(self.h, int(coord.shape[0]), coord.data_ptr(), box.data_ptr(),
                                       atype.data_ptr(), float(e_ref), force_ref.data_ptr(), float(pe), float(pf),
                                       loss.data_ptr(), st))

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None) -> None:
        _check(self.lib.dp_adam_step(self.h, float(lr), float(beta1), float(beta2), float(eps), stream))

    def set_profiling(self, on: bool) -> None:
        _check(self.lib.dp_set_profiling(self.h, 1 if on else 0))

    def stage_times(self):
        """[(stage, ms)] of every call since profiling was switched on."""
        names = (ctypes.c_char_p * 8192)()
        ms = (ctypes.c_float * 8192)()
        k = self.lib.dp_stage_times(self.h, names, ms, 8192)
        if k < 0:
            _check(k)
        return [(names[i].decode(), float(ms[i])) for i in range(k)]

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.dp_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
