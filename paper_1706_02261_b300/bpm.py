"""Python binding of libbpm.so (include/bpm.h): argument marshalling only.

Every function mirrors the C entry point of the same name; device buffers are
torch CUDA tensors (complex64 fields, float16 index volumes, float32 intensity
volumes) and streams are torch CUDA streams.  All arithmetic runs in the
library's CUDA kernels; when the library is missing this module raises on
import rather than falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbpm.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "bpm.h")
HEADERS = [HEADER, os.path.join(os.path.dirname(_HERE), "include", "bpm_corrector.h")]

BPM_OK = 0
BPM_ERR_ARG = -1
BPM_ERR_ALIGN = -2
BPM_ERR_CUDA = -3
BPM_ERR_TIMEOUT = -4
BPM_ERR_NAN = -5
BPM_ERR_UNSUPPORTED = -6
BPM_FLAG_SYNC = 0x1
BPM_FLAG_MULTI_LAUNCH = 0x2
BPM_FLAG_GRAPH = 0x4
BPM_FLAG_ADAPTIVE = 0x8

# transform lengths of each grid side (nx, ny in this set, nx ny <= 2^22);
# batched plans take square grids of BATCH_N
SUPPORTED_N = (64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048)
BATCH_N = (64, 128, 192, 256, 384, 512, 1024)


class BpmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class bpm_instance_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("n0", ctypes.c_double),
                ("tilt_x", ctypes.c_double), ("tilt_y", ctypes.c_double)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libbpm.so not found at {LIB_PATH}; build it with "
                      f"`python -m paper_1706_02261_b300.build` (nvcc, sm_103a)")
_lib = ctypes.CDLL(LIB_PATH)
_vp, _i, _u, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double
_pp = ctypes.POINTER(ctypes.c_void_p)
_lib.bpm_plan.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(bpm_instance_desc), _i, _u, _vp]
_lib.bpm_propagate.argtypes = [_vp, _pp, _pp, _pp, _pp, _i, _i, _vp]
_lib.bpm_multiplex_psf.argtypes = [_vp, _i, _i, _vp, _vp, _d, _vp, _vp]
_lib.bpm_multiplex_annular.argtypes = [_vp, _i, _i, _vp, _vp, _d, _d, _vp, _vp]
_lib.bpm_light_sheet.argtypes = [_vp, _i, _d, _d, _vp, _vp]
_lib.bpm_check.argtypes = [_vp]
_lib.bpm_free.argtypes = [_vp]
_lib.bpm_last_error.restype = ctypes.c_char_p
_lib.bpm_plan_info.argtypes = [_vp, ctypes.POINTER(_i), _i]
_lib.bpm_debug_set_barrier_timeout.argtypes = [_vp, ctypes.c_ulonglong, _u]
_lib.bpm_debug_stall_exchange.argtypes = [_vp, _i]
_lib.bpm_autotune.argtypes = [_vp, _pp, _pp, _pp, _pp, _i, _vp]
_lib.bpm_set_schedule.argtypes = [_vp, _i]
_lib.bpm_propagate_host.argtypes = [_vp, _vp, _vp, _i, _vp, _vp, _i, _vp]
_lib.bpm_propagate_static.argtypes = [ctypes.POINTER(bpm_instance_desc), _vp, _vp, _vp, _vp, _i, _i, _vp]
_lib.bpm_propagate_window.argtypes = [_vp, _pp, _pp, _pp, _pp, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), _vp]
_lib.bpm_propagate_reverse.argtypes = [_vp, _vp, _vp, _vp, _vp, _i, _i, _vp]
_lib.bpm_phase_conjugate.argtypes = [_vp, _i, _vp, _vp]
_lib.bpm_propagate_absorbing.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _vp]
_lib.bpm_demultiplex.argtypes = [_vp, _i, _vp, _i, _i, _i, ctypes.POINTER(_i), _i, _i, _i, _vp, _vp]
for _f in ("bpm_plan", "bpm_propagate", "bpm_multiplex_psf", "bpm_light_sheet", "bpm_check",
           "bpm_free", "bpm_plan_info", "bpm_debug_set_barrier_timeout", "bpm_debug_stall_exchange", "bpm_propagate_static", "bpm_autotune", "bpm_propagate_host",
           "bpm_set_schedule"):
    getattr(_lib, _f).restype = _i


def declared_symbols() -> list:
    """Names of the functions declared in include/bpm.h and include/bpm_corrector.h."""
    txt = "".join(open(h).read() for h in HEADERS)
    return sorted(set(re.findall(r"^(?:int|const char \*)\s*(bpm_\w+)\s*\(", txt, re.M)))


def library() -> ctypes.CDLL:
    return _lib


def bpm_last_error() -> str:
    return _lib.bpm_last_error().decode()


def _check(rc: int):
    if rc != BPM_OK:
        raise BpmError(rc, bpm_last_error())
    return rc


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _arr(ptrs):
    a = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        a[i] = p.value if isinstance(p, ctypes.c_void_p) else p
    return a


@dataclass
class Instance:
    """One propagation problem: grid n x ny (n = nx, the row length; ny
    defaults to n) x nz, spacings in um, vacuum wavelength, n0."""
    n: int
    nz: int
    dx: float
    dz: float
    lam: float = 0.5
    n0: float = 1.33
    dy: float | None = None
    ny: int | None = None

    @property
    def nx(self) -> int:
        return self.n

    @property
    def rows(self) -> int:
        return self.ny or self.n

    def desc(self) -> bpm_instance_desc:
        return bpm_instance_desc(self.n, self.rows, self.nz, self.dx, self.dy or self.dx, self.dz,
                                 self.lam, self.n0, 0.0, 0.0)


def bpm_plan(instances, flags: int = 0, stream=None) -> ctypes.c_void_p:
    if isinstance(instances, Instance):
        instances = [instances]
    descs = (bpm_instance_desc * len(instances))(*[i.desc() for i in instances])
    h = ctypes.c_void_p()
    _check(_lib.bpm_plan(ctypes.byref(h), descs, len(instances), flags, _stream_handle(stream)))
    return h


def bpm_propagate(plan, dn, e_in, e_out, inten=None, z_begin: int = 0, z_end: int = 2 ** 31 - 1,
                  stream=None) -> int:
    """dn, e_in, e_out, inten: tensors or lists of tensors (one per instance)."""
    single = not isinstance(e_in, (list, tuple))
    dn, e_in, e_out = ([dn], [e_in], [e_out]) if single else (dn, e_in, e_out)
    if inten is not None and single:
        inten = [inten]
    a_dn = _arr([_ptr(t) or ctypes.c_void_p(0) for t in dn])
    a_in = _arr([_ptr(t) for t in e_in])
    a_out = _arr([_ptr(t) for t in e_out])
    a_i = _arr([_ptr(t) if t is not None else ctypes.c_void_p(0) for t in inten]) if inten is not None else None
    return _check(_lib.bpm_propagate(plan, a_dn, a_in, a_out, a_i, z_begin, z_end, _stream_handle(stream)))


def bpm_propagate_window(plan, dn, e_in, e_out, inten, w_begin, w_end, z_begin: int = 0,
                         z_end: int = 2 ** 31 - 1, stream=None) -> int:
    """bpm_propagate writing |E|^2 only for slices [w_begin, w_end) of each
    instance into inten (w_end - w_begin slices).  Single tensors or lists;
    w_begin, w_end: ints or lists of ints (one per instance)."""
    single = not isinstance(e_in, (list, tuple))
    dn, e_in, e_out, inten = ([dn], [e_in], [e_out], [inten]) if single else (dn, e_in, e_out, inten)
    wb = [w_begin] if single else list(w_begin)
    we = [w_end] if single else list(w_end)
    a_dn = _arr([_ptr(t) or ctypes.c_void_p(0) for t in dn])
    a_in = _arr([_ptr(t) for t in e_in])
    a_out = _arr([_ptr(t) for t in e_out])
    a_i = _arr([_ptr(t) if t is not None else ctypes.c_void_p(0) for t in inten])
    c_wb = (_i * len(wb))(*wb)
    c_we = (_i * len(we))(*we)
    return _check(_lib.bpm_propagate_window(plan, a_dn, a_in, a_out, a_i, z_begin, z_end, c_wb, c_we,
                                            _stream_handle(stream)))


def bpm_propagate_reverse(plan, dn, e_in, e_out, inten=None, z_begin: int = 0, z_end: int = 2 ** 31 - 1,
                          stream=None) -> int:
    """Slices z_end-1 down to z_begin (propagation towards -z), single-instance plans."""
    return _check(_lib.bpm_propagate_reverse(plan, _ptr(dn), _ptr(e_in), _ptr(e_out), _ptr(inten), z_begin, z_end,
                                             _stream_handle(stream)))


def bpm_propagate_absorbing(plan, dn, kappa, e_in, e_out, inten=None, z_begin: int = 0, z_end: int = 2 ** 31 - 1,
                            stream=None) -> int:
    """Complex index n0 + dn + i kappa (FP16 volumes), single-instance plans."""
    return _check(_lib.bpm_propagate_absorbing(plan, _ptr(dn), _ptr(kappa), _ptr(e_in), _ptr(e_out), _ptr(inten),
                                               z_begin, z_end, _stream_handle(stream)))


def bpm_phase_conjugate(plan, inst: int, e, stream=None) -> int:
    """e <- conj(e) on the device."""
    return _check(_lib.bpm_phase_conjugate(plan, inst, _ptr(e), _stream_handle(stream)))


def bpm_demultiplex(plan, inst: int, inten, w_begin: int, foci, patch, out, stream=None) -> int:
    """Cut patch = (px, py, pz) around each focus (rows of foci: ix, iy, iz
    voxel indices) out of the intensity window inten [w_nz][ny][nx] that starts
    at slice w_begin; out: float tensor [n_foci][pz][py][px]."""
    f = np.ascontiguousarray(np.asarray(foci, dtype=np.int32).reshape(-1, 3))
    px, py, pz = patch
    return _check(_lib.bpm_demultiplex(plan, inst, _ptr(inten), w_begin, int(inten.shape[0]), f.shape[0],
                                       f.ctypes.data_as(ctypes.POINTER(_i)), px, py, pz, _ptr(out),
                                       _stream_handle(stream)))


def bpm_propagate_host(plan, dn_host, e_in, e_out_host, inten_host=None, chunk: int = 64, stream=None) -> int:
    """Whole propagation with host index/intensity volumes (pinned torch CPU
    tensors or numpy arrays); e_in may be a host or a CUDA tensor."""
    def hp(t):
        if t is None:
            return None
        if isinstance(t, np.ndarray):
            return ctypes.c_void_p(t.ctypes.data)
        return ctypes.c_void_p(t.data_ptr())
    on_dev = int(hasattr(e_in, "is_cuda") and e_in.is_cuda)
    return _check(_lib.bpm_propagate_host(plan, hp(dn_host), hp(e_in), on_dev, hp(e_out_host), hp(inten_host),
                                          chunk, _stream_handle(stream)))


def bpm_autotune(plan, dn, e_in, e_out, inten=None, z_probe: int = 8, stream=None) -> int:
    """Pick the fastest configuration on these buffers: the cluster size of a
    batched plan (lists, one entry per instance) or the transform schedule of a
    single-field plan (tensors or one-entry lists)."""
    if not isinstance(e_in, (list, tuple)):
        dn, e_in, e_out = [dn], [e_in], [e_out]
        inten = [inten] if inten is not None else None
    a_dn = _arr([_ptr(t) for t in dn])
    a_in = _arr([_ptr(t) for t in e_in])
    a_out = _arr([_ptr(t) for t in e_out])
    a_i = _arr([_ptr(t) if t is not None else ctypes.c_void_p(0) for t in inten]) if inten is not None else None
    return _check(_lib.bpm_autotune(plan, a_dn, a_in, a_out, a_i, z_probe, _stream_handle(stream)))


def bpm_multiplex_psf(plan, inst: int, xyz: np.ndarray, phase: np.ndarray, NA: float, e_out,
                      stream=None) -> int:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    phase = np.ascontiguousarray(phase, dtype=np.float64).reshape(-1)
    assert phase.size == xyz.shape[0]
    return _check(_lib.bpm_multiplex_psf(plan, inst, phase.size, ctypes.c_void_p(xyz.ctypes.data),
                                         ctypes.c_void_p(phase.ctypes.data), NA, _ptr(e_out),
                                         _stream_handle(stream)))


def bpm_multiplex_annular(plan, inst: int, xyz: np.ndarray, phase: np.ndarray, NA_in: float, NA_out: float, e_out,
                          stream=None) -> int:
    """Bessel beams / lattices: emitters through the annulus NA_in <= |k_perp|/k0 <= NA_out."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    phase = np.ascontiguousarray(phase, dtype=np.float64).reshape(-1)
    assert phase.size == xyz.shape[0]
    return _check(_lib.bpm_multiplex_annular(plan, inst, phase.size, ctypes.c_void_p(xyz.ctypes.data),
                                             ctypes.c_void_p(phase.ctypes.data), NA_in, NA_out, _ptr(e_out),
                                             _stream_handle(stream)))


def bpm_light_sheet(plan, inst: int, NA: float, zf: float, e_out, stream=None) -> int:
    return _check(_lib.bpm_light_sheet(plan, inst, NA, zf, _ptr(e_out), _stream_handle(stream)))


def bpm_check(plan) -> int:
    return _lib.bpm_check(plan)


def bpm_free(plan) -> int:
    return _check(_lib.bpm_free(plan))


def bpm_plan_info(plan) -> dict:
    out = (ctypes.c_int * 7)()
    _check(_lib.bpm_plan_info(plan, out, 7))
    return {"team_ctas": out[0], "threads": out[1], "smem_bytes": out[2], "persistent": out[3],
            "launches_per_call": out[4], "schedule": out[5], "schedules": out[6]}


def bpm_set_schedule(plan, schedule: int) -> int:
    """Transform schedule of a single-field plan (0 .. plan_info()['schedules'] - 1)."""
    return _check(_lib.bpm_set_schedule(plan, schedule))


def bpm_debug_set_barrier_timeout(plan, timeout_ns: int, extra_arrivals: int = 0) -> int:
    return _check(_lib.bpm_debug_set_barrier_timeout(plan, timeout_ns, extra_arrivals))


def bpm_debug_stall_exchange(plan, on: bool) -> int:
    return _check(_lib.bpm_debug_stall_exchange(plan, 1 if on else 0))


def bpm_propagate_static(instance: "Instance", dn, e_in, e_out, inten=None, z_begin: int = 0,
                         z_end: int = 2 ** 31 - 1, stream=None) -> int:
    """Allocation-free propagation of one instance (square grids up to 256 x 256);
    synchronises the stream and returns the device status."""
    desc = instance.desc()
    return _check(_lib.bpm_propagate_static(ctypes.byref(desc), _ptr(dn), _ptr(e_in), _ptr(e_out),
                                            _ptr(inten), z_begin, z_end, _stream_handle(stream)))


# ---- learned coarse-step corrector (include/bpm_corrector.h) ----------------
_fp = ctypes.POINTER(ctypes.c_float)
_lib.bpm_corrector_create.argtypes = [ctypes.POINTER(_vp), _i, _i, _i, _i, _vp]
_lib.bpm_corrector_param_count.argtypes = [_vp]
_lib.bpm_corrector_set_residual_scale.argtypes = [_vp, ctypes.c_float]
_lib.bpm_corrector_set_params.argtypes = [_vp, _vp, _i, _vp]
_lib.bpm_corrector_get_params.argtypes = [_vp, _vp, _i, _i, _vp]
_lib.bpm_corrector_forward.argtypes = [_vp, _vp, _vp, _i, _i, _i, _vp]
_lib.bpm_corrector_loss_grad.argtypes = [_vp, _vp, _vp, _i, _i, _i, _fp, _vp]
_lib.bpm_corrector_adam.argtypes = [_vp, ctypes.c_float, _vp]
_lib.bpm_corrector_train_step.argtypes = [_vp, _vp, _vp, _i, _i, _i, ctypes.c_float, _fp, _vp]
_lib.bpm_corrector_pack.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_float, _vp, _vp, _i, _i, _i, _vp]
_lib.bpm_corrector_apply.argtypes = [_vp, _vp, _vp, ctypes.c_float, _i, _i, _vp]
_lib.bpm_coarsen_index.argtypes = [_vp, _i, _i, _i, _i, _vp, _vp]
_lib.bpm_corrector_free.argtypes = [_vp]
_lib.bpm_corrector_set_tensor_cores.argtypes = [_vp, _i]
_lib.bpm_corrector_set_train_tensor_cores.argtypes = [_vp, _i]
_lib.bpm_corrector_check.argtypes = [_vp, _vp]
_lib.bpm_corrector_last_error.restype = ctypes.c_char_p
for _f in ("bpm_corrector_create", "bpm_corrector_param_count", "bpm_corrector_set_params",
           "bpm_corrector_get_params", "bpm_corrector_forward", "bpm_corrector_loss_grad", "bpm_corrector_adam",
           "bpm_corrector_train_step", "bpm_corrector_pack", "bpm_corrector_apply", "bpm_coarsen_index",
           "bpm_corrector_free", "bpm_corrector_set_residual_scale"):
    getattr(_lib, _f).restype = _i


def _ccheck(rc: int):
    if rc != BPM_OK:
        raise BpmError(rc, _lib.bpm_corrector_last_error().decode())
    return rc


class Corrector:
    """Owner of a bpm_corrector_t (argument marshalling only)."""

    def __init__(self, in_channels: int, max_batch: int, max_h: int, max_w: int, stream=None):
        self.h = ctypes.c_void_p()
        _ccheck(_lib.bpm_corrector_create(ctypes.byref(self.h), in_channels, max_batch, max_h, max_w,
                                          _stream_handle(stream)))
        self.in_channels = in_channels
        self.n_params = _lib.bpm_corrector_param_count(self.h)

    def set_params(self, theta: np.ndarray, stream=None):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == self.n_params
        _ccheck(_lib.bpm_corrector_set_params(self.h, ctypes.c_void_p(a.ctypes.data), a.size, _stream_handle(stream)))

    def set_residual_scale(self, sigma: float):
        _ccheck(_lib.bpm_corrector_set_residual_scale(self.h, sigma))

    def get_params(self, which: int = 0, stream=None) -> np.ndarray:
        a = np.zeros(self.n_params, np.float32)
        _ccheck(_lib.bpm_corrector_get_params(self.h, ctypes.c_void_p(a.ctypes.data), a.size, which,
                                              _stream_handle(stream)))
        return a

    def forward(self, x, out, stream=None):
        b, _, hh, ww = x.shape
        _ccheck(_lib.bpm_corrector_forward(self.h, _ptr(x), _ptr(out), b, hh, ww, _stream_handle(stream)))

    def loss_grad(self, x, target, stream=None) -> float:
        b, _, hh, ww = x.shape
        loss = ctypes.c_float()
        _ccheck(_lib.bpm_corrector_loss_grad(self.h, _ptr(x), _ptr(target), b, hh, ww, ctypes.byref(loss),
                                             _stream_handle(stream)))
        return float(loss.value)

    def adam(self, lr: float, stream=None):
        _ccheck(_lib.bpm_corrector_adam(self.h, lr, _stream_handle(stream)))

    def train_step(self, x, target, lr: float, want_loss: bool = False, stream=None):
        b, _, hh, ww = x.shape
        loss = ctypes.c_float()
        _ccheck(_lib.bpm_corrector_train_step(self.h, _ptr(x), _ptr(target), b, hh, ww, lr,
                                              ctypes.byref(loss) if want_loss else None, _stream_handle(stream)))
        return float(loss.value) if want_loss else None

    def pack(self, fields, dn, dn_scale: float, x, targets=None, t=None, stream=None):
        b, hh, ww = fields.shape
        _ccheck(_lib.bpm_corrector_pack(self.h, _ptr(fields), _ptr(targets), _ptr(dn), dn_scale, _ptr(x), _ptr(t),
                                        b, hh, ww, _stream_handle(stream)))

    def apply(self, field, dn=None, dn_scale: float = 0.0, stream=None):
        hh, ww = field.shape
        _ccheck(_lib.bpm_corrector_apply(self.h, _ptr(field), _ptr(dn), dn_scale, hh, ww, _stream_handle(stream)))

    def set_tensor_cores(self, on: bool):
        """Inference on the tensor cores (BF16 activations) or on the FP32 pipes."""
        _ccheck(_lib.bpm_corrector_set_tensor_cores(self.h, int(bool(on))))

    def set_train_tensor_cores(self, on: bool):
        """Loss and gradients on the tensor cores (BF16 operands) or on the FP32 pipes."""
        _ccheck(_lib.bpm_corrector_set_train_tensor_cores(self.h, int(bool(on))))

    def check(self, stream=None):
        _ccheck(_lib.bpm_corrector_check(self.h, _stream_handle(stream)))

    def free(self):
        if self.h:
            _lib.bpm_corrector_free(self.h)
            self.h = ctypes.c_void_p()


def bpm_coarsen_index(dn, factor: int, out, stream=None) -> int:
    nz, ny, nx = dn.shape
    return _ccheck(_lib.bpm_coarsen_index(_ptr(dn), nz, ny, nx, factor, _ptr(out), _stream_handle(stream)))
