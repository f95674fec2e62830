"""Python binding of libtlbm.so (the C ABI in include/tlbm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  PyTorch provides device memory and streams.  The functions keep the
C names; `Sim` is a small convenience wrapper that owns a torch allocation for
the bound device block.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

from . import build as _build

TLBM_OK = 0
TLBM_ERR_ARG = -1
TLBM_ERR_OOM = -2
TLBM_ERR_CUDA = -3
TLBM_ERR_DIVERGED = -4
TLBM_ERR_TIMEOUT = -5
TLBM_ERR_UNBOUND = -6
TLBM_ERR_UNSUPPORTED = -7

TLBM_D2Q9_D2Q5 = 0
TLBM_D3Q19_D3Q7 = 1
TLBM_FP64, TLBM_FP32, TLBM_FP16_OFFSET, TLBM_BF16_OFFSET = 0, 1, 2, 3
TLBM_RB, TLBM_SIDE_HEATED = 0, 1
TLBM_OUT_F64, TLBM_OUT_F32 = 0, 1
TLBM_STREAM_PULL, TLBM_STREAM_INPLACE = 0, 1

PRECISIONS = {"fp64": TLBM_FP64, "fp32": TLBM_FP32, "fp16": TLBM_FP16_OFFSET, "bf16": TLBM_BF16_OFFSET}


class tlbm_params(C.Structure):
    _fields_ = [
        ("walls", C.c_int), ("periodic_mask", C.c_int), ("u_is_ma", C.c_int),
        ("a_T", C.c_double), ("nu", C.c_double), ("alpha", C.c_double), ("gbeta", C.c_double),
        ("s_rho", C.c_double), ("s_e", C.c_double), ("s_eps", C.c_double), ("s_j", C.c_double),
        ("s_q", C.c_double), ("s_pi", C.c_double), ("s_m", C.c_double),
        ("q_e", C.c_double), ("q_v", C.c_double),
        ("body_force", C.c_double * 3), ("Th", C.c_double), ("Tc", C.c_double),
        ("store_scale", C.c_double), ("streaming", C.c_int),
    ]


class tlbm_instance(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("Ra", C.c_double),
                ("Pr", C.c_double), ("Ma", C.c_double), ("seed", C.c_uint64)]


class TlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tlbm error {code}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()

_SIGS = {
    "tlbm_default_params": (None, [C.POINTER(tlbm_params)]),
    "tlbm_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                              C.c_double, C.c_double, C.c_int, C.POINTER(tlbm_params)]),
    "tlbm_required_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "tlbm_bind_memory": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "tlbm_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tlbm_init": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double]),
    "tlbm_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "tlbm_macros": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "tlbm_nusselt": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "tlbm_energy": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "tlbm_get_populations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tlbm_set_populations": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "tlbm_get_populations_window": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                              C.c_void_p, C.c_void_p]),
    "tlbm_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int64)]),
    "tlbm_derived": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int)]),
    "tlbm_set_variant": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "tlbm_get_variant": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int)] * 5),
    "tlbm_reduce_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "tlbm_set_staged": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "tlbm_batch_set_rows": (C.c_int, [C.c_void_p, C.c_int]),
    "tlbm_batch_get_rows": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "tlbm_get_staged": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "tlbm_fp64_fma_rate": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "tlbm_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "tlbm_bounds_violations": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "tlbm_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "tlbm_set_wait_limit": (C.c_int, [C.c_void_p, C.c_double]),
    "tlbm_batch_set_wait_limit": (C.c_int, [C.c_void_p, C.c_double]),
    "tlbm_set_graph": (C.c_int, [C.c_void_p, C.c_int]),
    "tlbm_init_fields": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tlbm_conv3x3_pack_weights": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "tlbm_conv3x3_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                       C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "tlbm_conv3x3_backward_data": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.c_int, C.c_void_p, C.c_void_p]),
    "tlbm_conv3x3_status": (C.c_int, [C.POINTER(C.c_ulonglong)]),
    "tlbm_conv3x3_weight_elems": (C.c_int, [C.c_int]),
    "tlbm_conv3x3_workspace_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "tlbm_conv3x3_backward_weight": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                               C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_size_t,
                                               C.c_void_p]),
    "tlbm_relu_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tlbm_to_bf16": (C.c_int, [C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p]),
    "tlbm_mse_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p]),
    "tlbm_adam_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_float, C.c_float,
                                 C.c_float, C.c_float, C.c_int, C.c_void_p]),
    "tlbm_upsample_bilinear": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "tlbm_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_int, C.c_int,
                                    C.POINTER(tlbm_params)]),
    "tlbm_batch_required_bytes": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "tlbm_batch_bind_memory": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "tlbm_batch_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tlbm_batch_init": (C.c_int, [C.c_void_p, C.c_double]),
    "tlbm_batch_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "tlbm_batch_set_variant": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "tlbm_batch_get_variant": (C.c_int, [C.c_void_p] + [C.POINTER(C.c_int)] * 5),
    "tlbm_batch_autotune": (C.c_int, [C.c_void_p, C.c_int]),
    "tlbm_batch_set_staged": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "tlbm_batch_get_staged": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                        C.POINTER(C.c_longlong)]),
    "tlbm_batch_set_persistent": (C.c_int, [C.c_void_p, C.c_int]),
    "tlbm_batch_instance": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "tlbm_batch_nusselt": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "tlbm_batch_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "tlbm_batch_macros": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int]),
    "tlbm_batch_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "tlbm_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "tlbm_batch_destroy": (None, [C.c_void_p]),
    "tlbm_last_error": (C.c_char_p, [C.c_void_p]),
    "tlbm_launch_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "tlbm_destroy": (None, [C.c_void_p]),
}


def _debug_bounds() -> bool:
    return os.environ.get("TLBM_DEBUG_BOUNDS") == "1"


def library_path() -> str:
    """libtlbm.so, or libtlbm_debug.so (every kernel access bounds-checked)
    when the environment sets TLBM_DEBUG_BOUNDS=1."""
    return _build.LIB_DEBUG if _debug_bounds() else _build.LIB


def lib(build_if_missing: bool = True):
    """Load the library (building it first if it is missing or stale).  Raises
    if it cannot be built or loaded: there is no fallback path."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if build_if_missing:
                _build.build(debug=_debug_bounds())
            if not os.path.exists(path):
                raise RuntimeError(f"{os.path.basename(path)} not found at {path}; run the build first")
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name, None)
                if fn is None:
                    continue
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(h, rc):
    if rc != TLBM_OK:
        msg = lib().tlbm_last_error(h)
        raise TlbmError(rc, msg.decode() if msg else "")
    return rc


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ C names

def tlbm_default_params(**overrides) -> tlbm_params:
    p = tlbm_params()
    lib().tlbm_default_params(C.byref(p))
    for k, v in overrides.items():
        if k == "body_force":
            for a in range(3):
                p.body_force[a] = float(v[a])
        else:
            setattr(p, k, v)
    return p


def tlbm_create(nx, ny, nz, lattice, Ra, Pr, Ma, precision, params: tlbm_params | None = None):
    h = C.c_void_p()
    rc = lib().tlbm_create(C.byref(h), int(nx), int(ny), int(nz), int(lattice), float(Ra), float(Pr),
                           float(Ma), int(precision), C.byref(params) if params is not None else None)
    _check(None, rc)
    return h


def tlbm_required_bytes(h) -> int:
    n = C.c_size_t()
    _check(h, lib().tlbm_required_bytes(h, C.byref(n)))
    return n.value


def tlbm_bind_memory(h, dev_ptr: int, nbytes: int):
    _check(h, lib().tlbm_bind_memory(h, C.c_void_p(dev_ptr), nbytes))


def tlbm_set_stream(h, stream_handle: int):
    _check(h, lib().tlbm_set_stream(h, C.c_void_p(stream_handle)))


def tlbm_init(h, seed: int, noise_amp: float):
    _check(h, lib().tlbm_init(h, C.c_uint64(seed), float(noise_amp)))


def tlbm_step(h, n: int):
    _check(h, lib().tlbm_step(h, C.c_int64(n)))


def tlbm_macros(h, rho=None, ux=None, uy=None, uz=None, T=None, out_dtype=TLBM_OUT_F64):
    _check(h, lib().tlbm_macros(h, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(uz), _ptr(T), int(out_dtype)))


def tlbm_nusselt(h, allow_diverged: bool = False) -> float:
    """allow_diverged: return the value of a diverged state instead of raising."""
    v = C.c_double()
    rc = lib().tlbm_nusselt(h, C.byref(v))
    if not (allow_diverged and rc == TLBM_ERR_DIVERGED):
        _check(h, rc)
    return v.value


def tlbm_energy(h, allow_diverged: bool = False):
    e, m = C.c_double(), C.c_double()
    rc = lib().tlbm_energy(h, C.byref(e), C.byref(m))
    if not (allow_diverged and rc == TLBM_ERR_DIVERGED):
        _check(h, rc)
    return e.value, m.value


def tlbm_get_populations(h, host_f, host_g):
    """host_f, host_g: C-contiguous float64 numpy arrays (or None)."""
    fp = None if host_f is None else C.c_void_p(host_f.ctypes.data)
    gp = None if host_g is None else C.c_void_p(host_g.ctypes.data)
    _check(h, lib().tlbm_get_populations(h, fp, gp))


def tlbm_get_populations_window(h, x0, y0, z0, wx, wy, wz, host_f, host_g):
    fp = None if host_f is None else C.c_void_p(host_f.ctypes.data)
    gp = None if host_g is None else C.c_void_p(host_g.ctypes.data)
    _check(h, lib().tlbm_get_populations_window(h, x0, y0, z0, wx, wy, wz, fp, gp))


def tlbm_set_populations(h, host_f, host_g):
    _check(h, lib().tlbm_set_populations(h, C.c_void_p(host_f.ctypes.data), C.c_void_p(host_g.ctypes.data)))


def tlbm_status(h):
    d, s = C.c_int(), C.c_int64()
    _check(h, lib().tlbm_status(h, C.byref(d), C.byref(s)))
    return bool(d.value), s.value


def tlbm_derived(h) -> list:
    buf = (C.c_double * 64)()
    n = C.c_int()
    _check(h, lib().tlbm_derived(h, buf, 64, C.byref(n)))
    return list(buf[: n.value])


def tlbm_set_variant(h, vec=0, form=0, block_x=0, block_y=0, rows=0):
    _check(h, lib().tlbm_set_variant(h, int(vec), int(form), int(block_x), int(block_y), int(rows)))


def tlbm_init_fields(h, T, ux=None, uy=None, uz=None):
    """Warm start from device FP32 tensors of nx*ny*nz values."""
    _check(h, lib().tlbm_init_fields(h, _ptr(T), _ptr(ux), _ptr(uy), _ptr(uz)))


def _cs(stream):
    return C.c_void_p(stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else 0))


def _c(rc):
    if rc != TLBM_OK:
        raise TlbmError(rc, "invalid arguments or CUDA failure")


def tlbm_conv3x3_pack_weights(w, cout, cin, a, stream=None):
    _c(lib().tlbm_conv3x3_pack_weights(_ptr(w), cout, cin, _ptr(a), _cs(stream)))


def tlbm_conv3x3_forward(x, a, bias, y, y_act, B, cin, cout, H, W, relu, stream=None):
    _c(lib().tlbm_conv3x3_forward(_ptr(x), _ptr(a), _ptr(bias), _ptr(y), _ptr(y_act), B, cin, cout, H, W,
                                  int(relu), _cs(stream)))


def tlbm_conv3x3_backward_data(dy, w_bf16, dx, B, cin, cout, H, W, at_workspace, stream=None):
    _c(lib().tlbm_conv3x3_backward_data(_ptr(dy), _ptr(w_bf16), _ptr(dx), B, cin, cout, H, W, _ptr(at_workspace),
                                        _cs(stream)))


def tlbm_conv3x3_weight_elems(cin: int) -> int:
    return int(lib().tlbm_conv3x3_weight_elems(cin))


def tlbm_conv3x3_status() -> int:
    n = C.c_ulonglong()
    _c(lib().tlbm_conv3x3_status(C.byref(n)))
    return n.value


def tlbm_conv3x3_workspace_bytes(B, cin, cout, H, W) -> int:
    n = C.c_size_t()
    _c(lib().tlbm_conv3x3_workspace_bytes(B, cin, cout, H, W, C.byref(n)))
    return n.value


def tlbm_conv3x3_backward_weight(x, dy_bf16, dy, dw, db, B, cin, cout, H, W, workspace, stream=None):
    _c(lib().tlbm_conv3x3_backward_weight(_ptr(x), _ptr(dy_bf16), _ptr(dy), _ptr(dw), _ptr(db), B, cin, cout, H, W,
                                          _ptr(workspace), workspace.numel() * workspace.element_size(),
                                          _cs(stream)))


def tlbm_relu_backward(dx, y, n, g, g_bf16, stream=None):
    _c(lib().tlbm_relu_backward(_ptr(dx), _ptr(y), int(n), _ptr(g), _ptr(g_bf16), _cs(stream)))


def tlbm_to_bf16(a, n, b, stream=None):
    _c(lib().tlbm_to_bf16(_ptr(a), int(n), _ptr(b), _cs(stream)))


def tlbm_mse_loss(y, target, n, g, g_bf16, loss_dev, partial_dev, stream=None):
    _c(lib().tlbm_mse_loss(_ptr(y), _ptr(target), int(n), _ptr(g), _ptr(g_bf16), _ptr(loss_dev), _ptr(partial_dev),
                           _cs(stream)))


def tlbm_adam_step(w, g, m, v, n, lr, b1, b2, eps, t, stream=None):
    _c(lib().tlbm_adam_step(_ptr(w), _ptr(g), _ptr(m), _ptr(v), int(n), float(lr), float(b1), float(b2), float(eps),
                            int(t), _cs(stream)))


def tlbm_upsample_bilinear(x, channels, h, w, factor, out, stream=None):
    _c(lib().tlbm_upsample_bilinear(_ptr(x), channels, h, w, factor, _ptr(out), _cs(stream)))


def tlbm_set_graph(h, steps):
    _check(h, lib().tlbm_set_graph(h, int(steps)))


def tlbm_set_staged(h, tile_width=0, stages=0):
    _check(h, lib().tlbm_set_staged(h, int(tile_width), int(stages)))


def tlbm_get_staged(h):
    """(tile width, stages, blocks) of the staged kernel, zeros for the register kernels."""
    tw, ns, nb = C.c_int(), C.c_int(), C.c_int()
    _check(h, lib().tlbm_get_staged(h, C.byref(tw), C.byref(ns), C.byref(nb)))
    return tw.value, ns.value, nb.value


def tlbm_fp64_fma_rate(stream=None) -> float:
    """Measured FP64 FMA rate of the current device in FLOP/s."""
    v = C.c_double()
    rc = lib().tlbm_fp64_fma_rate(_cs(stream), C.byref(v))
    if rc != 0:
        raise TlbmError(rc, "tlbm_fp64_fma_rate failed")
    return v.value


def tlbm_set_wait_limit(h, seconds):
    _check(h, lib().tlbm_set_wait_limit(h, float(seconds)))


def tlbm_bounds_violations(h) -> int:
    n = C.c_int64()
    _check(h, lib().tlbm_bounds_violations(h, C.byref(n)))
    return n.value


def tlbm_save(h, path):
    _check(h, lib().tlbm_save(h, os.fsencode(path)))


def tlbm_load(h, path):
    _check(h, lib().tlbm_load(h, os.fsencode(path)))


def tlbm_get_variant(h):
    """(vec, form, block_x, block_y, rows)"""
    v = [C.c_int() for _ in range(5)]
    _check(h, lib().tlbm_get_variant(h, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def tlbm_reduce_noalloc(h, state_ptr=None) -> list:
    """The six FP64 diagnostic sums of a state with no device allocation (see
    include/tlbm.h); state_ptr is a device address or None for the current state."""
    out = (C.c_double * 6)()
    _check(h, lib().tlbm_reduce_noalloc(h, None if state_ptr is None else C.c_void_p(state_ptr), out))
    return list(out)


def tlbm_last_error(h) -> str:
    m = lib().tlbm_last_error(h)
    return m.decode() if m else ""


def tlbm_launch_count(h) -> int:
    n = C.c_int64()
    _check(h, lib().tlbm_launch_count(h, C.byref(n)))
    return n.value


def tlbm_destroy(h):
    if h:
        lib().tlbm_destroy(h)


# ------------------------------------------------------------------ convenience

class Sim:
    """One cell on the current CUDA device; device memory is a torch uint8
    tensor bound to the handle."""

    def __init__(self, nx, ny, nz=1, lattice=TLBM_D2Q9_D2Q5, Ra=1e5, Pr=0.71, Ma=0.1, precision=TLBM_FP32,
                 stream=None, **params):
        import torch

        self.lattice = lattice
        self.nx, self.ny = nx, ny
        self.nz = nz if lattice == TLBM_D3Q19_D3Q7 else 1
        self.qf = 9 if lattice == TLBM_D2Q9_D2Q5 else 19
        self.qg = 5 if lattice == TLBM_D2Q9_D2Q5 else 7
        self.N = self.nx * self.ny * self.nz
        self.precision = precision
        self.params = tlbm_default_params(**params)
        self.h = tlbm_create(nx, ny, self.nz, lattice, Ra, Pr, Ma, precision, self.params)
        self.nbytes = tlbm_required_bytes(self.h)
        self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        tlbm_bind_memory(self.h, self.mem.data_ptr(), self.nbytes)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        tlbm_set_stream(self.h, s.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            tlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx) if self.lattice == TLBM_D3Q19_D3Q7 else (self.ny, self.nx)

    def init(self, seed, noise_amp):
        tlbm_init(self.h, seed, noise_amp)

    def step(self, n=1):
        tlbm_step(self.h, n)

    def macros(self, dtype=None) -> dict:
        import torch

        dtype = dtype or torch.float64
        out = {k: torch.empty(self.shape, dtype=dtype, device="cuda") for k in ("rho", "ux", "uy", "uz", "T")}
        tlbm_macros(self.h, out["rho"], out["ux"], out["uy"], out["uz"] if self.lattice else None, out["T"],
                    TLBM_OUT_F64 if dtype == torch.float64 else TLBM_OUT_F32)
        if not self.lattice:
            out["uz"].zero_()
        return out

    def nusselt(self, allow_diverged=False):
        return tlbm_nusselt(self.h, allow_diverged)

    def energy(self, allow_diverged=False):
        return tlbm_energy(self.h, allow_diverged)

    def status(self):
        return tlbm_status(self.h)

    def derived(self) -> dict:
        v = tlbm_derived(self.h)
        d = dict(U=v[0], H=v[1], nu=v[2], alpha=v[3], gbeta=v[4], a_T=v[5], omega=v[6])
        d["S"] = v[7:7 + self.qf]
        d["Q"] = v[7 + self.qf:7 + self.qf + self.qg]
        return d

    def get_populations(self):
        import numpy as np

        f = np.zeros((self.qf,) + self.shape)
        g = np.zeros((self.qg,) + self.shape)
        tlbm_get_populations(self.h, f, g)
        return f, g

    def get_populations_into(self, f, g):
        """Fill preallocated C-contiguous float64 arrays (e.g. pinned host memory)."""
        tlbm_get_populations(self.h, f, g)

    def get_window(self, x0, y0, z0, wx, wy, wz=1):
        import numpy as np

        shp = (wz, wy, wx) if self.lattice == TLBM_D3Q19_D3Q7 else (wy, wx)
        f = np.zeros((self.qf,) + shp)
        g = np.zeros((self.qg,) + shp)
        tlbm_get_populations_window(self.h, x0, y0, z0, wx, wy, wz, f, g)
        return f, g

    def set_populations(self, f, g):
        import numpy as np

        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.size == self.qf * self.N and g.size == self.qg * self.N
        tlbm_set_populations(self.h, f, g)

    def set_variant(self, vec=0, form=0, block_x=0, block_y=0, rows=0):
        tlbm_set_variant(self.h, vec, form, block_x, block_y, rows)

    def set_staged(self, tile_width=0, stages=0):
        tlbm_set_staged(self.h, tile_width, stages)

    def set_wait_limit(self, seconds):
        tlbm_set_wait_limit(self.h, seconds)

    def save(self, path):
        tlbm_save(self.h, path)

    def load(self, path):
        tlbm_load(self.h, path)

    @property
    def variant(self):
        return tlbm_get_variant(self.h)

    @property
    def staged(self):
        return tlbm_get_staged(self.h)

    @property
    def launches(self):
        return tlbm_launch_count(self.h)


# ------------------------------------------------------------------ batched ensemble

def _bcheck(b, rc):
    if rc != TLBM_OK:
        msg = lib().tlbm_batch_last_error(b)
        raise TlbmError(rc, msg.decode() if msg else "")
    return rc


def tlbm_batch_create(instances, lattice, precision, params: tlbm_params | None = None):
    """instances: sequence of (nx, ny, nz, Ra, Pr, Ma, seed)."""
    arr = (tlbm_instance * len(instances))()
    for k, (nx, ny, nz, Ra, Pr, Ma, seed) in enumerate(instances):
        arr[k] = tlbm_instance(int(nx), int(ny), int(nz), float(Ra), float(Pr), float(Ma), int(seed))
    b = C.c_void_p()
    rc = lib().tlbm_batch_create(C.byref(b), len(instances), C.cast(arr, C.c_void_p), int(lattice), int(precision),
                                 C.byref(params) if params is not None else None)
    _bcheck(None, rc)
    return b


def tlbm_batch_required_bytes(b) -> int:
    n = C.c_size_t()
    _bcheck(b, lib().tlbm_batch_required_bytes(b, C.byref(n)))
    return n.value


def tlbm_batch_bind_memory(b, dev_ptr: int, nbytes: int):
    _bcheck(b, lib().tlbm_batch_bind_memory(b, C.c_void_p(dev_ptr), nbytes))


def tlbm_batch_set_stream(b, stream_handle: int):
    _bcheck(b, lib().tlbm_batch_set_stream(b, C.c_void_p(stream_handle)))


def tlbm_batch_init(b, noise_amp: float):
    _bcheck(b, lib().tlbm_batch_init(b, float(noise_amp)))


def tlbm_batch_step(b, n: int):
    _bcheck(b, lib().tlbm_batch_step(b, C.c_int64(n)))


def tlbm_batch_set_variant(b, vec=0, form=0, block_x=0, block_y=0, graph_steps=16):
    _bcheck(b, lib().tlbm_batch_set_variant(b, int(vec), int(form), int(block_x), int(block_y), int(graph_steps)))


def tlbm_batch_get_variant(b):
    v = [C.c_int() for _ in range(5)]
    _bcheck(b, lib().tlbm_batch_get_variant(b, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def tlbm_batch_set_staged(b, consumer_warps: int = 8, stages: int = 0):
    _bcheck(b, lib().tlbm_batch_set_staged(b, int(consumer_warps), int(stages)))


def tlbm_batch_get_staged(b):
    nc, ns, tiles = C.c_int(), C.c_int(), C.c_longlong()
    _bcheck(b, lib().tlbm_batch_get_staged(b, C.byref(nc), C.byref(ns), C.byref(tiles)))
    return nc.value, ns.value, tiles.value


def tlbm_batch_autotune(b, trials: int = 5):
    _bcheck(b, lib().tlbm_batch_autotune(b, int(trials)))


def tlbm_batch_set_persistent(b, steps_per_launch: int):
    _bcheck(b, lib().tlbm_batch_set_persistent(b, int(steps_per_launch)))


def tlbm_batch_set_rows(b, rows: int):
    _bcheck(b, lib().tlbm_batch_set_rows(b, int(rows)))


def tlbm_batch_get_rows(b) -> int:
    r = C.c_int()
    _bcheck(b, lib().tlbm_batch_get_rows(b, C.byref(r)))
    return r.value


def tlbm_batch_set_wait_limit(b, seconds):
    _bcheck(b, lib().tlbm_batch_set_wait_limit(b, float(seconds)))


def tlbm_batch_instance(b, idx: int):
    h = C.c_void_p()
    _bcheck(b, lib().tlbm_batch_instance(b, int(idx), C.byref(h)))
    return h


def tlbm_batch_nusselt(b, n: int, allow_diverged: bool = False) -> list:
    out = (C.c_double * n)()
    rc = lib().tlbm_batch_nusselt(b, out)
    if not (allow_diverged and rc == TLBM_ERR_DIVERGED):
        _bcheck(b, rc)
    return list(out)


def tlbm_batch_status(b, n: int) -> list:
    out = (C.c_int * n)()
    _bcheck(b, lib().tlbm_batch_status(b, out))
    return [bool(v) for v in out]


def tlbm_batch_macros(b, idx, rho=None, ux=None, uy=None, uz=None, T=None, out_dtype=TLBM_OUT_F64):
    _bcheck(b, lib().tlbm_batch_macros(b, int(idx), _ptr(rho), _ptr(ux), _ptr(uy), _ptr(uz), _ptr(T),
                                       int(out_dtype)))


def tlbm_batch_launch_count(b) -> int:
    n = C.c_int64()
    _bcheck(b, lib().tlbm_batch_launch_count(b, C.byref(n)))
    return n.value


def tlbm_batch_last_error(b) -> str:
    m = lib().tlbm_batch_last_error(b)
    return m.decode() if m else ""


def tlbm_batch_destroy(b):
    if b:
        lib().tlbm_batch_destroy(b)


class Batch:
    """An ensemble of independent cells stepped together; device memory is a
    torch uint8 tensor bound to the batch."""

    def __init__(self, instances, lattice=TLBM_D2Q9_D2Q5, precision=TLBM_FP32, stream=None, **params):
        import torch

        self.instances = list(instances)
        self.n = len(self.instances)
        self.lattice = lattice
        self.params = tlbm_default_params(**params)
        self.b = tlbm_batch_create(self.instances, lattice, precision, self.params)
        self.nbytes = tlbm_batch_required_bytes(self.b)
        self.mem = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        tlbm_batch_set_stream(self.b, s.cuda_stream)
        tlbm_batch_bind_memory(self.b, self.mem.data_ptr(), self.nbytes)

    def close(self):
        if getattr(self, "b", None):
            tlbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, noise_amp):
        tlbm_batch_init(self.b, noise_amp)

    def step(self, n=1):
        tlbm_batch_step(self.b, n)

    def set_variant(self, vec=0, form=0, block_x=0, block_y=0, graph_steps=16):
        tlbm_batch_set_variant(self.b, vec, form, block_x, block_y, graph_steps)

    @property
    def variant(self):
        return tlbm_batch_get_variant(self.b)

    def autotune(self, trials=5):
        tlbm_batch_autotune(self.b, trials)

    def set_staged(self, consumer_warps=8, stages=0):
        """Shared-memory staged form (consumer_warps 4 or 8 in 2D, 4 or 7 in 3D; 0 off)."""
        tlbm_batch_set_staged(self.b, consumer_warps, stages)

    @property
    def staged(self):
        """(consumer warps, stages, tiles per step); (0, 0, 0) for the register kernels."""
        return tlbm_batch_get_staged(self.b)

    def set_persistent(self, steps_per_launch):
        tlbm_batch_set_persistent(self.b, steps_per_launch)

    def set_rows(self, rows):
        tlbm_batch_set_rows(self.b, rows)

    @property
    def rows(self):
        return tlbm_batch_get_rows(self.b)

    def set_wait_limit(self, seconds):
        tlbm_batch_set_wait_limit(self.b, seconds)

    def nusselt(self, allow_diverged=False):
        return tlbm_batch_nusselt(self.b, self.n, allow_diverged)

    def status(self):
        return tlbm_batch_status(self.b, self.n)

    def instance(self, idx):
        return tlbm_batch_instance(self.b, idx)

    def get_populations(self, idx):
        import numpy as np

        nx, ny, nz = self.instances[idx][:3]
        shape = (nz, ny, nx) if self.lattice == TLBM_D3Q19_D3Q7 else (ny, nx)
        qf, qg = (9, 5) if self.lattice == TLBM_D2Q9_D2Q5 else (19, 7)
        f = np.zeros((qf,) + shape)
        g = np.zeros((qg,) + shape)
        tlbm_get_populations(self.instance(idx), f, g)
        return f, g

    @property
    def launches(self):
        return tlbm_batch_launch_count(self.b)
