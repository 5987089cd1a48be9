"""ctypes binding of the cmb3d C ABI (include/cmb3d.h).

Argument marshalling only: every step of a realization runs in the CUDA
kernels of libcmb3d.so.  Functions carry the C names; device buffers may be
passed as torch CUDA tensors or raw integer addresses, host arrays as numpy
arrays.  A missing library raises immediately: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcmb3d.so")

CMB3D_OK = 0
CMB3D_EINVAL = -1
CMB3D_ENOMEM = -2
CMB3D_ECUDA = -3
CMB3D_ENOSPEC = -4
CMB3D_ETIMEOUT = -5
CMB3D_EUNSUPPORTED = -6

CMB3D_TRILINEAR = 1
CMB3D_TRICUBIC = 3

CMB3D_FLAG_NONE = 0
CMB3D_FLAG_NO_SORT = 1 << 0
CMB3D_FLAG_ALLOW_WRAP = 1 << 1
CMB3D_FLAG_STAGE_TIMING = 1 << 2
CMB3D_FLAG_THREE_PASS = 1 << 3
CMB3D_FLAG_FUSED_YX = 1 << 4
CMB3D_FLAG_AUTOTUNE = 1 << 5
CMB3D_FLAG_FP16_GEMM = 1 << 6
CMB3D_FLAG_NO_PRUNE = 1 << 7
CMB3D_FLAG_PIPELINE = 1 << 8
CMB3D_FLAG_FUSED_XG = 1 << 9

CMB3D_SPEC_PK = 0
CMB3D_SPEC_CL = 1

CMB3D_STAGE_DRAW_ZFFT = 0
CMB3D_STAGE_YFFT = 1
CMB3D_STAGE_XC2R = 2
CMB3D_STAGE_GATHER = 3
CMB3D_STAGE_YX_FUSED = 4
CMB3D_NUM_STAGES = 5
STAGE_NAMES = ("draw_zfft", "yfft", "xc2r", "gather", "yx_fused")

_vp = C.c_void_p
_i32 = C.c_int
_i64 = C.c_int64
_u32 = C.c_uint32
_u64 = C.c_uint64
_dp = C.POINTER(C.c_double)

# name -> (restype, argtypes); the full exported surface of include/cmb3d.h
PROTOTYPES = {
    "cmb3d_plan": (_i32, [C.POINTER(_vp), _i32, C.c_double, C.c_double, _dp, _i64, _i32, _u32]),
    "cmb3d_plan_2d": (_i32, [C.POINTER(_vp), _i32, _i32, _i32, C.c_double, C.c_double, C.c_double, _dp, _i64,
                             _i32, _u32]),
    "cmb3d_gamma_sqrt_table": (_i32, [_i32, _i32, _i32, C.c_double, _dp, _dp, _i32, C.POINTER(C.c_float)]),
    "cmb3d_set_spectrum": (_i32, [_vp, _i32, _dp, _dp, _i32, _i32, _dp]),
    "cmb3d_fit_pk": (_i32, [_dp, _dp, _i32, _i32, C.c_double, C.c_double, _i32, _dp, _dp, _dp]),
    "cmb3d_lp_system": (_i32, [_dp, _dp, _i32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                               C.c_double, C.POINTER(_i32), C.POINTER(_i32), _dp, _dp, _dp, _dp]),
    "cmb3d_fit_pk_lp": (_i32, [_dp, _dp, _i32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                               C.c_double, _i32, _dp, _dp, C.POINTER(_i32), _dp, _dp]),
    "cmb3d_get_pk": (_i32, [_vp, _dp, _dp, _i32]),
    "cmb3d_cl_matrix": (_i32, [_dp, _i32, _dp, _i32, C.c_double, _dp]),
    "cmb3d_realize_sample": (_i32, [_vp, _u64, _vp, _vp]),
    "cmb3d_realize_sample_to_host": (_i32, [_vp, _u64, _vp, _vp]),
    "cmb3d_realize_samples_to_host": (_i32, [_vp, C.POINTER(_u64), _i32, C.POINTER(_vp), _vp]),
    "cmb3d_realize_sample_batch": (_i32, [C.POINTER(_vp), C.POINTER(_u64), C.POINTER(_vp), _i32, _vp]),
    "cmb3d_batch_debug": (None, [_u32, _i32, _i32]),
    "cmb3d_debug_alloc_limit": (None, [_i64]),
    "cmb3d_debug_poison_boxes": (_i32, [_vp]),
    "cmb3d_draw_spectrum": (_i32, [_vp, _u64, _vp, _vp]),
    "cmb3d_realize_field": (_i32, [_vp, _u64, _vp, _vp]),
    "cmb3d_philox4x32_10": (_i32, [_vp, _u64, _vp, _i64, _vp]),
    "cmb3d_stage_times": (_i32, [_vp, _dp, C.POINTER(_i64), _i32, _i32]),
    "cmb3d_realize_sample_noalloc": (_i32, [_i32, C.c_double, C.c_double, _vp, _i64, _i32, _vp, _u64, _vp, _vp]),
    "cmb3d_plan_info": (_i32, [_vp, C.POINTER(_i32), C.POINTER(_i64), C.POINTER(_i64)]),
    "cmb3d_plan_prune_info": (_i32, [_vp, C.POINTER(_i64), C.POINTER(_i64)]),
    "cmb3d_plan_x_stored": (_i32, [_vp, C.POINTER(_i64)]),
    "cmb3d_pixel_tables_host": (_i32, [_i32, C.c_double, C.c_double, C.c_void_p, _i64, _i32, C.c_uint32,
                                       C.POINTER(_i64)]),
    "cmb3d_plan_schedule": (_i32, [_vp, C.POINTER(_i32)]),
    "cmb3d_batch_schedule": (_i32, [_vp, C.POINTER(_i32), C.POINTER(_i32)]),
    "cmb3d_plan_set_schedule": (_i32, [_vp, C.POINTER(_i32)]),
    "cmb3d_mlp_create": (_i32, [C.POINTER(_vp), _i32, _i32, _i32, _i32, _dp, _vp, _vp, _vp, _i32, _u64]),
    "cmb3d_mlp_train": (_i32, [_vp, _vp, _i64, _i32, _i32, C.c_float, _u64, _vp, _vp]),
    "cmb3d_mlp_predict": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "cmb3d_mlp_loss_grad": (_i32, [_vp, _vp, _i64, _dp, _vp, _vp]),
    "cmb3d_mlp_params": (_i32, [_vp, _vp, _vp, C.POINTER(_i64)]),
    "cmb3d_mlp_destroy": (None, [_vp]),
    "cmb3d_mlp_refine": (_i32, [_vp, _vp, _vp, _i64, _i32, _i32, _vp, _vp]),
    "cmb3d_mlp_gemm": (_i32, [_i32, _i32, _i32, _vp, _i64, _i64, _vp, _i64, _i64, C.c_float, _vp, _i32, _vp, _i64,
                              _i64, _vp]),
    "cmb3d_mlp_error_detail": (C.c_char_p, []),
    "cmb3d_destroy": (None, [_vp]),
    "cmb3d_strerror": (C.c_char_p, [_i32]),
    "cmb3d_error_detail": (C.c_char_p, []),
}

_lib = None


class Cmb3dError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        lib = load()
        msg = lib.cmb3d_strerror(status).decode()
        detail = lib.cmb3d_error_detail().decode()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))


def load(path: str | None = None):
    """Load libcmb3d.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"cmb3d native library not found at {p}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(p)
    for name, (res, args) in PROTOTYPES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(status: int, where: str) -> None:
    if status != CMB3D_OK:
        raise Cmb3dError(status, where)


def _dev_ptr(x) -> int | None:
    """Device address of a torch CUDA tensor, or an integer address as given."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if hasattr(x, "is_cuda") and not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        return x.data_ptr()
    raise TypeError(f"cannot take a device address of {type(x)!r}")


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------
# C-named wrappers
# --------------------------------------------------------------------------

def cmb3d_plan(N: int, L: float, r: float, pix_xyz, interp: int = CMB3D_TRILINEAR,
               flags: int = CMB3D_FLAG_NONE) -> int:
    lib = load()
    pix = _f64(pix_xyz).reshape(-1, 3)
    h = _vp()
    ptr = pix.ctypes.data_as(_dp) if pix.size else None
    _check(lib.cmb3d_plan(C.byref(h), int(N), float(L), float(r), ptr, pix.shape[0], int(interp), int(flags)),
           "cmb3d_plan")
    return h.value


def cmb3d_plan_2d(N: int, M: int, h: int, L: float, r: float, z0: float, pix_xyz, interp: int = CMB3D_TRILINEAR,
                  flags: int = CMB3D_FLAG_NONE) -> int:
    lib = load()
    pix = _f64(pix_xyz).reshape(-1, 3)
    hd = _vp()
    ptr = pix.ctypes.data_as(_dp) if pix.size else None
    _check(lib.cmb3d_plan_2d(C.byref(hd), int(N), int(M), int(h), float(L), float(r), float(z0), ptr, pix.shape[0],
                             int(interp), int(flags)), "cmb3d_plan_2d")
    return hd.value


def cmb3d_gamma_sqrt_table(N: int, M: int, h: int, L: float, k, pk) -> np.ndarray:
    """float32 [(2 (N/2)^2 + 1), h, h]: the 2-D method's per-q square roots."""
    lib = load()
    ka, pa = _f64(k), _f64(pk)
    out = np.zeros((2 * (N // 2) ** 2 + 1, h, h), dtype=np.float32)
    _check(lib.cmb3d_gamma_sqrt_table(int(N), int(M), int(h), float(L), ka.ctypes.data_as(_dp),
                                      pa.ctypes.data_as(_dp), ka.size, out.ctypes.data_as(C.POINTER(C.c_float))),
           "cmb3d_gamma_sqrt_table")
    return out


def cmb3d_set_spectrum(plan: int, kind: int, x, y, nkbins: int = 256) -> float:
    lib = load()
    xa, ya = _f64(x), _f64(y)
    if xa.shape != ya.shape or xa.ndim != 1:
        raise ValueError("x and y must be 1-D arrays of equal length")
    err = C.c_double(0.0)
    _check(lib.cmb3d_set_spectrum(plan, int(kind), xa.ctypes.data_as(_dp), ya.ctypes.data_as(_dp), xa.size,
                                  int(nkbins), C.byref(err)), "cmb3d_set_spectrum")
    return err.value


def cmb3d_fit_pk(ell, cl, N: int, L: float, r: float, nk: int = 256):
    """Host-only C_l -> P_inf(k) inversion; returns (knodes, pk, max relative C_l error)."""
    lib = load()
    ea, ca = _f64(ell), _f64(cl)
    if ea.shape != ca.shape or ea.ndim != 1:
        raise ValueError("ell and cl must be 1-D arrays of equal length")
    kn = np.empty(int(nk))
    pk = np.empty(int(nk))
    err = C.c_double(0.0)
    _check(lib.cmb3d_fit_pk(ea.ctypes.data_as(_dp), ca.ctypes.data_as(_dp), ea.size, int(N), float(L), float(r),
                            int(nk), kn.ctypes.data_as(_dp), pk.ctypes.data_as(_dp), C.byref(err)), "cmb3d_fit_pk")
    return kn, pk, err.value


def _lp_args(ell, cl, R, theta_max, beam, dr, dk, kmax):
    ea, ca = _f64(ell), _f64(cl)
    if ea.shape != ca.shape or ea.ndim != 1:
        raise ValueError("ell and cl must be 1-D arrays of equal length")
    return (ea, ca, (ea.ctypes.data_as(_dp), ca.ctypes.data_as(_dp), ea.size, float(R), float(theta_max),
                     float(beam), float(dr), float(dk), float(kmax)))


def cmb3d_lp_system(ell, cl, R: float, theta_max: float, beam: float = 0.0, dr: float = 0.0, dk: float = 0.0,
                    kmax: float = 0.0):
    """The linear program of the paper's inversion (Sec. II.B) without solving
    it: (r [m], knodes [nk + 1], A [m, nk], b [m])."""
    lib = load()
    ea, ca, head = _lp_args(ell, cl, R, theta_max, beam, dr, dk, kmax)
    m, nk = _i32(0), _i32(0)
    _check(lib.cmb3d_lp_system(*head, C.byref(m), C.byref(nk), None, None, None, None), "cmb3d_lp_system")
    r, kn = np.empty(m.value), np.empty(nk.value + 1)
    A, b = np.empty((m.value, nk.value)), np.empty(m.value)
    _check(lib.cmb3d_lp_system(*head, C.byref(m), C.byref(nk), r.ctypes.data_as(_dp), kn.ctypes.data_as(_dp),
                               A.ctypes.data_as(_dp), b.ctypes.data_as(_dp)), "cmb3d_lp_system")
    return r, kn, A, b


def cmb3d_fit_pk_lp(ell, cl, R: float, theta_max: float, beam: float = 0.0, dr: float = 0.0, dk: float = 0.0,
                    kmax: float = 0.0):
    """The paper's LP inversion (Sec. II.B), host only: returns (knodes, pk,
    objective c^T x, max |A x - b| / |b_0|)."""
    lib = load()
    ea, ca, head = _lp_args(ell, cl, R, theta_max, beam, dr, dk, kmax)
    m, nk = _i32(0), _i32(0)
    _check(lib.cmb3d_lp_system(*head, C.byref(m), C.byref(nk), None, None, None, None), "cmb3d_lp_system")
    cap = nk.value + 1
    kn, pk = np.empty(cap), np.empty(cap)
    obj, err, cnt = C.c_double(0.0), C.c_double(0.0), _i32(0)
    _check(lib.cmb3d_fit_pk_lp(*head, cap, kn.ctypes.data_as(_dp), pk.ctypes.data_as(_dp), C.byref(cnt),
                               C.byref(obj), C.byref(err)), "cmb3d_fit_pk_lp")
    return kn[:cnt.value], pk[:cnt.value], obj.value, err.value


def cmb3d_cl_matrix(ell, knodes, r: float) -> np.ndarray:
    """Forward-relation matrix A (len(ell) x len(knodes)): C_l = A @ P(knodes)."""
    lib = load()
    ea, ka = _f64(ell), _f64(knodes)
    out = np.empty((ea.size, ka.size))
    _check(lib.cmb3d_cl_matrix(ea.ctypes.data_as(_dp), ea.size, ka.ctypes.data_as(_dp), ka.size, float(r),
                               out.ctypes.data_as(_dp)), "cmb3d_cl_matrix")
    return out


def cmb3d_get_pk(plan: int, k) -> np.ndarray:
    lib = load()
    ka = _f64(k)
    out = np.empty_like(ka)
    _check(lib.cmb3d_get_pk(plan, ka.ctypes.data_as(_dp), out.ctypes.data_as(_dp), ka.size), "cmb3d_get_pk")
    return out


def cmb3d_realize_sample(plan: int, seed: int, out_dev, stream=None) -> None:
    lib = load()
    _check(lib.cmb3d_realize_sample(plan, int(seed) & 0xFFFFFFFFFFFFFFFF, _dev_ptr(out_dev), _stream_ptr(stream)),
           "cmb3d_realize_sample")


def cmb3d_realize_sample_to_host(plan: int, seed: int, out_host: np.ndarray, stream=None) -> None:
    lib = load()
    if out_host.dtype != np.float32 or not out_host.flags.c_contiguous:
        raise ValueError("out_host must be a contiguous float32 array")
    _check(lib.cmb3d_realize_sample_to_host(plan, int(seed) & 0xFFFFFFFFFFFFFFFF, out_host.ctypes.data,
                                            _stream_ptr(stream)), "cmb3d_realize_sample_to_host")


def cmb3d_realize_samples_to_host(plan: int, seeds, outs_host, stream=None) -> None:
    """Maps of seeds[i] into the host arrays outs_host[i] (contiguous float32;
    pinned memory lets each download overlap the next map's kernels)."""
    lib = load()
    n = len(seeds)
    if len(outs_host) != n:
        raise ValueError("seeds and outs_host must have equal lengths")
    for o in outs_host:
        if o.dtype != np.float32 or not o.flags.c_contiguous:
            raise ValueError("every output must be a contiguous float32 array")
    hs = (_u64 * max(n, 1))(*[int(s) & 0xFFFFFFFFFFFFFFFF for s in seeds])
    ho = (_vp * max(n, 1))(*[o.ctypes.data for o in outs_host])
    _check(lib.cmb3d_realize_samples_to_host(plan, hs, n, ho, _stream_ptr(stream)), "cmb3d_realize_samples_to_host")


def cmb3d_realize_sample_batch(plans, seeds, outs_dev, stream=None) -> None:
    lib = load()
    B = len(plans)
    if len(seeds) != B or len(outs_dev) != B:
        raise ValueError("plans, seeds and outs_dev must have equal lengths")
    hp = (_vp * B)(*plans)
    hs = (_u64 * B)(*[int(s) & 0xFFFFFFFFFFFFFFFF for s in seeds])
    ho = (_vp * B)(*[_dev_ptr(o) for o in outs_dev])
    _check(lib.cmb3d_realize_sample_batch(hp, hs, ho, B, _stream_ptr(stream)), "cmb3d_realize_sample_batch")


def cmb3d_batch_debug(spin_limit: int = 0, withhold_draw: bool = False, force_form: int = -1) -> None:
    load().cmb3d_batch_debug(int(spin_limit), int(bool(withhold_draw)), int(force_form))


def cmb3d_debug_alloc_limit(nbytes: int) -> None:
    load().cmb3d_debug_alloc_limit(int(nbytes))


def cmb3d_debug_poison_boxes(plan: int) -> None:
    _check(load().cmb3d_debug_poison_boxes(plan), "cmb3d_debug_poison_boxes")


def cmb3d_draw_spectrum(plan: int, seed: int, spec_dev, stream=None) -> None:
    lib = load()
    _check(lib.cmb3d_draw_spectrum(plan, int(seed) & 0xFFFFFFFFFFFFFFFF, _dev_ptr(spec_dev), _stream_ptr(stream)),
           "cmb3d_draw_spectrum")


def cmb3d_realize_field(plan: int, seed: int, field_dev, stream=None) -> None:
    lib = load()
    _check(lib.cmb3d_realize_field(plan, int(seed) & 0xFFFFFFFFFFFFFFFF, _dev_ptr(field_dev), _stream_ptr(stream)),
           "cmb3d_realize_field")


def cmb3d_philox4x32_10(ctr_dev, seed: int, out_dev, n: int, stream=None) -> None:
    lib = load()
    _check(lib.cmb3d_philox4x32_10(_dev_ptr(ctr_dev), int(seed) & 0xFFFFFFFFFFFFFFFF, _dev_ptr(out_dev), int(n),
                                   _stream_ptr(stream)), "cmb3d_philox4x32_10")


CMB3D_NOALLOC_MAX_N = 64


def cmb3d_realize_sample_noalloc(N: int, L: float, r: float, pix_dev, npix: int, interp: int, amp_dev, seed: int,
                                 out_dev, stream=None) -> None:
    """Plan-free map that allocates no device memory (box in a static device
    array; N <= CMB3D_NOALLOC_MAX_N)."""
    lib = load()
    _check(lib.cmb3d_realize_sample_noalloc(int(N), float(L), float(r), _dev_ptr(pix_dev), int(npix), int(interp),
                                            _dev_ptr(amp_dev), int(seed) & 0xFFFFFFFFFFFFFFFF, _dev_ptr(out_dev),
                                            _stream_ptr(stream)), "cmb3d_realize_sample_noalloc")


def cmb3d_stage_times(plan: int, reset: bool = True) -> tuple[np.ndarray, np.ndarray]:
    lib = load()
    ms = np.zeros(CMB3D_NUM_STAGES)
    cnt = np.zeros(CMB3D_NUM_STAGES, dtype=np.int64)
    _check(lib.cmb3d_stage_times(plan, ms.ctypes.data_as(_dp), cnt.ctypes.data_as(C.POINTER(_i64)),
                                 CMB3D_NUM_STAGES, int(bool(reset))), "cmb3d_stage_times")
    return ms, cnt


def cmb3d_plan_info(plan: int) -> tuple[int, int, int]:
    lib = load()
    n, npix, nbytes = _i32(), _i64(), _i64()
    _check(lib.cmb3d_plan_info(plan, C.byref(n), C.byref(npix), C.byref(nbytes)), "cmb3d_plan_info")
    return n.value, npix.value, nbytes.value


def cmb3d_pixel_tables_host(N: int, L: float, r: float, pix_xyz, interp: int, flags: int = 0) -> tuple:
    """(z-planes, rows, stored x reals, gather runs) a 3-D plan with these
    arguments would build; host only."""
    import numpy as np
    lib = load()
    pix = np.ascontiguousarray(pix_xyz, dtype=np.float64).reshape(-1, 3)
    out = (_i64 * 4)()
    _check(lib.cmb3d_pixel_tables_host(int(N), float(L), float(r), pix.ctypes.data if pix.size else None,
                                       int(pix.shape[0]), int(interp), int(flags), out), "cmb3d_pixel_tables_host")
    return tuple(int(v) for v in out)


def cmb3d_plan_x_stored(plan: int) -> int:
    """Reals the x pass of a sky map stores (the column blocks the stencils read)."""
    lib = load()
    reals = _i64()
    _check(lib.cmb3d_plan_x_stored(plan, C.byref(reals)), "cmb3d_plan_x_stored")
    return reals.value


def cmb3d_plan_prune_info(plan: int) -> tuple[int, int]:
    """(z-planes, (z, y) rows) the sky-map path transforms."""
    lib = load()
    planes, rows = _i64(), _i64()
    _check(lib.cmb3d_plan_prune_info(plan, C.byref(planes), C.byref(rows)), "cmb3d_plan_prune_info")
    return planes.value, rows.value


def cmb3d_plan_schedule(plan: int) -> tuple[int, int, int, int]:
    """(draw variant, y variant, x variant, fused variant); -1 marks unused."""
    lib = load()
    out = (_i32 * 4)()
    _check(lib.cmb3d_plan_schedule(plan, out), "cmb3d_plan_schedule")
    return tuple(out)


def cmb3d_batch_schedule(plan: int) -> tuple[int, int]:
    """(form, variant) of the batched path last built with `plan` first."""
    lib = load()
    f, v = _i32(), _i32()
    _check(lib.cmb3d_batch_schedule(plan, C.byref(f), C.byref(v)), "cmb3d_batch_schedule")
    return f.value, v.value


def cmb3d_plan_set_schedule(plan: int, sched) -> None:
    lib = load()
    arr = (_i32 * 4)(*[int(v) for v in sched])
    _check(lib.cmb3d_plan_set_schedule(plan, arr), "cmb3d_plan_set_schedule")


def cmb3d_destroy(plan: int) -> None:
    load().cmb3d_destroy(plan)


def cmb3d_strerror(status: int) -> str:
    return load().cmb3d_strerror(int(status)).decode()


def cmb3d_error_detail() -> str:
    return load().cmb3d_error_detail().decode()


class MlpError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        lib = load()
        super().__init__(f"{where}: {lib.cmb3d_strerror(status).decode()} ({lib.cmb3d_mlp_error_detail().decode()})")


def _mcheck(status: int, where: str) -> None:
    if status != CMB3D_OK:
        raise MlpError(status, where)


def _f32p(a):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return arr, arr.ctypes.data


def cmb3d_mlp_create(n_in, width, depth, n_out, afwd, mu=None, sd=None, out_bias=None, batch_cap=1024, seed=0):
    lib = load()
    A = _f64(afwd).reshape(n_in, n_out)
    keep = [_f32p(mu), _f32p(sd), _f32p(out_bias)]
    h = _vp()
    _mcheck(lib.cmb3d_mlp_create(C.byref(h), int(n_in), int(width), int(depth), int(n_out), A.ctypes.data_as(_dp),
                                 keep[0][1], keep[1][1], keep[2][1], int(batch_cap), int(seed)), "cmb3d_mlp_create")
    return h.value


def cmb3d_mlp_train(mlp, logcl_dev, n, epochs, batch, lr, seed=0, stream=None):
    lib = load()
    losses = np.zeros(max(int(epochs), 1), dtype=np.float32)
    _mcheck(lib.cmb3d_mlp_train(mlp, _dev_ptr(logcl_dev), int(n), int(epochs), int(batch), float(lr), int(seed),
                                losses.ctypes.data, _stream_ptr(stream)), "cmb3d_mlp_train")
    return losses[: int(epochs)]


def cmb3d_mlp_predict(mlp, logcl_dev, n, logpk_dev, stream=None):
    _mcheck(load().cmb3d_mlp_predict(mlp, _dev_ptr(logcl_dev), int(n), _dev_ptr(logpk_dev), _stream_ptr(stream)),
            "cmb3d_mlp_predict")


def cmb3d_mlp_loss_grad(mlp, logcl_dev, n, grad_dev=None, stream=None) -> float:
    loss = C.c_double(0.0)
    _mcheck(load().cmb3d_mlp_loss_grad(mlp, _dev_ptr(logcl_dev), int(n), C.byref(loss), _dev_ptr(grad_dev),
                                       _stream_ptr(stream)), "cmb3d_mlp_loss_grad")
    return loss.value


def cmb3d_mlp_params(mlp, set_values=None):
    lib = load()
    cnt = _i64()
    _mcheck(lib.cmb3d_mlp_params(mlp, None, None, C.byref(cnt)), "cmb3d_mlp_params")
    out = np.empty(cnt.value, dtype=np.float32)
    if set_values is not None:
        arr = np.ascontiguousarray(np.asarray(set_values, dtype=np.float32))
        _mcheck(lib.cmb3d_mlp_params(mlp, None, arr.ctypes.data, None), "cmb3d_mlp_params")
    _mcheck(lib.cmb3d_mlp_params(mlp, out.ctypes.data, None, None), "cmb3d_mlp_params")
    return out


def cmb3d_mlp_destroy(mlp) -> None:
    load().cmb3d_mlp_destroy(mlp)


def cmb3d_mlp_error_detail() -> str:
    return load().cmb3d_mlp_error_detail().decode()


def cmb3d_mlp_refine(mlp, logcl_dev, logpk_dev, n: int, pk_dev, iters: int = 300, power_iters: int = 30,
                     stream=None) -> None:
    """P >= 0 refined from exp(logpk) toward the NNLS optimum of the forward
    relation (FISTA, the network's GEMM kernel); result in pk_dev (not log)."""
    lib = load()
    _mcheck(lib.cmb3d_mlp_refine(mlp, _dev_ptr(logcl_dev), _dev_ptr(logpk_dev), int(n), int(iters), int(power_iters),
                                 _dev_ptr(pk_dev), _stream_ptr(stream)), "cmb3d_mlp_refine")


def cmb3d_mlp_gemm(M: int, N: int, K: int, a, a_strides, b, b_strides, out, out_strides, alpha: float = 1.0,
                   bias=None, gelu: bool = False, stream=None) -> None:
    """The network's BF16 x BF16 -> FP32 product kernel on device FP32 data
    (strides in elements): out[m, n] = f(alpha sum_k a[m, k] b[n, k] + bias[n])."""
    lib = load()
    _mcheck(lib.cmb3d_mlp_gemm(int(M), int(N), int(K), _dev_ptr(a), int(a_strides[0]), int(a_strides[1]), _dev_ptr(b),
                               int(b_strides[0]), int(b_strides[1]), float(alpha), _dev_ptr(bias), int(bool(gelu)),
                               _dev_ptr(out), int(out_strides[0]), int(out_strides[1]), _stream_ptr(stream)),
            "cmb3d_mlp_gemm")


# --------------------------------------------------------------------------
# Convenience object
# --------------------------------------------------------------------------

class Plan:
    """Owns a cmb3d plan handle; methods forward to the C functions."""

    def __init__(self, N, L, r, pix_xyz, interp=CMB3D_TRILINEAR, flags=CMB3D_FLAG_NONE):
        self.handle = cmb3d_plan(N, L, r, pix_xyz, interp, flags)
        self.N = int(N)
        self.npix = int(np.asarray(pix_xyz).reshape(-1, 3).shape[0])

    def set_pk(self, k, pk) -> None:
        cmb3d_set_spectrum(self.handle, CMB3D_SPEC_PK, k, pk)

    def set_cl(self, ell, cl, nkbins: int = 256) -> float:
        return cmb3d_set_spectrum(self.handle, CMB3D_SPEC_CL, ell, cl, nkbins)

    def realize_sample(self, seed, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.npix, dtype=torch.float32, device="cuda")
        cmb3d_realize_sample(self.handle, seed, out, stream)
        return out

    def realize_field(self, seed, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.N, self.N, self.N), dtype=torch.float32, device="cuda")
        cmb3d_realize_field(self.handle, seed, out, stream)
        return out

    def draw_spectrum(self, seed, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.N, self.N, self.N // 2, 2), dtype=torch.float32, device="cuda")
        cmb3d_draw_spectrum(self.handle, seed, out, stream)
        return out

    def close(self) -> None:
        if getattr(self, "handle", None):
            cmb3d_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Plan2D(Plan):
    """Plan of the 2-D Fourier method (h layers of N x N, z-period M, layer 0
    at z0); the same calls as Plan, with the field and hybrid spectrum shaped
    by the layers."""

    def __init__(self, N, M, h, L, r, z0, pix_xyz, interp=CMB3D_TRILINEAR, flags=CMB3D_FLAG_NONE):
        self.handle = cmb3d_plan_2d(N, M, h, L, r, z0, pix_xyz, interp, flags)
        self.N, self.M, self.h = int(N), int(M), int(h)
        self.npix = int(np.asarray(pix_xyz).reshape(-1, 3).shape[0])

    def realize_field(self, seed, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.h, self.N, self.N), dtype=torch.float32, device="cuda")
        cmb3d_realize_field(self.handle, seed, out, stream)
        return out

    def draw_spectrum(self, seed, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((self.h, self.N, self.N // 2, 2), dtype=torch.float32, device="cuda")
        cmb3d_draw_spectrum(self.handle, seed, out, stream)
        return out
