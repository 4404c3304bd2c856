"""Thin Python binding of liblcq (ctypes).  Argument marshalling only: every step of the
correction path runs in the library's CUDA kernels.  PyTorch supplies device memory
(input/output tensors) and the CUDA stream.

The names follow the C ABI in include/lcq.h: build_near_lists, gen_corrections,
apply_corrected_S / _D / _CFIE.  Importing this module raises if the library has not
been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblcq.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"liblcq.so not built ({LIB_PATH}); run "
                      "`python -c 'import __graft_entry__ as g; g.build()'` first")
_lib = C.CDLL(LIB_PATH)

LCQ_OK = 0
STATUS = {0: "ok", 1: "invalid argument", 2: "non-finite coordinates", 3: "degenerate patch",
          4: "max_depth reached", 5: "capacity exceeded", 6: "CUDA error", 7: "out of memory",
          8: "tables", 9: "timeout"}
KERNELS = {"S": 0, "D": 1, "CFIE": 2, "Sp": 3}


class LCQError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        super().__init__(f"{what}: {STATUS.get(status, status)} {detail}".strip())
        self.status = status


class Surface_t(C.Structure):
    _fields_ = [("n_patches", C.c_int64), ("deg", C.c_void_p), ("node_off", C.c_void_p),
                ("xyz", C.c_void_p)]


class Params_t(C.Structure):
    _fields_ = [("eps", C.c_double), ("eta", C.c_double), ("eta1", C.c_double),
                ("eps_loosen", C.c_double), ("max_depth", C.c_int32), ("m_max", C.c_int32),
                ("self_order", C.c_int32), ("leaf_order", C.c_int32), ("n_test_dirs", C.c_int32),
                ("test_dirs", C.c_void_p)]


class Physics_t(C.Structure):
    _fields_ = [("k_re", C.c_double), ("k_im", C.c_double), ("alpha_re", C.c_double),
                ("alpha_im", C.c_double), ("beta_re", C.c_double), ("beta_im", C.c_double),
                ("eps", C.c_double)]


_vp, _i64, _i32, _d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
_sig = {
    "lcq_params_default": (None, [_vp]),
    "lcq_create": (C.c_int, [_vp, C.c_int, _vp]),
    "lcq_destroy": (None, [_vp]),
    "lcq_ref_nodes": (C.c_int, [C.c_int, _vp, _vp, _vp]),
    "lcq_build_near_lists": (C.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "lcq_build_near_lists_batched": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp, _vp, _i64, _vp,
                                               _vp]),
    "lcq_near_info": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lcq_near_export": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "lcq_near_destroy": (None, [_vp]),
    "lcq_gen_corrections": (C.c_int, [_vp, _vp, _vp, C.c_int, _d, _d, _d, _d, _d, _d, C.c_int,
                                      _vp, _vp]),
    "lcq_gen_corrections_batched": (C.c_int, [_vp, _vp, _vp, C.c_int, C.c_int, _vp, C.c_int, _vp,
                                              _vp]),
    "lcq_corr_info": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lcq_corr_export": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lcq_corr_export_stats": (C.c_int, [_vp, _vp, _vp, _vp]),
    "lcq_apply_corrected_S": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _d, _vp]),
    "lcq_apply_corrected_D": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _d, _vp]),
    "lcq_apply_corrected_CFIE": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _d, _vp]),
    "lcq_apply_corrected_Sp": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _d, _vp]),
    "lcq_apply_corrected": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, _vp, C.c_int, _d, _vp]),
    "lcq_near_set_target_normals": (C.c_int, [_vp, _vp]),
    "lcq_corr_destroy": (None, [_vp]),
    "lcq_plan_create": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "lcq_plan_launch": (C.c_int, [_vp]),
    "lcq_plan_destroy": (None, [_vp]),
    "lcq_apply_adjoint": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _d, _vp]),
    "lcq_shape_gradient": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "lcq_sync": (C.c_int, [_vp, _i64]),
    "lcq_counters": (C.c_int, [_vp, _vp]),
    "lcq_stage_times": (C.c_int, [_vp, _vp, _vp]),
    "lcq_adaptive_corrections_noalloc": (C.c_int, [C.c_int, _vp, _i64, _vp, C.c_int, _d, _d, _d,
                                                   _d, _d, _d, C.c_int, _d, C.c_int, _vp, _vp]),
    "lcq_pipe_peaks": (C.c_int, [C.c_int, _vp, C.c_int]),
    "lcq_selftest": (C.c_int, [C.c_int, _vp, C.c_int]),
    "lcq_status_string": (C.c_char_p, [C.c_int]),
    "lcq_last_error": (C.c_char_p, [_vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

SYMBOLS = tuple(_sig)


def _ptr(a) -> int:
    if a is None:
        return 0
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def ref_nodes(deg: int):
    """Discretization nodes (u, v) and weights w of degree `deg` (host)."""
    n = (deg + 1) * (deg + 2) // 2
    u, v, w = np.empty(n), np.empty(n), np.empty(n)
    st = _lib.lcq_ref_nodes(deg, _ptr(u), _ptr(v), _ptr(w))
    if st:
        raise LCQError(st, "lcq_ref_nodes")
    return u, v, w


def params(eps: float, eta: float = -1.0, eta1: float = 1.25, eps_loosen: float = 1.0,
           max_depth: int = 24, m_max: int = 24, self_order: int = 0, leaf_order: int = 0,
           test_dirs=None):
    p = Params_t()
    _lib.lcq_params_default(C.byref(p))
    p.eps, p.eta, p.eta1, p.eps_loosen = eps, eta, eta1, eps_loosen
    p.max_depth, p.m_max, p.self_order, p.leaf_order = max_depth, m_max, self_order, leaf_order
    keep = None
    if test_dirs is not None:
        keep = np.ascontiguousarray(test_dirs, dtype=np.float64)
        p.n_test_dirs = keep.shape[0]
        p.test_dirs = keep.ctypes.data
    p._keep = keep
    return p


class Context:
    """lcq_create on a CUDA device with torch's current stream of that device."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.device = device
        self.torch_device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.torch_device)
        self.stream = stream
        h = C.c_void_p()
        st = _lib.lcq_create(C.byref(h), device, C.c_void_p(stream.cuda_stream))
        if st:
            raise LCQError(st, "lcq_create")
        self.h = h

    def check(self, st, what):
        if st:
            raise LCQError(st, what, _lib.lcq_last_error(self.h).decode())

    def sync(self, timeout_ms: int = -1):
        st = _lib.lcq_sync(self.h, timeout_ms)
        return st

    def counters(self):
        out = np.zeros(8, np.int64)
        self.check(_lib.lcq_counters(self.h, _ptr(out)), "lcq_counters")
        return out

    def stage_times(self):
        """(ms per stage [near, far order, smooth+annulus, adaptive, self, v2c], launches)."""
        ms = np.zeros(6, np.float32)
        nl = C.c_int64()
        self.check(_lib.lcq_stage_times(self.h, _ptr(ms), C.byref(nl)), "lcq_stage_times")
        return ms.astype(np.float64), int(nl.value)

    def close(self):
        if getattr(self, "h", None):
            _lib.lcq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DeviceSurface:
    """Surface description: host degrees and offsets, device SoA coordinates [3][N]."""

    def __init__(self, deg, node_off, xyz_dev):
        self.deg = np.ascontiguousarray(deg, dtype=np.int32)
        self.node_off = np.ascontiguousarray(node_off, dtype=np.int64)
        self.xyz = xyz_dev
        self.s = Surface_t(len(self.deg), self.deg.ctypes.data, self.node_off.ctypes.data,
                           xyz_dev.data_ptr())

    @property
    def n_points(self):
        return int(self.node_off[-1])


class NearLists:
    def __init__(self, ctx, h, keep):
        self.ctx, self.h, self._keep = ctx, h, keep
        a = [C.c_int64() for _ in range(4)]
        _lib.lcq_near_info(h, *[C.byref(x) for x in a])
        self.n_pairs, self.n_self, self.n_adaptive, self.nnz = (int(x.value) for x in a)

    def export(self, n_patches: int):
        pp = np.empty(n_patches + 1, np.int64)
        tg = np.empty(max(self.n_pairs, 1), np.int32)
        ad = np.empty(max(self.n_pairs, 1), np.uint8)
        cen = np.empty((n_patches, 3))
        rad = np.empty(n_patches)
        self.ctx.check(_lib.lcq_near_export(self.h, _ptr(pp), _ptr(tg), _ptr(ad), _ptr(cen),
                                            _ptr(rad)), "lcq_near_export")
        return pp, tg[:self.n_pairs], ad[:self.n_pairs].astype(bool), cen, rad

    def set_target_normals(self, normals):
        """Normals of the off-surface targets for S' (device float64 [3][NT])."""
        self._normals = normals
        self.ctx.check(_lib.lcq_near_set_target_normals(self.h, _ptr(normals)),
                       "lcq_near_set_target_normals")

    def close(self):
        if getattr(self, "h", None):
            _lib.lcq_near_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_near_lists(ctx: Context, surf: DeviceSurface, tgt_xyz, tgt_node, prm) -> NearLists:
    nt = int(tgt_node.shape[0])
    h = C.c_void_p()
    ctx.check(_lib.lcq_build_near_lists(ctx.h, C.byref(surf.s), _ptr(tgt_xyz), _ptr(tgt_node), nt,
                                        C.byref(prm), C.byref(h)), "lcq_build_near_lists")
    return NearLists(ctx, h, (surf, tgt_xyz, tgt_node))


def build_near_lists_batched(ctx: Context, surf: DeviceSurface, surface_patch_off, tgt_xyz,
                             tgt_node, prm, tgt_surface=None) -> NearLists:
    """Near lists of a batch of independent surfaces: surface s owns patches
    [surface_patch_off[s], surface_patch_off[s+1]); targets pair only with their own
    surface (off-surface targets: tgt_surface, device int32, or surface 0)."""
    off = np.ascontiguousarray(surface_patch_off, dtype=np.int64)
    nt = int(tgt_node.shape[0])
    h = C.c_void_p()
    ctx.check(_lib.lcq_build_near_lists_batched(ctx.h, C.byref(surf.s), len(off) - 1, _ptr(off),
                                                _ptr(tgt_xyz), _ptr(tgt_node), _ptr(tgt_surface),
                                                nt, C.byref(prm), C.byref(h)),
              "lcq_build_near_lists_batched")
    nl = NearLists(ctx, h, (surf, tgt_xyz, tgt_node, tgt_surface, off))
    nl.n_surfaces = len(off) - 1
    return nl


class Corrections:
    def __init__(self, ctx, h, near, kernel):
        self.ctx, self.h, self.near, self.kernel = ctx, h, near, kernel

    def info(self):
        nnz, nover, dt = C.c_int64(), C.c_int64(), C.c_int()
        self.ctx.check(_lib.lcq_corr_info(self.h, C.byref(nnz), C.byref(nover), C.byref(dt)),
                       "lcq_corr_info")
        return int(nnz.value), int(nover.value)

    def export(self, n_targets: int, out=None):
        """CSR (row_ptr, col, val) to host; `out` may supply preallocated arrays: pinned host
        arrays or device tensors (int64, int32, complex128)."""
        nnz = self.near.nnz
        if out is None:
            out = (np.empty(n_targets + 1, np.int64), np.empty(max(nnz, 1), np.int32),
                   np.empty(max(nnz, 1), np.complex128))
        rp, col, val = out
        self.ctx.check(_lib.lcq_corr_export(self.h, _ptr(rp), _ptr(col), _ptr(val)),
                       "lcq_corr_export")
        return (rp, None if col is None else col[:nnz], None if val is None else val[:nnz])

    def stats(self, n_patches: int):
        q = np.empty(n_patches, np.int32)
        qn = np.empty(n_patches, np.int32)
        lv = np.empty(max(self.near.n_pairs, 1), np.int32)
        self.ctx.check(_lib.lcq_corr_export_stats(self.h, _ptr(q), _ptr(qn), _ptr(lv)),
                       "lcq_corr_export_stats")
        return q, qn, lv[:self.near.n_pairs]

    def close(self):
        if getattr(self, "h", None):
            _lib.lcq_corr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PRECISIONS = {"fp64": 0, "mixed": 1}


class Plan:
    """A captured regeneration of `corr` (lcq_plan_create): launch() regenerates it in place
    from the current node coordinates of `surf` with one CUDA graph launch."""

    def __init__(self, ctx: Context, surf: DeviceSurface, near: NearLists, corr: Corrections):
        h = C.c_void_p()
        ctx.check(_lib.lcq_plan_create(ctx.h, C.byref(surf.s), near.h, corr.h, C.byref(h)),
                  "lcq_plan_create")
        self.ctx, self.h, self._keep = ctx, h, (surf, near, corr)

    def launch(self):
        self.ctx.check(_lib.lcq_plan_launch(self.h), "lcq_plan_launch")

    def close(self):
        if getattr(self, "h", None):
            _lib.lcq_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gen_corrections(ctx: Context, surf: DeviceSurface, near: NearLists, kernel: str, k,
                    prm, alpha=1.0, beta=0.0, precision: str = "fp64") -> Corrections:
    k, alpha, beta = complex(k), complex(alpha), complex(beta)
    h = C.c_void_p()
    ctx.check(_lib.lcq_gen_corrections(ctx.h, C.byref(surf.s), near.h, KERNELS[kernel], k.real,
                                       k.imag, alpha.real, alpha.imag, beta.real, beta.imag,
                                       PRECISIONS[precision], C.byref(prm), C.byref(h)),
              "lcq_gen_corrections")
    return Corrections(ctx, h, near, kernel)


def gen_corrections_batched(ctx: Context, surf: DeviceSurface, near: NearLists, kernel: str,
                            physics, prm, precision: str = "fp64") -> Corrections:
    """lcq_gen_corrections_batched; physics: one (k, alpha, beta, eps) per surface."""
    arr = (Physics_t * len(physics))()
    for i, (k, alpha, beta, eps) in enumerate(physics):
        k, alpha, beta = complex(k), complex(alpha), complex(beta)
        arr[i] = Physics_t(k.real, k.imag, alpha.real, alpha.imag, beta.real, beta.imag,
                           float(eps))
    h = C.c_void_p()
    ctx.check(_lib.lcq_gen_corrections_batched(ctx.h, C.byref(surf.s), near.h, KERNELS[kernel],
                                               len(physics), arr, PRECISIONS[precision],
                                               C.byref(prm), C.byref(h)),
              "lcq_gen_corrections_batched")
    return Corrections(ctx, h, near, kernel)


def _apply(fn, ctx, surf, near, corr, sigma, jump, out):
    ctx.check(fn(ctx.h, C.byref(surf.s), near.h, corr.h, _ptr(sigma), float(jump), _ptr(out)),
              fn.__name__)
    return out


def _out_like(ctx, near_nt):
    import torch
    return torch.empty(near_nt, dtype=torch.complex128, device=ctx.torch_device)


def apply_corrected_S(ctx, surf, near, corr, sigma, n_targets, jump=0.0):
    return _apply(_lib.lcq_apply_corrected_S, ctx, surf, near, corr, sigma, jump,
                  _out_like(ctx, n_targets))


def apply_corrected_D(ctx, surf, near, corr, sigma, n_targets, jump=0.0):
    return _apply(_lib.lcq_apply_corrected_D, ctx, surf, near, corr, sigma, jump,
                  _out_like(ctx, n_targets))


def apply_corrected_CFIE(ctx, surf, near, corr, sigma, n_targets, jump=0.0):
    return _apply(_lib.lcq_apply_corrected_CFIE, ctx, surf, near, corr, sigma, jump,
                  _out_like(ctx, n_targets))


def apply_adjoint(ctx, surf, near, corr, g, jump=0.0):
    """A^H g (device complex128 [N]) for the operator of apply_corrected_* with `jump`."""
    import torch
    out = torch.empty(surf.n_points, dtype=torch.complex128, device=ctx.torch_device)
    ctx.check(_lib.lcq_apply_adjoint(ctx.h, C.byref(surf.s), near.h, corr.h, _ptr(g), float(jump),
                                     _ptr(out)), "lcq_apply_adjoint")
    return out


def shape_gradient(ctx, surf, near, corr, sigma, g):
    """dL/dy (device float64 [3][N]) for dL = Re sum conj(g) du at off-surface targets."""
    import torch
    out = torch.empty((3, surf.n_points), dtype=torch.float64, device=ctx.torch_device)
    ctx.check(_lib.lcq_shape_gradient(ctx.h, C.byref(surf.s), near.h, corr.h, _ptr(sigma), _ptr(g),
                                      _ptr(out)), "lcq_shape_gradient")
    return out


def apply_corrected(ctx, surf, near, corr, sigma, n_targets, jump=0.0):
    """The corrected potential for the corrections' kernel; sigma complex128 or complex64."""
    import torch
    dt = {torch.complex128: 0, torch.complex64: 1}[sigma.dtype]
    out = _out_like(ctx, n_targets)
    ctx.check(_lib.lcq_apply_corrected(ctx.h, C.byref(surf.s), near.h, corr.h,
                                       KERNELS[corr.kernel], _ptr(sigma), dt, float(jump),
                                       _ptr(out)), "lcq_apply_corrected")
    return out


def apply_corrected_Sp(ctx, surf, near, corr, sigma, n_targets, jump=0.0):
    return _apply(_lib.lcq_apply_corrected_Sp, ctx, surf, near, corr, sigma, jump,
                  _out_like(ctx, n_targets))


def adaptive_corrections_noalloc(deg, y_dev, tgt_dev, kernel, k, q, eps, out, alpha=1.0, beta=0.0,
                                 max_depth=16, stream=None):
    """lcq_adaptive_corrections_noalloc: one patch's adaptive near corrections into the
    caller's `out` (device complex128 [n_targets][n]); the library allocates nothing."""
    import torch
    k, alpha, beta = complex(k), complex(alpha), complex(beta)
    if stream is None:
        stream = torch.cuda.current_stream(y_dev.device)
    return _lib.lcq_adaptive_corrections_noalloc(
        deg, _ptr(y_dev), int(tgt_dev.shape[1]), _ptr(tgt_dev), KERNELS[kernel], k.real, k.imag,
        alpha.real, alpha.imag, beta.real, beta.imag, int(q), float(eps), int(max_depth),
        C.c_void_p(stream.cuda_stream), _ptr(out))


PEAK_KEYS = ("fp64_fma_tflops", "fp32_fma_tflops", "mufu_sin_tops", "int32_tops",
             "mma_f64_tflops", "mma_f16_tflops", "mma_bf16_tflops", "mma_tf32_tflops")


def pipe_peaks(device: int = 0) -> dict:
    """Measured pipe throughputs on `device` (lcq_pipe_peaks), keyed by PEAK_KEYS."""
    out = np.zeros(len(PEAK_KEYS))
    st = _lib.lcq_pipe_peaks(device, _ptr(out), len(PEAK_KEYS))
    if st:
        raise LCQError(st, "lcq_pipe_peaks")
    return dict(zip(PEAK_KEYS, out.tolist()))


def selftest(device: int = 0) -> dict:
    """Device self-checks (lcq_selftest): sincos table error, tensor-core contraction error,
    two-float kernel value and sincos errors."""
    out = np.zeros(5)
    st = _lib.lcq_selftest(device, _ptr(out), 5)
    if st:
        raise LCQError(st, "lcq_selftest")
    return {"sincos_abs_err": float(out[0]), "tc_rel_err_d6": float(out[1]),
            "tc_rel_err_d10": float(out[2]), "ff_kernel_rel_err": float(out[3]),
            "ff_sincos_err": float(out[4])}
