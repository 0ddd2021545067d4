"""Thin Python binding of the C ABI in include/m2l.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: device memory and streams come from PyTorch, all
computation runs in libm2l.so.  Importing this module on a machine without the
built library raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libm2l.so")

M2L_OK, M2L_EINVAL, M2L_ENOMEM, M2L_ECUDA, M2L_ETIMEOUT, M2L_EUNSUPPORTED = range(6)
STATUS_NAMES = {0: "M2L_OK", 1: "M2L_EINVAL", 2: "M2L_ENOMEM", 3: "M2L_ECUDA", 4: "M2L_ETIMEOUT",
                5: "M2L_EUNSUPPORTED"}
M2L_K_INV_R, M2L_K_INV_R4, M2L_K_INV_SQRT_R2C2 = 0, 1, 2
M2L_FP64, M2L_FP32, M2L_TF32, M2L_BF16X3, M2L_TF32X3 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": M2L_FP64, "fp32": M2L_FP32, "tf32": M2L_TF32, "bf16x3": M2L_BF16X3, "tf32x3": M2L_TF32X3}


class M2LError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__("%s: %s: %s" % (fn, STATUS_NAMES.get(status, status), msg))
        self.status = status


class m2l_dlevel(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("width", ctypes.c_double), ("ncells_tgt", ctypes.c_int),
                ("ncells_src", ctypes.c_int), ("n_cones", ctypes.c_int), ("tgt_ijk", ctypes.c_void_p),
                ("src_ijk", ctypes.c_void_p), ("il_offsets", ctypes.c_void_p), ("il_sources", ctypes.c_void_p),
                ("nnz", ctypes.c_int)]


class m2l_kernel(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("c", ctypes.c_double)]


class m2l_level(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("width", ctypes.c_double), ("ncells_tgt", ctypes.c_int),
                ("ncells_src", ctypes.c_int), ("tgt_ijk", ctypes.c_void_p), ("src_ijk", ctypes.c_void_p),
                ("il_offsets", ctypes.c_void_p), ("il_sources", ctypes.c_void_p), ("nnz", ctypes.c_int)]


_lib = None


def lib():
    """The loaded libm2l.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libm2l.so is not built (run __graft_entry__.build() or "
                               "python paper_1210_7292_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sig = {
            "m2l_precompute": [m2l_kernel, I, D, D, ctypes.POINTER(P)],
            "m2l_ops_rebuild": [P, P],
            "m2l_ops_rebuild_tables": [P, P],
            "m2l_ops_rebuild_operators": [P, P],
            "m2l_ops_query": [P, P, P, P],
            "m2l_ops_copy_operators": [P, P],
            "m2l_ops_copy_lowrank": [P, I, P, P],
            "m2l_ops_info": [P, P, P, P, P, P],
            "m2l_apply_level": [P, ctypes.POINTER(m2l_level), P, P, I, I, P],
            "m2l_apply_level_adjoint": [P, ctypes.POINTER(m2l_level), P, P, I, I, P],
            "m2l_classify_level": [P, ctypes.POINTER(m2l_level), P],
            "m2l_apply_classified": [P, P, P, I, I, P],
            "m2l_plan_create": [P, ctypes.POINTER(m2l_level), I, P, ctypes.POINTER(P)],
            "m2l_plan_apply": [P, P, P, I, I, P],
            "m2l_plan_query": [P, P, P, P],
            "m2l_plan_classify": [P, ctypes.POINTER(m2l_level), P],
            "m2l_plan_kernel_info": [P, P, P, P],
            "m2l_fmm_create": [P, I, P, I, I, D, D, P, ctypes.POINTER(P)],
            "m2l_fmm_evaluate": [P, P, P, P, I, P],
            "m2l_fmm_query": [P, I, P, P, P],
            "m2l_fmm_info": [P, P, P, P],
            "m2l_ops_prepare": [P, I, P],
            "m2l_apply_batch": [P, ctypes.POINTER(m2l_level), P, P, I, I, I, P],
            "m2l_build_lists": [I, P, I, P, P, P, P, P],
            "m2l_apply_level_noalloc": [P, ctypes.POINTER(m2l_level), P, P, P],
            "m2l_batch_create": [P, I, P, P, I, I, P, ctypes.POINTER(P)],
            "m2l_batch_run": [P, P],
            "m2l_batch_info": [P, P, P, P],
            "m2l_batch_groups": [P, I, P, P, P, P],
            "m2l_sync_status": [P, P],
            "m2l_ops_set_debug": [P, I],
            "m2l_sa_create": [P, D, I, P, ctypes.POINTER(P)],
            "m2l_sa_info": [P, P, P, P],
            "m2l_sa_copy_factors": [P, P, P, P, P],
            "m2l_sa_apply_level": [P, ctypes.POINTER(m2l_level), P, P, I, I, P],
            "m2l_precompute_aca": [m2l_kernel, I, D, D, ctypes.POINTER(P)],
            "m2l_ops_aca_info": [P, P, P],
            "m2l_precompute_ex": [m2l_kernel, I, D, D, I, I, ctypes.POINTER(P)],
            "m2l_ops_truncation": [P, ctypes.POINTER(I)],
            "m2l_ops_svd_sweeps": [P, P],
            "m2l_dfmm_build_lists": [I, D, D, I, P, I, P, P, P, P, P, P],
            "m2l_dfmm_plan_create": [I, D, ctypes.POINTER(m2l_dlevel), P, ctypes.POINTER(P)],
            "m2l_dfmm_plan_info": [P, P, P, P, P, P],
            "m2l_dfmm_plan_apply": [P, P, P, I, P],
            "m2l_dfmm_plan_prepare": [P, I, P],
            "m2l_dfmm_plan_sync": [P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.m2l_ops_free.argtypes = [P]
        L.m2l_ops_free.restype = None
        L.m2l_plan_free.argtypes = [P]
        L.m2l_plan_free.restype = None
        L.m2l_batch_free.argtypes = [P]
        L.m2l_batch_free.restype = None
        L.m2l_fmm_free.argtypes = [P]
        L.m2l_fmm_free.restype = None
        L.m2l_sa_free.argtypes = [P]
        L.m2l_sa_free.restype = None
        L.m2l_dfmm_plan_free.argtypes = [P]
        L.m2l_dfmm_plan_free.restype = None
        L.m2l_last_error.argtypes = []
        L.m2l_last_error.restype = ctypes.c_char_p
        L.m2l_launch_count.argtypes = []
        L.m2l_launch_count.restype = ctypes.c_int64
        _lib = L
    return _lib


def _check(fn, status):
    if status != M2L_OK:
        raise M2LError(fn, status, lib().m2l_last_error().decode(errors="replace"))


def _stream_ptr(stream, device_index=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream() if device_index is None else torch.cuda.current_stream(device_index)
    elif device_index is not None:
        _check_device(device_index, ("stream", stream))
    return ctypes.c_void_p(stream.cuda_stream)


def _check_device(device_index, *named):
    """Raises ValueError unless every (name, tensor or stream) lives on CUDA
    device `device_index`, the device that owns the operators."""
    for what, t in named:
        if t is None:
            continue
        idx = t.device.index if hasattr(t, "device") else None
        if idx is None or int(idx) != int(device_index):
            raise ValueError("%s is on device %s, the operators on cuda:%d" % (what, idx, int(device_index)))


def _dev_ptr(t, dtype=None, what="tensor"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (what, dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


class Ops:
    """Owner of an m2l_ops handle (freed with the object).  `device` is the CUDA
    device that was current when the operators were built; the library refuses
    to use them from another one."""

    def __init__(self, handle, ell, device=None):
        self.handle = handle
        self.ell = ell
        self.n3 = ell ** 3
        if device is None:
            import torch
            device = torch.cuda.current_device()
        self.device = int(device)

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.m2l_ops_free(h)


class Level:
    """One level's device arrays, kept alive alongside the m2l_level struct."""

    def __init__(self, width, tgt_ijk, src_ijk, il_offsets, il_sources, level=0):
        import torch
        self.tgt_ijk, self.src_ijk = tgt_ijk, src_ijk
        self.il_offsets, self.il_sources = il_offsets, il_sources
        self.width = float(width)
        self.level = int(level)
        for name in ("tgt_ijk", "src_ijk", "il_offsets", "il_sources"):
            _dev_ptr(getattr(self, name), torch.int32, name)
        self.struct = m2l_level(self.level, self.width, int(tgt_ijk.shape[0]), int(src_ijk.shape[0]),
                                tgt_ijk.data_ptr(), src_ijk.data_ptr(), il_offsets.data_ptr(),
                                il_sources.data_ptr(), int(il_sources.numel()))

    @property
    def nnz(self):
        return int(self.struct.nnz)


M2L_TRUNC_FROBENIUS, M2L_TRUNC_SPECTRAL = 0, 1
_TRUNC = {"frobenius": M2L_TRUNC_FROBENIUS, "spectral": M2L_TRUNC_SPECTRAL}


def _trunc_code(truncation):
    if isinstance(truncation, str):
        if truncation not in _TRUNC:
            raise ValueError("truncation must be one of %s, got %r" % (sorted(_TRUNC), truncation))
        return _TRUNC[truncation]
    return int(truncation)


def m2l_precompute(kernel_type, ell, eps=0.0, width=0.0, c=0.0, truncation="frobenius") -> Ops:
    """Operators and tables; low-rank factors at accuracy eps under the
    truncation criterion ("frobenius" or "spectral") when eps > 0."""
    h = ctypes.c_void_p()
    _check("m2l_precompute_ex", lib().m2l_precompute_ex(m2l_kernel(int(kernel_type), float(c)), int(ell), float(eps),
                                                        float(width), _trunc_code(truncation), 0, ctypes.byref(h)))
    return Ops(h, int(ell))


def m2l_precompute_aca(kernel_type, ell, eps=0.0, width=0.0, c=0.0, truncation="frobenius") -> Ops:
    """m2l_precompute with the low-rank factors from ACA + truncated SVD."""
    h = ctypes.c_void_p()
    _check("m2l_precompute_ex", lib().m2l_precompute_ex(m2l_kernel(int(kernel_type), float(c)), int(ell), float(eps),
                                                        float(width), _trunc_code(truncation), 1, ctypes.byref(h)))
    return Ops(h, int(ell))


def m2l_ops_truncation(ops: Ops) -> str:
    """The truncation criterion ops were built with ("frobenius" or "spectral")."""
    v = ctypes.c_int()
    _check("m2l_ops_truncation", lib().m2l_ops_truncation(ops.handle, ctypes.byref(v)))
    return {c: n for n, c in _TRUNC.items()}[v.value]


def m2l_ops_svd_sweeps(ops: Ops):
    """Jacobi sweeps [16] of the SVD of each operator (or ACA core)."""
    sweeps = np.zeros(16, dtype=np.int32)
    _check("m2l_ops_svd_sweeps", lib().m2l_ops_svd_sweeps(ops.handle, sweeps.ctypes.data))
    return sweeps


def m2l_ops_aca_info(ops: Ops):
    """(ACA terms [16], Jacobi sweeps [16]) of ops from m2l_precompute_aca."""
    terms = np.zeros(16, dtype=np.int32)
    sweeps = np.zeros(16, dtype=np.int32)
    _check("m2l_ops_aca_info", lib().m2l_ops_aca_info(ops.handle, terms.ctypes.data, sweeps.ctypes.data))
    return terms, sweeps


def m2l_ops_rebuild(ops: Ops, stream=None):
    _check("m2l_ops_rebuild", lib().m2l_ops_rebuild(ops.handle, _stream_ptr(stream, ops.device)))


def m2l_ops_rebuild_tables(ops: Ops, stream=None):
    _check("m2l_ops_rebuild_tables", lib().m2l_ops_rebuild_tables(ops.handle, _stream_ptr(stream, ops.device)))


def m2l_ops_rebuild_operators(ops: Ops, stream=None):
    _check("m2l_ops_rebuild_operators", lib().m2l_ops_rebuild_operators(ops.handle, _stream_ptr(stream, ops.device)))


def m2l_ops_query(ops: Ops):
    """Returns (ranks [16] int32, sigma [48, ell^3] int16, lut [343] uint16) as numpy arrays."""
    ranks = np.zeros(16, dtype=np.int32)
    sigma = np.zeros((48, ops.n3), dtype=np.int16)
    lut = np.zeros(343, dtype=np.uint16)
    _check("m2l_ops_query", lib().m2l_ops_query(ops.handle, ranks.ctypes.data, sigma.ctypes.data, lut.ctypes.data))
    return ranks, sigma, lut


def m2l_ops_copy_operators(ops: Ops) -> np.ndarray:
    out = np.zeros((16, ops.n3, ops.n3), dtype=np.float64)
    _check("m2l_ops_copy_operators", lib().m2l_ops_copy_operators(ops.handle, out.ctypes.data))
    return out


def m2l_ops_copy_lowrank(ops: Ops, p: int):
    ranks, _, _ = m2l_ops_query(ops)
    r = int(ranks[p])
    U = np.zeros((ops.n3, r))
    V = np.zeros((ops.n3, r))
    _check("m2l_ops_copy_lowrank", lib().m2l_ops_copy_lowrank(ops.handle, int(p), U.ctypes.data, V.ctypes.data))
    return U, V


def m2l_ops_info(ops: Ops):
    ell, kt, hd = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    eps, w = ctypes.c_double(), ctypes.c_double()
    _check("m2l_ops_info", lib().m2l_ops_info(ops.handle, ctypes.byref(ell), ctypes.byref(kt), ctypes.byref(eps),
                                              ctypes.byref(w), ctypes.byref(hd)))
    return {"ell": ell.value, "kernel_type": kt.value, "eps": eps.value, "ref_width": w.value,
            "homogeneity_degree": hd.value}


def _vec_dtypes(precision, out_fp64):
    import torch
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    tin = torch.float64 if p == M2L_FP64 else torch.float32
    tout = torch.float64 if (p == M2L_FP64 or out_fp64) else torch.float32
    return p, tin, tout


def m2l_apply_level(ops: Ops, level: Level, multipoles, locals_, precision="fp32", locals_fp64=False, stream=None):
    p, tin, tout = _vec_dtypes(precision, locals_fp64)
    _check_shapes(ops, multipoles, locals_, level.struct.ncells_src, level.struct.ncells_tgt)
    _check_level_device(ops, level, multipoles, locals_)
    _check("m2l_apply_level", lib().m2l_apply_level(
        ops.handle, ctypes.byref(level.struct), _dev_ptr(multipoles, tin, "multipoles"),
        _dev_ptr(locals_, tout, "locals"), p, int(bool(locals_fp64)), _stream_ptr(stream, ops.device)))


def m2l_classify_level(ops: Ops, level: Level, stream=None):
    _check_level_device(ops, level)
    _check("m2l_classify_level", lib().m2l_classify_level(ops.handle, ctypes.byref(level.struct),
                                                          _stream_ptr(stream, ops.device)))
    ops._classified = (level.struct.ncells_src, level.struct.ncells_tgt)


def m2l_apply_classified(ops: Ops, multipoles, locals_, precision="fp32", locals_fp64=False, stream=None):
    p, tin, tout = _vec_dtypes(precision, locals_fp64)
    nin, nout = getattr(ops, "_classified", (multipoles.shape[0], locals_.shape[0]))
    _check_shapes(ops, multipoles, locals_, nin, nout)
    _check_device(ops.device, ("multipoles", multipoles), ("locals", locals_))
    _check("m2l_apply_classified", lib().m2l_apply_classified(
        ops.handle, _dev_ptr(multipoles, tin, "multipoles"), _dev_ptr(locals_, tout, "locals"), p,
        int(bool(locals_fp64)), _stream_ptr(stream, ops.device)))


def m2l_apply_level_adjoint(ops: Ops, level: Level, grad_locals, grad_multipoles, precision="fp32",
                            grad_fp64=False, stream=None):
    p, tin, tout = _vec_dtypes(precision, grad_fp64)
    _check_shapes(ops, grad_locals, grad_multipoles, level.struct.ncells_tgt, level.struct.ncells_src)
    _check_level_device(ops, level, grad_locals, grad_multipoles)
    _check("m2l_apply_level_adjoint", lib().m2l_apply_level_adjoint(
        ops.handle, ctypes.byref(level.struct), _dev_ptr(grad_locals, tin, "grad_locals"),
        _dev_ptr(grad_multipoles, tout, "grad_multipoles"), p, int(bool(grad_fp64)), _stream_ptr(stream, ops.device)))


def _check_level_device(ops, level, *vectors):
    """The level's arrays and the vectors must be on the operators' device."""
    _check_device(ops.device, *[(n, getattr(level, n)) for n in ("tgt_ijk", "src_ijk", "il_offsets", "il_sources")])
    _check_device(ops.device, *[("vector %d" % i, v) for i, v in enumerate(vectors)])


def _check_shapes(ops, vin, vout, nin, nout):
    if tuple(vin.shape) != (nin, ops.n3) or tuple(vout.shape) != (nout, ops.n3):
        raise ValueError("vector shapes %s -> %s, expected (%d, %d) -> (%d, %d)"
                         % (tuple(vin.shape), tuple(vout.shape), nin, ops.n3, nout, ops.n3))


class Plan:
    def __init__(self, handle, ops, n_in, n_out):
        self.handle, self.ops, self.n_in, self.n_out = handle, ops, n_in, n_out

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.m2l_plan_free(h)


def m2l_plan_create(ops: Ops, level: Level, adjoint=False, stream=None) -> Plan:
    h = ctypes.c_void_p()
    _check_level_device(ops, level)
    _check("m2l_plan_create", lib().m2l_plan_create(ops.handle, ctypes.byref(level.struct), int(bool(adjoint)),
                                                    _stream_ptr(stream, ops.device), ctypes.byref(h)))
    s = level.struct
    n_in, n_out = (s.ncells_tgt, s.ncells_src) if adjoint else (s.ncells_src, s.ncells_tgt)
    plan = Plan(h, ops, n_in, n_out)
    plan.adjoint = bool(adjoint)
    return plan


def m2l_plan_apply(plan: Plan, vin, vout, precision="fp32", out_fp64=False, stream=None):
    p, tin, tout = _vec_dtypes(precision, out_fp64)
    _check_shapes(plan.ops, vin, vout, plan.n_in, plan.n_out)
    _check_device(plan.ops.device, ("input vectors", vin), ("output vectors", vout))
    _check("m2l_plan_apply", lib().m2l_plan_apply(plan.handle, _dev_ptr(vin, tin, "input vectors"),
                                                  _dev_ptr(vout, tout, "output vectors"), p,
                                                  int(bool(out_fp64)), _stream_ptr(stream, plan.ops.device)))


def m2l_plan_classify(plan: Plan, level: Level, stream=None):
    """Re-classify `level` into `plan` on `stream` (no host synchronisation)."""
    _check_level_device(plan.ops, level)
    _check("m2l_plan_classify", lib().m2l_plan_classify(plan.handle, ctypes.byref(level.struct),
                                                        _stream_ptr(stream, plan.ops.device)))
    s = level.struct
    plan.n_in, plan.n_out = ((s.ncells_tgt, s.ncells_src) if getattr(plan, "adjoint", False)
                             else (s.ncells_src, s.ncells_tgt))
    plan.level = level   # the level's device arrays must outlive the stream's use of them


def m2l_ops_prepare(ops: Ops, precision="fp32", stream=None):
    """Build the operators' kernel layouts for `precision` on `stream`."""
    _check("m2l_ops_prepare", lib().m2l_ops_prepare(ops.handle, PRECISIONS[precision], _stream_ptr(stream, ops.device)))


def m2l_plan_query(plan: Plan):
    """Returns (counts [16] int64, records [nvalid, 3] int32: source, target, g)."""
    counts = np.zeros(16, dtype=np.int64)
    nvalid = ctypes.c_int64()
    _check("m2l_plan_query", lib().m2l_plan_query(plan.handle, counts.ctypes.data, None, ctypes.byref(nvalid)))
    rec = np.zeros((max(1, nvalid.value), 3), dtype=np.int32)
    _check("m2l_plan_query", lib().m2l_plan_query(plan.handle, None, rec.ctypes.data, ctypes.byref(nvalid)))
    return counts, rec[:nvalid.value]


def m2l_plan_kernel_info(plan: Plan):
    """{"dense": bool, "units": int, "unit_width": int}: whether the plan's
    tensor-core applies take the target-stationary kernel, and its unit layout."""
    d, u, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check("m2l_plan_kernel_info", lib().m2l_plan_kernel_info(plan.handle, ctypes.byref(d), ctypes.byref(u),
                                                              ctypes.byref(w)))
    return {"dense": bool(d.value), "units": u.value, "unit_width": w.value}


def m2l_apply_batch(ops_list, levels, multipoles, locals_, precision="fp32", locals_fp64=False, stream=None):
    n = len(ops_list)
    p, tin, tout = _vec_dtypes(precision, locals_fp64)
    arr_ops = (ctypes.c_void_p * n)(*[o.handle.value for o in ops_list])
    arr_lv = (m2l_level * n)(*[lv.struct for lv in levels])
    for o, lv, a, b in zip(ops_list, levels, multipoles, locals_):
        _check_shapes(o, a, b, lv.struct.ncells_src, lv.struct.ncells_tgt)
    arr_in = (ctypes.c_void_p * n)(*[_dev_ptr(t, tin, "multipoles").value for t in multipoles])
    arr_out = (ctypes.c_void_p * n)(*[_dev_ptr(t, tout, "locals").value for t in locals_])
    _check("m2l_apply_batch", lib().m2l_apply_batch(arr_ops, arr_lv, arr_in, arr_out, n, p, int(bool(locals_fp64)),
                                                    _stream_ptr(stream)))


class Batch:
    """Owner of an m2l_batch; keeps its plans and vectors alive."""

    def __init__(self, handle, plans, ins, outs):
        self.handle, self.plans, self.ins, self.outs = handle, plans, ins, outs

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.m2l_batch_free(h)


def m2l_batch_create(plans, ins, outs, precision="fp32", out_fp64=False, stream=None) -> Batch:
    """Persistent launches over a fixed set of planned translations: one for the
    CUDA-core precisions, one per order for the tensor-core ones."""
    n = len(plans)
    p, tin, tout = _vec_dtypes(precision, out_fp64)
    for pl, a, b in zip(plans, ins, outs):
        _check_shapes(pl.ops, a, b, pl.n_in, pl.n_out)
    arr_pl = (ctypes.c_void_p * n)(*[pl.handle.value for pl in plans])
    arr_in = (ctypes.c_void_p * n)(*[_dev_ptr(t, tin, "input vectors").value for t in ins])
    arr_out = (ctypes.c_void_p * n)(*[_dev_ptr(t, tout, "output vectors").value for t in outs])
    h = ctypes.c_void_p()
    _check("m2l_batch_create", lib().m2l_batch_create(arr_pl, n, arr_in, arr_out, p, int(bool(out_fp64)),
                                                      _stream_ptr(stream), ctypes.byref(h)))
    return Batch(h, list(plans), list(ins), list(outs))


def m2l_batch_run(batch: Batch, stream=None):
    _check("m2l_batch_run", lib().m2l_batch_run(batch.handle, _stream_ptr(stream)))


def m2l_batch_info(batch: Batch):
    nt, tiles, ms = ctypes.c_int(), ctypes.c_int64(), ctypes.c_double()
    _check("m2l_batch_info", lib().m2l_batch_info(batch.handle, ctypes.byref(nt), ctypes.byref(tiles),
                                                  ctypes.byref(ms)))
    return {"tile_width": nt.value, "tiles": tiles.value, "tuned_ms": ms.value}


def m2l_batch_groups(batch: Batch):
    """[(ell^3, tile width, epilogue groups)] of each launch group of the batch."""
    n = ctypes.c_int32()
    _check("m2l_batch_groups", lib().m2l_batch_groups(batch.handle, 0, None, None, None, ctypes.byref(n)))
    k = max(n.value, 1)
    e3, nt, eg = (np.zeros(k, dtype=np.int32) for _ in range(3))
    _check("m2l_batch_groups", lib().m2l_batch_groups(batch.handle, k, e3.ctypes.data, nt.ctypes.data,
                                                      eg.ctypes.data, ctypes.byref(n)))
    return [(int(e3[i]), int(nt[i]), int(eg[i])) for i in range(n.value)]


def m2l_build_lists(tgt_ijk, src_ijk, stream=None):
    """Returns (il_offsets, il_sources) as device int32 tensors."""
    import torch
    nt, ns = int(tgt_ijk.shape[0]), int(src_ijk.shape[0])
    off = torch.empty(nt + 1, dtype=torch.int32, device=tgt_ijk.device)
    nnz = ctypes.c_int64()
    L = lib()
    _check("m2l_build_lists", L.m2l_build_lists(nt, _dev_ptr(tgt_ijk, torch.int32, "tgt_ijk"), ns,
                                                _dev_ptr(src_ijk, torch.int32, "src_ijk"), _dev_ptr(off), None,
                                                ctypes.byref(nnz), _stream_ptr(stream)))
    src = torch.empty(max(1, nnz.value), dtype=torch.int32, device=tgt_ijk.device)
    _check("m2l_build_lists", L.m2l_build_lists(nt, _dev_ptr(tgt_ijk), ns, _dev_ptr(src_ijk), _dev_ptr(off),
                                                _dev_ptr(src), ctypes.byref(nnz), _stream_ptr(stream)))
    return off, src[:nnz.value]


def m2l_apply_level_noalloc(ops: Ops, level: Level, multipoles, locals_, stream=None):
    """FP32 level translation that allocates no device memory (see include/m2l.h)."""
    import torch
    _check_shapes(ops, multipoles, locals_, level.struct.ncells_src, level.struct.ncells_tgt)
    _check_level_device(ops, level, multipoles, locals_)
    _check("m2l_apply_level_noalloc", lib().m2l_apply_level_noalloc(
        ops.handle, ctypes.byref(level.struct), _dev_ptr(multipoles, torch.float32, "multipoles"),
        _dev_ptr(locals_, torch.float32, "locals"), _stream_ptr(stream, ops.device)))


def m2l_sync_status(ops: Ops, stream=None):
    _check("m2l_sync_status", lib().m2l_sync_status(ops.handle, _stream_ptr(stream, ops.device)))


M2L_DEBUG_STALL_PRODUCER = 1
M2L_DEBUG_NO_DENSE = 2


def m2l_ops_set_debug(ops: Ops, flags: int):
    _check("m2l_ops_set_debug", lib().m2l_ops_set_debug(ops.handle, int(flags)))


def m2l_last_error() -> str:
    return lib().m2l_last_error().decode(errors="replace")


def m2l_launch_count() -> int:
    return int(lib().m2l_launch_count())


class FMM:
    """A bbFMM matvec (tree, per-level lists and M2L plans) built by m2l_fmm_create."""

    def __init__(self, handle, ops_list, n, fp64, ell, leaf):
        self.handle, self.ops_list, self.n, self.fp64, self.ell, self.leaf = handle, ops_list, n, fp64, ell, leaf

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.m2l_fmm_free(h)


def m2l_fmm_create(ops, xyz, leaf_level, lo=-1.0, domain_width=2.0, stream=None) -> FMM:
    """ops: one Ops for every level (homogeneous kernel) or a dict / list by level
    2..leaf_level; xyz: device [n, 3] float64 or float32."""
    import torch
    if isinstance(ops, Ops):
        ops_list = [ops] * (leaf_level - 1)
    elif isinstance(ops, dict):
        ops_list = [ops[L] for L in range(2, leaf_level + 1)]
    else:
        ops_list = list(ops)
    if len(ops_list) != leaf_level - 1:
        raise ValueError("need operators for levels 2..%d" % leaf_level)
    fp64 = xyz.dtype == torch.float64
    if xyz.dtype not in (torch.float64, torch.float32) or xyz.dim() != 2 or xyz.shape[1] != 3:
        raise ValueError("xyz must be a [n, 3] float64 or float32 device tensor")
    arr = (ctypes.c_void_p * len(ops_list))(*[o.handle.value for o in ops_list])
    h = ctypes.c_void_p()
    _check("m2l_fmm_create", lib().m2l_fmm_create(arr, xyz.shape[0], _dev_ptr(xyz, xyz.dtype, "xyz"), int(fp64),
                                                  int(leaf_level), float(lo), float(domain_width),
                                                  _stream_ptr(stream), ctypes.byref(h)))
    return FMM(h, ops_list, xyz.shape[0], fp64, ops_list[0].ell, leaf_level)


def m2l_fmm_evaluate(fmm: FMM, xyz, charges, potentials, precision=None, stream=None):
    """potentials[i] = the FMM's approximation of sum_j K(x_i, x_j) q_j (j != i)."""
    import torch
    dt = torch.float64 if fmm.fp64 else torch.float32
    if precision is None:
        precision = "fp64" if fmm.fp64 else "fp32"
    for t, what in ((xyz, "xyz"), (charges, "charges"), (potentials, "potentials")):
        if t.shape[0] != fmm.n:
            raise ValueError("%s has %d rows, the FMM %d particles" % (what, t.shape[0], fmm.n))
    _check("m2l_fmm_evaluate", lib().m2l_fmm_evaluate(fmm.handle, _dev_ptr(xyz, dt, "xyz"),
                                                      _dev_ptr(charges, dt, "charges"),
                                                      _dev_ptr(potentials, dt, "potentials"),
                                                      PRECISIONS[precision], _stream_ptr(stream)))


def m2l_fmm_info(fmm: FMM):
    """(leaf level, kept cells per level [9], list entries per level [9])."""
    leaf = ctypes.c_int()
    nc = np.zeros(9, dtype=np.int64)
    nz = np.zeros(9, dtype=np.int64)
    _check("m2l_fmm_info", lib().m2l_fmm_info(fmm.handle, ctypes.byref(leaf), nc.ctypes.data, nz.ctypes.data))
    return leaf.value, nc, nz


def m2l_fmm_query(fmm: FMM, level: int):
    """Host (ijk [ncells, 3] int32, W [ncells, ell^3], F [ncells, ell^3]) of a level."""
    _, nc, _ = m2l_fmm_info(fmm)
    n = int(nc[level])
    dt = np.float64 if fmm.fp64 else np.float32
    ijk = np.zeros((max(n, 1), 3), dtype=np.int32)
    W = np.zeros((max(n, 1), fmm.ell ** 3), dtype=dt)
    F = np.zeros((max(n, 1), fmm.ell ** 3), dtype=dt)
    _check("m2l_fmm_query", lib().m2l_fmm_query(fmm.handle, int(level), ijk.ctypes.data, W.ctypes.data,
                                                F.ctypes.data))
    return ijk[:n], W[:n], F[:n]


class SA:
    """SA / SArcmp factors of one operator set (Sec. 4.1), built by m2l_sa_create."""

    def __init__(self, handle, ops, eps, recompress):
        self.handle, self.ops, self.eps, self.recompress = handle, ops, eps, recompress

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.m2l_sa_free(h)


def m2l_sa_create(ops: Ops, eps, recompress=False, stream=None) -> SA:
    h = ctypes.c_void_p()
    _check("m2l_sa_create", lib().m2l_sa_create(ops.handle, float(eps), int(bool(recompress)), _stream_ptr(stream),
                                                ctypes.byref(h)))
    return SA(h, ops, float(eps), bool(recompress))


def m2l_sa_info(sa: SA):
    """(rank r, number of recompressed cores, r_t per t-slot [343] (0: C_t kept whole))."""
    r, nrc = ctypes.c_int(), ctypes.c_int()
    rt = np.zeros(343, dtype=np.int32)
    _check("m2l_sa_info", lib().m2l_sa_info(sa.handle, ctypes.byref(r), ctypes.byref(nrc), rt.ctypes.data))
    return r.value, nrc.value, rt


def m2l_sa_copy_factors(sa: SA):
    """Host FP64 (U [n3, r], B [n3, r], X [343, r, r], Y [343, r, r])."""
    r, _, _ = m2l_sa_info(sa)
    n3 = sa.ops.n3
    Ut = np.zeros((r, n3))
    B = np.zeros((n3, r))
    X = np.zeros((343, r, r))
    Y = np.zeros((343, r, r))
    _check("m2l_sa_copy_factors", lib().m2l_sa_copy_factors(sa.handle, Ut.ctypes.data, B.ctypes.data,
                                                            X.ctypes.data, Y.ctypes.data))
    return Ut.T.copy(), B, X, Y


def m2l_sa_apply_level(sa: SA, level: Level, multipoles, locals_, precision="fp32", locals_fp64=False,
                       stream=None):
    p, tin, tout = _vec_dtypes(precision, locals_fp64)
    _check_shapes(sa.ops, multipoles, locals_, level.struct.ncells_src, level.struct.ncells_tgt)
    _check_level_device(sa.ops, level, multipoles, locals_)
    _check("m2l_sa_apply_level", lib().m2l_sa_apply_level(
        sa.handle, ctypes.byref(level.struct), _dev_ptr(multipoles, tin, "multipoles"),
        _dev_ptr(locals_, tout, "locals"), p, int(bool(locals_fp64)), _stream_ptr(stream, sa.ops.device)))


# ---------------------------------------------------------------- directional FMM (Helmholtz)
def m2l_dfmm_build_lists(level, wavenumber, tgt_ijk, src_ijk=None, domain_width=2.0, stream=None):
    """Directional far-field lists of one level: (n_cones, offsets [ntgt * n_cones + 1],
    sources [nnz]) as device int32 tensors (CSR over target expansions x * n_cones + c)."""
    import torch
    if src_ijk is None:
        src_ijk = tgt_ijk
    for t, what in ((tgt_ijk, "tgt_ijk"), (src_ijk, "src_ijk")):
        _dev_ptr(t, torch.int32, what)
    nt, ns = int(tgt_ijk.shape[0]), int(src_ijk.shape[0])
    C = ctypes.c_int()
    nnz = ctypes.c_int64()
    args = (int(level), float(wavenumber), float(domain_width), nt, _dev_ptr(tgt_ijk), ns, _dev_ptr(src_ijk),
            ctypes.byref(C))
    _check("m2l_dfmm_build_lists", lib().m2l_dfmm_build_lists(*args, None, None, ctypes.byref(nnz),
                                                              _stream_ptr(stream)))
    off = torch.empty(nt * C.value + 1, dtype=torch.int32, device=tgt_ijk.device)
    _check("m2l_dfmm_build_lists", lib().m2l_dfmm_build_lists(*args, _dev_ptr(off), None, ctypes.byref(nnz),
                                                              _stream_ptr(stream)))
    src = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=tgt_ijk.device)
    if nnz.value > 0:
        _check("m2l_dfmm_build_lists", lib().m2l_dfmm_build_lists(*args, _dev_ptr(off), _dev_ptr(src),
                                                                  ctypes.byref(nnz), _stream_ptr(stream)))
    return C.value, off, src[:nnz.value]


class DLevel:
    """One level's directional lists (device arrays kept alive with the struct)."""

    def __init__(self, width, tgt_ijk, src_ijk, n_cones, il_offsets, il_sources, level=0):
        import torch
        self.tgt_ijk, self.src_ijk, self.il_offsets, self.il_sources = tgt_ijk, src_ijk, il_offsets, il_sources
        for name in ("tgt_ijk", "src_ijk", "il_offsets", "il_sources"):
            _dev_ptr(getattr(self, name), torch.int32, name)
        self.n_cones = int(n_cones)
        self.struct = m2l_dlevel(int(level), float(width), int(tgt_ijk.shape[0]), int(src_ijk.shape[0]),
                                 self.n_cones, tgt_ijk.data_ptr(), src_ijk.data_ptr(), il_offsets.data_ptr(),
                                 il_sources.data_ptr(), int(il_sources.numel()))


class DPlan:
    """Owner of an m2l_dplan handle."""

    def __init__(self, handle, ell, n_cones, ntgt, nsrc):
        self.handle, self.ell, self.n_cones, self.ntgt, self.nsrc = handle, ell, n_cones, ntgt, nsrc
        self.n3 = ell ** 3

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.m2l_dfmm_plan_free(h)


def m2l_dfmm_plan_create(ell, wavenumber, level: DLevel, stream=None) -> DPlan:
    h = ctypes.c_void_p()
    _check("m2l_dfmm_plan_create", lib().m2l_dfmm_plan_create(int(ell), float(wavenumber), ctypes.byref(level.struct),
                                                              _stream_ptr(stream), ctypes.byref(h)))
    return DPlan(h, ell, level.n_cones, level.struct.ncells_tgt, level.struct.ncells_src)


def m2l_dfmm_plan_info(plan: DPlan):
    """(T_sym [nsym, 3] int32, n_p [nsym] int64, n_cones, nnz) on the host."""
    nsym, C, nnz = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check("m2l_dfmm_plan_info", lib().m2l_dfmm_plan_info(plan.handle, ctypes.byref(nsym), ctypes.byref(C),
                                                          ctypes.byref(nnz), None, None))
    tsym = np.zeros((max(nsym.value, 1), 3), dtype=np.int32)
    n_p = np.zeros(max(nsym.value, 1), dtype=np.int64)
    _check("m2l_dfmm_plan_info", lib().m2l_dfmm_plan_info(plan.handle, None, None, None, tsym.ctypes.data,
                                                          n_p.ctypes.data))
    return tsym[:nsym.value], n_p[:nsym.value], C.value, nnz.value


def m2l_dfmm_plan_apply(plan: DPlan, multipoles, locals_, precision="fp32", stream=None):
    """locals_ += M2L(multipoles); complex tensors [ncells * n_cones, ell^3] (or
    [ncells, n_cones, ell^3]), complex128 for "fp64", complex64 for the others
    ("fp32" on the CUDA cores; "tf32", "bf16x3", "tf32x3" on the tensor cores)."""
    import torch
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    dt = torch.complex128 if p == M2L_FP64 else torch.complex64
    for t, n, what in ((multipoles, plan.nsrc, "multipoles"), (locals_, plan.ntgt, "locals")):
        if t.numel() != n * plan.n_cones * plan.n3:
            raise ValueError("%s must hold %d x %d x %d values" % (what, n, plan.n_cones, plan.n3))
    _check("m2l_dfmm_plan_apply", lib().m2l_dfmm_plan_apply(plan.handle, _dev_ptr(multipoles, dt, "multipoles"),
                                                            _dev_ptr(locals_, dt, "locals"), p, _stream_ptr(stream)))


def m2l_dfmm_plan_prepare(plan: DPlan, precision, stream=None):
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check("m2l_dfmm_plan_prepare", lib().m2l_dfmm_plan_prepare(plan.handle, p, _stream_ptr(stream)))


def m2l_dfmm_plan_sync(plan: DPlan, stream=None):
    _check("m2l_dfmm_plan_sync", lib().m2l_dfmm_plan_sync(plan.handle, _stream_ptr(stream)))
