"""Python binding of libstag, the GB300 (sm_103a) even-odd improved-staggered solver library.

The functions carry the C ABI's names (``include/stag.h``) and only marshal
arguments: PyTorch CUDA tensors become device pointers and the current
PyTorch stream becomes the ``cudaStream_t``.  Every step of the computation
runs in the library's own CUDA kernels; there is no CPU fallback, and
importing this package fails loudly if ``libstag.so`` has not been built
(``python -c "import __graft_entry__ as g; g.build()"``).

Field tensors are complex128 CUDA tensors in the canonical layout: links
``[V][4][3][3]``, single-parity colour vectors ``[V/2][3]`` (or
``[nrhs][V/2][3]``), sites lexicographic with x fastest, a parity field
indexed by lex // 2.
"""

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# STAG_LIBRARY may name another build of the library (the bounds-checked
# libstag_debug.so next to this file); default libstag.so
LIB_PATH = os.environ.get("STAG_LIBRARY") or os.path.join(_HERE, "libstag.so")

STAG_OK = 0
STAG_EINVAL = -1
STAG_ENOMEM = -2
STAG_ECUDA = -3
STAG_ENOTCONV = -4
STAG_EBREAKDOWN = -5
STAG_ENOTUNITARY = -6
STAG_ETIMEOUT = -7

STAG_FP64, STAG_FP32, STAG_FP16, STAG_FX16, STAG_DF64, STAG_FX16L32 = 0, 1, 2, 3, 4, 5
STAG_PLAIN64, STAG_MIXED32, STAG_MIXED16, STAG_MIXEDFX16, STAG_LEARNED, STAG_MIXED16L = 0, 1, 2, 3, 4, 5

PREC = {"fp64": STAG_FP64, "fp32": STAG_FP32, "fp16": STAG_FP16, "fx16": STAG_FX16, "df64": STAG_DF64,
        "fx16l": STAG_FX16L32}
MODE = {
    "plain64": STAG_PLAIN64,
    "mixed32": STAG_MIXED32,
    "mixed16": STAG_MIXED16,
    "mixedfx16": STAG_MIXEDFX16,
    "learned": STAG_LEARNED,
    "mixed16l": STAG_MIXED16L,
}

# every entry point declared in include/stag.h
EXPORTS = (
    "stag_default_params",
    "stag_load_links",
    "stag_free_lattice",
    "stag_lattice_info",
    "stag_tuned_shape",
    "stag_dslash",
    "stag_apply_m",
    "stag_apply_m_noalloc",
    "stag_cg",
    "stag_multishift_cg",
    "stag_batch_solve",
    "stag_net_create",
    "stag_net_free",
    "stag_net_num_params",
    "stag_net_get_params",
    "stag_net_set_params",
    "stag_net_apply",
    "stag_net_loss_grad",
    "stag_net_train",
    "stag_tc_selftest",
    "stag_build_links",
    "stag_gauge_force",
    "stag_fermion_force",
    "stag_strerror",
    "stag_profile_enable",
    "stag_profile_select",
    "stag_profile_reset",
    "stag_profile_read",
    "stag_launch_count",
    "stag_tuned_mrhs",
    "stag_tuned_mrhs_epi",
    "stag_tuned_mrhs_variant",
    "stag_tune_key",
    "stag_tune_cache_get",
    "stag_tune_cache_put",
    "stag_tune_cache_load",
    "stag_tune_cache_save",
    "stag_tune_cache_clear",
    "stag_tune_cache_size",
    "stag_dd_create",
    "stag_dd_free",
    "stag_dd_info",
    "stag_dd_dslash",
    "stag_dd_apply_m",
    "stag_dd_cg",
    "stag_bounds_violations",
)


class StagError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


class LinkOpts(ctypes.Structure):
    _fields_ = [
        ("recon_long", ctypes.c_int),
        ("long_coeff", ctypes.c_double),
        ("prec_mask", ctypes.c_uint),
        ("autotune", ctypes.c_int),
    ]


class SolveParams(ctypes.Structure):
    _fields_ = [
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("mode", ctypes.c_int),
        ("delta", ctypes.c_double),
        ("use_initial_guess", ctypes.c_int),
        ("check_interval", ctypes.c_int),
        ("ms_tol", ctypes.c_double),
        ("precond", ctypes.c_void_p),
    ]


class BatchItem(ctypes.Structure):
    _fields_ = [
        ("lat", ctypes.c_void_p),
        ("x", ctypes.c_void_p),
        ("b", ctypes.c_void_p),
        ("nrhs", ctypes.c_int),
        ("mass", ctypes.c_double),
    ]


class TrainPair(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_void_p), ("r", ctypes.c_void_p), ("e", ctypes.c_void_p)]


class TrainParams(ctypes.Structure):
    _fields_ = [
        ("epochs", ctypes.c_int),
        ("batch", ctypes.c_int),
        ("lr", ctypes.c_double),
        ("seed", ctypes.c_ulonglong),
        ("pair_prec", ctypes.c_int),
        ("loss", ctypes.c_int),
        ("mass", ctypes.c_double),
    ]


LOSS = {"error": 0, "residual": 1}


class SolveInfo(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("reliable_updates", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("status", ctypes.c_int),
        ("true_rel_resid", ctypes.c_double),
        ("seconds", ctypes.c_double),
        ("precond_fallback", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: the CUDA library must be built first "
            '(python -c "import __graft_entry__ as g; g.build()")'
        )
    lib = ctypes.CDLL(path)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "stag_default_params": (None, [ctypes.POINTER(SolveParams)]),
        "stag_load_links": (ci, [ctypes.POINTER(vp), ctypes.POINTER(ci), vp, vp, ctypes.POINTER(LinkOpts), vp]),
        "stag_free_lattice": (ci, [vp]),
        "stag_lattice_info": (ci, [vp, ctypes.POINTER(ci), ctypes.POINTER(ctypes.c_longlong)]),
        "stag_tuned_shape": (ci, [vp, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(cd)]),
        "stag_dslash": (ci, [vp, vp, vp, ci, ci, ci, vp]),
        "stag_apply_m": (ci, [vp, vp, vp, cd, cd, ci, vp]),
        "stag_apply_m_noalloc": (ci, [vp, vp, vp, cd, cd, vp]),
        "stag_cg": (ci, [vp, vp, vp, cd, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), vp]),
        "stag_multishift_cg": (
            ci,
            [vp, ctypes.POINTER(vp), vp, cd, ctypes.POINTER(cd), ci, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), vp],
        ),
        "stag_batch_solve": (ci, [ctypes.POINTER(BatchItem), ci, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), vp]),
        "stag_net_create": (ci, [ctypes.POINTER(vp), ctypes.POINTER(ci), ci, ctypes.c_ulonglong]),
        "stag_net_free": (ci, [vp]),
        "stag_net_num_params": (ctypes.c_longlong, [vp]),
        "stag_net_get_params": (ci, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_longlong, ci]),
        "stag_net_set_params": (ci, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_longlong]),
        "stag_net_apply": (ci, [vp, vp, vp, vp, vp]),
        "stag_net_loss_grad": (
            ci,
            [vp, vp, vp, vp, ci, cd, ctypes.POINTER(cd), ctypes.POINTER(ctypes.c_float), ctypes.c_longlong, vp],
        ),
        "stag_net_train": (ci, [vp, ctypes.POINTER(TrainPair), ci, ctypes.POINTER(TrainParams), ctypes.POINTER(cd), vp]),
        "stag_tc_selftest": (ci, [ctypes.POINTER(cd)]),
        "stag_build_links": (ci, [ctypes.POINTER(ci), vp, vp, vp, cd, cd, cd, vp]),
        "stag_gauge_force": (ci, [ctypes.POINTER(ci), vp, vp, cd, cd, cd, cd, vp]),
        "stag_fermion_force": (ci, [ctypes.POINTER(ci), vp, ci, vp, vp, ctypes.POINTER(cd), cd, cd, cd, vp, vp]),
        "stag_strerror": (ctypes.c_char_p, [ci]),
        "stag_profile_enable": (ci, [ci]),
        "stag_profile_select": (ci, [ctypes.c_char_p, ci]),
        "stag_profile_reset": (ci, []),
        "stag_profile_read": (ci, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(cd)]),
        "stag_launch_count": (ctypes.c_longlong, []),
        "stag_tuned_mrhs": (ci, [vp, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(cd)]),
        "stag_tuned_mrhs_epi": (ci, [vp, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(cd)]),
        "stag_tuned_mrhs_variant": (ci, [vp, ci, ci, ci]),
        "stag_tune_key": (ci, [ctypes.c_char_p, ci, ctypes.c_char_p, ci, ci, ci, ctypes.POINTER(ci)]),
        "stag_tune_cache_get": (ci, [ctypes.c_char_p, ctypes.POINTER(ci), ctypes.POINTER(cd)]),
        "stag_tune_cache_put": (ci, [ctypes.c_char_p, ci, cd]),
        "stag_tune_cache_load": (ci, [ctypes.c_char_p]),
        "stag_tune_cache_save": (ci, [ctypes.c_char_p]),
        "stag_tune_cache_clear": (ci, []),
        "stag_tune_cache_size": (ctypes.c_longlong, []),
        "stag_dd_create": (ci, [ctypes.POINTER(vp), ctypes.POINTER(ci), ci, ci, vp, vp, ctypes.POINTER(LinkOpts), vp]),
        "stag_dd_free": (ci, [vp]),
        "stag_dd_info": (ci, [vp, ctypes.POINTER(ci), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ci)]),
        "stag_dd_dslash": (ci, [vp, vp, vp, ci, vp, vp]),
        "stag_dd_apply_m": (ci, [vp, vp, vp, cd, vp, vp]),
        "stag_dd_cg": (ci, [vp, vp, vp, cd, ctypes.POINTER(SolveParams), ctypes.POINTER(SolveInfo), vp, vp]),
        "stag_bounds_violations": (ci, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ci),
                                        ctypes.POINTER(ctypes.c_longlong), ci]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def strerror(status):
    return _lib.stag_strerror(int(status)).decode()


def _check(status, where):
    if status != STAG_OK:
        raise StagError(status, where)


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t, name, numel=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda or t.dtype != torch.complex128 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _prec(p):
    return PREC[p] if isinstance(p, str) else int(p)


def default_params(**kw):
    p = SolveParams()
    _lib.stag_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "mode" and isinstance(v, str):
            v = MODE[v]
        if k == "precond" and isinstance(v, NetHandle):
            v = v.ptr.value
        setattr(p, k, v)
    return p


class LatticeHandle:
    """Owns a ``stag_lattice_t``; released by :func:`stag_free_lattice` or on GC."""

    def __init__(self, ptr, dims):
        self.ptr = ctypes.c_void_p(ptr)
        self.dims = tuple(dims)
        V = 1
        for d in dims:
            V *= d
        self.V = V
        self.Vh = V // 2

    def free(self):
        if self.ptr and self.ptr.value:
            _check(_lib.stag_free_lattice(self.ptr), "stag_free_lattice")
            self.ptr = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def stag_load_links(dims, fat, lng, recon_long=18, long_coeff=-1.0 / 24.0, prec_mask=0, autotune=True, stream=None):
    """Copy canonical fat/long links into a new lattice handle (see stag.h)."""
    dims = tuple(int(d) for d in dims)
    V = dims[0] * dims[1] * dims[2] * dims[3]
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*dims)
    o = LinkOpts(int(recon_long), float(long_coeff), int(prec_mask), 1 if autotune else 0)
    st = _lib.stag_load_links(
        ctypes.byref(h), d, _ptr(fat, "fat", V * 36), _ptr(lng, "lng", V * 36), ctypes.byref(o), _stream(stream)
    )
    _check(st, "stag_load_links")
    return LatticeHandle(h.value, dims)


def stag_free_lattice(h):
    h.free()


def stag_tuned_shape(h, prec, kernel=0):
    """(threads per block, min blocks per SM, us per launch) kept by the autotuner."""
    b, m, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(_lib.stag_tuned_shape(h.ptr, _prec(prec), int(kernel), ctypes.byref(b), ctypes.byref(m), ctypes.byref(us)), "stag_tuned_shape")
    return b.value, m.value, us.value


def stag_lattice_info(h):
    d = (ctypes.c_int * 4)()
    vh = ctypes.c_longlong()
    _check(_lib.stag_lattice_info(h.ptr, d, ctypes.byref(vh)), "stag_lattice_info")
    return tuple(d), vh.value


def stag_dslash(h, out, inp, out_parity, prec="fp64", nrhs=1, stream=None):
    """out = D inp on parity out_parity (canonical [nrhs][V/2][3] complex128)."""
    n = h.Vh * 3 * nrhs
    st = _lib.stag_dslash(
        h.ptr, _ptr(out, "out", n), _ptr(inp, "inp", n), int(out_parity), _prec(prec), int(nrhs), _stream(stream)
    )
    _check(st, "stag_dslash")
    return out


def stag_apply_m(h, out, inp, mass, shift=0.0, prec="fp64", stream=None):
    """out = (m^2 + shift) inp - D_eo D_oe inp on even sites."""
    n = h.Vh * 3
    st = _lib.stag_apply_m(
        h.ptr, _ptr(out, "out", n), _ptr(inp, "inp", n), float(mass), float(shift), _prec(prec), _stream(stream)
    )
    _check(st, "stag_apply_m")
    return out


def stag_apply_m_noalloc(h, out, inp, mass, shift=0.0, stream=None):
    """FP64 out = (m^2 + shift) inp - D_eo D_oe inp without any device allocation
    (scratch in the library's static device array; V/2 <= NOALLOC_MAX_VH)."""
    n = h.Vh * 3
    st = _lib.stag_apply_m_noalloc(h.ptr, _ptr(out, "out", n), _ptr(inp, "inp", n), float(mass), float(shift), _stream(stream))
    _check(st, "stag_apply_m_noalloc")
    return out


NOALLOC_MAX_VH = 65536


def stag_cg(h, x, b, mass, params=None, stream=None, raise_on_error=True, **kw):
    """Solve M x = b; returns the solve info as a dict (status included)."""
    p = params if params is not None else default_params(**kw)
    info = SolveInfo()
    n = h.Vh * 3
    st = _lib.stag_cg(h.ptr, _ptr(x, "x", n), _ptr(b, "b", n), float(mass), ctypes.byref(p), ctypes.byref(info), _stream(stream))
    if raise_on_error and st not in (STAG_OK,):
        raise StagError(st, "stag_cg")
    d = info.as_dict()
    d["return"] = st
    return d


def stag_multishift_cg(h, xs, b, mass, shifts, params=None, stream=None, raise_on_error=True, **kw):
    """Solve (M + shifts[s]) xs[s] = b for all shifts; returns a list of info dicts."""
    p = params if params is not None else default_params(**kw)
    ns = len(shifts)
    n = h.Vh * 3
    ptrs = (ctypes.c_void_p * ns)(*[_ptr(x, f"xs[{i}]", n).value for i, x in enumerate(xs)])
    sh = (ctypes.c_double * ns)(*[float(s) for s in shifts])
    infos = (SolveInfo * ns)()
    st = _lib.stag_multishift_cg(h.ptr, ptrs, _ptr(b, "b", n), float(mass), sh, ns, ctypes.byref(p), infos, _stream(stream))
    if raise_on_error and st != STAG_OK:
        raise StagError(st, "stag_multishift_cg")
    out = [i.as_dict() for i in infos]
    for d in out:
        d["return"] = st
    return out


def stag_batch_solve(items, params=None, stream=None, raise_on_error=True, **kw):
    """Solve many systems on several lattices together.

    items: sequence of (handle, x, b, nrhs, mass) with x, b complex128 CUDA
    tensors [nrhs][V/2][3].  Returns one info dict per system, item by item."""
    p = params if params is not None else default_params(**kw)
    arr = (BatchItem * len(items))()
    total = 0
    for i, (h, x, b, nrhs, mass) in enumerate(items):
        n = h.Vh * 3 * int(nrhs)
        arr[i] = BatchItem(h.ptr.value, _ptr(x, f"x[{i}]", n).value, _ptr(b, f"b[{i}]", n).value, int(nrhs), float(mass))
        total += int(nrhs)
    infos = (SolveInfo * total)()
    st = _lib.stag_batch_solve(arr, len(items), ctypes.byref(p), infos, _stream(stream))
    if raise_on_error and st != STAG_OK:
        raise StagError(st, "stag_batch_solve")
    out = [i.as_dict() for i in infos]
    for d in out:
        d["return"] = st
    return out


class NetHandle:
    """Owns a ``stag_net_t`` (the learned preconditioner's parameters)."""

    def __init__(self, ptr, channels):
        self.ptr = ctypes.c_void_p(ptr)
        self.channels = tuple(channels)

    def free(self):
        if self.ptr and self.ptr.value:
            _check(_lib.stag_net_free(self.ptr), "stag_net_free")
            self.ptr = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def stag_net_create(channels=(1, 16, 16, 16, 1), seed=1):
    ch = (ctypes.c_int * len(channels))(*channels)
    h = ctypes.c_void_p()
    _check(_lib.stag_net_create(ctypes.byref(h), ch, len(channels) - 1, int(seed)), "stag_net_create")
    return NetHandle(h.value, channels)


def stag_net_free(net):
    net.free()


def stag_net_num_params(net):
    return int(_lib.stag_net_num_params(net.ptr))


def stag_net_get_params(net, rounded=False):
    import numpy as np

    n = stag_net_num_params(net)
    out = np.empty(n, dtype=np.float32)
    _check(
        _lib.stag_net_get_params(net.ptr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), n, 1 if rounded else 0),
        "stag_net_get_params",
    )
    return out


def stag_net_set_params(net, values):
    import numpy as np

    v = np.ascontiguousarray(values, dtype=np.float32)
    _check(_lib.stag_net_set_params(net.ptr, v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), v.size), "stag_net_set_params")


def stag_net_apply(net, h, z, r, stream=None):
    n = h.Vh * 3
    _check(_lib.stag_net_apply(net.ptr, h.ptr, _ptr(z, "z", n), _ptr(r, "r", n), _stream(stream)), "stag_net_apply")
    return z


def stag_net_loss_grad(net, h, r, e, loss="residual", mass=0.0, stream=None):
    """Loss of one (r, e) pair and its gradient (host float32 array).  loss:
    "residual" (||M z^ - r^||^2 / ||r^||^2, needs the pair's mass) or "error"."""
    import numpy as np

    n = h.Vh * 3
    npar = stag_net_num_params(net)
    g = np.empty(npar, dtype=np.float32)
    out = ctypes.c_double()
    _check(
        _lib.stag_net_loss_grad(net.ptr, h.ptr, _ptr(r, "r", n), _ptr(e, "e", n), LOSS[loss], float(mass),
                                ctypes.byref(out),
                                g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), npar, _stream(stream)),
        "stag_net_loss_grad",
    )
    return out.value, g


def stag_net_train(net, pairs, epochs=1, batch=4, lr=1e-3, seed=1, loss="residual", mass=0.0, stream=None):
    """pairs: sequence of (handle, r, e) with r, e complex128 or complex64 CUDA tensors [V/2][3].
    loss: "residual" (needs the pairs' mass) or "error".
    Returns the per-pair losses (epochs * len(pairs), visiting order)."""
    import numpy as np

    arr = (TrainPair * len(pairs))()
    prec = None
    for i, (h, r, e) in enumerate(pairs):
        for t, nm in ((r, "r"), (e, "e")):
            if not t.is_cuda or not t.is_contiguous() or t.numel() != h.Vh * 3:
                raise ValueError(f"pair {i}: {nm} must be a contiguous CUDA tensor of V/2*3 entries")
        p = STAG_FP64 if r.dtype == torch.complex128 else STAG_FP32 if r.dtype == torch.complex64 else None
        if p is None or e.dtype != r.dtype or (prec is not None and p != prec):
            raise ValueError("pairs must all be complex128 or all complex64")
        prec = p
        arr[i] = TrainPair(h.ptr.value, r.data_ptr(), e.data_ptr())
    tp = TrainParams(int(epochs), int(batch), float(lr), int(seed), prec, LOSS[loss], float(mass))
    losses = np.empty(len(pairs) * int(epochs), dtype=np.float64)
    _check(
        _lib.stag_net_train(net.ptr, arr, len(pairs), ctypes.byref(tp),
                            losses.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream(stream)),
        "stag_net_train",
    )
    return losses


def stag_build_links(dims, thin, fat=None, lng=None, c1=1.0, c_staple=0.125, c3=-1.0 / 24.0, stream=None):
    """Fat and Naik links from thin links on the GPU (FP64).  thin: contiguous
    complex128 CUDA tensor of V*4*9 entries (canonical [V][4][3][3]); fat and
    lng are allocated like thin when not given.  Returns (fat, lng)."""
    V = int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])
    n = V * 36
    fat = torch.empty_like(thin) if fat is None else fat
    lng = torch.empty_like(thin) if lng is None else lng
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(_lib.stag_build_links(d, _ptr(thin, "thin", n), _ptr(fat, "fat", n), _ptr(lng, "lng", n),
                                 float(c1), float(c_staple), float(c3), _stream(stream)), "stag_build_links")
    return fat, lng


def stag_gauge_force(dims, thin, beta, c_pl, c_rt, c_pg, force=None, stream=None):
    """Symanzik one-loop gauge force (FP64) from thin links (contiguous complex128
    CUDA tensor, canonical [V][4][3][3]); returns the force tensor, same layout."""
    V = int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])
    n = V * 36
    force = torch.empty_like(thin) if force is None else force
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(_lib.stag_gauge_force(d, _ptr(thin, "thin", n), _ptr(force, "force", n), float(beta), float(c_pl),
                                 float(c_rt), float(c_pg), _stream(stream)), "stag_gauge_force")
    return force


def stag_fermion_force(dims, thin, xs, ys, alphas, c1=1.0, c_staple=0.125, c3=-1.0 / 24.0, force=None, stream=None):
    """Fermion force (FP64) through the fat and Naik link construction.  thin:
    canonical [V][4][3][3] complex128 CUDA tensor; xs: even-site solutions X_i
    and ys: odd-site Y_i = D_oe X_i, contiguous [n][V/2][3] complex128 CUDA
    tensors; alphas: n weights.  Returns the force, canonical [V][4][3][3]."""
    V = int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])
    n = V * 36
    nt = len(alphas)
    force = torch.empty_like(thin) if force is None else force
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    a = (ctypes.c_double * max(nt, 1))(*[float(v) for v in alphas])
    nf = nt * (V // 2) * 3
    _check(_lib.stag_fermion_force(d, _ptr(thin, "thin", n), nt, _ptr(xs, "xs", nf), _ptr(ys, "ys", nf), a,
                                   float(c1), float(c_staple), float(c3), _ptr(force, "force", n), _stream(stream)),
           "stag_fermion_force")
    return force


def stag_tc_selftest():
    """Max relative error of one tensor-core tile against the CUDA cores (0 expected)."""
    err = ctypes.c_double()
    _check(_lib.stag_tc_selftest(ctypes.byref(err)), "stag_tc_selftest")
    return err.value


def stag_strerror(status):
    return strerror(status)


def stag_profile_enable(on=True):
    _check(_lib.stag_profile_enable(1 if on else 0), "stag_profile_enable")


def stag_profile_select(families="", every=1):
    """Time only the listed kernel families (comma-separated; "" = all), one
    launch in `every` of each."""
    _check(_lib.stag_profile_select(families.encode(), int(every)), "stag_profile_select")


def stag_profile_reset():
    _check(_lib.stag_profile_reset(), "stag_profile_reset")


def stag_profile_read(family):
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(_lib.stag_profile_read(family.encode(), ctypes.byref(n), ctypes.byref(ms)), "stag_profile_read")
    return n.value, ms.value


def stag_launch_count():
    return int(_lib.stag_launch_count())


def stag_tuned_mrhs(h, prec, nrhs, epilogue=False):
    """(threads per site, min blocks per SM, us per launch) of the tuned
    launch variant of the N-right-hand-side plain kernel, or with
    epilogue=True of its epilogue form (us 0: not timed)."""
    t, m, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    fn = _lib.stag_tuned_mrhs_epi if epilogue else _lib.stag_tuned_mrhs
    _check(fn(h.ptr, _prec(prec), int(nrhs), ctypes.byref(t), ctypes.byref(m), ctypes.byref(us)),
           "stag_tuned_mrhs_epi" if epilogue else "stag_tuned_mrhs")
    return t.value, m.value, us.value


def stag_tuned_mrhs_epi(h, prec, nrhs):
    return stag_tuned_mrhs(h, prec, nrhs, epilogue=True)


def stag_tuned_mrhs_variant(h, prec, nrhs, epilogue=False):
    """Index (0..5) of the tuned variant of the N-right-hand-side plain kernel
    or of its epilogue form."""
    v = int(_lib.stag_tuned_mrhs_variant(h.ptr, _prec(prec), int(nrhs), 1 if epilogue else 0))
    if v < 0:
        raise StagError(v, "stag_tuned_mrhs_variant")
    return v


def stag_tune_key(kernel, prec, nl, nrhs, dims):
    buf = ctypes.create_string_buffer(256)
    d = (ctypes.c_int * 4)(*[int(v) for v in dims])
    _check(_lib.stag_tune_key(buf, 256, kernel.encode(), _prec(prec), int(nl), int(nrhs), d), "stag_tune_key")
    return buf.value.decode()


def stag_tune_cache_get(key):
    """(variant, us) stored under key, or (-1, 0.0)."""
    v, us = ctypes.c_int(), ctypes.c_double()
    _check(_lib.stag_tune_cache_get(key.encode(), ctypes.byref(v), ctypes.byref(us)), "stag_tune_cache_get")
    return v.value, us.value


def stag_tune_cache_put(key, variant, us):
    _check(_lib.stag_tune_cache_put(key.encode(), int(variant), float(us)), "stag_tune_cache_put")


def stag_tune_cache_load(path):
    _check(_lib.stag_tune_cache_load(os.fsencode(path)), "stag_tune_cache_load")


def stag_tune_cache_save(path):
    _check(_lib.stag_tune_cache_save(os.fsencode(path)), "stag_tune_cache_save")


def stag_tune_cache_clear():
    _check(_lib.stag_tune_cache_clear(), "stag_tune_cache_clear")


def stag_tune_cache_size():
    return int(_lib.stag_tune_cache_size())


# ---------------------------------------------------------------- one lattice over several ranks
DD_HALO = 4  # STAG_DD_HALO

_EXCH_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_void_p)
_ALLRED_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                              ctypes.c_void_p)


class StagComm(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("exchange", _EXCH_FN), ("allreduce_sum", _ALLRED_FN)]


class _CudaBytes:
    """A raw device range seen by torch without a copy (__cuda_array_interface__)."""

    def __init__(self, ptr, n, typestr="|u1"):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def _view(ptr, nbytes, dtype=torch.uint8):
    typestr = {torch.uint8: "|u1", torch.float64: "<f8"}[dtype]
    n = nbytes // (8 if dtype == torch.float64 else 1)
    return torch.as_tensor(_CudaBytes(ptr, n, typestr), device="cuda")


class Communicator:
    """The caller side of stag_comm: subclasses implement

      exchange(send_lo, send_hi, recv_lo, recv_hi)  uint8 CUDA tensors: send_lo
          to the rank below, send_hi to the rank above, receive the rank
          below's send_hi into recv_lo and the rank above's send_lo into recv_hi
      allreduce(t)                                   float64 CUDA tensor, in place

    The library's callbacks wrap the raw device ranges as tensors and run the
    subclass's work on the library's stream (so it is ordered after the
    kernels that wrote the data and before those that read the result)."""

    def __init__(self, rank, size):
        self.rank, self.size = int(rank), int(size)
        self.error = None
        self._ex = _EXCH_FN(self._exchange_cb)
        self._ar = _ALLRED_FN(self._allreduce_cb)
        self.struct = StagComm(None, self._ex, self._ar)

    def _exchange_cb(self, ctx, slo, shi, rlo, rhi, nbytes, stream):
        try:
            st = torch.cuda.ExternalStream(int(stream)) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(st):
                self.exchange(*[_view(p, nbytes) for p in (slo, shi, rlo, rhi)])
            return 0
        except Exception as e:  # reported as a failed call (STAG_ECUDA); kept for the caller
            self.error = e
            return 1

    def _allreduce_cb(self, ctx, values, n, stream):
        try:
            st = torch.cuda.ExternalStream(int(stream)) if stream else torch.cuda.default_stream()
            with torch.cuda.stream(st):
                self.allreduce(_view(ctypes.cast(values, ctypes.c_void_p).value, 8 * n, torch.float64))
            return 0
        except Exception as e:
            self.error = e
            return 1


class TorchDistComm(Communicator):
    """stag_comm over torch.distributed (default group): NCCL moves the
    device buffers directly; gloo stages them through host memory.  The
    halo sent to the rank below travels with tag 1, the one sent above with
    tag 2, so that two ranks (each the other's lower and upper neighbour)
    keep them apart."""

    def __init__(self):
        import torch.distributed as dist

        super().__init__(dist.get_rank(), dist.get_world_size())
        self.dist = dist
        self.host = dist.get_backend() != "nccl"

    def exchange(self, send_lo, send_hi, recv_lo, recv_hi):
        dist, R, r = self.dist, self.size, self.rank
        if R == 1:
            recv_lo.copy_(send_hi)
            recv_hi.copy_(send_lo)
            return
        lo, hi = (r - 1) % R, (r + 1) % R
        if self.host:
            s_lo, s_hi = send_lo.cpu(), send_hi.cpu()
            b_lo, b_hi = torch.empty_like(s_lo), torch.empty_like(s_hi)
            reqs = [dist.isend(s_lo, lo, tag=1), dist.isend(s_hi, hi, tag=2),
                    dist.irecv(b_lo, lo, tag=2), dist.irecv(b_hi, hi, tag=1)]
            for q in reqs:
                q.wait()
            recv_lo.copy_(b_lo)
            recv_hi.copy_(b_hi)
        else:
            ops = [dist.P2POp(dist.isend, send_lo, lo), dist.P2POp(dist.isend, send_hi, hi),
                   dist.P2POp(dist.irecv, recv_lo, lo), dist.P2POp(dist.irecv, recv_hi, hi)]
            for q in dist.batch_isend_irecv(ops):
                q.wait()

    def allreduce(self, t):
        if self.host:
            h = t.cpu()
            self.dist.all_reduce(h)
            t.copy_(h)
        else:
            self.dist.all_reduce(t)


class DDHandle:
    """Owns a ``stag_dd_t`` (one rank's part of a lattice split along t)."""

    def __init__(self, ptr, gdims, rank, nranks):
        self.ptr = ctypes.c_void_p(ptr)
        self.gdims, self.rank, self.nranks = tuple(gdims), rank, nranks
        d = (ctypes.c_int * 4)()
        vh, t0 = ctypes.c_longlong(), ctypes.c_int()
        _check(_lib.stag_dd_info(self.ptr, d, ctypes.byref(vh), ctypes.byref(t0)), "stag_dd_info")
        self.local_dims, self.Vh, self.t_offset = tuple(d), vh.value, t0.value

    def free(self):
        if self.ptr and self.ptr.value:
            _check(_lib.stag_dd_free(self.ptr), "stag_dd_free")
            self.ptr = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def stag_dd_create(gdims, rank, nranks, fat_ext, lng_ext, recon_long=18, long_coeff=-1.0 / 24.0, stream=None):
    """One rank's handle; fat_ext, lng_ext: the extended slab's links (see dd_slab), complex128 CUDA."""
    g = tuple(int(v) for v in gdims)
    T = g[3] // int(nranks)
    n = g[0] * g[1] * g[2] * (T + 2 * DD_HALO) * 36
    h = ctypes.c_void_p()
    o = LinkOpts(int(recon_long), float(long_coeff), 1 << STAG_FP64, 1)
    _check(_lib.stag_dd_create(ctypes.byref(h), (ctypes.c_int * 4)(*g), int(rank), int(nranks),
                               _ptr(fat_ext, "fat_ext", n), _ptr(lng_ext, "lng_ext", n), ctypes.byref(o),
                               _stream(stream)), "stag_dd_create")
    return DDHandle(h.value, g, int(rank), int(nranks))


def _dd_call(name, status, comm):
    if status != STAG_OK:
        err = StagError(status, name)
        if comm.error is not None:
            raise err from comm.error
        raise err


def stag_dd_dslash(dd, out, inp, out_parity, comm, stream=None):
    n = dd.Vh * 3
    st = _lib.stag_dd_dslash(dd.ptr, _ptr(out, "out", n), _ptr(inp, "inp", n), int(out_parity),
                             ctypes.byref(comm.struct), _stream(stream))
    _dd_call("stag_dd_dslash", st, comm)
    return out


def stag_dd_apply_m(dd, out, inp, mass, comm, stream=None):
    n = dd.Vh * 3
    st = _lib.stag_dd_apply_m(dd.ptr, _ptr(out, "out", n), _ptr(inp, "inp", n), float(mass),
                              ctypes.byref(comm.struct), _stream(stream))
    _dd_call("stag_dd_apply_m", st, comm)
    return out


def stag_dd_cg(dd, x, b, mass, comm, params=None, stream=None, raise_on_error=True, **kw):
    """FP64 CG on the split lattice; x, b: the rank's own even sites.  Returns the info dict."""
    kw.setdefault("mode", "plain64")
    p = params if params is not None else default_params(**kw)
    info = SolveInfo()
    n = dd.Vh * 3
    st = _lib.stag_dd_cg(dd.ptr, _ptr(x, "x", n), _ptr(b, "b", n), float(mass), ctypes.byref(p), ctypes.byref(info),
                         ctypes.byref(comm.struct), _stream(stream))
    if raise_on_error and st != STAG_OK:
        _dd_call("stag_dd_cg", st, comm)
    d = info.as_dict()
    d["return"] = st
    return d


def dd_slab(links, gdims, rank, nranks):
    """The extended slab of canonical [V][4][3][3] links a rank's handle takes:
    global slices rank*T - DD_HALO .. rank*T + T + DD_HALO - 1, periodic in t
    (works on numpy arrays and torch tensors of the global field)."""
    Lx, Ly, Lz, Lt = (int(v) for v in gdims)
    T = Lt // int(nranks)
    slab = Lx * Ly * Lz
    ts = [(rank * T - DD_HALO + k) % Lt for k in range(T + 2 * DD_HALO)]
    shp = links.shape
    per_t = links.reshape((Lt, slab) + tuple(shp[1:]))
    idx = torch.tensor(ts) if isinstance(links, torch.Tensor) else ts
    out = per_t[idx]
    return out.reshape((len(ts) * slab,) + tuple(shp[1:]))


def dd_own_sites(field, gdims, rank, nranks):
    """A rank's own sites of a global single-parity field [V/2][3] (or [..][V/2][3])."""
    Lx, Ly, Lz, Lt = (int(v) for v in gdims)
    T = Lt // int(nranks)
    S = Lx // 2 * Ly * Lz
    return field[..., rank * T * S:(rank + 1) * T * S, :]


def stag_bounds_violations(clear=False):
    """(count, first code, first index) of the bounds-checked build; count -1 in the normal build."""
    n, c, i = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_longlong()
    _check(_lib.stag_bounds_violations(ctypes.byref(n), ctypes.byref(c), ctypes.byref(i), 1 if clear else 0),
           "stag_bounds_violations")
    return n.value, c.value, i.value
