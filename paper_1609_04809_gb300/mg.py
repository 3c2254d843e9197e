"""ctypes binding of libmg.so (include/mg.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels. PyTorch is used for device
memory (the library allocates through callbacks into torch's caching allocator) and
for the caller's CUDA stream. If libmg.so has not been built, loading it raises
ImportError: there is no fallback.
"""
import ctypes
import os

import numpy as np

from . import _build

MG_OK, MG_PENDING = 0, 1
MG_EINVAL, MG_ENOMEM, MG_ENOCONV, MG_ECUDA, MG_ETIMEOUT, MG_EBUDGET, MG_ENOTFOUND = -1, -2, -3, -4, -5, -6, -7
MG_Q1, MG_RQ1, MG_P1, MG_P2 = 0, 1, 2, 3
MG_JACOBI, MG_CHEBYSHEV, MG_GAUSS_SEIDEL = 0, 1, 2
MG_FP64, MG_MIXED = 0, 1
MG_STORAGE_AUTO, MG_STORAGE_CSR, MG_STORAGE_ELL, MG_STORAGE_DIA, MG_STORAGE_SELL, MG_STORAGE_STENCIL = 0, 1, 2, 3, 4, 5
MG_STORAGE_COEF = 6
MG_TRANSFER_NONE, MG_TRANSFER_GRID, MG_TRANSFER_SELL = 0, 1, 2
MG_MAX_LEVELS = 16
(MG_K_SMOOTH, MG_K_RESID, MG_K_RESTRICT, MG_K_PROLONG, MG_K_COARSE, MG_K_OUTER, MG_K_UPDATE,
 MG_K_SMOOTH0, MG_K_KRYLOV) = range(9)
MG_K_COUNT = 9
KCLASS_NAMES = ["smooth", "resid", "restrict", "prolong", "coarse", "outer", "update", "smooth0", "krylov"]


class MgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("mg status %d: %s" % (status, msg))
        self.status = status


class mg_problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("element", ctypes.c_int), ("n_cells", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("k_cell", ctypes.POINTER(ctypes.c_double)),
                ("mass", ctypes.c_double)]


class mg_options(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("omega", ctypes.c_double), ("cheb_degree", ctypes.c_int),
                ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("cheb_hi", ctypes.c_double),
                ("cheb_ratio", ctypes.c_double), ("power_iters", ctypes.c_int),
                ("power_seed", ctypes.c_uint64), ("precision", ctypes.c_int), ("storage", ctypes.c_int),
                ("max_iters", ctypes.c_int), ("use_graph", ctypes.c_int), ("use_pdl", ctypes.c_int),
                ("coarse_tail", ctypes.c_int), ("fuse_first", ctypes.c_int)]


class mg_rhs(ctypes.Structure):
    _fields_ = [("n_modes", ctypes.c_int), ("amp", ctypes.POINTER(ctypes.c_double)),
                ("freq", ctypes.POINTER(ctypes.c_int)), ("f_const", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class mg_device(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p), ("stream", ctypes.c_void_p)]


class mg_info(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("precision", ctypes.c_int),
                ("n", ctypes.c_int64 * MG_MAX_LEVELS), ("nnz", ctypes.c_int64 * MG_MAX_LEVELS),
                ("storage", ctypes.c_int * MG_MAX_LEVELS), ("galerkin", ctypes.c_int * MG_MAX_LEVELS),
                ("lambda_", ctypes.c_double * MG_MAX_LEVELS), ("device_bytes", ctypes.c_size_t),
                ("kernels_per_cycle", ctypes.c_int), ("tail_levels", ctypes.c_int),
                ("transfer", ctypes.c_int * MG_MAX_LEVELS)]


class mg_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int),
                ("rows_per_thread", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("options", mg_options)]


class mg_serve_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_uint64), ("cycles", ctypes.c_uint64), ("active", ctypes.c_int),
                ("queued", ctypes.c_int), ("operator_sets", ctypes.c_int), ("mean_batch", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("device_bytes_in_use", ctypes.c_size_t),
                ("device_bytes_peak", ctypes.c_size_t), ("gpu_ms", ctypes.c_double), ("setup_ms", ctypes.c_double),
                ("span_ms", ctypes.c_double)]


# every entry point declared in include/mg.h, with its ctypes signature
_P = ctypes.POINTER
_vp = ctypes.c_void_p
_dp = _P(ctypes.c_double)
SIGNATURES = {
    "mg_options_default": (None, [_P(mg_options)]),
    "mg_ndofs": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "mg_load_vector": (ctypes.c_int, [_P(mg_problem), _P(mg_rhs), _dp]),
    "mg_load_vector_separable": (ctypes.c_int, [_P(mg_problem), _P(mg_rhs), _dp]),
    "mg_assemble_operator": (ctypes.c_int, [_P(mg_problem), ctypes.c_int, ctypes.c_int, _P(ctypes.c_int64),
                                            _P(ctypes.c_int64), _P(ctypes.c_int64), _P(ctypes.c_int32), _dp]),
    "mg_setup": (ctypes.c_int, [_P(mg_problem), _P(mg_options), _P(mg_device), _P(_vp)]),
    "mg_hierarchy_free": (ctypes.c_int, [_vp]),
    "mg_get_info": (ctypes.c_int, [_vp, _P(mg_info)]),
    "mg_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _P(ctypes.c_int), _dp]),
    "mg_solve_host": (ctypes.c_int, [_vp, _dp, _dp, ctypes.c_double, _P(ctypes.c_int), _dp]),
    "mg_pcg": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, _P(ctypes.c_int), _dp]),
    "mg_pcg_host": (ctypes.c_int, [_vp, _dp, _dp, ctypes.c_double, _P(ctypes.c_int), _dp]),
    "mg_heat": (ctypes.c_int, [_vp, _vp, _dp, ctypes.c_int, _vp, ctypes.c_double, ctypes.c_int, _P(ctypes.c_int)]),
    "mg_heat_host": (ctypes.c_int, [_vp, _dp, _dp, ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int,
                                    _P(ctypes.c_int)]),
    "mg_constant_stencil": (ctypes.c_int, [_P(mg_problem), ctypes.c_int, _P(ctypes.c_int)]),
    "mg_cycle": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _dp]),
    "mg_export_operator": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P(ctypes.c_int64),
                                          _P(ctypes.c_int64), _P(ctypes.c_int64), _P(ctypes.c_int32), _dp]),
    "mg_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_uint, ctypes.c_uint]),
    "mg_profile_read": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _dp, _P(ctypes.c_int64), _dp, _dp]),
    "mg_residual_norm_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _vp, _dp]),
    "mg_serve_config_default": (None, [_P(mg_serve_config)]),
    "mg_serve_create": (ctypes.c_int, [_P(mg_serve_config), _P(mg_device), _P(_vp)]),
    "mg_serve_submit": (ctypes.c_int, [_vp, _P(mg_problem), _dp, ctypes.c_double, _P(ctypes.c_uint64)]),
    "mg_serve_submit_rhs": (ctypes.c_int, [_vp, _P(mg_problem), _P(mg_rhs), ctypes.c_double,
                                           _P(ctypes.c_uint64)]),
    "mg_serve_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, _dp, _P(ctypes.c_int)]),
    "mg_serve_wait": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_double, _dp, _P(ctypes.c_int), _dp,
                                     ctypes.c_int]),
    "mg_serve_get_stats": (ctypes.c_int, [_vp, _P(mg_serve_stats)]),
    "mg_serve_reset_stats": (ctypes.c_int, [_vp]),
    "mg_serve_tune": (ctypes.c_int, [_vp, _P(mg_problem), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     _P(ctypes.c_int), _P(ctypes.c_int)]),
    "mg_serve_destroy": (ctypes.c_int, [_vp]),
    "mg_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Open libmg.so (built in-tree by ``__graft_entry__.build()``); ImportError if absent."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise ImportError("libmg.so is not built (%s); run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error():
    return lib().mg_last_error().decode()


def _check(st, ok=(MG_OK,)):
    if st not in ok:
        raise MgError(st, last_error())
    return st


def _as_dp(a):
    return a.ctypes.data_as(_dp)


# ---------------------------------------------------------------------------------
# torch-backed device memory
# ---------------------------------------------------------------------------------
class TorchDevice:
    """mg_device whose alloc/free keep torch uint8 tensors alive, on torch's current stream."""

    def __init__(self, stream=None):
        import torch
        self._torch = torch
        self._live = {}

        self.allocations = 0  # calls of the alloc callback

        def _alloc(nbytes, ctx):
            self.allocations += 1
            try:
                t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
            except Exception:
                return None
            self._live[t.data_ptr()] = t
            return t.data_ptr()

        def _free(ptr, nbytes, ctx):
            self._live.pop(ptr, None)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        s = stream if stream is not None else torch.cuda.current_stream()
        self.struct = mg_device(self._alloc_cb, self._free_cb, None, ctypes.c_void_p(s.cuda_stream))

    def bytes_held(self):
        return sum(t.numel() for t in self._live.values())


# ---------------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------------
def mg_options_default(**overrides):
    o = mg_options()
    lib().mg_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def mg_ndofs(dim, element, n_cells):
    return int(lib().mg_ndofs(dim, element, n_cells))


def _problem(dim, element, n_cells, n_levels, k_cell=None, mass=0.0):
    keep = None
    p = mg_problem(dim, element, n_cells, n_levels, None, float(mass))
    if k_cell is not None:
        keep = np.ascontiguousarray(k_cell, dtype=np.float64)
        p.k_cell = _as_dp(keep)
    return p, keep


def _rhs(modes=None, f_const=1.0):
    if not modes:
        return mg_rhs(0, None, None, float(f_const)), None
    amp = np.array([m[0] for m in modes], dtype=np.float64)
    freq = np.zeros((len(modes), 3), dtype=np.intc)
    for i, m in enumerate(modes):
        freq[i, :len(m[1])] = m[1]
    freq = np.ascontiguousarray(freq.reshape(-1))
    return mg_rhs(len(modes), _as_dp(amp), freq.ctypes.data_as(_P(ctypes.c_int)), 0.0), (amp, freq)


def mg_load_vector(dim, element, n_cells, modes=None, f_const=1.0, n_levels=1):
    """Load vector of the finest grid for f = -Laplace(sum of sine modes) or f = f_const."""
    p, _k = _problem(dim, element, n_cells, n_levels)
    f, _keep = _rhs(modes, f_const)
    b = np.zeros(mg_ndofs(dim, element, n_cells))
    _check(lib().mg_load_vector(ctypes.byref(p), ctypes.byref(f), _as_dp(b)))
    return b


def mg_assemble_operator(dim, element, n_cells, n_levels, level, which=0, k_cell=None, mass=0.0):
    """Host-assembled level operator (no GPU) as (rowptr, col, val): which 0 = A (+ mass M), 1 = P, 2 = R."""
    L = lib()
    p, _k = _problem(dim, element, n_cells, n_levels, k_cell, mass)
    nrows, nnz = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(L.mg_assemble_operator(ctypes.byref(p), level, which, ctypes.byref(nrows), ctypes.byref(nnz),
                                  None, None, None))
    rowptr = np.zeros(nrows.value + 1, dtype=np.int64)
    col = np.zeros(max(nnz.value, 1), dtype=np.int32)
    val = np.zeros(max(nnz.value, 1))
    _check(L.mg_assemble_operator(ctypes.byref(p), level, which, ctypes.byref(nrows), ctypes.byref(nnz),
                                  rowptr.ctypes.data_as(_P(ctypes.c_int64)),
                                  col.ctypes.data_as(_P(ctypes.c_int32)), _as_dp(val)))
    return rowptr, col[:nnz.value], val[:nnz.value]


def mg_constant_stencil(dim, element, n_cells, n_levels, level, k_cell=None, mass=0.0):
    """Host check (no GPU): is every row of the level matrix the same stencil? (bool)"""
    p, _k = _problem(dim, element, n_cells, n_levels, k_cell, mass)
    out = ctypes.c_int(0)
    _check(lib().mg_constant_stencil(ctypes.byref(p), level, ctypes.byref(out)))
    return bool(out.value)


def mg_load_vector_separable(dim, n_cells, modes=None, f_const=1.0):
    """The Q1 load vector with the Gauss rule factorised per mode and axis (equal up to rounding)."""
    p, _k = _problem(dim, MG_Q1, n_cells, 1)
    f, _keep = _rhs(modes, f_const)
    b = np.zeros(mg_ndofs(dim, MG_Q1, n_cells))
    _check(lib().mg_load_vector_separable(ctypes.byref(p), ctypes.byref(f), _as_dp(b)))
    return b


def mg_setup(dim, element, n_cells, n_levels, options=None, k_cell=None, device=None, mass=0.0):
    """Build a hierarchy; returns the opaque handle (int). device: TorchDevice or None (cudaMalloc).
    mass: sigma of the operator A + sigma M (Crank-Nicolson, sigma = 2/dt)."""
    p, _k = _problem(dim, element, n_cells, n_levels, k_cell, mass)
    o = options if options is not None else mg_options_default()
    h = _vp()
    dptr = ctypes.byref(device.struct) if device is not None else None
    _check(lib().mg_setup(ctypes.byref(p), ctypes.byref(o), dptr, ctypes.byref(h)))
    return h.value


def mg_hierarchy_free(h):
    return _check(lib().mg_hierarchy_free(h))


def mg_get_info(h):
    info = mg_info()
    _check(lib().mg_get_info(h, ctypes.byref(info)))
    L = info.n_levels
    return dict(n_levels=L, precision=info.precision, n=list(info.n[:L]), nnz=list(info.nnz[:L]),
                storage=list(info.storage[:L]), galerkin=list(info.galerkin[:L]),
                lambda_=list(info.lambda_[:L]), device_bytes=int(info.device_bytes),
                kernels_per_cycle=info.kernels_per_cycle, tail_levels=info.tail_levels,
                transfer=list(info.transfer[:L]))


def mg_solve(h, b_dev, x_dev, rel_tol, max_iters=100):
    """b_dev, x_dev: CUDA float64 tensors (x_dev updated in place). Returns (status, iters, hist)."""
    it = ctypes.c_int(0)
    hist = np.zeros(max_iters + 1)
    st = lib().mg_solve(h, ctypes.c_void_p(b_dev.data_ptr()), ctypes.c_void_p(x_dev.data_ptr()),
                        float(rel_tol), ctypes.byref(it), _as_dp(hist))
    _check(st, (MG_OK, MG_ENOCONV))
    return st, it.value, hist[:it.value + 1].copy()


def mg_solve_host(h, b_host, x_host, rel_tol, max_iters=100):
    """b_host, x_host: float64 numpy arrays (x_host updated in place; pinned memory is fastest)."""
    assert b_host.dtype == np.float64 and x_host.dtype == np.float64
    assert b_host.flags.c_contiguous and x_host.flags.c_contiguous
    it = ctypes.c_int(0)
    hist = np.zeros(max_iters + 1)
    st = lib().mg_solve_host(h, _as_dp(b_host), _as_dp(x_host), float(rel_tol), ctypes.byref(it), _as_dp(hist))
    _check(st, (MG_OK, MG_ENOCONV))
    return st, it.value, hist[:it.value + 1].copy()


def mg_pcg(h, b_dev, x_dev, rel_tol, max_iters=100):
    """CG preconditioned by one V-cycle; arguments and result as mg_solve."""
    it = ctypes.c_int(0)
    hist = np.zeros(max_iters + 1)
    st = lib().mg_pcg(h, ctypes.c_void_p(b_dev.data_ptr()), ctypes.c_void_p(x_dev.data_ptr()),
                      float(rel_tol), ctypes.byref(it), _as_dp(hist))
    _check(st, (MG_OK, MG_ENOCONV))
    return st, it.value, hist[:it.value + 1].copy()


def mg_pcg_host(h, b_host, x_host, rel_tol, max_iters=100):
    """mg_pcg with float64 numpy arrays (x_host updated in place)."""
    assert b_host.dtype == np.float64 and x_host.dtype == np.float64
    assert b_host.flags.c_contiguous and x_host.flags.c_contiguous
    it = ctypes.c_int(0)
    hist = np.zeros(max_iters + 1)
    st = lib().mg_pcg_host(h, _as_dp(b_host), _as_dp(x_host), float(rel_tol), ctypes.byref(it), _as_dp(hist))
    _check(st, (MG_OK, MG_ENOCONV))
    return st, it.value, hist[:it.value + 1].copy()


MG_METHOD_DC, MG_METHOD_PCG = 0, 1


def mg_heat(h, bF_dev, g, u_dev, rel_tol, method=MG_METHOD_DC):
    """Crank-Nicolson steps k = 0..len(g)-2 on a hierarchy set up with mass = 2/dt.
    bF_dev, u_dev: CUDA float64 tensors (u updated in place). Returns (status, iters per step)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    n_steps = len(g) - 1
    its = np.zeros(max(n_steps, 1), dtype=np.intc)
    st = lib().mg_heat(h, ctypes.c_void_p(bF_dev.data_ptr()), _as_dp(g), n_steps, ctypes.c_void_p(u_dev.data_ptr()),
                       float(rel_tol), int(method), its.ctypes.data_as(_P(ctypes.c_int)))
    _check(st, (MG_OK, MG_ENOCONV))
    return st, its[:n_steps].copy()


def mg_heat_host(h, bF_host, g, u_host, rel_tol, method=MG_METHOD_DC):
    """mg_heat with float64 numpy arrays (u_host updated in place)."""
    g = np.ascontiguousarray(g, dtype=np.float64)
    assert bF_host.dtype == np.float64 and u_host.dtype == np.float64 and u_host.flags.c_contiguous
    bF_host = np.ascontiguousarray(bF_host)
    n_steps = len(g) - 1
    its = np.zeros(max(n_steps, 1), dtype=np.intc)
    st = lib().mg_heat_host(h, _as_dp(bF_host), _as_dp(g), n_steps, _as_dp(u_host), float(rel_tol), int(method),
                            its.ctypes.data_as(_P(ctypes.c_int)))
    _check(st, (MG_OK, MG_ENOCONV))
    return st, its[:n_steps].copy()


def mg_cycle(h, b_dev, x_dev, n_cycles):
    rel = ctypes.c_double(0.0)
    _check(lib().mg_cycle(h, ctypes.c_void_p(b_dev.data_ptr()), ctypes.c_void_p(x_dev.data_ptr()),
                          int(n_cycles), ctypes.byref(rel)))
    return rel.value


def mg_export_operator(h, level, which, precision=MG_FP64):
    """Level operator as (rowptr, col, val): which 0 = A, 1 = P, 2 = R."""
    L = lib()
    nrows, nnz = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(L.mg_export_operator(h, level, which, precision, ctypes.byref(nrows), ctypes.byref(nnz),
                                None, None, None))
    rowptr = np.zeros(nrows.value + 1, dtype=np.int64)
    col = np.zeros(max(nnz.value, 1), dtype=np.int32)
    val = np.zeros(max(nnz.value, 1))
    _check(L.mg_export_operator(h, level, which, precision, ctypes.byref(nrows), ctypes.byref(nnz),
                                rowptr.ctypes.data_as(_P(ctypes.c_int64)),
                                col.ctypes.data_as(_P(ctypes.c_int32)), _as_dp(val)))
    return rowptr, col[:nnz.value], val[:nnz.value]


def mg_residual_norm_noalloc(h, b_dev, x_dev, r_dev):
    """r_dev = b - A x on the finest level and ||r||_2, with no device allocation (see mg.h).

    The C entry point cannot check sizes or devices, so the tensors are checked here: each
    must be a contiguous float64 CUDA tensor of the hierarchy's finest DOF count on the
    current device (ValueError otherwise, before anything is launched)."""
    import torch
    n = mg_get_info(h)["n"][-1]
    dev = torch.cuda.current_device()
    for name, t in (("b", b_dev), ("x", x_dev), ("r", r_dev)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == dev and t.dtype == torch.float64
                and t.is_contiguous() and t.numel() == n):
            raise ValueError("mg_residual_norm_noalloc: %s must be a contiguous float64 CUDA tensor of %d "
                             "elements on device %d" % (name, n, dev))
    nr = ctypes.c_double(0.0)
    _check(lib().mg_residual_norm_noalloc(h, ctypes.c_void_p(b_dev.data_ptr()), ctypes.c_void_p(x_dev.data_ptr()),
                                          ctypes.c_void_p(r_dev.data_ptr()), ctypes.byref(nr)))
    return nr.value


def mg_profile_enable(h, enable=True, classes=None, levels=None):
    """Time launches with CUDA events; classes / levels: iterables of MG_K_* / level indices (None: all)."""
    cm = 0xFFFFFFFF if classes is None else sum(1 << c for c in classes)
    lm = 0xFFFFFFFF if levels is None else sum(1 << l for l in levels)
    return _check(lib().mg_profile_enable(h, int(bool(enable)), cm, lm))


def mg_profile_read(h, kclass, level):
    """(total ms, launches, algorithmic bytes per launch, algorithmic flops per launch)."""
    ms, n, b, f = ctypes.c_double(0), ctypes.c_int64(0), ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().mg_profile_read(h, kclass, level, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                                 ctypes.byref(f)))
    return ms.value, n.value, b.value, f.value


# ---------------------------------------------------------------------------------
# A small object wrapper
# ---------------------------------------------------------------------------------
class Hierarchy:
    """Owns an mg_hierarchy built on torch device memory."""

    def __init__(self, dim, element, n_cells, n_levels, k_cell=None, device=None, mass=0.0, **opts):
        self.options = mg_options_default(**opts)
        self.device = device if device is not None else TorchDevice()
        self.dim, self.element, self.n_cells, self.n_levels = dim, element, n_cells, n_levels
        self.n = mg_ndofs(dim, element, n_cells)
        self.h = mg_setup(dim, element, n_cells, n_levels, self.options, k_cell, self.device, mass)

    def close(self):
        if getattr(self, "h", None):
            mg_hierarchy_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return mg_get_info(self.h)

    def solve(self, b_dev, x_dev, rel_tol):
        return mg_solve(self.h, b_dev, x_dev, rel_tol, self.options.max_iters)

    def solve_host(self, b_host, x_host, rel_tol):
        return mg_solve_host(self.h, b_host, x_host, rel_tol, self.options.max_iters)

    def heat(self, bF_dev, g, u_dev, rel_tol, method=MG_METHOD_DC):
        return mg_heat(self.h, bF_dev, g, u_dev, rel_tol, method)

    def heat_host(self, bF_host, g, u_host, rel_tol, method=MG_METHOD_DC):
        return mg_heat_host(self.h, bF_host, g, u_host, rel_tol, method)

    def pcg(self, b_dev, x_dev, rel_tol):
        return mg_pcg(self.h, b_dev, x_dev, rel_tol, self.options.max_iters)

    def pcg_host(self, b_host, x_host, rel_tol):
        return mg_pcg_host(self.h, b_host, x_host, rel_tol, self.options.max_iters)

    def cycle(self, b_dev, x_dev, n_cycles):
        return mg_cycle(self.h, b_dev, x_dev, n_cycles)

    def export(self, level, which=0, precision=MG_FP64):
        return mg_export_operator(self.h, level, which, precision)


# ---------------------------------------------------------------------------------
# Serving (mg_serve_*)
# ---------------------------------------------------------------------------------
def mg_serve_config_default(**overrides):
    c = mg_serve_config()
    lib().mg_serve_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        if hasattr(c, k):
            setattr(c, k, v)
        else:
            setattr(c.options, k, v)
    return c


class Server:
    """A continuous-batching multigrid server (one mg_server); torch supplies the budget memory."""

    def __init__(self, hbm_budget_bytes, device=None, **overrides):
        self.config = mg_serve_config_default(hbm_budget_bytes=int(hbm_budget_bytes), **overrides)
        self.device = device if device is not None else TorchDevice()
        h = _vp()
        _check(lib().mg_serve_create(ctypes.byref(self.config), ctypes.byref(self.device.struct), ctypes.byref(h)))
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            lib().mg_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, dim, n_cells, n_levels, b_host, rel_tol):
        """Copy b_host (float64, n DOFs) into a new request; returns its ticket."""
        p, _k = _problem(dim, MG_Q1, n_cells, n_levels)
        b = np.ascontiguousarray(b_host, dtype=np.float64)
        t = ctypes.c_uint64(0)
        _check(lib().mg_serve_submit(self.h, ctypes.byref(p), _as_dp(b), float(rel_tol), ctypes.byref(t)))
        return t.value

    def submit_rhs(self, dim, n_cells, n_levels, modes, rel_tol, f_const=1.0):
        """Request whose load vector the server assembles from sine modes (or f = f_const)."""
        p, _k = _problem(dim, MG_Q1, n_cells, n_levels)
        f, _keep = _rhs(modes, f_const)
        t = ctypes.c_uint64(0)
        _check(lib().mg_serve_submit_rhs(self.h, ctypes.byref(p), ctypes.byref(f), float(rel_tol), ctypes.byref(t)))
        return t.value

    def poll(self, ticket, n=None):
        """None while pending, else (status, x or None, iters)."""
        x = np.zeros(n) if n else None
        it = ctypes.c_int(0)
        st = lib().mg_serve_poll(self.h, ctypes.c_uint64(ticket), _as_dp(x) if x is not None else None,
                                 ctypes.byref(it))
        if st == MG_PENDING:
            return None
        if st in (MG_EINVAL, MG_ENOTFOUND, MG_ECUDA):
            raise MgError(st, last_error())
        return st, x, it.value

    def wait(self, ticket, n, timeout_s=600.0, hist_len=0):
        """Block until the request finishes: (status, x, iters, hist)."""
        x = np.zeros(n)
        it = ctypes.c_int(0)
        hist = np.zeros(max(hist_len, 1))
        st = lib().mg_serve_wait(self.h, ctypes.c_uint64(ticket), float(timeout_s), _as_dp(x), ctypes.byref(it),
                                 _as_dp(hist), int(hist_len))
        if st in (MG_EINVAL, MG_ENOTFOUND, MG_ECUDA, MG_ETIMEOUT):
            raise MgError(st, last_error())
        return st, x, it.value, hist[:min(hist_len, it.value + 1)].copy()

    def stats(self):
        s = mg_serve_stats()
        _check(lib().mg_serve_get_stats(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in mg_serve_stats._fields_}

    def reset_stats(self):
        _check(lib().mg_serve_reset_stats(self.h))

    def tune(self, shapes, repeats=2, rel_tol=1e-8):
        """shapes: list of (dim, n_cells, n_levels). Returns the chosen (rows_per_thread, blocks_per_sm)."""
        arr = (mg_problem * len(shapes))(*[mg_problem(d, MG_Q1, n, l, None, 0.0) for d, n, l in shapes])
        r, b = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().mg_serve_tune(self.h, arr, len(shapes), int(repeats), float(rel_tol), ctypes.byref(r),
                                   ctypes.byref(b)))
        return r.value, b.value
