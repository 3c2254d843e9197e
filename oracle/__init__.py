"""FP64 CPU oracle for the geometric multigrid solve.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference leg may import, call, link or execute anything in this
package. It shares no code with the CUDA library (``paper_1609_04809_gb300``), and
neither imports the other.

The numerics live in ``mg_oracle.c`` (plain C, FP64, one sequential sum per row,
compiled with ``-ffp-contract=off``); the exact reference-element tables come from
``elements.py`` (rational arithmetic). This module only marshals arrays.

Which parts of the paper each function follows:
  * ``Hierarchy``: the mesh hierarchy by uniform refinement and the system matrix on
    every level (Sec. 5.1), Q1 / rotated-Q1 stiffness matrices, grid transfers with
    R = P^T (Sec. 5.4).
  * ``Hierarchy.solve``: V-cycles of the paper's V-cycle algorithm (Sec. 5.3) inside a
    defect-correction loop that stops at a relative residual.
  * ``Hierarchy.pcg``: conjugate gradients preconditioned by one V-cycle (Sec. 1: multigrid
    as a preconditioner of a Krylov method), Saad's Alg. 9.1.
  * ``load_vector``: the load vector of the sparse FE system.
  * ``assemble_mass``, ``heat_B``, ``heat_rhs``, ``heat``: Crank-Nicolson time stepping of
    the heat equation (Sec. 6 "Model Problem") on the shifted operator A + (2/dt) M.
  * ``colours`` / ``gs_sweep``: the multicolour Gauss-Seidel smoother (the paper's
    Gauss-Seidel step, Eq. GS, on DOFs numbered colour-wise, Sec. 4 "DOF Reordering").
"""
import ctypes
import os
import subprocess

import numpy as np

from . import elements

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

Q1, RQ1, P1, P2 = 0, 1, 2, 3
JACOBI, CHEBYSHEV, GAUSS_SEIDEL = 0, 1, 2

_lib = None


def build(force=False):
    """Compile mg_oracle.c into oracle/_build/liboracle.so (gcc, FP64, no contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _CSR(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.POINTER(ctypes.c_int64)),
                ("col", ctypes.POINTER(ctypes.c_int32)),
                ("val", ctypes.POINTER(ctypes.c_double))]


class _Opts(ctypes.Structure):
    _fields_ = [("smoother", ctypes.c_int), ("omega", ctypes.c_double),
                ("cheb_degree", ctypes.c_int), ("nu_pre", ctypes.c_int),
                ("nu_post", ctypes.c_int), ("cheb_hi", ctypes.c_double),
                ("cheb_ratio", ctypes.c_double), ("max_iters", ctypes.c_int)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        dp, ip, vp = P(ctypes.c_double), P(ctypes.c_int), ctypes.c_void_p
        L.orc_ndofs.restype = ctypes.c_int64
        L.orc_ndofs.argtypes = [ctypes.c_int] * 3
        L.orc_assemble.argtypes = [ctypes.c_int] * 3 + [dp, dp, P(_CSR)]
        L.orc_prolongation.argtypes = [ctypes.c_int] * 3 + [dp, P(_CSR)]
        L.orc_csr_free.argtypes = [P(_CSR)]
        L.orc_load_vector.argtypes = [ctypes.c_int] * 4 + [dp, ip, ctypes.c_double, dp, dp]
        L.orc_l2_error.restype = ctypes.c_double
        L.orc_l2_error.argtypes = [ctypes.c_int] * 4 + [dp, ip, dp, dp]
        L.orc_setup.restype = vp
        L.orc_setup.argtypes = [ctypes.c_int] * 4 + [dp, dp, dp, ctypes.c_int, ctypes.c_uint64, dp, ctypes.c_double]
        L.orc_assemble_mass.argtypes = [ctypes.c_int] * 3 + [dp, P(_CSR)]
        L.orc_heat_rhs.argtypes = [P(_CSR), dp, dp, ctypes.c_double, dp]
        L.orc_load_vector_tet.argtypes = [ctypes.c_int] * 3 + [dp, ip, ctypes.c_double, dp, dp]
        L.orc_free.argtypes = [vp]
        L.orc_solve.restype = ctypes.c_int
        L.orc_solve.argtypes = [vp, P(_Opts), dp, dp, ctypes.c_double, dp, ip]
        L.orc_vcycle.argtypes = [vp, P(_Opts), dp, dp]
        L.orc_pcg.restype = ctypes.c_int
        L.orc_pcg.argtypes = [vp, P(_Opts), dp, dp, ctypes.c_double, dp, ip]
        L.orc_n_levels.argtypes = [vp]
        L.orc_level_N.argtypes = [vp, ctypes.c_int]
        L.orc_level_galerkin.argtypes = [vp, ctypes.c_int]
        L.orc_level_lambda.restype = ctypes.c_double
        L.orc_level_lambda.argtypes = [vp, ctypes.c_int]
        for nm in ("orc_level_A", "orc_level_P", "orc_level_R"):
            getattr(L, nm).restype = P(_CSR)
            getattr(L, nm).argtypes = [vp, ctypes.c_int]
        L.orc_spmv.argtypes = [P(_CSR), dp, dp]
        L.orc_lu_factor.restype = ctypes.c_int
        L.orc_lu_factor.argtypes = [dp, ctypes.c_int, ip]
        L.orc_lu_solve.argtypes = [dp, ctypes.c_int, ip, dp, dp]
        L.orc_n_colours.restype = ctypes.c_int
        L.orc_n_colours.argtypes = [ctypes.c_int] * 2
        L.orc_colour.restype = ctypes.c_int
        L.orc_colour.argtypes = [ctypes.c_int] * 3 + [ctypes.c_int64]
        L.orc_gs_sweep.argtypes = [P(_CSR), dp, ip, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
        L.orc_power_lambda.restype = ctypes.c_double
        L.orc_power_lambda.argtypes = [P(_CSR), dp, ctypes.c_int, ctypes.c_uint64]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


class CSR:
    """A copied CSR matrix (rowptr int64, col int32 ascending per row, val float64)."""

    def __init__(self, rowptr, col, val, shape):
        self.rowptr, self.col, self.val, self.shape = rowptr, col, val, shape

    @classmethod
    def _from_c(cls, c):
        n, nnz = c.nrows, c.nnz
        rowptr = np.ctypeslib.as_array(c.rowptr, shape=(n + 1,)).copy()
        col = (np.ctypeslib.as_array(c.col, shape=(nnz,)).copy() if nnz else np.zeros(0, np.int32))
        val = (np.ctypeslib.as_array(c.val, shape=(nnz,)).copy() if nnz else np.zeros(0))
        return cls(rowptr, col, val, (c.nrows, c.ncols))

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=self.shape)

    def dense(self):
        return self.to_scipy().toarray()


def set_threads(n):
    """Threads of the oracle's row loops (the results do not depend on it)."""
    lib().orc_set_threads(int(n))


def get_threads():
    return int(lib().orc_get_threads())


def ndofs(dim, elem, N):
    return int(lib().orc_ndofs(dim, elem, N))


def kref(dim, elem):
    """Unit-cell element stiffness as nearest doubles (row-major); P1/P2: one Kuhn tetrahedron."""
    if elem == Q1:
        return np.array(elements.q1_stiffness(dim), dtype=np.float64)
    if elem in (P1, P2):
        assert dim == 3
        return np.array(elements.tet_stiffness(1 if elem == P1 else 2), dtype=np.float64)
    assert dim == 3
    return np.array(elements.rq1_stiffness(), dtype=np.float64)


def _rq1_w():
    return np.array(elements.rq1_prolong_table(), dtype=np.float64)


def _rq1_basis():
    return np.array(elements.rq1_basis_table(), dtype=np.float64)


def assemble(dim, elem, N, k_cell=None):
    """Stiffness matrix on N^dim cells with Dirichlet DOFs eliminated (CSR copy)."""
    L = lib()
    c = _CSR()
    K = kref(dim, elem)
    kc = _f64(k_cell)
    if L.orc_assemble(dim, elem, N, _dp(K), _dp(kc), ctypes.byref(c)) != 0:
        raise MemoryError("oracle assembly failed")
    try:
        return CSR._from_c(c)
    finally:
        L.orc_csr_free(ctypes.byref(c))


def mref(dim, elem):
    """Unit-cell element mass matrix as nearest doubles (Q1, or a Kuhn tetrahedron for P1/P2)."""
    if elem in (P1, P2):
        return np.array(elements.tet_mass(1 if elem == P1 else 2), dtype=np.float64)
    if elem != Q1:
        raise ValueError("the mass matrix is built for Q1, P1 and P2")
    return np.array(elements.q1_mass(dim), dtype=np.float64)


def node_coords(elem, N):
    """Coordinates (n x 3) of the DOFs of a tetrahedral element (P1: vertices; P2: points of
    the grid of 2N cells), lexicographic with x fastest."""
    M = N if elem == P1 else 2 * N
    w = np.arange(1, M) / M
    z, y, x = np.meshgrid(w, w, w, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def assemble_mass(dim, elem, N):
    """Consistent mass matrix on N^dim cells, Dirichlet DOFs eliminated (CSR copy)."""
    L = lib()
    c = _CSR()
    Mr = mref(dim, elem)
    if L.orc_assemble_mass(dim, elem, N, _dp(Mr), ctypes.byref(c)) != 0:
        raise MemoryError("oracle assembly failed")
    try:
        return CSR._from_c(c)
    finally:
        L.orc_csr_free(ctypes.byref(c))


def heat_B(dim, elem, N, sigma, k_cell=None):
    """B = sigma M - A of the scaled Crank-Nicolson step (entrywise, same pattern)."""
    A = assemble(dim, elem, N, k_cell)
    M = assemble_mass(dim, elem, N)
    assert np.array_equal(A.rowptr, M.rowptr) and np.array_equal(A.col, M.col)
    return CSR(A.rowptr, A.col, sigma * M.val - A.val, A.shape)


def heat_rhs(B, u, bF, t):
    """rhs = B u + t bF (one Crank-Nicolson right-hand side, see mg_oracle.c)."""
    rhs = np.zeros(B.shape[0])
    lib().orc_heat_rhs(ctypes.byref(_c_csr(B)), _dp(_f64(u)), _dp(_f64(bF)), float(t), _dp(rhs))
    return rhs


def heat(H, B, bF, g, u0, tol, method="dc"):
    """Crank-Nicolson steps n = 0 .. len(g)-2 of (A + sigma M) u^{n+1} = B u^n + (g_n + g_{n+1}) bF,
    each solved from u^n by defect correction ("dc") or V-cycle CG ("pcg"). Returns (u, iters)."""
    u = np.array(u0, dtype=np.float64)
    its = []
    for k in range(len(g) - 1):
        rhs = heat_rhs(B, u, bF, g[k] + g[k + 1])
        solve = H.solve if method == "dc" else H.pcg
        u, hist, it, conv = solve(rhs, tol, x0=u)
        if not conv:
            raise RuntimeError("oracle heat step %d did not converge" % k)
        its.append(it)
    return u, its


def prolongation(dim, elem, Nc):
    """P from Nc to 2 Nc cells per axis (fine rows, coarse columns)."""
    L = lib()
    c = _CSR()
    W = _rq1_w()
    if L.orc_prolongation(dim, elem, Nc, _dp(W), ctypes.byref(c)) != 0:
        raise MemoryError("oracle prolongation failed")
    try:
        return CSR._from_c(c)
    finally:
        L.orc_csr_free(ctypes.byref(c))


def _modes(modes):
    """modes: list of (amp, (k1, k2[, k3])) or None."""
    if not modes:
        return 0, None, None
    amp = np.array([m[0] for m in modes], dtype=np.float64)
    kf = np.zeros((len(modes), 3), dtype=np.int32)
    for i, m in enumerate(modes):
        kf[i, :len(m[1])] = m[1]
    return len(modes), amp, np.ascontiguousarray(kf.reshape(-1))


def load_vector(dim, elem, N, modes=None, fconst=1.0):
    """b_i = int f phi_i by 3-point Gauss per axis per cell.

    ``modes``: the manufactured solution u = sum amp * prod sin(k_d pi x_d), f = -Lap u;
    ``None``: f = fconst.
    """
    L = lib()
    nm, amp, kf = _modes(modes)
    b = np.zeros(ndofs(dim, elem, N))
    if elem in (P1, P2):  # b = M f_I (see mg_oracle.c)
        L.orc_load_vector_tet(elem, N, nm, _dp(amp), _ip(kf), float(fconst), _dp(mref(dim, elem)), _dp(b))
        return b
    L.orc_load_vector(dim, elem, N, nm, _dp(amp), _ip(kf), float(fconst), _dp(_rq1_basis()), _dp(b))
    return b


def l2_error(dim, elem, N, modes, x):
    L = lib()
    nm, amp, kf = _modes(modes)
    x = _f64(x)
    return float(L.orc_l2_error(dim, elem, N, nm, _dp(amp), _ip(kf), _dp(_rq1_basis()), _dp(x)))


def _c_csr(A):
    return _CSR(A.shape[0], A.shape[1], len(A.val),
                A.rowptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                A.col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(A.val))


def n_colours(dim, elem):
    return int(lib().orc_n_colours(dim, elem))


def colours(dim, elem, N):
    """Gauss-Seidel colour of every DOF (parity colouring, see mg_oracle.c)."""
    n = ndofs(dim, elem, N)
    L = lib()
    return np.array([L.orc_colour(dim, elem, N, i) for i in range(n)], dtype=np.intc)


def gs_sweep(A, colour, ncol, b, x, backward=False):
    """One multicolour Gauss-Seidel sweep (returns the new x; x is not modified)."""
    c = _c_csr(A)
    d = A.to_scipy().diagonal()
    dinv = np.array([1.0 / v for v in d])
    x = np.array(x, dtype=np.float64)
    colour = np.ascontiguousarray(colour, dtype=np.intc)
    lib().orc_gs_sweep(ctypes.byref(c), _dp(dinv), _ip(colour), ncol, int(backward), _dp(_f64(b)), _dp(x))
    return x


def spmv(A, x):
    """y = A x with the oracle's sequential row sums."""
    c = _c_csr(A)
    x = _f64(x)
    y = np.zeros(A.shape[0])
    lib().orc_spmv(ctypes.byref(c), _dp(x), _dp(y))
    return y


def lu_solve_dense(a, b):
    """Dense LU with partial pivoting (first maximal |a| wins) and the two triangular solves."""
    a = np.array(a, dtype=np.float64, order="C")
    n = a.shape[0]
    piv = np.zeros(n, dtype=np.intc)
    if lib().orc_lu_factor(_dp(a), n, _ip(piv)) != 0:
        raise np.linalg.LinAlgError("singular")
    x = np.zeros(n)
    b = _f64(b)
    lib().orc_lu_solve(_dp(a), n, _ip(piv), _dp(b), _dp(x))
    return x


class Options:
    """Multigrid options (same meaning as the library's mg_options)."""

    def __init__(self, smoother=JACOBI, omega=0.8, cheb_degree=2, nu_pre=2, nu_post=2,
                 cheb_hi=1.1, cheb_ratio=4.0, max_iters=100, power_iters=20, power_seed=1609):
        self.smoother, self.omega, self.cheb_degree = smoother, omega, cheb_degree
        self.nu_pre, self.nu_post = nu_pre, nu_post
        self.cheb_hi, self.cheb_ratio, self.max_iters = cheb_hi, cheb_ratio, max_iters
        self.power_iters, self.power_seed = power_iters, power_seed

    def _c(self):
        return _Opts(self.smoother, self.omega, self.cheb_degree, self.nu_pre, self.nu_post,
                     self.cheb_hi, self.cheb_ratio, self.max_iters)


class Hierarchy:
    """Levels 0 (coarsest) .. L (finest, N cells per axis) of the oracle's multigrid."""

    def __init__(self, dim, elem, N, n_levels, k_cell=None, opts=None, mass=0.0):
        """mass: sigma of the shifted operator A + sigma M on every level (0: A alone)."""
        self.opts = opts or Options()
        L = lib()
        self.dim, self.elem, self.N, self.n_levels = dim, elem, N, n_levels
        self.n = ndofs(dim, elem, N)
        K, W, kc = kref(dim, elem), _rq1_w(), _f64(k_cell)
        piters = self.opts.power_iters if self.opts.smoother == CHEBYSHEV else 0
        Mr = mref(dim, elem) if mass else None
        self._h = L.orc_setup(dim, elem, N, n_levels, _dp(K), _dp(W), _dp(kc), piters,
                              self.opts.power_seed, _dp(Mr), float(mass))
        if not self._h:
            raise ValueError("oracle setup failed (bad sizes or out of memory)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    def level_N(self, l):
        return lib().orc_level_N(self._h, l)

    def galerkin(self, l):
        return bool(lib().orc_level_galerkin(self._h, l))

    def lam(self, l):
        return float(lib().orc_level_lambda(self._h, l))

    def A(self, l):
        return CSR._from_c(lib().orc_level_A(self._h, l).contents)

    def P(self, l):
        return CSR._from_c(lib().orc_level_P(self._h, l).contents)

    def R(self, l):
        return CSR._from_c(lib().orc_level_R(self._h, l).contents)

    def vcycle(self, r):
        r = _f64(r)
        c = np.zeros(self.n)
        lib().orc_vcycle(self._h, ctypes.byref(self.opts._c()), _dp(r), _dp(c))
        return c

    def solve(self, b, tol, x0=None, max_iters=None):
        """Defect correction with V-cycles. Returns (x, hist, iters, converged)."""
        o = self.opts._c()
        if max_iters is not None:
            o.max_iters = max_iters
        b = _f64(b)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        hist = np.zeros(o.max_iters + 1)
        it = ctypes.c_int(0)
        st = lib().orc_solve(self._h, ctypes.byref(o), _dp(b), _dp(x), float(tol), _dp(hist),
                             ctypes.byref(it))
        return x, hist[:it.value + 1].copy(), it.value, st == 0

    def pcg(self, b, tol, x0=None, max_iters=None):
        """CG preconditioned by one V-cycle. Returns (x, hist, iters, converged)."""
        o = self.opts._c()
        if max_iters is not None:
            o.max_iters = max_iters
        b = _f64(b)
        x = np.zeros(self.n) if x0 is None else np.array(x0, dtype=np.float64)
        hist = np.zeros(o.max_iters + 1)
        it = ctypes.c_int(0)
        st = lib().orc_pcg(self._h, ctypes.byref(o), _dp(b), _dp(x), float(tol), _dp(hist), ctypes.byref(it))
        return x, hist[:it.value + 1].copy(), it.value, st == 0
