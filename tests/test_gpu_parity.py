"""GPU parity: the CUDA multigrid path against the FP64 oracle, through the C ABI.

Tolerances (written per test):
  * FP64 path: residual history |h_gpu - h_orc| <= 1e-12 * h_orc on every entry,
    equal iteration counts, final solution ||x_gpu - x_orc|| <= 1e-9 ||x_orc||. The
    kernels evaluate every product and sum of the oracle's definition in the same
    order with the same rounding, so the iterates are expected to agree bit for bit;
    the only reordered sum is the norm inside the stopping test.
  * mixed path (FP32 V-cycle in FP64 defect correction): the true FP64 relative
    residual, recomputed by the oracle from its own matrix, is <= tol, and the
    solution differs from the oracle's by the stated bound.
"""
import numpy as np
import pytest

from paper_1609_04809_gb300 import mg
from paper_1609_04809_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HIST_RTOL = 1e-12
X_RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    torch.cuda.set_device(0)


def _orc_opts(orc, smoother, omega, nu_pre, nu_post, degree=2, max_iters=100):
    return orc.Options(smoother=smoother, omega=omega, nu_pre=nu_pre, nu_post=nu_post,
                       cheb_degree=degree, max_iters=max_iters)


def _run_both(orc, dim, elem, N, L, b, smoother=0, omega=0.8, nu_pre=2, nu_post=2, degree=2, tol=1e-10,
              k=None, precision=mg.MG_FP64, storage=mg.MG_STORAGE_AUTO, use_graph=1, max_iters=100, x0=None):
    H = mg.Hierarchy(dim, elem, N, L, k_cell=k, smoother=smoother, omega=omega, nu_pre=nu_pre,
                     nu_post=nu_post, cheb_degree=degree, precision=precision, storage=storage,
                     use_graph=use_graph, max_iters=max_iters)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd) if x0 is None else torch.from_numpy(x0.copy()).cuda()
    st, it, hist = H.solve(bd, xd, tol)
    x = xd.cpu().numpy()
    O = orc.Hierarchy(dim, elem, N, L, k_cell=k,
                      opts=_orc_opts(orc, smoother, omega, nu_pre, nu_post, degree, max_iters))
    xo, ho, ito, conv = O.solve(b, tol, x0=x0)
    return H, O, (st, it, hist, x), (conv, ito, ho, xo)


def _assert_fp64_parity(g, o, bitwise=True):
    st, it, hist, x = g
    conv, ito, ho, xo = o
    assert (st == mg.MG_OK) == conv
    assert it == ito, (it, ito)
    assert np.all(np.abs(hist - ho) <= HIST_RTOL * ho), np.max(np.abs(hist - ho) / ho)
    nx = np.linalg.norm(xo)
    assert np.linalg.norm(x - xo) <= X_RTOL * max(nx, 1e-300)
    if bitwise:
        assert np.array_equal(x, xo), np.max(np.abs(x - xo))


# small cases: several 256-row tiles and a ragged tail, every element / smoother
SMALL = [
    # id, dim, elem, N, L, smoother, omega, nu_pre, nu_post
    ("q1_2d_64_jacobi", 2, 0, 64, 5, 0, 0.8, 2, 2),          # the 2D workload at full size
    ("q1_2d_96_cheb", 2, 0, 96, 4, 1, 0.8, 1, 1),
    ("q1_3d_32_cheb", 3, 0, 32, 4, 1, 0.8, 1, 1),
    ("q1_3d_24_jacobi", 3, 0, 24, 3, 0, 0.8, 2, 2),
    ("rq1_16_jacobi", 3, 1, 16, 4, 0, 0.7, 2, 2),
    ("rq1_12_cheb", 3, 1, 12, 3, 1, 0.7, 1, 1),
]


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_fp64_matches_oracle_manufactured(orc, case):
    _, dim, elem, N, L, sm, om, n1, n2 = case
    b = orc.load_vector(dim, elem, N, modes=W.manufactured_modes(dim))
    H, O, g, o = _run_both(orc, dim, elem, N, L, b, smoother=sm, omega=om, nu_pre=n1, nu_post=n2)
    _assert_fp64_parity(g, o)
    if sm == 1:
        info = H.info()
        for l in range(1, L):
            assert info["lambda_"][l] == O.lam(l)


@pytest.mark.parametrize("storage", [mg.MG_STORAGE_DIA, mg.MG_STORAGE_ELL, mg.MG_STORAGE_CSR])
@pytest.mark.parametrize("graph", [1, 0])
def test_fp64_every_storage_and_graph_mode(orc, storage, graph):
    dim, elem, N, L = 3, 0, 16, 3
    b = W.random_vector(mg.mg_ndofs(dim, elem, N), seed=11)
    H, O, g, o = _run_both(orc, dim, elem, N, L, b, smoother=1, nu_pre=1, nu_post=1, storage=storage,
                           use_graph=graph)
    assert H.info()["storage"][L - 1] == storage
    _assert_fp64_parity(g, o)


@pytest.mark.parametrize("dim,N,L,sm", [(3, 32, 4, 1), (2, 64, 5, 0), (3, 16, 3, 0)])
@pytest.mark.parametrize("precision", [mg.MG_FP64, mg.MG_MIXED])
def test_coarse_level_tail_changes_no_bit(orc, dim, N, L, sm, precision):
    """Levels of at most 4096 rows run as one cluster launch; results are identical."""
    b = W.random_vector(mg.mg_ndofs(dim, 0, N), seed=14)
    bd = torch.from_numpy(b).cuda()
    xs, its = [], []
    for tail in (0, 1):
        H = mg.Hierarchy(dim, 0, N, L, smoother=sm, nu_pre=1 if sm else 2, nu_post=1 if sm else 2,
                         precision=precision, coarse_tail=tail)
        assert (H.info()["tail_levels"] > 0) == bool(tail)
        x = torch.zeros_like(bd)
        st, it, hist = H.solve(bd, x, 1e-10)
        assert st == mg.MG_OK
        xs.append(x.cpu().numpy())
        its.append(it)
    assert its[0] == its[1] and np.array_equal(xs[0], xs[1])
    # the default measures both launch plans at setup and keeps the faster; same bits again
    H = mg.Hierarchy(dim, 0, N, L, smoother=sm, nu_pre=1 if sm else 2, nu_post=1 if sm else 2,
                     precision=precision)
    x = torch.zeros_like(bd)
    H.solve(bd, x, 1e-10)
    assert np.array_equal(x.cpu().numpy(), xs[0])
    if precision == mg.MG_FP64:  # and both equal the oracle
        O = orc.Hierarchy(dim, 0, N, L, opts=_orc_opts(orc, sm, 0.8, 1 if sm else 2, 1 if sm else 2))
        xo, ho, ito, conv = O.solve(b, 1e-10)
        assert np.array_equal(xs[1], xo)


def test_coarse_level_tail_with_long_smoothing_fits_its_operation_list():
    """Chebyshev of degree 8 with 3+3 steps records 52 operations per level: fewer levels join the tail."""
    b = torch.from_numpy(W.random_vector(mg.mg_ndofs(3, 0, 32), seed=15)).cuda()
    xs = []
    for tail in (0, 1):
        H = mg.Hierarchy(3, 0, 32, 4, smoother=1, cheb_degree=8, nu_pre=3, nu_post=3, coarse_tail=tail)
        x = torch.zeros_like(b)
        st, it, hist = H.solve(b, x, 1e-10)
        assert st == mg.MG_OK
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])


@pytest.mark.parametrize("precision", [mg.MG_FP64, mg.MG_MIXED])
def test_programmatic_dependent_launch_changes_no_bit(precision):
    dim, elem, N, L = 3, 0, 32, 4
    b = torch.from_numpy(W.random_vector(mg.mg_ndofs(dim, elem, N), seed=13)).cuda()
    xs = []
    for pdl in (0, 1):
        H = mg.Hierarchy(dim, elem, N, L, smoother=1, nu_pre=1, nu_post=1, precision=precision, use_pdl=pdl)
        x = torch.zeros_like(b)
        H.solve(b, x, 1e-10)
        xs.append(x.cpu().numpy())
    assert np.array_equal(xs[0], xs[1])


@pytest.mark.parametrize("storage", [mg.MG_STORAGE_ELL, mg.MG_STORAGE_CSR])
def test_rq1_storage(orc, storage):
    dim, elem, N, L = 3, 1, 8, 3
    b = W.random_vector(mg.mg_ndofs(dim, elem, N), seed=12)
    H, O, g, o = _run_both(orc, dim, elem, N, L, b, omega=0.7, storage=storage)
    _assert_fp64_parity(g, o)


def test_variable_coefficient_with_galerkin_levels(orc):
    dim, elem, N, L = 3, 0, 32, 4  # blocks of 4 cells: the 4^3-cell level straddles blocks
    k = W.k_blocks(N, dim=3, blocks_per_axis=8, seed=20260101)
    b = orc.load_vector(dim, elem, N)
    H, O, g, o = _run_both(orc, dim, elem, N, L, b, smoother=1, nu_pre=1, nu_post=1, k=k)
    assert H.info()["galerkin"] == [1, 0, 0, 0]
    _assert_fp64_parity(g, o)


def test_device_operators_equal_host_operators(orc):
    for dim, elem, N, L, fmt in [(3, 0, 8, 3, mg.MG_STORAGE_DIA), (2, 0, 16, 3, mg.MG_STORAGE_DIA),
                                 (3, 1, 8, 3, mg.MG_STORAGE_ELL), (3, 0, 8, 2, mg.MG_STORAGE_CSR)]:
        H = mg.Hierarchy(dim, elem, N, L, storage=fmt)
        O = orc.Hierarchy(dim, elem, N, L)
        for l in range(L):
            for which in ((0, 1, 2) if l else (0,)):
                a = H.export(l, which)
                m = (O.A, O.P, O.R)[which](l)
                for u, v in zip(a, (m.rowptr, m.col, m.val)):
                    assert np.array_equal(u, v), (dim, elem, l, which)


def test_edge_cases(orc):
    # one level: the V-cycle is the exact LU solve
    b = W.random_vector(mg.mg_ndofs(2, 0, 8), seed=1)
    H, O, g, o = _run_both(orc, 2, 0, 8, 1, b, tol=1e-12)
    _assert_fp64_parity(g, o, bitwise=False)
    assert g[1] <= 2
    # the smallest grids: one interior DOF (2D Q1, N=2), twelve faces (rotated Q1, N=2)
    for dim, elem, N, L in [(2, 0, 2, 1), (3, 1, 2, 1), (3, 0, 4, 2), (3, 1, 4, 2)]:
        b = W.random_vector(mg.mg_ndofs(dim, elem, N), seed=N)
        H, O, g, o = _run_both(orc, dim, elem, N, L, b, omega=0.7, tol=1e-11)
        _assert_fp64_parity(g, o, bitwise=False)
    # zero right-hand side: converged before any cycle
    n = mg.mg_ndofs(3, 0, 8)
    H, O, g, o = _run_both(orc, 3, 0, 8, 2, np.zeros(n))
    assert g[0] == mg.MG_OK and g[1] == 0 and np.all(g[3] == 0)
    # no pre-smoothing
    b = W.random_vector(n, seed=5)
    H, O, g, o = _run_both(orc, 3, 0, 8, 3, b, nu_pre=0, nu_post=2)
    _assert_fp64_parity(g, o)
    # max_iters reached: MG_ENOCONV with the last iterate, identical to the oracle's
    H, O, g, o = _run_both(orc, 3, 0, 8, 3, b, max_iters=3, tol=1e-14)
    assert g[0] == mg.MG_ENOCONV and not o[0]
    _assert_fp64_parity(g, o)
    # warm start from a nonzero guess
    x0 = W.random_vector(n, seed=6)
    H, O, g, o = _run_both(orc, 3, 0, 8, 3, b, x0=x0)
    _assert_fp64_parity(g, o)


def test_host_entry_point_and_fixed_cycles(orc):
    dim, elem, N, L = 3, 0, 16, 3
    n = mg.mg_ndofs(dim, elem, N)
    b = W.random_vector(n, seed=21)
    H = mg.Hierarchy(dim, elem, N, L, smoother=1, nu_pre=1, nu_post=1, max_iters=4)
    bd = torch.from_numpy(b).cuda()
    xd = torch.zeros_like(bd)
    st, it, hist = H.solve(bd, xd, 0.0)  # runs max_iters cycles
    assert st == mg.MG_ENOCONV and it == 4
    xh = np.zeros(n)
    st2, it2, hist2 = H.solve_host(b, xh, 0.0)
    assert np.array_equal(xh, xd.cpu().numpy()) and np.array_equal(hist, hist2)
    xc = torch.zeros_like(bd)
    rel = H.cycle(bd, xc, 4)
    assert np.array_equal(xc.cpu().numpy(), xh)
    assert rel == hist[3]


def test_profiled_launch_counts(orc):
    dim, elem, N, L = 3, 0, 16, 3
    b = torch.from_numpy(W.random_vector(mg.mg_ndofs(dim, elem, N), seed=2)).cuda()
    # one launch per operation (at 16^3 every level would otherwise join the tail launch)
    H = mg.Hierarchy(dim, elem, N, L, smoother=1, nu_pre=1, nu_post=1, coarse_tail=0)
    mg.mg_profile_enable(H.h, True)  # every class and level
    x = torch.zeros_like(b)
    H.cycle(b, x, 3)
    total = sum(mg.mg_profile_read(H.h, k, l)[1] for k in range(mg.MG_K_COUNT) for l in range(L))
    assert total == 3 * H.info()["kernels_per_cycle"]
    ms, cnt, byts, flops = mg.mg_profile_read(H.h, mg.MG_K_SMOOTH, L - 1)
    # 21 stored diagonals (the face-neighbour couplings of 3D Q1 vanish) plus vectors
    assert H.info()["storage"][L - 1] == mg.MG_STORAGE_DIA
    assert cnt == 3 * 3 and ms > 0 and byts >= 21 * 15 ** 3 * 8 + 3 * 15 ** 3 * 8
    assert flops >= 2 * 21 * 15 ** 3
    # with the tail the whole V-cycle is one cluster launch, profiled as the coarse solve
    T = mg.Hierarchy(dim, elem, N, L, smoother=1, nu_pre=1, nu_post=1, coarse_tail=1)
    mg.mg_profile_enable(T.h, True)
    T.cycle(b, torch.zeros_like(b), 3)
    total = sum(mg.mg_profile_read(T.h, k, l)[1] for k in range(mg.MG_K_COUNT) for l in range(L))
    assert total == 3 * T.info()["kernels_per_cycle"] < 3 * H.info()["kernels_per_cycle"]
    assert mg.mg_profile_read(T.h, mg.MG_K_COARSE, 0)[1] == 3
    assert all(mg.mg_profile_read(T.h, mg.MG_K_SMOOTH, l)[1] == 0 for l in range(L))


@pytest.mark.parametrize("dim,elem,N,L,sm", [(3, 0, 32, 4, 1), (3, 1, 16, 4, 0), (2, 0, 128, 6, 0)])
def test_mixed_precision_reaches_fp64_tolerance(orc, dim, elem, N, L, sm):
    b = orc.load_vector(dim, elem, N, modes=W.manufactured_modes(dim))
    H, O, g, o = _run_both(orc, dim, elem, N, L, b, smoother=sm, omega=0.7 if elem else 0.8,
                           nu_pre=1 if sm else 2, nu_post=1 if sm else 2, precision=mg.MG_MIXED)
    st, it, hist, x = g
    assert st == mg.MG_OK
    A = O.A(L - 1)
    r = b - orc.spmv(A, x)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    xo = o[3]
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    assert it <= o[1] + 2
