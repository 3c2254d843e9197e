"""GPU parity of P1 / P2 on the Kuhn tetrahedra of the cube grid against the FP64 oracle.

The level operators, transfers and load vectors are built on the host bit for bit like
the oracle's (tests/test_abi_host.py); the sweeps and transfers then follow the oracle's
arithmetic, so FP64 solves agree bit for bit. P1 runs on DIA storage (7 stored
diagonals, 15 with a mass shift), P2 on ELL or CSR.
"""
import numpy as np
import pytest

from paper_1609_04809_gb300 import mg
from paper_1609_04809_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    torch.cuda.set_device(0)


def _both(orc, elem, N, L, b, smoother=0, omega=0.7, nu=2, storage=mg.MG_STORAGE_AUTO, tol=1e-10,
          precision=mg.MG_FP64, method="dc", k=None, use_graph=1):
    H = mg.Hierarchy(3, elem, N, L, k_cell=k, smoother=smoother, omega=omega, nu_pre=nu, nu_post=nu,
                     storage=storage, precision=precision, use_graph=use_graph)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, hist = (H.pcg if method == "pcg" else H.solve)(bd, x, tol)
    O = orc.Hierarchy(3, elem, N, L, k_cell=k, opts=orc.Options(smoother=smoother, omega=omega, nu_pre=nu, nu_post=nu))
    xo, ho, ito, conv = (O.pcg if method == "pcg" else O.solve)(b, tol)
    return H, O, (st, it, hist, x.cpu().numpy()), (conv, ito, ho, xo)


CASES = [
    # id, elem, N, L, smoother, nu
    ("p1_32_jacobi", 2, 32, 4, 0, 2),
    ("p1_32_cheb", 2, 32, 4, 1, 1),
    ("p1_24_gs", 2, 24, 3, 2, 2),
    ("p2_16_jacobi", 3, 16, 4, 0, 2),
    ("p2_12_cheb", 3, 12, 3, 1, 1),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_tet_fp64_bitwise(orc, case):
    _, elem, N, L, sm, nu = case
    b = orc.load_vector(3, elem, N, modes=W.manufactured_modes(3))
    assert np.array_equal(b, mg.mg_load_vector(3, elem, N, modes=W.manufactured_modes(3)))
    H, O, g, o = _both(orc, elem, N, L, b, smoother=sm, nu=nu)
    assert g[0] == mg.MG_OK and o[0] and g[1] == o[1]
    assert np.array_equal(g[3], o[3])
    assert np.all(np.abs(g[2] - o[2]) <= 1e-12 * o[2])
    if elem == mg.MG_P1:
        assert H.info()["storage"][L - 1] == mg.MG_STORAGE_DIA


@pytest.mark.parametrize("elem,N,L,storage", [(2, 16, 3, mg.MG_STORAGE_ELL), (2, 16, 3, mg.MG_STORAGE_CSR),
                                              (3, 8, 3, mg.MG_STORAGE_ELL), (3, 8, 3, mg.MG_STORAGE_CSR)])
@pytest.mark.parametrize("graph", [1, 0])
def test_tet_every_storage_and_graph_mode(orc, elem, N, L, storage, graph):
    b = W.random_vector(mg.mg_ndofs(3, elem, N), seed=71)
    H, O, g, o = _both(orc, elem, N, L, b, storage=storage, use_graph=graph)
    assert H.info()["storage"][L - 1] == storage
    assert g[1] == o[1] and np.array_equal(g[3], o[3])


def test_tet_variable_coefficient_galerkin_levels(orc):
    N, L = 32, 4
    k = W.k_blocks(N, dim=3, blocks_per_axis=8, seed=20260101)
    b = orc.load_vector(3, mg.MG_P1, N)
    H, O, g, o = _both(orc, mg.MG_P1, N, L, b, smoother=1, nu=1, k=k)
    assert H.info()["galerkin"] == [1, 0, 0, 0]
    assert g[1] == o[1] and np.array_equal(g[3], o[3])


@pytest.mark.parametrize("elem,N,L", [(2, 32, 4), (3, 16, 4)])
def test_tet_pcg(orc, elem, N, L):
    b = orc.load_vector(3, elem, N, modes=W.manufactured_modes(3))
    H, O, g, o = _both(orc, elem, N, L, b, smoother=1, nu=1, method="pcg")
    assert g[0] == mg.MG_OK and abs(g[1] - o[1]) <= 1
    m = min(len(g[2]), len(o[2]))
    assert np.all(np.abs(g[2][:m] - o[2][:m]) <= 1e-10 * o[2][:m])
    assert np.linalg.norm(g[3] - o[3]) <= 1e-9 * np.linalg.norm(o[3])


@pytest.mark.parametrize("elem,N,L", [(2, 32, 4), (3, 16, 4)])
def test_tet_mixed_precision(orc, elem, N, L):
    b = orc.load_vector(3, elem, N, modes=W.manufactured_modes(3))
    H, O, g, o = _both(orc, elem, N, L, b, smoother=1, nu=1, precision=mg.MG_MIXED)
    assert g[0] == mg.MG_OK
    assert np.linalg.norm(b - orc.spmv(O.A(L - 1), g[3])) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(g[3] - o[3]) <= 1e-8 * np.linalg.norm(o[3])


@pytest.mark.parametrize("sm,nu", [(1, 1), (2, 3)])
def test_tet_heat_steps_bitwise(orc, sm, nu):
    """Crank-Nicolson on P1 (the paper's model problem with its own element family; with
    Gauss-Seidel 3+3, the paper's smoother)."""
    N, L = 16, 3
    wl = W.heat_workload(dim=3, n_cells=N, n_levels=L, dt=0.01, t_end=0.05)
    sigma = wl["sigma"]
    H = mg.Hierarchy(3, mg.MG_P1, N, L, mass=sigma, smoother=sm, nu_pre=nu, nu_post=nu)
    assert H.info()["storage"][L - 1] == mg.MG_STORAGE_DIA
    bF = mg.mg_load_vector(3, mg.MG_P1, N, modes=wl["source_modes"])
    u = torch.from_numpy(wl["u0"].copy()).cuda()
    st, its = H.heat(torch.from_numpy(bF).cuda(), wl["g"], u, 1e-10)
    O = orc.Hierarchy(3, mg.MG_P1, N, L, mass=sigma, opts=orc.Options(smoother=sm, nu_pre=nu, nu_post=nu))
    bFo = orc.load_vector(3, orc.P1, N, modes=wl["source_modes"])
    uo, ito = orc.heat(O, orc.heat_B(3, orc.P1, N, sigma), bFo, wl["g"], wl["u0"], 1e-10)
    assert st == mg.MG_OK and list(its) == list(ito) and np.array_equal(u.cpu().numpy(), uo)


@pytest.mark.parametrize("elem,N,L,nu,storage", [(2, 32, 4, 2, mg.MG_STORAGE_DIA), (2, 16, 3, 3, mg.MG_STORAGE_CSR),
                                                 (3, 16, 4, 2, mg.MG_STORAGE_AUTO), (3, 8, 3, 1, mg.MG_STORAGE_ELL)])
def test_tet_gauss_seidel_bitwise(orc, elem, N, L, nu, storage):
    """P1 (four colours) and P2 (fifteen colours) Gauss-Seidel, every storage of the copy."""
    b = orc.load_vector(3, elem, N, modes=W.manufactured_modes(3))
    H, O, g, o = _both(orc, elem, N, L, b, smoother=mg.MG_GAUSS_SEIDEL, nu=nu, storage=storage)
    assert g[0] == mg.MG_OK and g[1] == o[1] and np.array_equal(g[3], o[3])


@pytest.mark.parametrize("name", ["p1_3d_128_cheb", "p2_3d_64_cheb"])
def test_tet_full_size_workloads(orc, name):
    """The 2M-DOF tetrahedral workloads: converged in FP64 (the true residual by the
    no-allocation residual), and the nodal error of the manufactured solution is at the
    level of the element's order."""
    c = W.TET_CONFIGS[name]
    elem, N, L = c["element"], c["n_cells"], c["n_levels"]
    b = orc.load_vector(3, elem, N, modes=W.manufactured_modes(3))
    H = mg.Hierarchy(3, elem, N, L, smoother=c["smoother"], omega=c["omega"], nu_pre=c["nu_pre"], nu_post=c["nu_post"])
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, hist = H.solve(bd, x, 1e-10)
    assert st == mg.MG_OK and it <= 40  # P1: 23 V(1,1) Chebyshev cycles at 128^3
    r = torch.empty_like(bd)
    assert mg.mg_residual_norm_noalloc(H.h, bd, x, r) <= 1.0001e-10 * np.linalg.norm(b)
    X = orc.node_coords(elem, N)
    err = np.max(np.abs(x.cpu().numpy() - np.prod(np.sin(np.pi * X), axis=1)))
    assert err < (4e-4 if elem == mg.MG_P1 else 2e-6), err  # about 2.5e-4 and 2e-7 extrapolated


@pytest.mark.parametrize("elem,N,L", [(3, 8, 3), (1, 8, 3), (0, 16, 3), (2, 16, 3)])
@pytest.mark.parametrize("precision", [mg.MG_FP64, mg.MG_MIXED])
def test_sell_storage(orc, elem, N, L, precision):
    """SELL-32 (rows sorted by length, slices of 32) on every element: FP64 bitwise; mixed
    converged; exported operator equal to the host one; CG and the no-allocation residual
    read it too."""
    b = W.random_vector(mg.mg_ndofs(3, elem, N), seed=91)
    H, O, g, o = _both(orc, elem, N, L, b, storage=mg.MG_STORAGE_SELL, precision=precision, omega=0.7)
    assert H.info()["storage"][L - 1] == mg.MG_STORAGE_SELL
    assert g[0] == mg.MG_OK
    if precision == mg.MG_FP64:
        assert g[1] == o[1] and np.array_equal(g[3], o[3])
        rp, col, val = mg.mg_export_operator(H.h, L - 1, 0, mg.MG_FP64)
        A = O.A(L - 1)
        assert np.array_equal(rp, A.rowptr) and np.array_equal(col, A.col) and np.array_equal(val, A.val)
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        st, it, hist = H.pcg(bd, x, 1e-10)
        xo, ho, ito, conv = O.pcg(b, 1e-10)
        assert st == mg.MG_OK and np.linalg.norm(x.cpu().numpy() - xo) <= 1e-9 * np.linalg.norm(xo)
        r = torch.empty_like(bd)
        nr = mg.mg_residual_norm_noalloc(H.h, bd, x, r)
        assert abs(nr - np.linalg.norm(b - orc.spmv(A, x.cpu().numpy()))) <= 1e-12 * np.linalg.norm(b)
    else:
        assert np.linalg.norm(b - orc.spmv(O.A(L - 1), g[3])) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("elem,N,L", [(1, 16, 3), (2, 16, 3), (3, 16, 3), (3, 8, 3)])
@pytest.mark.parametrize("precision", [mg.MG_FP64, mg.MG_MIXED])
def test_explicit_transfers(orc, elem, N, L, precision):
    """Rotated Q1, P1, P2: P and R stored explicitly in SELL-32 (rows sorted by length;
    the prolongation of rotated Q1 has rows without entries next to the boundary); the
    device transfers exported as CSR equal the host operators; FP64 solves bitwise, mixed
    converged to the FP64 residual."""
    b = W.random_vector(mg.mg_ndofs(3, elem, N), seed=93)
    H, O, g, o = _both(orc, elem, N, L, b, precision=precision)
    assert H.info()["transfer"] == [mg.MG_TRANSFER_NONE] + [mg.MG_TRANSFER_SELL] * (L - 1)
    assert g[0] == mg.MG_OK
    if precision == mg.MG_FP64:
        assert g[1] == o[1] and np.array_equal(g[3], o[3])
        for l in range(1, L):
            for which, M in ((1, O.P(l)), (2, O.R(l))):
                rp, col, val = mg.mg_export_operator(H.h, l, which, mg.MG_FP64)
                assert np.array_equal(rp, M.rowptr) and np.array_equal(col, M.col) and np.array_equal(val, M.val)
    else:
        assert np.linalg.norm(b - orc.spmv(O.A(L - 1), g[3])) <= 1e-10 * np.linalg.norm(b)


def test_q1_transfers_from_the_grid():
    H = mg.Hierarchy(3, mg.MG_Q1, 16, 3)
    assert H.info()["transfer"] == [mg.MG_TRANSFER_NONE, mg.MG_TRANSFER_GRID, mg.MG_TRANSFER_GRID]
