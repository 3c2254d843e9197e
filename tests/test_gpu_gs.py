"""GPU parity of the multicolour Gauss-Seidel smoother against the FP64 oracle.

The FP64 path evaluates every row of every colour with the oracle's arithmetic (row sums
column-ascending by fused multiply-adds, x_i + dinv_i (b_i - s)), and rows of one colour
are uncoupled, so the iterates agree bit for bit with the oracle's sequential sweep in
colour order. The mixed path (FP32 V-cycle, FP64 defect correction) is gated by the
true FP64 relative residual, recomputed by the oracle from its own matrix.
"""
import numpy as np
import pytest

from paper_1609_04809_gb300 import mg
from paper_1609_04809_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GS = mg.MG_GAUSS_SEIDEL


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    torch.cuda.set_device(0)


def _both(orc, dim, elem, N, L, b, nu=(2, 2), storage=mg.MG_STORAGE_AUTO, k=None, tol=1e-10,
          precision=mg.MG_FP64, use_graph=1):
    H = mg.Hierarchy(dim, elem, N, L, k_cell=k, smoother=GS, nu_pre=nu[0], nu_post=nu[1],
                     storage=storage, precision=precision, use_graph=use_graph)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, hist = H.solve(bd, x, tol)
    O = orc.Hierarchy(dim, elem, N, L, k_cell=k,
                      opts=orc.Options(smoother=orc.GAUSS_SEIDEL, nu_pre=nu[0], nu_post=nu[1]))
    xo, ho, ito, conv = O.solve(b, tol)
    return H, O, (st, it, hist, x.cpu().numpy()), (conv, ito, ho, xo)


CASES = [
    # id, dim, elem, N, L, nu
    ("q1_2d_64", 2, 0, 64, 5, (2, 2)),
    ("q1_2d_96_v33", 2, 0, 96, 4, (3, 3)),    # the paper's three smoothing steps each way
    ("q1_3d_32", 3, 0, 32, 4, (2, 2)),
    ("q1_3d_24_v12", 3, 0, 24, 3, (1, 2)),
    ("rq1_16", 3, 1, 16, 4, (2, 2)),
    ("rq1_12_v33", 3, 1, 12, 3, (3, 3)),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_gs_fp64_bitwise(orc, case):
    _, dim, elem, N, L, nu = case
    b = orc.load_vector(dim, elem, N, modes=W.manufactured_modes(dim))
    H, O, g, o = _both(orc, dim, elem, N, L, b, nu=nu)
    st, it, hist, x = g
    conv, ito, ho, xo = o
    assert st == mg.MG_OK and conv and it == ito
    assert np.array_equal(x, xo)
    assert np.all(np.abs(hist - ho) <= 1e-12 * ho)


@pytest.mark.parametrize("dim,elem,N,L,storage", [(3, 0, 16, 3, mg.MG_STORAGE_DIA), (3, 0, 16, 3, mg.MG_STORAGE_ELL),
                                                   (3, 0, 16, 3, mg.MG_STORAGE_CSR), (2, 0, 40, 3, mg.MG_STORAGE_CSR),
                                                   (3, 1, 8, 3, mg.MG_STORAGE_ELL), (3, 1, 8, 3, mg.MG_STORAGE_CSR)])
@pytest.mark.parametrize("graph", [1, 0])
def test_gs_every_storage_and_graph_mode(orc, dim, elem, N, L, storage, graph):
    b = W.random_vector(mg.mg_ndofs(dim, elem, N), seed=31)
    H, O, g, o = _both(orc, dim, elem, N, L, b, storage=storage, use_graph=graph)
    assert H.info()["storage"][L - 1] == storage
    assert g[1] == o[1] and np.array_equal(g[3], o[3])


def test_gs_galerkin_levels(orc):
    dim, N, L = 3, 32, 4
    k = W.k_blocks(N, dim=3, blocks_per_axis=8, seed=20260101)
    b = orc.load_vector(dim, 0, N)
    H, O, g, o = _both(orc, dim, 0, N, L, b, k=k)
    assert H.info()["galerkin"] == [1, 0, 0, 0]
    assert g[0] == mg.MG_OK and g[1] == o[1] and np.array_equal(g[3], o[3])


def test_gs_vcycle_alone_bitwise(orc):
    """One V-cycle on a random defect (no outer loop): the colour order of pre- and post-smoothing."""
    dim, elem, N, L = 3, 0, 32, 4
    r = W.random_vector(mg.mg_ndofs(dim, elem, N), seed=32)
    H = mg.Hierarchy(dim, elem, N, L, smoother=GS, nu_pre=1, nu_post=1)
    rd = torch.from_numpy(r).cuda()
    c = torch.zeros_like(rd)
    H.cycle(rd, c, 1)
    O = orc.Hierarchy(dim, elem, N, L, opts=orc.Options(smoother=orc.GAUSS_SEIDEL, nu_pre=1, nu_post=1))
    assert np.array_equal(c.cpu().numpy(), O.vcycle(r))


@pytest.mark.parametrize("dim,elem,N,L", [(3, 0, 32, 4), (3, 1, 16, 4), (2, 0, 128, 6)])
def test_gs_mixed_precision_reaches_fp64_tolerance(orc, dim, elem, N, L):
    b = orc.load_vector(dim, elem, N, modes=W.manufactured_modes(dim))
    H, O, g, o = _both(orc, dim, elem, N, L, b, precision=mg.MG_MIXED)
    st, it, hist, x = g
    assert st == mg.MG_OK
    A = O.A(L - 1)
    assert np.linalg.norm(b - orc.spmv(A, x)) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - o[3]) <= 1e-8 * np.linalg.norm(o[3])
    assert it <= o[1] + 2


def test_gs_rejected_by_serving():
    with pytest.raises(mg.MgError) as e:
        mg.Server(1 << 30, smoother=GS)
    assert e.value.status == mg.MG_EINVAL and "Gauss-Seidel" in str(e.value)


def test_gs_full_size_128(orc):
    """The 128^3 Q1 workload with Gauss-Seidel V(1,1) at full size, as bench --smoother
    gauss-seidel runs it (DIA, colour pairs): bit for bit the oracle's iterates."""
    c = W.CONFIGS["q1_3d_128_cheb"]
    b = orc.load_vector(3, 0, c["n_cells"], modes=W.manufactured_modes(3))
    H, O, g, o = _both(orc, 3, 0, c["n_cells"], c["n_levels"], b, nu=(1, 1))
    assert H.info()["storage"][c["n_levels"] - 1] == mg.MG_STORAGE_DIA
    st, it, hist, x = g
    conv, ito, ho, xo = o
    assert st == mg.MG_OK and conv and it == ito
    assert np.array_equal(x, xo)
