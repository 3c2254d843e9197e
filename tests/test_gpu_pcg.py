"""GPU parity of V-cycle-preconditioned CG against the FP64 oracle.

Tolerance. Every vector operation of an iteration is evaluated as in the oracle; only the
inner products differ in summation order (a fixed block tree on the GPU, Neumaier's
compensated sum in the oracle). Their relative difference is at most about
(log2 n + 2) u = 3e-15 for n = 2e6, so alpha and beta differ by that much per
iteration. With a V-cycle preconditioner (condition number of B A below 2) the
perturbation of r_k relative to ||r_k|| stays near k * 3e-15 = 1e-13 over the 5-15
iterations these solves take. The tests allow 1e-10 relative per history entry (1000x
margin), equal iteration counts (one more or fewer only where the oracle's last entry
is within 2% of the tolerance), and ||x - x_orc|| <= 1e-9 ||x_orc||.
"""
import numpy as np
import pytest

from paper_1609_04809_gb300 import mg
from paper_1609_04809_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HIST_RTOL = 1e-10
X_RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    torch.cuda.set_device(0)


def _pcg_both(orc, dim, elem, N, L, b, smoother=0, omega=0.8, nu=2, tol=1e-10, precision=mg.MG_FP64,
              storage=mg.MG_STORAGE_AUTO, use_graph=1, k=None):
    H = mg.Hierarchy(dim, elem, N, L, k_cell=k, smoother=smoother, omega=omega, nu_pre=nu, nu_post=nu,
                     precision=precision, storage=storage, use_graph=use_graph)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, hist = H.pcg(bd, x, tol)
    O = orc.Hierarchy(dim, elem, N, L, k_cell=k,
                      opts=orc.Options(smoother=smoother, omega=omega, nu_pre=nu, nu_post=nu))
    xo, ho, ito, conv = O.pcg(b, tol)
    return H, O, (st, it, hist, x.cpu().numpy()), (conv, ito, ho, xo)


def _assert_parity(g, o, tol):
    st, it, hist, x = g
    conv, ito, ho, xo = o
    assert st == mg.MG_OK and conv
    if it != ito:
        assert abs(it - ito) == 1 and abs(ho[-1] - tol) <= 0.02 * tol
    m = min(len(hist), len(ho))
    assert np.all(np.abs(hist[:m] - ho[:m]) <= HIST_RTOL * ho[:m]), np.max(np.abs(hist[:m] - ho[:m]) / ho[:m])
    assert np.linalg.norm(x - xo) <= X_RTOL * np.linalg.norm(xo)


CASES = [
    # id, dim, elem, N, L, smoother, omega, nu
    ("q1_2d_64_jacobi", 2, 0, 64, 5, 0, 0.8, 2),
    ("q1_3d_32_cheb", 3, 0, 32, 4, 1, 0.8, 1),
    ("q1_3d_32_gs", 3, 0, 32, 4, 2, 0.8, 1),
    ("q1_3d_24_jacobi", 3, 0, 24, 3, 0, 0.8, 2),
    ("rq1_16_jacobi", 3, 1, 16, 4, 0, 0.7, 2),
    ("rq1_12_gs", 3, 1, 12, 3, 2, 0.7, 2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pcg_fp64_matches_oracle(orc, case):
    _, dim, elem, N, L, sm, om, nu = case
    b = orc.load_vector(dim, elem, N, modes=W.manufactured_modes(dim))
    H, O, g, o = _pcg_both(orc, dim, elem, N, L, b, smoother=sm, omega=om, nu=nu)
    _assert_parity(g, o, 1e-10)


@pytest.mark.parametrize("storage", [mg.MG_STORAGE_DIA, mg.MG_STORAGE_ELL, mg.MG_STORAGE_CSR])
@pytest.mark.parametrize("graph", [1, 0])
def test_pcg_every_storage_and_graph_mode(orc, storage, graph):
    b = W.random_vector(mg.mg_ndofs(3, 0, 16), seed=51)
    H, O, g, o = _pcg_both(orc, 3, 0, 16, 3, b, smoother=1, nu=1, storage=storage, use_graph=graph)
    assert H.info()["storage"][2] == storage
    _assert_parity(g, o, 1e-10)


def test_pcg_variable_coefficient(orc):
    N, L = 32, 4
    k = W.k_blocks(N, dim=3, blocks_per_axis=8, seed=20260101)
    b = orc.load_vector(3, 0, N)
    H, O, g, o = _pcg_both(orc, 3, 0, N, L, b, smoother=1, nu=1, k=k)
    _assert_parity(g, o, 1e-10)
    # and CG needs fewer V-cycles than the defect correction on the jumping coefficient
    bd = torch.from_numpy(b).cuda()
    st, it_dc, _ = H.solve(bd, torch.zeros_like(bd), 1e-10)
    assert g[1] < it_dc


@pytest.mark.parametrize("smoother", [0, 1, 2])
def test_pcg_mixed_precision_reaches_fp64_tolerance(orc, smoother):
    dim, elem, N, L = 3, 0, 32, 4
    b = orc.load_vector(dim, elem, N, modes=W.manufactured_modes(dim))
    H, O, g, o = _pcg_both(orc, dim, elem, N, L, b, smoother=smoother, nu=1 if smoother else 2,
                           precision=mg.MG_MIXED)
    st, it, hist, x = g
    assert st == mg.MG_OK and it <= o[1] + 2
    assert np.linalg.norm(b - orc.spmv(O.A(L - 1), x)) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x - o[3]) <= 1e-8 * np.linalg.norm(o[3])


def test_pcg_is_deterministic_and_host_api_agrees():
    b = W.random_vector(mg.mg_ndofs(3, 0, 32), seed=52)
    H = mg.Hierarchy(3, 0, 32, 4, smoother=1, nu_pre=1, nu_post=1)
    bd = torch.from_numpy(b).cuda()
    xs = []
    for _ in range(2):
        x = torch.zeros_like(bd)
        H.pcg(bd, x, 1e-11)
        xs.append(x.cpu().numpy())
    xh = np.zeros_like(b)
    H.pcg_host(b, xh, 1e-11)
    assert np.array_equal(xs[0], xs[1]) and np.array_equal(xs[0], xh)


def test_pcg_rejects_an_unsymmetric_vcycle():
    H = mg.Hierarchy(3, 0, 16, 3, nu_pre=2, nu_post=1)
    b = torch.ones(mg.mg_ndofs(3, 0, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MgError) as e:
        H.pcg(b, torch.zeros_like(b), 1e-8)
    assert e.value.status == mg.MG_EINVAL


def test_pcg_full_size_128(orc):
    """The 128^3 Chebyshev workload at full size, as the bench runs it."""
    c = W.CONFIGS["q1_3d_128_cheb"]
    b = orc.load_vector(3, 0, c["n_cells"], modes=W.manufactured_modes(3))
    H, O, g, o = _pcg_both(orc, 3, 0, c["n_cells"], c["n_levels"], b, smoother=c["smoother"], omega=c["omega"],
                           nu=c["nu_pre"])
    _assert_parity(g, o, 1e-10)
    # fewer V-cycles than the defect correction of the same hierarchy
    bd = torch.from_numpy(b).cuda()
    st, it_dc, _ = H.solve(bd, torch.zeros_like(bd), 1e-10)
    assert g[1] <= it_dc
