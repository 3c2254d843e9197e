"""Edge cases of the widened solve paths (Gauss-Seidel, CG, Crank-Nicolson, tetrahedra),
each against the oracle."""
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


def _pcg(orc, dim, elem, N, L, b, x0=None, tol=1e-10, max_iters=100, sm=1, nu=1):
    H = mg.Hierarchy(dim, elem, N, L, smoother=sm, nu_pre=nu, nu_post=nu, max_iters=max_iters)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd) if x0 is None else torch.from_numpy(x0.copy()).cuda()
    st, it, hist = H.pcg(bd, x, tol)
    O = orc.Hierarchy(dim, elem, N, L, opts=orc.Options(smoother=sm, nu_pre=nu, nu_post=nu, max_iters=max_iters))
    xo, ho, ito, conv = O.pcg(b, tol, x0=x0)
    return (st, it, hist, x.cpu().numpy()), (conv, ito, ho, xo)


def test_pcg_edge_cases(orc):
    n = mg.mg_ndofs(3, 0, 8)
    # zero right-hand side: converged before the first V-cycle
    g, o = _pcg(orc, 3, 0, 8, 2, np.zeros(n))
    assert g[0] == mg.MG_OK and g[1] == 0 and o[1] == 0 and np.all(g[3] == 0)
    # one level: M^-1 = A^-1, one iteration
    b = W.random_vector(n, seed=81)
    g, o = _pcg(orc, 3, 0, 8, 1, b, tol=1e-12)
    assert g[0] == mg.MG_OK and g[1] == o[1] == 1
    assert np.linalg.norm(g[3] - o[3]) <= 1e-12 * np.linalg.norm(o[3])
    # max_iters reached: MG_ENOCONV, the last iterate near the oracle's
    g, o = _pcg(orc, 3, 0, 16, 3, W.random_vector(mg.mg_ndofs(3, 0, 16), seed=82), tol=1e-15, max_iters=3)
    assert g[0] == mg.MG_ENOCONV and not o[0] and g[1] == o[1] == 3
    assert np.linalg.norm(g[3] - o[3]) <= 1e-10 * np.linalg.norm(o[3])
    # warm start
    nb = mg.mg_ndofs(3, 0, 16)
    b = W.random_vector(nb, seed=83)
    g, o = _pcg(orc, 3, 0, 16, 3, b, x0=W.random_vector(nb, seed=84))
    assert g[0] == mg.MG_OK and abs(g[1] - o[1]) <= 1
    assert np.linalg.norm(g[3] - o[3]) <= 1e-9 * np.linalg.norm(o[3])


def test_gs_edge_cases(orc):
    # smoothing on one side only (nu_pre = 0): GS runs backward after the correction
    n = mg.mg_ndofs(3, 0, 16)
    b = W.random_vector(n, seed=85)
    H = mg.Hierarchy(3, 0, 16, 3, smoother=mg.MG_GAUSS_SEIDEL, nu_pre=0, nu_post=2)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, hist = H.solve(bd, x, 1e-10)
    O = orc.Hierarchy(3, 0, 16, 3, opts=orc.Options(smoother=orc.GAUSS_SEIDEL, nu_pre=0, nu_post=2))
    xo, ho, ito, conv = O.solve(b, 1e-10)
    assert st == mg.MG_OK and it == ito and np.array_equal(x.cpu().numpy(), xo)
    # 2D Q1 (four colours, none mergeable) and rotated Q1 (six)
    for dim, elem, N, L in [(2, 0, 32, 4), (3, 1, 8, 3)]:
        n = mg.mg_ndofs(dim, elem, N)
        b = W.random_vector(n, seed=86)
        H = mg.Hierarchy(dim, elem, N, L, smoother=mg.MG_GAUSS_SEIDEL, nu_pre=1, nu_post=1)
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        H.solve(bd, x, 1e-10)
        O = orc.Hierarchy(dim, elem, N, L, opts=orc.Options(smoother=orc.GAUSS_SEIDEL, nu_pre=1, nu_post=1))
        assert np.array_equal(x.cpu().numpy(), O.solve(b, 1e-10)[0])


def test_heat_edge_cases(orc):
    wl = W.heat_workload(dim=3, n_cells=8, n_levels=2, dt=0.01, t_end=0.01)
    H = mg.Hierarchy(3, 0, 8, 2, mass=wl["sigma"])
    bF = mg.mg_load_vector(3, 0, 8, modes=wl["source_modes"])
    u = torch.from_numpy(wl["u0"].copy()).cuda()
    # no steps: u unchanged
    st, its = H.heat(torch.from_numpy(bF).cuda(), wl["g"][:1], u, 1e-10)
    assert st == mg.MG_OK and len(its) == 0 and np.array_equal(u.cpu().numpy(), wl["u0"])
    # one step with a zero source from u = 0: stays exactly zero
    z = torch.zeros_like(u)
    st, its = H.heat(torch.zeros_like(u), np.zeros(2), z, 1e-10)
    assert st == mg.MG_OK and np.all(z.cpu().numpy() == 0)
    # one step equals the oracle's
    st, its = H.heat(torch.from_numpy(bF).cuda(), wl["g"], u, 1e-10)
    O = orc.Hierarchy(3, 0, 8, 2, mass=wl["sigma"], opts=orc.Options())
    bFo = orc.load_vector(3, orc.Q1, 8, modes=wl["source_modes"])
    uo, ito = orc.heat(O, orc.heat_B(3, orc.Q1, 8, wl["sigma"]), bFo, wl["g"], wl["u0"], 1e-10)
    assert np.array_equal(u.cpu().numpy(), uo) and list(its) == list(ito)


@pytest.mark.parametrize("elem,N,L", [(2, 2, 1), (2, 4, 2), (3, 2, 1), (3, 4, 2)])
def test_tet_smallest_grids(orc, elem, N, L):
    """P1 on 2 cells: one DOF; P2 on 2 cells: 27 DOFs (one level: the LU solve)."""
    n = mg.mg_ndofs(3, elem, N)
    b = W.random_vector(n, seed=87)
    H = mg.Hierarchy(3, elem, N, L, omega=0.7)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, hist = H.solve(bd, x, 1e-12)
    xd = np.linalg.solve(orc.assemble(3, elem, N).dense(), b)
    assert st == mg.MG_OK and np.linalg.norm(x.cpu().numpy() - xd) <= 1e-10 * np.linalg.norm(xd)
