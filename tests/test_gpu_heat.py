"""GPU parity of Crank-Nicolson time stepping (the paper's heat model problem, Sec. 6).

Every step forms rhs = (sigma M - A) u + (g_k + g_{k+1}) bF with the oracle's row order and
solves (A + sigma M) u' = rhs from u by the multigrid defect correction, whose FP64
iterates agree with the oracle's bit for bit; so do the time steps. With CG as the step
solver the inner products are summed in another order (tolerance derived in
test_gpu_pcg.py); the mixed path is gated by the distance to the oracle's solution.
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


def _heat_both(orc, dim, N, L, dt, t_end, smoother=0, nu=2, tol=1e-10, method=mg.MG_METHOD_DC,
               precision=mg.MG_FP64, k=None):
    wl = W.heat_workload(dim=dim, n_cells=N, n_levels=L, dt=dt, t_end=t_end)
    sigma = wl["sigma"]
    H = mg.Hierarchy(dim, 0, N, L, k_cell=k, mass=sigma, smoother=smoother, nu_pre=nu, nu_post=nu,
                     precision=precision)
    bF = mg.mg_load_vector(dim, 0, N, modes=wl["source_modes"])
    u = torch.from_numpy(wl["u0"].copy()).cuda()
    st, its = H.heat(torch.from_numpy(bF).cuda(), wl["g"], u, tol, method)
    O = orc.Hierarchy(dim, 0, N, L, k_cell=k, mass=sigma, opts=orc.Options(smoother=smoother, nu_pre=nu, nu_post=nu))
    B = orc.heat_B(dim, 0, N, sigma, k)
    uo, ito = orc.heat(O, B, orc.load_vector(dim, 0, N, modes=wl["source_modes"]), wl["g"], wl["u0"], tol,
                       "pcg" if method == mg.MG_METHOD_PCG else "dc")
    return wl, H, (st, its, u.cpu().numpy()), (ito, uo)


@pytest.mark.parametrize("dim,N,L,sm,nu", [(2, 32, 4, 0, 2), (3, 16, 3, 1, 1), (3, 16, 3, 2, 2), (2, 48, 3, 2, 3)])
def test_heat_dc_fp64_bitwise(orc, dim, N, L, sm, nu):
    wl, H, g, o = _heat_both(orc, dim, N, L, dt=0.01, t_end=0.1, smoother=sm, nu=nu)
    st, its, u = g
    assert st == mg.MG_OK and list(its) == list(o[0])
    assert np.array_equal(u, o[1])


def test_heat_variable_coefficient_galerkin_levels(orc):
    N, L = 32, 4
    k = W.k_blocks(N, dim=3, blocks_per_axis=8, seed=20260101)
    wl, H, g, o = _heat_both(orc, 3, N, L, dt=0.01, t_end=0.05, smoother=1, nu=1, k=k)
    assert H.info()["galerkin"] == [1, 0, 0, 0]
    assert g[0] == mg.MG_OK and list(g[1]) == list(o[0]) and np.array_equal(g[2], o[1])


def test_heat_pcg_steps(orc):
    wl, H, g, o = _heat_both(orc, 3, 16, 3, dt=0.01, t_end=0.1, smoother=1, nu=1, method=mg.MG_METHOD_PCG)
    st, its, u = g
    assert st == mg.MG_OK
    assert np.all(np.abs(np.array(its) - np.array(o[0])) <= 1)
    assert np.linalg.norm(u - o[1]) <= 1e-9 * np.linalg.norm(o[1])


@pytest.mark.parametrize("method", [mg.MG_METHOD_DC, mg.MG_METHOD_PCG])
def test_heat_mixed_precision(orc, method):
    wl, H, g, o = _heat_both(orc, 3, 32, 4, dt=0.01, t_end=0.1, smoother=1, nu=1, method=method,
                             precision=mg.MG_MIXED)
    assert g[0] == mg.MG_OK
    assert np.linalg.norm(g[2] - o[1]) <= 1e-8 * np.linalg.norm(o[1])


def test_heat_host_api_and_device_api_agree():
    wl = W.heat_workload(dim=3, n_cells=32, n_levels=4, dt=0.01, t_end=0.05)
    H = mg.Hierarchy(3, 0, 32, 4, mass=wl["sigma"], smoother=1, nu_pre=1, nu_post=1)
    bF = mg.mg_load_vector(3, 0, 32, modes=wl["source_modes"])
    u = torch.from_numpy(wl["u0"].copy()).cuda()
    H.heat(torch.from_numpy(bF).cuda(), wl["g"], u, 1e-10)
    uh = wl["u0"].copy()
    H.heat_host(bF, wl["g"], uh, 1e-10)
    assert np.array_equal(u.cpu().numpy(), uh)


def test_heat_needs_a_mass_shift():
    H = mg.Hierarchy(3, 0, 16, 3)
    v = torch.zeros(mg.mg_ndofs(3, 0, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MgError) as e:
        H.heat(v, np.ones(3), v, 1e-8)
    assert e.value.status == mg.MG_EINVAL


def test_heat_workload_full_size_first_steps(orc):
    """The 128^3 heat workload (dt = 0.01): its first three steps equal the oracle's bit for bit."""
    wl, H, g, o = _heat_both(orc, 3, 128, 6, dt=0.01, t_end=0.03, smoother=1, nu=1)
    assert g[0] == mg.MG_OK and list(g[1]) == list(o[0]) and np.array_equal(g[2], o[1])


def test_heat_solution_tracks_the_exact_solution():
    """64^3, dt = 0.01 to t = 0.5: u_h is within the discretisation error of u(t)."""
    wl = W.heat_workload(dim=3, n_cells=64, n_levels=5, dt=0.01, t_end=0.5)
    H = mg.Hierarchy(3, 0, 64, 5, mass=wl["sigma"], smoother=1, nu_pre=1, nu_post=1)
    bF = mg.mg_load_vector(3, 0, 64, modes=wl["source_modes"])
    u = torch.from_numpy(wl["u0"].copy()).cuda()
    st, its = H.heat(torch.from_numpy(bF).cuda(), wl["g"], u, 1e-10)
    exact = W.q1_nodal_sine(3, 64, amp=wl["exact_amp"])
    err = np.max(np.abs(u.cpu().numpy() - exact)) / np.max(np.abs(exact))
    assert st == mg.MG_OK and err < 2e-3 and np.all(its <= 8)
