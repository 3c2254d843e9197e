"""Failure detection without a GPU fault: inputs that hold a NaN or an infinity are
rejected on the host side of every entry point (MG_EINVAL, the hierarchy stays usable),
and a bounded wait on a serving request that is still running ends with MG_ETIMEOUT
while the request itself carries on to its result."""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_nonfinite_right_hand_side_is_rejected(orc, bad):
    dim, N, L = 3, 16, 3
    n = mg.mg_ndofs(dim, mg.MG_Q1, N)
    b = orc.load_vector(dim, orc.Q1, N, modes=W.manufactured_modes(dim))
    H = mg.Hierarchy(dim, mg.MG_Q1, N, L, smoother=mg.MG_CHEBYSHEV, nu_pre=1, nu_post=1)
    bad_b = b.copy()
    bad_b[n // 2] = bad
    for call in (lambda bd, x: H.solve(bd, x, 1e-10), lambda bd, x: H.pcg(bd, x, 1e-10)):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        with pytest.raises(mg.MgError) as e:
            call(torch.from_numpy(bad_b).cuda(), x)
        assert e.value.status == mg.MG_EINVAL and "right-hand side" in str(e.value)
    with pytest.raises(mg.MgError) as e:
        H.solve_host(bad_b, np.zeros(n), 1e-10)
    assert e.value.status == mg.MG_EINVAL
    # a non-finite initial guess
    x0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    x0[3] = float(bad)
    with pytest.raises(mg.MgError) as e:
        H.solve(torch.from_numpy(b).cuda(), x0, 1e-10)
    assert e.value.status == mg.MG_EINVAL and "initial guess" in str(e.value)
    # the hierarchy is still usable and still matches the oracle bit for bit
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, it, hist = H.solve(torch.from_numpy(b).cuda(), x, 1e-10)
    O = orc.Hierarchy(dim, orc.Q1, N, L, opts=orc.Options(smoother=orc.CHEBYSHEV, nu_pre=1, nu_post=1))
    xo, ho, ito, conv = O.solve(b, 1e-10)
    assert st == mg.MG_OK and conv and it == ito and np.array_equal(x.cpu().numpy(), xo)


def test_nonfinite_heat_state_is_rejected():
    wl = W.heat_workload(dim=3, n_cells=8, n_levels=2, dt=0.01, t_end=0.02)
    H = mg.Hierarchy(3, mg.MG_Q1, 8, 2, mass=wl["sigma"])
    bF = torch.from_numpy(oracle.load_vector(3, oracle.Q1, 8, modes=wl["source_modes"])).cuda()
    u = torch.from_numpy(wl["u0"].copy()).cuda()
    u[0] = float("nan")
    with pytest.raises(mg.MgError) as e:
        H.heat(bF, wl["g"], u, 1e-10)
    assert e.value.status == mg.MG_EINVAL


def test_serving_rejects_nonfinite_right_hand_sides():
    S = mg.Server(1 << 30)
    try:
        n = mg.mg_ndofs(2, mg.MG_Q1, 32)
        b = np.ones(n)
        b[7] = np.nan
        with pytest.raises(mg.MgError) as e:
            S.submit(2, 32, 4, b, 1e-8)
        assert e.value.status == mg.MG_EINVAL and "right-hand side" in str(e.value)
        with pytest.raises(mg.MgError) as e:
            S.submit_rhs(2, 32, 4, [(float("inf"), (1, 2))], 1e-8)
        assert e.value.status == mg.MG_EINVAL
        with pytest.raises(mg.MgError) as e:
            S.submit_rhs(2, 32, 4, None, 1e-8, f_const=float("nan"))
        assert e.value.status == mg.MG_EINVAL
        # the server still serves
        bo = oracle.load_vector(2, oracle.Q1, 32, modes=W.random_modes(2, seed=3))
        st, x, it, _ = S.wait(S.submit(2, 32, 4, bo, 1e-8), n)
        assert st == mg.MG_OK
        assert np.linalg.norm(bo - oracle.spmv(oracle.assemble(2, oracle.Q1, 32), x)) <= 1e-8 * np.linalg.norm(bo)
    finally:
        S.close()


def test_serving_wait_times_out_and_the_request_completes():
    """A request on a new 128^3 shape needs its operator set assembled first (seconds of
    host work), so a 1 ms wait runs out; the request is not dropped and a later wait
    returns its result."""
    S = mg.Server(4 << 30)
    try:
        N, L = 128, 6
        n = mg.mg_ndofs(3, mg.MG_Q1, N)
        t = S.submit_rhs(3, N, L, W.random_modes(3, seed=11), 1e-8)
        with pytest.raises(mg.MgError) as e:
            S.wait(t, n, timeout_s=1e-3)
        assert e.value.status == mg.MG_ETIMEOUT
        assert S.poll(t, n) is None  # still pending, still known
        st, x, it, _ = S.wait(t, n, timeout_s=600.0)
        assert st == mg.MG_OK and it > 0 and np.all(np.isfinite(x))
        with pytest.raises(mg.MgError) as e:  # returned once, then forgotten
            S.poll(t, n)
        assert e.value.status == mg.MG_ENOTFOUND
    finally:
        S.close()
