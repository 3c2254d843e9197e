"""GPU tests of the continuous-batching server (mg_serve_*).

Tolerances: a served request runs the same per-row arithmetic as mg_solve in mixed
precision, so with equal iteration counts the iterates are identical (checked bit for
bit); the residual norm is reduced in a different order, which only matters for the
reported history (checked to 1e-12 relative). A request's result is the same bit for bit
alone and in any mix. Every served solution meets its tolerance in the true FP64
residual, recomputed by the oracle from its own matrix.
"""
import time

import numpy as np
import pytest

import oracle
from paper_1609_04809_gb300 import mg
from paper_1609_04809_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-8
GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    torch.cuda.set_device(0)


def _levels(dim, N):
    """Coarsest grid 4 cells per axis (9 or 27 DOFs)."""
    return int(np.log2(N)) - 1


def _rhs(dim, N, seed):
    """The request's right-hand side, assembled by the oracle."""
    return oracle.load_vector(dim, oracle.Q1, N, modes=W.random_modes(dim, seed=seed))


def _true_rel_residual(dim, N, L, b, x):
    """||b - A x|| / ||b|| with A assembled and applied by the oracle."""
    A = oracle.assemble(dim, oracle.Q1, N)
    return np.linalg.norm(b - oracle.spmv(A, x)) / np.linalg.norm(b)


def test_served_request_equals_single_solve():
    """Served requests keep the levels of at least 32768 rows as the constant stencil and
    the smaller ones in DIA, the storage mg_setup gives MG_STORAGE_STENCIL: the same bits
    as mg_solve with it (2D 256^2 and 3D 64^3 have stencil levels, the others none)."""
    S = mg.Server(2 * GB)
    try:
        for dim, N, seed in [(3, 32, 1), (2, 128, 2), (2, 256, 3), (3, 64, 4)]:
            L = _levels(dim, N)
            b = _rhs(dim, N, seed)
            st, x, it, hist = S.wait(S.submit(dim, N, L, b, TOL), b.size, hist_len=100)
            assert st == mg.MG_OK
            H = mg.Hierarchy(dim, mg.MG_Q1, N, L, smoother=mg.MG_CHEBYSHEV, nu_pre=1, nu_post=1,
                             precision=mg.MG_MIXED, storage=mg.MG_STORAGE_STENCIL)
            assert (mg.MG_STORAGE_STENCIL in H.info()["storage"]) == (b.size >= 32768)
            bd = torch.from_numpy(b).cuda()
            xd = torch.zeros_like(bd)
            st2, it2, hist2 = H.solve(bd, xd, TOL)
            assert st2 == mg.MG_OK and it == it2
            assert np.array_equal(x, xd.cpu().numpy())
            assert np.all(np.abs(hist - hist2) <= 1e-12 * hist2)
            assert _true_rel_residual(dim, N, L, b, x) <= TOL
    finally:
        S.close()


MIX = [(3, 32, 11), (2, 256, 12), (3, 16, 13), (2, 64, 14), (3, 64, 15), (2, 128, 16), (2, 512, 17)]


def test_same_result_alone_and_in_the_mix():
    S = mg.Server(4 * GB, max_active=16)
    try:
        alone = {}
        for dim, N, seed in MIX[:3]:
            b = _rhs(dim, N, seed)
            alone[seed] = S.wait(S.submit(dim, N, _levels(dim, N), b, TOL), b.size)
        # now everything at once, with the first three submitted again among the others
        tickets = []
        for dim, N, seed in MIX + MIX[:3]:
            b = _rhs(dim, N, seed)
            tickets.append((dim, N, seed, b, S.submit(dim, N, _levels(dim, N), b, TOL)))
        for dim, N, seed, b, t in tickets:
            st, x, it, _ = S.wait(t, b.size)
            assert st == mg.MG_OK, (dim, N)
            assert _true_rel_residual(dim, N, _levels(dim, N), b, x) <= TOL
            if seed in alone:
                st0, x0, it0, _ = alone[seed]
                assert it == it0 and np.array_equal(x, x0), (dim, N)
        stats = S.stats()
        assert stats["completed"] == len(MIX) + 6
        assert stats["mean_batch"] > 1.0  # requests shared the launches
        assert stats["operator_sets"] == len(set((d, n) for d, n, _ in MIX))
    finally:
        S.close()


def test_continuous_admission_under_a_small_budget():
    # room for the plan buffers and only a few 3D 64^3 requests at a time
    budget = 160 << 20
    S = mg.Server(budget, max_active=64)
    try:
        dim, N = 3, 64
        L = _levels(dim, N)
        bs = [_rhs(dim, N, 40 + k) for k in range(8)]
        ts = []
        for k, b in enumerate(bs):
            ts.append(S.submit(dim, N, L, b, TOL))
            if k == 3:
                time.sleep(0.05)  # later arrivals join requests already on the GPU
        for b, t in zip(bs, ts):
            st, x, it, _ = S.wait(t, b.size)
            assert st == mg.MG_OK
            assert _true_rel_residual(dim, N, L, b, x) <= TOL
        stats = S.stats()
        assert stats["device_bytes_peak"] <= budget
        assert stats["completed"] == 8
    finally:
        S.close()


def test_request_that_never_fits_is_rejected():
    S = mg.Server(64 << 20, max_active=8)
    try:
        b = _rhs(2, 1024, 3)
        st, x, it, _ = S.wait(S.submit(2, 1024, _levels(2, 1024), b, TOL), b.size)
        assert st == mg.MG_EBUDGET
        # the server still works for a request that fits
        b2 = _rhs(2, 64, 4)
        st2, x2, it2, _ = S.wait(S.submit(2, 64, _levels(2, 64), b2, TOL), b2.size)
        assert st2 == mg.MG_OK
    finally:
        S.close()


def test_iteration_limit_and_history():
    S = mg.Server(1 * GB, max_iters=2)
    try:
        b = _rhs(3, 32, 5)
        st, x, it, hist = S.wait(S.submit(3, 32, _levels(3, 32), b, 1e-14), b.size, hist_len=10)
        assert st == mg.MG_ENOCONV and it == 2 and len(hist) == 3
        H = mg.Hierarchy(3, mg.MG_Q1, 32, _levels(3, 32), smoother=mg.MG_CHEBYSHEV, nu_pre=1, nu_post=1,
                         precision=mg.MG_MIXED, max_iters=2)
        bd = torch.from_numpy(b).cuda()
        xd = torch.zeros_like(bd)
        st2, it2, hist2 = H.solve(bd, xd, 1e-14)
        assert st2 == mg.MG_ENOCONV and np.array_equal(x, xd.cpu().numpy())
    finally:
        S.close()


def test_server_side_right_hand_side():
    S = mg.Server(1 * GB)
    try:
        modes = W.random_modes(2, seed=8)
        b = oracle.load_vector(2, oracle.Q1, 128, modes=modes)
        r1 = S.wait(S.submit(2, 128, 6, b, TOL), b.size)
        r2 = S.wait(S.submit_rhs(2, 128, 6, modes, TOL), b.size)
        # the server factorises the same quadrature rule: equal up to rounding
        assert r1[0] == r2[0] == mg.MG_OK
        assert np.linalg.norm(r1[1] - r2[1]) <= 1e-9 * np.linalg.norm(r1[1])
        assert _true_rel_residual(2, 128, 6, b, r2[1]) <= TOL * (1 + 1e-6)
    finally:
        S.close()


def test_invalid_requests():
    S = mg.Server(256 << 20)
    try:
        with pytest.raises(mg.MgError):
            S.submit(2, 64, 1, np.zeros(63 * 63), TOL)  # one level
        with pytest.raises(mg.MgError):
            S.submit(2, 64, 2, np.zeros(63 * 63), TOL)  # coarsest 32^2 cells: too many DOFs for the LU
        with pytest.raises(mg.MgError):
            S.submit(2, 64, 5, np.zeros(63 * 63), 0.0)  # tolerance must be positive
        with pytest.raises(mg.MgError) as e:
            S.poll(123456)
        assert e.value.status == mg.MG_ENOTFOUND
    finally:
        S.close()
