"""Constant-stencil storage of the FP32 levels of a mixed-precision hierarchy (Q1, P1):
every row of a rediscretised constant-coefficient level is the same stencil, so the
level keeps one value per stencil position and masks the boundary neighbours from the
grid coordinates. The FP32 V-cycle is a preconditioner inside the FP64 defect
correction; the bar is the FP64 residual, recomputed by the oracle from its own matrix,
and the distance to the stored-matrix (DIA) solve."""
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


def _solve(orc, dim, elem, N, L, b, storage, sm=1, nu=1, omega=0.8, k=None):
    """Mixed solve to 1e-10; nr is ||b - A x|| with A assembled and applied by the oracle."""
    H = mg.Hierarchy(dim, elem, N, L, k_cell=k, smoother=sm, omega=omega, nu_pre=nu, nu_post=nu,
                     precision=mg.MG_MIXED, storage=storage)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, hist = H.solve(bd, x, 1e-10)
    x = x.cpu().numpy()
    nr = np.linalg.norm(b - orc.spmv(orc.assemble(dim, elem, N, k_cell=k), x))
    return H, st, it, nr, x


@pytest.mark.parametrize("dim,elem,N,L,sm", [(3, mg.MG_Q1, 96, 5, 1), (2, mg.MG_Q1, 256, 5, 0),
                                             (3, mg.MG_P1, 64, 4, 1)])
def test_stencil_levels_solve_like_stored_ones(orc, dim, elem, N, L, sm):
    b = W.random_vector(mg.mg_ndofs(dim, elem, N), seed=97)
    Hs, st, it, nr, xs = _solve(orc, dim, elem, N, L, b, mg.MG_STORAGE_STENCIL, sm=sm)
    Hd, st_d, it_d, nr_d, xd = _solve(orc, dim, elem, N, L, b, mg.MG_STORAGE_DIA, sm=sm)
    info = Hs.info()
    for l in range(L):
        want = mg.MG_STORAGE_STENCIL if l >= 1 and info["n"][l] >= 32768 else mg.MG_STORAGE_DIA
        assert info["storage"][l] == want, (l, info["storage"])
    assert mg.MG_STORAGE_STENCIL in info["storage"]
    assert info["device_bytes"] < Hd.info()["device_bytes"]  # no matrix stored on those levels
    assert st == st_d == mg.MG_OK
    assert nr <= 1e-10 * np.linalg.norm(b) and abs(it - it_d) <= 1
    assert np.linalg.norm(xs - xd) <= 1e-6 * np.linalg.norm(xd)  # both within cond(A) x 1e-10


def test_stencil_export_is_the_host_operator_rounded(orc):
    """The exported FP32 stencil level has the oracle's operator structure; off-diagonal
    values are the FP64 ones rounded to FP32, the diagonal the row-sum-preserving rounding
    of an interior row (equal on interior rows, within FP32 rounding on the others)."""
    dim, elem, N, L = 3, mg.MG_Q1, 64, 4
    H = mg.Hierarchy(dim, elem, N, L, precision=mg.MG_MIXED, storage=mg.MG_STORAGE_STENCIL)
    assert H.info()["storage"][L - 1] == mg.MG_STORAGE_STENCIL
    rp, col, val = mg.mg_export_operator(H.h, L - 1, 0, mg.MG_MIXED)
    Ao = orc.assemble(dim, elem, N)
    hp, hc, hv = Ao.rowptr, Ao.col, Ao.val
    assert np.array_equal(rp, hp) and np.array_equal(col, hc)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    off = col != rows
    assert np.array_equal(val[off], hv[off].astype(np.float32).astype(np.float64))
    assert np.all(np.abs(val[~off] - hv[~off]) <= 1e-6 * np.abs(hv[~off]))
    # the FP64 operator of the outer residual stays stored and exact
    rp64, col64, val64 = mg.mg_export_operator(H.h, L - 1, 0, mg.MG_FP64)
    assert np.array_equal(rp64, hp) and np.array_equal(col64, hc) and np.array_equal(val64, hv)


def test_stencil_needs_a_constant_stencil_and_falls_back_to_dia(orc):
    """A per-cell coefficient makes the rows differ: every level keeps DIA. Requests the
    storage cannot serve are rejected."""
    dim, elem, N, L = 3, mg.MG_Q1, 64, 4
    k = W.k_blocks(N, dim=3, blocks_per_axis=8, seed=5)
    b = orc.load_vector(dim, elem, N)
    H, st, it, nr, x = _solve(orc, dim, elem, N, L, b, mg.MG_STORAGE_STENCIL, k=k)
    assert H.info()["storage"] == [mg.MG_STORAGE_DIA] * L
    assert st == mg.MG_OK and nr <= 1e-10 * np.linalg.norm(b)
    for kw in (dict(precision=mg.MG_FP64), dict(precision=mg.MG_MIXED, smoother=mg.MG_GAUSS_SEIDEL)):
        with pytest.raises(mg.MgError):
            mg.Hierarchy(dim, elem, 16, 3, storage=mg.MG_STORAGE_STENCIL, **kw)
    with pytest.raises(mg.MgError):
        mg.Hierarchy(3, mg.MG_P2, 8, 2, storage=mg.MG_STORAGE_STENCIL, precision=mg.MG_MIXED)


def _solve_rq1(orc, N, L, b, storage):
    H = mg.Hierarchy(3, mg.MG_RQ1, N, L, smoother=mg.MG_JACOBI, omega=0.7, nu_pre=2, nu_post=2,
                     precision=mg.MG_MIXED, storage=storage)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, hist = H.solve(bd, x, 1e-10)
    x = x.cpu().numpy()
    return H, st, it, np.linalg.norm(b - orc.spmv(orc.assemble(3, orc.RQ1, N), x)), x


def test_rq1_face_stencil_levels_solve_like_stored_ones(orc):
    """Rotated Q1 with a constant coefficient: every face row is 6h, +h at the two
    opposite faces, -h at the eight other faces of its cells. 48^3 and 24^3 cells are
    stencil levels (n >= 32768), the smaller ones keep ELL."""
    N, L = 48, 4
    b = W.random_vector(mg.mg_ndofs(3, mg.MG_RQ1, N), seed=41)
    Hs, st, it, nr, xs = _solve_rq1(orc, N, L, b, mg.MG_STORAGE_STENCIL)
    He, st_e, it_e, nr_e, xe = _solve_rq1(orc, N, L, b, mg.MG_STORAGE_ELL)
    assert Hs.info()["storage"] == [mg.MG_STORAGE_ELL] * 2 + [mg.MG_STORAGE_STENCIL] * 2
    assert Hs.info()["device_bytes"] < He.info()["device_bytes"]
    assert st == st_e == mg.MG_OK
    assert nr <= 1e-10 * np.linalg.norm(b) and abs(it - it_e) <= 1
    assert np.linalg.norm(xs - xe) <= 1e-6 * np.linalg.norm(xe)


def test_rq1_face_stencil_export_is_the_oracle_operator(orc):
    N, L = 48, 4
    H = mg.Hierarchy(3, mg.MG_RQ1, N, L, precision=mg.MG_MIXED, storage=mg.MG_STORAGE_STENCIL, omega=0.7)
    assert H.info()["storage"][L - 1] == mg.MG_STORAGE_STENCIL
    rp, col, val = mg.mg_export_operator(H.h, L - 1, 0, mg.MG_MIXED)
    Ao = orc.assemble(3, orc.RQ1, N)
    assert np.array_equal(rp, Ao.rowptr) and np.array_equal(col, Ao.col)
    assert np.all(np.abs(val - Ao.val) <= 1e-6 * (6.0 / N))
    # the FP64 operator of the outer residual stays stored and exact
    rp64, col64, val64 = mg.mg_export_operator(H.h, L - 1, 0, mg.MG_FP64)
    assert np.array_equal(rp64, Ao.rowptr) and np.array_equal(col64, Ao.col) and np.array_equal(val64, Ao.val)


def test_stencil_with_mass_shift_heat_steps():
    """Crank-Nicolson: A + sigma M is one 27-point stencil too; heat steps on stencil levels
    agree with the stored-matrix steps to the solve tolerance."""
    N, L = 64, 4
    wl = W.heat_workload(dim=3, n_cells=N, n_levels=L, dt=0.01, t_end=0.03)
    bF = torch.from_numpy(mg.mg_load_vector(3, mg.MG_Q1, N, modes=wl["source_modes"])).cuda()
    us = []
    for storage in (mg.MG_STORAGE_STENCIL, mg.MG_STORAGE_DIA):
        H = mg.Hierarchy(3, mg.MG_Q1, N, L, mass=wl["sigma"], precision=mg.MG_MIXED, storage=storage)
        assert (mg.MG_STORAGE_STENCIL in H.info()["storage"]) == (storage == mg.MG_STORAGE_STENCIL)
        u = torch.from_numpy(wl["u0"].copy()).cuda()
        st, its = H.heat(bF, wl["g"], u, 1e-10)
        assert st == mg.MG_OK
        us.append(u.cpu().numpy())
    assert np.linalg.norm(us[0] - us[1]) <= 1e-7 * np.linalg.norm(us[1])
