"""Per-cell coefficient storage of the FP32 levels of a mixed-precision 3D Q1 hierarchy:
a level rediscretised with a per-cell coefficient k_e is sum_e k_e h K_ref, so the sweep
forms each row from the eight cells around its vertex and stores one value per cell.
The FP32 V-cycle is a preconditioner inside the FP64 defect correction; the bar is the
FP64 residual recomputed by the oracle from its own matrix, and the distance to the
stored-matrix (DIA) solve."""
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


def _solve(orc, N, L, b, storage, k, sm=mg.MG_CHEBYSHEV, nu=1):
    H = mg.Hierarchy(3, mg.MG_Q1, N, L, k_cell=k, smoother=sm, nu_pre=nu, nu_post=nu, omega=0.8,
                     precision=mg.MG_MIXED, storage=storage)
    bd = torch.from_numpy(b).cuda()
    x = torch.zeros_like(bd)
    st, it, hist = H.solve(bd, x, 1e-10)
    x = x.cpu().numpy()
    nr = np.linalg.norm(b - orc.spmv(orc.assemble(3, orc.Q1, N, k_cell=k), x))
    return H, st, it, nr, x


@pytest.mark.parametrize("N,sm,nu", [(96, mg.MG_CHEBYSHEV, 1), (96, mg.MG_JACOBI, 2), (128, mg.MG_CHEBYSHEV, 2)])
def test_coef_levels_solve_like_stored_ones(orc, N, sm, nu):
    """96^3 cells, k on 12^3-cell blocks: 96^3 and 48^3 are coefficient levels, 24^3 is
    small (DIA), 12^3 and 6^3 straddle the blocks (Galerkin, DIA). 128^3 cells, k on
    16^3-cell blocks: the 128^3 level is swept three planes per thread, so the pairs the
    march carries from plane to plane are exercised (at 96^3 each thread owns one plane)."""
    L = 5
    k = W.k_blocks(N, dim=3, blocks_per_axis=8, seed=20260101)
    b = orc.load_vector(3, orc.Q1, N)
    Hc, st, it, nr, xc = _solve(orc, N, L, b, mg.MG_STORAGE_COEF, k, sm, nu)
    Hd, st_d, it_d, nr_d, xd = _solve(orc, N, L, b, mg.MG_STORAGE_DIA, k, sm, nu)
    info = Hc.info()
    if N == 96:
        assert info["galerkin"] == [1, 1, 0, 0, 0]
    assert info["storage"] == [mg.MG_STORAGE_DIA] * 3 + [mg.MG_STORAGE_COEF] * 2
    assert info["device_bytes"] < Hd.info()["device_bytes"]
    assert st == st_d == mg.MG_OK
    assert nr <= 1e-10 * np.linalg.norm(b) and nr_d <= 1e-10 * np.linalg.norm(b)
    assert it <= it_d + 1
    assert np.linalg.norm(xc - xd) <= 1e-6 * np.linalg.norm(xd)
    # one V-cycle from x = 0: the two storages apply the same operator up to FP32
    # rounding, so the first iterate agrees far below the first cycle's reduction
    bd = torch.from_numpy(b).cuda()
    x1c, x1d = torch.zeros_like(bd), torch.zeros_like(bd)
    Hc.cycle(bd, x1c, 1)
    Hd.cycle(bd, x1d, 1)
    x1c, x1d = x1c.cpu().numpy(), x1d.cpu().numpy()
    assert np.linalg.norm(x1c - x1d) <= 1e-4 * np.linalg.norm(x1d)


def test_coef_export_is_the_oracle_operator_in_fp32(orc):
    """The operator a coefficient level applies, exported: the oracle's structure, every
    entry within FP32 rounding of the oracle's FP64 value (relative to the row's diagonal)."""
    N, L = 64, 4
    k = W.k_blocks(N, dim=3, blocks_per_axis=4, seed=3)
    H = mg.Hierarchy(3, mg.MG_Q1, N, L, k_cell=k, precision=mg.MG_MIXED, storage=mg.MG_STORAGE_COEF,
                     smoother=mg.MG_CHEBYSHEV, nu_pre=1, nu_post=1)
    assert H.info()["storage"][L - 1] == mg.MG_STORAGE_COEF
    rp, col, val = mg.mg_export_operator(H.h, L - 1, 0, mg.MG_MIXED)
    Ao = orc.assemble(3, orc.Q1, N, k_cell=k)
    assert np.array_equal(rp, Ao.rowptr) and np.array_equal(col, Ao.col)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    diag = Ao.val[col == rows]
    assert np.all(np.abs(val - Ao.val) <= 4e-7 * diag[rows])
    # the FP64 operator of the outer residual stays stored and exact
    rp64, col64, val64 = mg.mg_export_operator(H.h, L - 1, 0, mg.MG_FP64)
    assert np.array_equal(val64, Ao.val)


def test_coef_auto_and_constant_coefficient(orc):
    """With k = 1 the coefficient form holds too; storage AUTO times it against DIA and the
    constant stencil and keeps the fastest. Any choice solves to the FP64 tolerance."""
    N, L = 64, 4
    b = orc.load_vector(3, orc.Q1, N, modes=W.manufactured_modes(3))
    H, st, it, nr, x = _solve(orc, N, L, b, mg.MG_STORAGE_COEF, None)
    assert H.info()["storage"][L - 1] == mg.MG_STORAGE_COEF
    assert st == mg.MG_OK and nr <= 1e-10 * np.linalg.norm(b)
    H, st, it, nr, x = _solve(orc, N, L, b, mg.MG_STORAGE_AUTO, None)
    assert st == mg.MG_OK and nr <= 1e-10 * np.linalg.norm(b)


def test_coef_storage_rejected_where_it_does_not_apply():
    k = W.k_blocks(32, dim=3, blocks_per_axis=4, seed=1)
    for kw in (dict(precision=mg.MG_FP64), dict(precision=mg.MG_MIXED, smoother=mg.MG_GAUSS_SEIDEL),
               dict(precision=mg.MG_MIXED, mass=200.0)):
        with pytest.raises(mg.MgError) as e:
            mg.Hierarchy(3, mg.MG_Q1, 32, 3, k_cell=k, storage=mg.MG_STORAGE_COEF, **kw)
        assert e.value.status == mg.MG_EINVAL
    for dim, elem in ((2, mg.MG_Q1), (3, mg.MG_RQ1), (3, mg.MG_P1)):
        with pytest.raises(mg.MgError):
            mg.Hierarchy(dim, elem, 32, 3, storage=mg.MG_STORAGE_COEF, precision=mg.MG_MIXED)
