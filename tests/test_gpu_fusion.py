"""The first pre-smoothing step of a level starts from x = 0, so the kernel that makes the
level's right-hand side can take it (the restriction from the finer level; on the finest
level of a mixed hierarchy the FP64 outer residual). Taken there or as a sweep of its own
(mg_options.fuse_first = 1 or 0), every product and sum is the same, so the iterates and
the residual history must agree bit for bit: on stored (DIA, SELL) and formed (stencil,
per-cell coefficient) levels, structured and explicit (SELL) transfers, Jacobi and
Chebyshev, FP64 and mixed precision."""
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


def _run(dim, elem, N, L, fuse, k=None, **opts):
    """Three V-cycles from x = 0, a solve to 1e-9 and (symmetric V-cycles) a CG solve."""
    H = mg.Hierarchy(dim, elem, N, L, k_cell=k, fuse_first=fuse, **opts)
    n = mg.mg_ndofs(dim, elem, N)
    rng = np.random.default_rng(7)
    b = torch.from_numpy(rng.standard_normal(n)).cuda()
    x = torch.zeros_like(b)
    H.cycle(b, x, 3)
    xs = torch.zeros_like(b)
    st, it, hist = H.solve(b, xs, 1e-9)
    pcg = None
    if opts.get("nu_pre", 2) == opts.get("nu_post", 2) and opts.get("smoother") != mg.MG_GAUSS_SEIDEL:
        xp = torch.zeros_like(b)
        pst, pit, phist = H.pcg(b, xp, 1e-9)
        pcg = (pst, pit, np.asarray(phist)[:pit + 1], xp.cpu().numpy())
    info = H.info()
    H.close()
    return x.cpu().numpy(), st, it, np.asarray(hist), xs.cpu().numpy(), info, pcg


CASES = [
    # dim, element, cells, levels, precision, smoother, nu, storage, k blocks per axis
    (3, mg.MG_Q1, 64, 4, mg.MG_FP64, mg.MG_CHEBYSHEV, 2, mg.MG_STORAGE_AUTO, 0),
    (3, mg.MG_Q1, 64, 4, mg.MG_FP64, mg.MG_JACOBI, 1, mg.MG_STORAGE_AUTO, 0),
    (3, mg.MG_Q1, 64, 4, mg.MG_MIXED, mg.MG_CHEBYSHEV, 2, mg.MG_STORAGE_STENCIL, 0),
    (3, mg.MG_Q1, 64, 4, mg.MG_MIXED, mg.MG_JACOBI, 2, mg.MG_STORAGE_DIA, 0),
    (3, mg.MG_Q1, 128, 5, mg.MG_MIXED, mg.MG_CHEBYSHEV, 2, mg.MG_STORAGE_COEF, 8),
    (2, mg.MG_Q1, 256, 6, mg.MG_MIXED, mg.MG_CHEBYSHEV, 2, mg.MG_STORAGE_AUTO, 0),
    (3, mg.MG_RQ1, 32, 4, mg.MG_MIXED, mg.MG_CHEBYSHEV, 2, mg.MG_STORAGE_AUTO, 0),
    (3, mg.MG_RQ1, 32, 4, mg.MG_FP64, mg.MG_JACOBI, 2, mg.MG_STORAGE_AUTO, 0),
    (3, mg.MG_P1, 32, 4, mg.MG_MIXED, mg.MG_CHEBYSHEV, 1, mg.MG_STORAGE_AUTO, 0),
]


@pytest.mark.parametrize("dim,elem,N,L,prec,sm,nu,storage,kb", CASES)
def test_fused_first_step_equals_the_separate_sweep(dim, elem, N, L, prec, sm, nu, storage, kb):
    k = W.k_blocks(N, dim=3, blocks_per_axis=kb, seed=20260101) if kb else None
    opts = dict(smoother=sm, nu_pre=nu, nu_post=nu, omega=0.8, precision=prec, storage=storage, coarse_tail=0)
    xf, stf, itf, hf, sf, info_f, pf = _run(dim, elem, N, L, 1, k, **opts)
    x0, st0, it0, h0, s0, info_0, p0 = _run(dim, elem, N, L, 0, k, **opts)
    assert info_f["storage"] == info_0["storage"]
    assert info_f["kernels_per_cycle"] < info_0["kernels_per_cycle"]
    assert np.array_equal(xf, x0), np.max(np.abs(xf - x0))
    assert stf == st0 == mg.MG_OK and itf == it0
    assert np.array_equal(hf[:itf + 1], h0[:it0 + 1])
    assert np.array_equal(sf, s0)
    # CG preconditioned by the V-cycle: on a mixed hierarchy its residual kernels (init and
    # update) take the finest first step too
    assert pf[0] == p0[0] == mg.MG_OK and pf[1] == p0[1]
    assert np.array_equal(pf[2], p0[2]) and np.array_equal(pf[3], p0[3])


def test_nothing_to_fuse_for_gauss_seidel_or_no_presmoothing():
    """Gauss-Seidel sweeps in place from a zeroed x, and nu_pre = 0 has no first step:
    fuse_first changes nothing there."""
    for opts in (dict(smoother=mg.MG_GAUSS_SEIDEL, nu_pre=1, nu_post=1),
                 dict(smoother=mg.MG_JACOBI, nu_pre=0, nu_post=2)):
        a = _run(3, mg.MG_Q1, 32, 3, 1, None, coarse_tail=0, **opts)
        b = _run(3, mg.MG_Q1, 32, 3, 0, None, coarse_tail=0, **opts)
        assert a[5]["kernels_per_cycle"] == b[5]["kernels_per_cycle"]
        assert a[2] == b[2] and np.array_equal(a[3][:a[2] + 1], b[3][:b[2] + 1])
        assert np.array_equal(a[0], b[0])
