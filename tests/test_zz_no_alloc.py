"""mg_residual_norm_noalloc: the residual entry point for callers that cannot allocate.

It must give the same residual norm as the regular path (mg_cycle reports
||b - A x|| / ||b|| of the iterate it starts from) and the same residual vector as
b - A x evaluated by the oracle on its own matrix, on two calls in a row (the second
call reuses the fixed scratch array the first one left behind), and it must allocate
nothing: neither the hierarchy's allocator nor torch's sees an allocation during a call.
This file is collected last so that a run stopping at the first failure has already run
every other test.
"""
import numpy as np
import pytest

from paper_1609_04809_gb300 import mg
from paper_1609_04809_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("dim,elem,N,L,storage", [(3, 0, 32, 4, mg.MG_STORAGE_DIA), (2, 0, 64, 5, mg.MG_STORAGE_DIA),
                                                  (3, 1, 16, 4, mg.MG_STORAGE_ELL), (3, 0, 16, 3, mg.MG_STORAGE_CSR)])
def test_noalloc_residual_matches_regular_path(orc, dim, elem, N, L, storage):
    H = mg.Hierarchy(dim, elem, N, L, storage=storage, omega=0.7 if elem else 0.8)
    n = H.n
    b = W.random_vector(n, seed=31)
    bd = torch.from_numpy(b).cuda()
    A = orc.assemble(dim, elem, N)
    xs = [W.random_vector(n, seed=32), W.random_vector(n, seed=33) * 1e-3]
    for x in xs:  # two calls in a row on the shared scratch
        xd = torch.from_numpy(x).cuda()
        rd = torch.empty_like(bd)
        torch.cuda.synchronize()
        before = (H.device.allocations, torch.cuda.memory_stats().get("allocation.all.allocated", 0))
        nr = mg.mg_residual_norm_noalloc(H.h, bd, xd, rd)
        torch.cuda.synchronize()
        after = (H.device.allocations, torch.cuda.memory_stats().get("allocation.all.allocated", 0))
        assert after == before, (before, after)  # the call allocated nothing
        # the regular entry point: mg_cycle reports the relative residual of its start iterate
        xc = xd.clone()
        rel = H.cycle(bd, xc, 1)
        assert abs(nr / np.linalg.norm(b) - rel) <= RTOL * rel, (nr / np.linalg.norm(b), rel)
        r_ref = b - orc.spmv(A, x)
        r = rd.cpu().numpy()
        assert np.max(np.abs(r - r_ref)) <= RTOL * np.max(np.abs(r_ref))
        assert abs(nr - np.linalg.norm(r_ref)) <= RTOL * nr
    H.close()


def test_noalloc_binding_rejects_tensors_it_cannot_use():
    """The C entry point cannot check its pointers; the binding refuses CPU tensors, the
    wrong dtype, the wrong length and non-contiguous views before launching anything."""
    H = mg.Hierarchy(2, 0, 16, 3)
    n = H.n
    good = torch.zeros(n, dtype=torch.float64, device="cuda")
    bad = [torch.zeros(n, dtype=torch.float64), torch.zeros(n, dtype=torch.float32, device="cuda"),
           torch.zeros(n - 1, dtype=torch.float64, device="cuda"),
           torch.zeros(2 * n, dtype=torch.float64, device="cuda")[::2]]
    for t in bad:
        for args in ((t, good, good), (good, t, good), (good, good, t)):
            with pytest.raises(ValueError):
                mg.mg_residual_norm_noalloc(H.h, *args)
    assert mg.mg_residual_norm_noalloc(H.h, good, good, torch.empty_like(good)) == 0.0
    H.close()
