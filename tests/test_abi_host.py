"""CPU checks of libmg.so: it loads, exports every declared symbol, and its host-side
setup (assembly, grid transfers, Galerkin levels, load vector) reproduces the oracle
bit for bit. No GPU is touched."""
import os
import re
import subprocess

import numpy as np
import pytest

import __graft_entry__
from paper_1609_04809_gb300 import mg
from paper_1609_04809_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build_library()
    return mg.lib()


def _declared(header):
    with open(os.path.join(ROOT, "include", header)) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", mg.lib_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (mg_\w+)", out))
    declared = [s for h in os.listdir(os.path.join(ROOT, "include")) for s in _declared(h)]
    assert declared, "no declarations found"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    bound = set(mg.SIGNATURES)
    assert set(declared) <= bound, sorted(set(declared) - bound)


def test_defaults_and_ndofs(lib):
    o = mg.mg_options_default()
    assert (o.smoother, o.omega, o.nu_pre, o.nu_post, o.precision, o.max_iters) == (0, 0.8, 2, 2, 0, 100)
    # the last fields of the struct: a layout mismatch between mg.h and the binding would
    # shift them
    assert (o.use_graph, o.use_pdl, o.coarse_tail, o.fuse_first) == (1, 1, 2, 1)
    assert mg.mg_ndofs(2, mg.MG_Q1, 64) == 63 ** 2
    assert mg.mg_ndofs(3, mg.MG_Q1, 128) == 127 ** 3
    assert mg.mg_ndofs(3, mg.MG_RQ1, 96) == 3 * 95 * 96 * 96 == 2626560
    assert mg.mg_ndofs(2, mg.MG_RQ1, 8) == -1


def _csr_equal(a, b):
    rp, c, v = a
    return (np.array_equal(rp, b.rowptr) and np.array_equal(c, b.col)
            and np.array_equal(v.view(np.uint64), b.val.view(np.uint64)))


CASES = [
    (2, 0, 16, 3, None),
    (3, 0, 8, 3, None),
    (3, 1, 8, 3, None),
    (3, 0, 16, 4, "blocks4"),  # coefficient blocks of 4 cells: the 2-cell level is Galerkin
    (3, 1, 8, 3, "blocks2"),
    (3, 2, 8, 3, None),        # P1 on Kuhn tetrahedra
    (3, 2, 16, 4, "blocks4"),
    (3, 3, 4, 2, None),        # P2
    (3, 3, 8, 3, "blocks2"),
]


def _k(dim, N, kind):
    if kind is None:
        return None
    per = {"blocks4": N // 4, "blocks2": N // 2}[kind]
    return W.k_blocks(N, dim=dim, blocks_per_axis=per, seed=3)


@pytest.mark.parametrize("dim,elem,N,L,kind", CASES)
def test_host_operators_bitwise_equal_oracle(lib, orc, dim, elem, N, L, kind):
    k = _k(dim, N, kind)
    H = orc.Hierarchy(dim, elem, N, L, k_cell=k)
    for l in range(L):
        assert _csr_equal(mg.mg_assemble_operator(dim, elem, N, L, l, 0, k), H.A(l)), ("A", l)
        if l >= 1:
            assert _csr_equal(mg.mg_assemble_operator(dim, elem, N, L, l, 1, k), H.P(l)), ("P", l)
            assert _csr_equal(mg.mg_assemble_operator(dim, elem, N, L, l, 2, k), H.R(l)), ("R", l)


@pytest.mark.parametrize("dim,elem,N,L,kind", [(2, 0, 16, 3, None), (3, 0, 8, 3, None), (3, 0, 16, 3, "blocks2"),
                                               (3, 0, 16, 3, "blocks4"), (3, 2, 8, 3, None), (3, 3, 4, 2, None)])
def test_shifted_operators_bitwise_equal_oracle(lib, orc, dim, elem, N, L, kind):
    """A + sigma M on every level (Crank-Nicolson with dt = 0.01), Galerkin levels included."""
    sigma = 200.0
    k = _k(dim, N, kind)
    H = orc.Hierarchy(dim, elem, N, L, k_cell=k, mass=sigma)
    for l in range(L):
        assert _csr_equal(mg.mg_assemble_operator(dim, elem, N, L, l, 0, k, mass=sigma), H.A(l)), ("A", l)


def test_mass_shift_is_rejected_for_rotated_q1_and_negative_sigma(lib):
    with pytest.raises(mg.MgError):
        mg.mg_assemble_operator(3, 1, 4, 2, 1, 0, mass=1.0)
    with pytest.raises(mg.MgError):
        mg.mg_assemble_operator(3, 0, 4, 2, 1, 0, mass=-1.0)


@pytest.mark.parametrize("dim,elem,N", [(2, 0, 32), (3, 0, 12), (3, 1, 6), (3, 2, 8), (3, 3, 4)])
def test_load_vector_bitwise_equal_oracle(lib, orc, dim, elem, N):
    for modes in (W.manufactured_modes(dim), W.random_modes(dim, seed=4), None):
        b1 = mg.mg_load_vector(dim, elem, N, modes=modes, f_const=1.0)
        b2 = orc.load_vector(dim, elem, N, modes=modes, fconst=1.0)
        assert np.array_equal(b1.view(np.uint64), b2.view(np.uint64))


@pytest.mark.parametrize("dim,N", [(2, 64), (3, 16)])
def test_separable_load_vector_equals_quadrature(lib, orc, dim, N):
    for modes in (W.random_modes(dim, seed=6), W.manufactured_modes(dim), None):
        b1 = mg.mg_load_vector_separable(dim, N, modes=modes, f_const=2.5)
        b2 = orc.load_vector(dim, orc.Q1, N, modes=modes, fconst=2.5)
        assert np.max(np.abs(b1 - b2)) <= 1e-13 * np.max(np.abs(b2))


def test_invalid_arguments_are_rejected(lib):
    with pytest.raises(mg.MgError) as e:
        mg.mg_assemble_operator(3, mg.MG_Q1, 12, 4, 0)  # 12 / 8 is not an integer
    assert e.value.status == mg.MG_EINVAL
    with pytest.raises(mg.MgError):
        mg.mg_assemble_operator(2, mg.MG_RQ1, 8, 2, 0)  # rotated Q1 is 3D only
    with pytest.raises(mg.MgError):
        mg.mg_assemble_operator(3, mg.MG_Q1, 8, 2, 1, which=5)


def _constant_stencil_ref(A, dim, N):
    """The constant-stencil condition written out on an oracle matrix: every entry within
    the 3^d box of its grid point, equal to the interior row's value at its position (zero
    where that row has none), and every in-grid neighbour with a nonzero stencil value
    present."""
    n1 = N - 1
    n = A.rowptr.size - 1
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))

    def coords(idx):
        c = [idx % n1, (idx // n1) % n1] + ([idx // (n1 * n1)] if dim == 3 else [])
        return np.stack(c, axis=1)

    ci, cj = coords(rows), coords(A.col.astype(np.int64))
    d = cj - ci
    if np.any(np.abs(d) > 1):
        return False
    pos = (d[:, 0] + 1) + 3 * (d[:, 1] + 1) + (9 * (d[:, 2] + 1) if dim == 3 else 0)
    i0 = 1 + n1 * (1 + (n1 if dim == 3 else 0))
    sel = rows == i0
    st, has = np.zeros(27), np.zeros(27, bool)
    st[pos[sel]], has[pos[sel]] = A.val[sel], True
    if not np.array_equal(A.val, np.where(has[pos], st[pos], 0.0)):
        return False
    present = np.zeros((n, 27), bool)
    present[rows, pos] = True
    allc = coords(np.arange(n))
    for p in range(27 if dim == 3 else 9):
        if not has[p] or st[p] == 0.0:
            continue
        dd = np.array([p % 3 - 1, (p // 3) % 3 - 1] + ([p // 9 - 1] if dim == 3 else []))
        inside = np.all((allc + dd >= 0) & (allc + dd <= n1 - 1), axis=1)
        if np.any(inside & ~present[:, p]):
            return False
    return True


@pytest.mark.parametrize("dim,elem,N,L,kind,mass", [
    (3, 0, 16, 3, None, 0.0), (2, 0, 32, 3, None, 0.0), (3, 0, 16, 3, "blocks4", 0.0),
    (3, 0, 16, 3, None, 200.0), (3, 2, 16, 3, None, 0.0), (3, 2, 16, 3, None, 200.0),
    (3, 2, 16, 4, "blocks4", 0.0)])
def test_constant_stencil_check_agrees_with_the_oracle_operator(lib, orc, dim, elem, N, L, kind, mass):
    """The library's host check behind MG_STORAGE_STENCIL against the condition written out
    on the oracle's matrices: constant coefficients (with or without the mass shift) give
    one stencil per level; per-cell coefficients and Galerkin levels do not."""
    k = _k(dim, N, kind)
    H = orc.Hierarchy(dim, elem, N, L, k_cell=k, mass=mass)
    for l in range(L):
        Nl = N >> (L - 1 - l)
        got = mg.mg_constant_stencil(dim, elem, N, L, l, k, mass=mass)
        want = Nl >= 4 and _constant_stencil_ref(H.A(l), dim, Nl)
        assert got == want, (l, got, want)
        if kind is None and Nl >= 4:
            assert got
    if kind is not None:
        assert not mg.mg_constant_stencil(dim, elem, N, L, L - 1, k, mass=mass)


def test_constant_stencil_only_for_vertex_elements(lib):
    assert not mg.mg_constant_stencil(3, mg.MG_RQ1, 16, 3, 2)
    assert not mg.mg_constant_stencil(3, mg.MG_P2, 8, 3, 2)
    # a grid of 2 cells per axis has no interior row with all neighbours inside
    assert not mg.mg_constant_stencil(3, mg.MG_Q1, 8, 3, 0)
    assert mg.mg_constant_stencil(3, mg.MG_Q1, 16, 3, 0)
