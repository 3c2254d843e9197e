"""Pins of the FP64 oracle to mathematics that does not come from the oracle itself.

Each test checks the oracle against a closed form, an independent computation
(quadrature in numpy, a symbolic derivation, a library routine), an invariant, or a
special case that reduces to a textbook operator. Together they fail on a dropped term,
a wrong sign or index, or a transposed operand anywhere in assembly, transfers, the
smoothers, the coarse solve or the V-cycle.
"""
import itertools

import numpy as np
import pytest
import scipy.fft
import scipy.sparse as sp

from paper_1609_04809_gb300 import workloads as W

# ------------------------------------------------------------------------------------
# Element matrices
# ------------------------------------------------------------------------------------


def _q1_quadrature_stiffness(dim):
    """Unit-cell Q1 stiffness by 2-point Gauss (exact for these bilinear products)."""
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    nl = 2 ** dim
    K = np.zeros((nl, nl))
    for q in itertools.product(range(2), repeat=dim):
        xi = g[list(q)]
        grads = np.zeros((nl, dim))
        for a in range(nl):
            bits = [(a >> d) & 1 for d in range(dim)]
            for d in range(dim):
                val = 1.0
                for e in range(dim):
                    if e == d:
                        val *= 1.0 if bits[e] else -1.0
                    else:
                        val *= xi[e] if bits[e] else 1.0 - xi[e]
                grads[a, d] = val
        K += (0.5 ** dim) * grads @ grads.T
    return K


@pytest.mark.parametrize("dim", [2, 3])
def test_q1_element_matches_gauss_quadrature(orc, dim):
    K = orc.kref(dim, orc.Q1).reshape(2 ** dim, 2 ** dim)
    np.testing.assert_allclose(K, _q1_quadrature_stiffness(dim), rtol=0, atol=4e-16)


def test_q1_element_textbook_values(orc):
    # unit square: diagonal 2/3, edge neighbours -1/6, opposite corner -1/3
    K2 = orc.kref(2, orc.Q1).reshape(4, 4)
    assert K2[0, 0] == 2 / 3 and K2[0, 1] == -1 / 6 and K2[0, 2] == -1 / 6 and K2[0, 3] == -1 / 3
    # unit cube: diagonal 1/3, edge-adjacent 0, face-diagonal and body-diagonal -1/12
    K3 = orc.kref(3, orc.Q1).reshape(8, 8)
    assert K3[0, 0] == 1 / 3 and K3[0, 1] == 0.0 and K3[0, 3] == -1 / 12 and K3[0, 7] == -1 / 12


def test_rq1_element_symbolic(orc):
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    mons = [sympy.Integer(1), x, y, z, x ** 2 - y ** 2, y ** 2 - z ** 2]
    faces = [(x, 0), (x, 1), (y, 0), (y, 1), (z, 0), (z, 1)]

    def mean(f, var, v):
        others = [s for s in (x, y, z) if s != var]
        return sympy.integrate(f.subs(var, v), (others[0], 0, 1), (others[1], 0, 1))

    M = sympy.Matrix(6, 6, lambda i, j: mean(mons[j], *faces[i]))
    C = M.inv()
    phi = [sum(C[m, a] * mons[m] for m in range(6)) for a in range(6)]
    K = sympy.Matrix(6, 6, lambda a, b: sympy.integrate(
        sum(sympy.diff(phi[a], v) * sympy.diff(phi[b], v) for v in (x, y, z)),
        (x, 0, 1), (y, 0, 1), (z, 0, 1)))
    Korc = orc.kref(3, orc.RQ1).reshape(6, 6)
    assert np.array_equal(np.array(K, dtype=float), Korc)
    # the known closed form: 3 on the diagonal, 1 for the opposite face, -1 otherwise
    expect = -np.ones((6, 6))
    for a in range(6):
        expect[a, a] = 3
        expect[a, a ^ 1] = 1
    assert np.array_equal(Korc, expect)


# ------------------------------------------------------------------------------------
# Assembled matrices
# ------------------------------------------------------------------------------------


def _kron_q1(dim, N):
    h = 1.0 / N
    n1 = N - 1
    K1 = sp.diags([-np.ones(n1 - 1), 2 * np.ones(n1), -np.ones(n1 - 1)], [-1, 0, 1]) / h
    M1 = sp.diags([np.ones(n1 - 1), 4 * np.ones(n1), np.ones(n1 - 1)], [-1, 0, 1]) * (h / 6)
    if dim == 2:  # index = ix + n1*iy: the y factor is the outer Kronecker factor
        return (sp.kron(M1, K1) + sp.kron(K1, M1)).toarray()
    return (sp.kron(sp.kron(M1, M1), K1) + sp.kron(sp.kron(M1, K1), M1)
            + sp.kron(sp.kron(K1, M1), M1)).toarray()


@pytest.mark.parametrize("dim,N", [(2, 8), (2, 13), (3, 6), (3, 9)])
def test_q1_matrix_is_kronecker_sum(orc, dim, N):
    A = orc.assemble(dim, orc.Q1, N).dense()
    K = _kron_q1(dim, N)
    assert np.max(np.abs(A - K)) <= 1e-15 * np.max(np.abs(K))


def test_q1_closed_form_stencils(orc):
    N = 8
    A2 = orc.assemble(2, orc.Q1, N).dense()
    i = 3 + 7 * 3  # interior vertex (4, 4)
    row = A2[i].reshape(7, 7)
    np.testing.assert_allclose(row[2:5, 2:5], np.array([[-1, -1, -1], [-1, 8, -1], [-1, -1, -1]]) / 3,
                               rtol=0, atol=1e-15)
    h = 1.0 / N
    A3 = orc.assemble(3, orc.Q1, N).dense()
    i = 3 + 7 * (3 + 7 * 3)
    row = A3[i].reshape(7, 7, 7)[2:5, 2:5, 2:5]
    for dz, dy, dx in itertools.product(range(3), repeat=3):
        nz = abs(dz - 1) + abs(dy - 1) + abs(dx - 1)
        expect = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}[nz]
        assert abs(row[dz, dy, dx] - expect) <= 1e-16


def _kfield(N, dim=3, per_axis=2, seed=7):
    return W.k_blocks(N, dim=dim, blocks_per_axis=per_axis, seed=seed)


@pytest.mark.parametrize("case", ["q1_2d", "q1_3d", "rq1", "q1_vark", "rq1_vark"])
def test_symmetric_bitwise(orc, case):
    if case == "q1_2d":
        A = orc.assemble(2, orc.Q1, 9)
    elif case == "q1_3d":
        A = orc.assemble(3, orc.Q1, 6)
    elif case == "rq1":
        A = orc.assemble(3, orc.RQ1, 4)
    elif case == "q1_vark":
        A = orc.assemble(3, orc.Q1, 8, k_cell=_kfield(8))
    else:
        A = orc.assemble(3, orc.RQ1, 4, k_cell=_kfield(4))
    D = A.dense()
    assert np.array_equal(D, D.T)
    # every column index sorted and unique within its row
    for i in range(A.shape[0]):
        c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_q1_zero_row_sums_away_from_boundary(orc):
    N = 8
    k = _kfield(N)
    A = orc.assemble(3, orc.Q1, N, k_cell=k).dense()
    n1 = N - 1
    for iz, iy, ix in itertools.product(range(1, n1 - 1), repeat=3):
        i = ix + n1 * (iy + n1 * iz)
        assert abs(A[i].sum()) <= 1e-14 * A[i, i]


def test_rq1_interior_row(orc):
    N = 4
    h = 1.0 / N
    A = orc.assemble(3, orc.RQ1, N)
    # x-face at i=2 (x = 1/2), cells j=1, k=1: both neighbouring cells are interior
    i = (2 - 1) + (N - 1) * (1 + N * 1)
    cols = A.col[A.rowptr[i]:A.rowptr[i + 1]]
    vals = A.val[A.rowptr[i]:A.rowptr[i + 1]]
    assert len(cols) == 11
    d = dict(zip(cols.tolist(), vals.tolist()))
    assert d[i] == 6 * h
    assert d[i - 1] == h and d[i + 1] == h  # opposite x-faces of the two cells
    assert sorted(v for c, v in d.items() if c not in (i, i - 1, i + 1)) == [-h] * 8
    assert abs(vals.sum()) <= 1e-15


# ------------------------------------------------------------------------------------
# Transfers
# ------------------------------------------------------------------------------------


def _lin(x, y, z=0.0):
    return 1.0 + 2.0 * x + 3.0 * y + 5.0 * z


@pytest.mark.parametrize("dim,Nc", [(2, 4), (2, 8), (3, 4)])
def test_q1_prolongation_reproduces_linear_functions(orc, dim, Nc):
    """Nodal interpolation is exact for multilinear functions (rows away from the boundary)."""
    Nf = 2 * Nc
    P = orc.prolongation(dim, orc.Q1, Nc).dense()
    H, h = 1.0 / Nc, 1.0 / Nf
    ncn, nfn = Nc - 1, Nf - 1
    coords_c = list(itertools.product(range(1, Nc), repeat=dim))  # (.., y, x) order below
    uc = np.zeros(ncn ** dim)
    for I, c in enumerate(_lex(dim, Nc)):
        uc[I] = _lin(*(np.array(c) * H))
    uf = P @ uc
    for i, c in enumerate(_lex(dim, Nf)):
        if all(2 <= v <= Nf - 2 for v in c):
            assert abs(uf[i] - _lin(*(np.array(c) * h))) <= 1e-14
    assert len(coords_c) == ncn ** dim and P.shape == (nfn ** dim, ncn ** dim)


def _lex(dim, N):
    """Interior vertex coordinates (x, y[, z]) in the DOF order (x fastest)."""
    rng = range(1, N)
    if dim == 2:
        return [(x, y) for y in rng for x in rng]
    return [(x, y, z) for z in rng for y in rng for x in rng]


def _rq1_faces(N):
    """(family, center coordinates, cells) of every interior face in the DOF order."""
    h = 1.0 / N
    out = []
    for f in range(3):
        rng = []
        for k in range(N if f != 2 else N - 1):
            for j in range(N if f != 1 else N - 1):
                for i in range(N if f != 0 else N - 1):
                    rng.append((i, j, k))
        for (i, j, k) in rng:
            ijk = [i, j, k]
            ijk[f] += 1  # face position 1..N-1 along the normal
            c = [(v + 0.5) * h for v in ijk]
            c[f] = ijk[f] * h
            out.append((f, tuple(ijk), tuple(c)))
    return out


def _face_mean_quad(f, pos, h):
    """Exact mean over the face of u = lin + 7(x^2-y^2) + 11(y^2-z^2)."""
    lo = [v * h for v in pos]
    m1 = []
    m2 = []
    for d in range(3):
        if d == f:
            m1.append(lo[d])
            m2.append(lo[d] ** 2)
        else:
            a, b = lo[d], lo[d] + h
            m1.append(0.5 * (a + b))
            m2.append((a * a + a * b + b * b) / 3.0)
    return 1 + 2 * m1[0] + 3 * m1[1] + 5 * m1[2] + 7 * (m2[0] - m2[1]) + 11 * (m2[1] - m2[2])


@pytest.mark.parametrize("Nc", [3, 4])
def test_rq1_prolongation_reproduces_local_space(orc, Nc):
    """Face averaging is exact on span{1,x,y,z,x^2-y^2,y^2-z^2} away from the boundary."""
    Nf = 2 * Nc
    P = orc.prolongation(3, orc.RQ1, Nc).dense()
    Hc, hf = 1.0 / Nc, 1.0 / Nf
    uc = np.array([_face_mean_quad(f, pos, Hc) for f, pos, _ in _rq1_faces(Nc)])
    uf = P @ uc
    checked = 0
    for i, (f, pos, _) in enumerate(_rq1_faces(Nf)):
        # coarse cells touched: every face of them must be interior
        cells = []
        for side in ([pos[f] // 2 - 1, pos[f] // 2] if pos[f] % 2 == 0 else [(pos[f] - 1) // 2]):
            c = [pos[d] // 2 for d in range(3)]
            c[f] = side
            cells.append(c)
        if all(1 <= v <= Nc - 2 for c in cells for v in c):
            assert abs(uf[i] - _face_mean_quad(f, pos, hf)) <= 1e-13
            checked += 1
    assert checked > 0


@pytest.mark.parametrize("dim,elem,Nc", [(2, 0, 4), (3, 0, 3), (3, 1, 3)])
def test_restriction_is_transpose(orc, dim, elem, Nc):
    H = orc.Hierarchy(dim, elem, 2 * Nc, 2)
    P, R = H.P(1).dense(), H.R(1).dense()
    assert np.array_equal(R, P.T)


@pytest.mark.parametrize("dim,N", [(2, 16), (3, 8)])
def test_q1_galerkin_identity(orc, dim, N):
    """For Q1 with nested spaces, R A_h P equals the rediscretised coarse matrix."""
    H = orc.Hierarchy(dim, orc.Q1, N, 2)
    Af, Ac, P = H.A(1).to_scipy(), H.A(0).dense(), H.P(1).to_scipy()
    G = (P.T @ Af @ P).toarray()
    assert np.max(np.abs(G - Ac)) <= 1e-14 * np.max(np.abs(Ac))


def test_galerkin_levels_for_unresolved_coefficient(orc):
    """Coarse levels whose cells straddle coefficient blocks use R A P (checked with scipy)."""
    N = 16
    k = W.k_blocks(N, dim=3, blocks_per_axis=4, seed=11)  # blocks of 4 cells
    H = orc.Hierarchy(3, orc.Q1, N, 4, k_cell=k)  # N = 2, 4, 8, 16
    assert [H.galerkin(l) for l in range(4)] == [True, False, False, False]
    Af, P = H.A(1).to_scipy(), H.P(1).to_scipy()
    G = (P.T @ Af @ P).toarray()
    Ac = H.A(0).dense()
    assert np.max(np.abs(G - Ac)) <= 1e-14 * np.max(np.abs(Ac))
    # resolved level: rediscretisation equals R A P as well
    A2, P2 = H.A(2).to_scipy(), H.P(2).to_scipy()
    G1 = (P2.T @ A2 @ P2).toarray()
    assert np.max(np.abs(G1 - H.A(1).dense())) <= 1e-13 * np.max(np.abs(G1))


# ------------------------------------------------------------------------------------
# Coarse solve, load vector
# ------------------------------------------------------------------------------------


def test_dense_lu_matches_numpy(orc):
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 30):
        a = rng.standard_normal((n, n)) + n * np.eye(n) * (rng.random() < 0.5)
        b = rng.standard_normal(n)
        x = orc.lu_solve_dense(a, b)
        np.testing.assert_allclose(x, np.linalg.solve(a, b), rtol=1e-11, atol=1e-12)
    A0 = orc.assemble(3, orc.RQ1, 3).dense()  # the 54-DOF coarsest rotated-Q1 level
    b = rng.standard_normal(A0.shape[0])
    np.testing.assert_allclose(orc.lu_solve_dense(A0, b), np.linalg.solve(A0, b), rtol=1e-12)


@pytest.mark.parametrize("dim,elem,N", [(2, 0, 8), (3, 0, 4), (3, 1, 4)])
def test_load_vector_constant_f(orc, dim, elem, N):
    """f = 1: int phi_i = h^d for a Q1 vertex, 2 * h^3/6 for a rotated-Q1 face."""
    b = orc.load_vector(dim, elem, N, modes=None, fconst=1.0)
    h = 1.0 / N
    expect = h ** dim if elem == 0 else h ** 3 / 3
    np.testing.assert_allclose(b, expect, rtol=2e-15)


def test_load_vector_matches_numpy_quadrature(orc):
    N = 8
    modes = W.random_modes(2, n_modes=3, seed=5)
    b = orc.load_vector(2, orc.Q1, N, modes=modes)
    g = np.array([0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)])
    w = np.array([5, 8, 5]) / 18.0
    h = 1.0 / N

    def f(x, y):
        return sum(a * np.pi ** 2 * (k[0] ** 2 + k[1] ** 2) * np.sin(k[0] * np.pi * x)
                   * np.sin(k[1] * np.pi * y) for a, k in modes)

    ref = np.zeros((N + 1, N + 1))  # vertex grid, [y, x]
    for cy, cx in itertools.product(range(N), repeat=2):
        for qy, qx in itertools.product(range(3), repeat=2):
            xi, eta = g[qx], g[qy]
            val = f((cx + xi) * h, (cy + eta) * h) * w[qx] * w[qy] * h * h
            ref[cy, cx] += val * (1 - xi) * (1 - eta)
            ref[cy, cx + 1] += val * xi * (1 - eta)
            ref[cy + 1, cx] += val * (1 - xi) * eta
            ref[cy + 1, cx + 1] += val * xi * eta
    np.testing.assert_allclose(b, ref[1:N, 1:N].reshape(-1), rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------------------------
# Solves
# ------------------------------------------------------------------------------------


def _dst_solve_q1(dim, N, b):
    """Exact solution of the constant-coefficient Q1 system by type-I DST diagonalisation."""
    h = 1.0 / N
    j = np.arange(1, N)
    c = np.cos(j * np.pi / N)
    kap = (2.0 / h) * (1.0 - c)
    mu = (h / 6.0) * (4.0 + 2.0 * c)
    shape = (N - 1,) * dim
    B = b.reshape(shape)  # axes (z,) y, x
    if dim == 2:
        lam = np.add.outer(kap, np.zeros(N - 1)) * mu[None, :] + mu[:, None] * kap[None, :]
    else:
        K, M = kap, mu
        lam = (K[:, None, None] * M[None, :, None] * M[None, None, :]
               + M[:, None, None] * K[None, :, None] * M[None, None, :]
               + M[:, None, None] * M[None, :, None] * K[None, None, :])
    bh = scipy.fft.dstn(B, type=1, norm="ortho")
    return scipy.fft.idstn(bh / lam, type=1, norm="ortho").reshape(-1)


@pytest.mark.parametrize("dim,N,L", [(2, 64, 5), (3, 16, 3)])
def test_mg_matches_dst_exact_solution(orc, dim, N, L):
    H = orc.Hierarchy(dim, orc.Q1, N, L, opts=orc.Options(omega=0.8))
    b = orc.load_vector(dim, orc.Q1, N, modes=W.random_modes(dim, seed=2))
    x, hist, it, conv = H.solve(b, 1e-13)
    assert conv
    xe = _dst_solve_q1(dim, N, b)
    assert np.linalg.norm(x - xe) <= 1e-10 * np.linalg.norm(xe)


@pytest.mark.parametrize("dim,elem,N,L,smoother", [(2, 0, 16, 3, 0), (3, 0, 8, 3, 0),
                                                    (3, 1, 4, 2, 0), (3, 0, 8, 3, 1),
                                                    (3, 1, 8, 3, 1), (2, 0, 16, 3, 2),
                                                    (3, 0, 8, 3, 2), (3, 1, 8, 3, 2)])
def test_mg_matches_dense_solve(orc, dim, elem, N, L, smoother):
    opts = orc.Options(smoother=smoother, omega=0.7 if elem else 0.8,
                       nu_pre=1 if smoother else 2, nu_post=1 if smoother else 2)
    H = orc.Hierarchy(dim, elem, N, L, opts=opts)
    b = W.random_vector(H.n, seed=N)
    x, hist, it, conv = H.solve(b, 1e-12)
    assert conv and np.all(np.diff(hist) < 0)
    xd = np.linalg.solve(H.A(L - 1).dense(), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def _level_colours(H, l):
    from oracle import colours
    return colours(H.dim, H.elem, H.level_N(l))


def _colour_triangles(A, col):
    """Strictly lower / upper parts of dense A in the order (colour, index)."""
    n = A.shape[0]
    key = col.astype(np.int64) * n + np.arange(n)
    before = key[None, :] < key[:, None]  # column j is visited before row i
    after = key[None, :] > key[:, None]
    return np.where(before, A, 0.0), np.where(after, A, 0.0)


def _vcycle_operator(H, opts, l):
    """Dense B_l with V(r) = B_l r, from the closed-form error propagation of each step."""
    A = H.A(l).dense()
    if l == 0:
        return np.linalg.inv(A)
    n = A.shape[0]
    Dinv = np.diag(1.0 / np.diag(A))
    I = np.eye(n)
    if opts.smoother == 0:
        S = np.linalg.matrix_power(I - opts.omega * Dinv @ A, opts.nu_pre)
        T = np.linalg.matrix_power(I - opts.omega * Dinv @ A, opts.nu_post)
    elif opts.smoother == 2:  # Gauss-Seidel in colour order: forward before, backward after
        Lo, Up = _colour_triangles(A, _level_colours(H, l))
        D = np.diag(np.diag(A))
        S = np.linalg.matrix_power(I - np.linalg.solve(D + Lo, A), opts.nu_pre)
        T = np.linalg.matrix_power(I - np.linalg.solve(D + Up, A), opts.nu_post)
    else:  # Chebyshev: error polynomial T_k((theta - t)/delta) / T_k(theta/delta)
        hi = opts.cheb_hi * H.lam(l)
        lo = hi / opts.cheb_ratio
        th, de = (hi + lo) / 2, (hi - lo) / 2
        Z = (th * I - Dinv @ A) / de
        Tk = np.polynomial.chebyshev.chebval(th / de, [0] * opts.cheb_degree + [1])
        Pk = np.zeros_like(Z)
        Tm, Tc = I, Z  # T_0, T_1
        if opts.cheb_degree == 1:
            Pk = Tc
        else:
            for _ in range(opts.cheb_degree - 1):
                Tm, Tc = Tc, 2 * Z @ Tc - Tm
            Pk = Tc
        S = np.linalg.matrix_power(Pk / Tk, opts.nu_pre)
        T = np.linalg.matrix_power(Pk / Tk, opts.nu_post)
    P, R = H.P(l).dense(), H.R(l).dense()
    Bc = _vcycle_operator(H, opts, l - 1)
    E = T @ (I - P @ Bc @ R @ A) @ S
    return (I - E) @ np.linalg.inv(A)


@pytest.mark.parametrize("dim,elem,N,L,smoother", [(2, 0, 16, 3, 0), (2, 0, 16, 3, 1),
                                                    (3, 1, 4, 2, 0), (3, 1, 4, 2, 1),
                                                    (2, 0, 16, 3, 2), (3, 0, 8, 3, 2), (3, 1, 4, 2, 2),
                                                    (3, 2, 8, 3, 2), (3, 3, 4, 2, 2)])
def test_vcycle_equals_closed_form_operator(orc, dim, elem, N, L, smoother):
    opts = orc.Options(smoother=smoother, omega=0.7, nu_pre=2 if not smoother else 1,
                       nu_post=1 if not smoother else 2, cheb_degree=3 if smoother else 2)
    H = orc.Hierarchy(dim, elem, N, L, opts=opts)
    r = W.random_vector(H.n, seed=9)
    c = H.vcycle(r)
    Bop = _vcycle_operator(H, opts, L - 1)
    np.testing.assert_allclose(c, Bop @ r, rtol=0, atol=1e-11 * np.max(np.abs(c)))


def test_reported_residual_norm_is_accurate(orc):
    """hist[0] = ||b - A x0|| / ||b|| to a few ulps (checked with an exactly rounded sum)."""
    import math
    N, L = 512, 8
    H = orc.Hierarchy(2, orc.Q1, N, L)
    b = W.random_vector(H.n, seed=3) * 1e3
    x0 = W.random_vector(H.n, seed=4)
    x, hist, it, conv = H.solve(b, 0.0, x0=x0, max_iters=0)
    r = b - orc.spmv(H.A(L - 1), x0)
    exact = math.sqrt(math.fsum(r * r)) / math.sqrt(math.fsum(b * b))
    assert abs(hist[0] - exact) <= 4e-16 * exact


def test_power_iteration_bounds(orc):
    N = 16
    opts = orc.Options(smoother=orc.CHEBYSHEV)
    H = orc.Hierarchy(3, orc.Q1, N, 3, opts=opts)
    A = H.A(2).to_scipy()
    d = A.diagonal()
    Ds = sp.diags(1.0 / np.sqrt(d))
    lam_max = np.linalg.eigvalsh((Ds @ A @ Ds).toarray()).max()
    lam = H.lam(2)
    assert 0.8 * lam_max <= lam <= lam_max * (1 + 1e-12)
    assert lam_max <= 2.0  # Gershgorin for a zero-row-sum M-matrix under Jacobi scaling
    H2 = orc.Hierarchy(3, orc.Q1, N, 3, opts=opts)
    assert H2.lam(2) == lam  # reproducible bit for bit


def _power_lambda_numpy(A, steps, seed):
    """lambda_hat of the stated reading, written out in numpy: start v = 1 + 0.2 (u - 1/2)
    with u_i the i-th SplitMix64(seed) draw, v /= ||v||; then `steps` times w = D^-1 A v,
    lambda = ||w||, v = w / lambda."""
    n = A.shape[0]
    dinv = 1.0 / A.diagonal()
    v = 1.0 + 0.2 * (W.uniform01(seed, n) - 0.5)
    v = v / np.linalg.norm(v)
    lam = 0.0
    for _ in range(steps):
        w = dinv * (A @ v)
        lam = np.linalg.norm(w)
        v = w / lam
    return lam


@pytest.mark.parametrize("dim,N,L", [(2, 32, 3), (3, 16, 3)])
def test_power_iteration_follows_the_stated_reading(orc, dim, N, L):
    """The Chebyshev bound: 20 power steps on D^-1 A from the seeded start vector (seed
    1609), on the Kronecker-form matrix of every smoothed level. A different step count,
    seed, start vector or normalisation moves lambda_hat far beyond the rounding bound."""
    H = orc.Hierarchy(dim, orc.Q1, N, L, opts=orc.Options(smoother=orc.CHEBYSHEV))
    for l in range(1, L):
        A = sp.csr_matrix(_kron_q1(dim, H.level_N(l)))
        want = _power_lambda_numpy(A, 20, 1609)
        assert abs(H.lam(l) - want) <= 1e-13 * want, (l, H.lam(l), want)
        for other in (_power_lambda_numpy(A, 19, 1609), _power_lambda_numpy(A, 20, 1608)):
            assert abs(H.lam(l) - other) > 1e-11 * want


@pytest.mark.slow
@pytest.mark.parametrize("dim,elem,Ns", [(2, 0, (16, 32, 64)), (3, 0, (8, 16, 32)),
                                         (3, 1, (4, 8, 16))])
def test_l2_error_is_second_order(orc, dim, elem, Ns):
    modes = W.manufactured_modes(dim)
    errs = []
    for N in Ns:
        L = int(np.log2(N)) - (1 if elem == 0 else 1)
        L = max(2, min(L, 4))
        H = orc.Hierarchy(dim, elem, N, L, opts=orc.Options(omega=0.7 if elem else 0.8))
        b = orc.load_vector(dim, elem, N, modes=modes)
        x, hist, it, conv = H.solve(b, 1e-12)
        assert conv
        errs.append(orc.l2_error(dim, elem, N, modes, x))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((orders > 1.9) & (orders < 2.1)), orders


@pytest.mark.slow
def test_contraction_is_h_independent(orc):
    rates = []
    for N, L in ((64, 5), (128, 6), (256, 7)):
        H = orc.Hierarchy(2, orc.Q1, N, L, opts=orc.Options(omega=0.8))
        b = W.random_vector(H.n, seed=1)
        x, hist, it, conv = H.solve(b, 1e-10)
        assert conv
        rates.append((hist[-1] / hist[1]) ** (1.0 / (len(hist) - 2)))
    rates = np.array(rates)
    assert np.all(rates < 0.2) and rates.max() / rates.min() < 1.2, rates


# ---------------------------------------------------------------------------------
# Multicolour Gauss-Seidel (the paper's smoother, Eq. GS, on colour-wise numbered DOFs)
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("dim,elem,N", [(2, 0, 8), (2, 0, 9), (3, 0, 8), (3, 1, 6), (3, 1, 5)])
def test_gs_colouring_is_valid_and_counts_parity_classes(orc, dim, elem, N):
    A = orc.assemble(dim, elem, N).to_scipy().tocoo()
    col = orc.colours(dim, elem, N)
    off = A.row != A.col
    assert not np.any(col[A.row[off]] == col[A.col[off]])  # no coupling inside a colour
    n1 = N - 1
    odd, even = (n1 + 1) // 2, n1 // 2  # positions 1..N-1 with parity 1 / 0
    cnt = np.bincount(col, minlength=orc.n_colours(dim, elem))
    if elem == orc.Q1:
        for c in range(1 << dim):
            want = 1
            for d in range(dim):
                want *= odd if (c >> d) & 1 else even
            assert cnt[c] == want
    else:
        assert list(cnt) == [even * N * N, odd * N * N] * 3


def test_gs_colouring_valid_on_galerkin_levels(orc):
    k = W.k_blocks(16, dim=3, blocks_per_axis=16, seed=20260101)  # one value per cell
    H = orc.Hierarchy(3, orc.Q1, 16, 3, k_cell=k, opts=orc.Options(smoother=orc.GAUSS_SEIDEL))
    assert H.galerkin(0) and H.galerkin(1)
    for l in range(3):
        A = H.A(l).to_scipy().tocoo()
        col = orc.colours(3, orc.Q1, H.level_N(l))
        off = (A.row != A.col) & (A.data != 0)
        assert not np.any(col[A.row[off]] == col[A.col[off]])


@pytest.mark.parametrize("dim,elem,N", [(2, 0, 12), (3, 0, 6), (3, 1, 4), (3, 2, 6), (3, 3, 3)])
@pytest.mark.parametrize("backward", [False, True])
def test_gs_sweep_is_a_triangular_solve(orc, dim, elem, N, backward):
    """x' = x + (D + L)^-1 (b - A x), L the couplings to earlier colours (later ones backward)."""
    import scipy.sparse.linalg as sla
    Ao = orc.assemble(dim, elem, N)
    A = Ao.to_scipy().tocsr()
    col = orc.colours(dim, elem, N)
    n = A.shape[0]
    order = np.lexsort((np.arange(n), col))  # colour-wise numbering, index order inside
    Ap = A[order][:, order]
    T = sp.triu(Ap, format="csr") if backward else sp.tril(Ap, format="csr")
    b = W.random_vector(n, seed=21)
    x = W.random_vector(n, seed=22)
    r = (b - A @ x)[order]
    dx = np.empty(n)
    dx[order] = sla.spsolve_triangular(T, r, lower=not backward)
    want = x + dx
    got = orc.gs_sweep(Ao, col, orc.n_colours(dim, elem), b, x, backward=backward)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("dim,elem,N", [(2, 0, 12), (3, 0, 6), (3, 1, 4)])
def test_gs_sweep_contracts_the_energy_error(orc, dim, elem, N):
    Ao = orc.assemble(dim, elem, N)
    A = Ao.dense()
    col = orc.colours(dim, elem, N)
    b = W.random_vector(A.shape[0], seed=23)
    xs = np.linalg.solve(A, b)
    x = W.random_vector(A.shape[0], seed=24)
    en = lambda e: float(np.sqrt(e @ A @ e))
    for backward in (False, True, False):
        x1 = orc.gs_sweep(Ao, col, orc.n_colours(dim, elem), b, x, backward=backward)
        assert en(x1 - xs) < en(x - xs)
        x = x1
    # the exact solution is a fixed point
    x2 = orc.gs_sweep(Ao, col, orc.n_colours(dim, elem), b, xs)
    assert np.linalg.norm(x2 - xs) <= 1e-12 * np.linalg.norm(xs)


@pytest.mark.parametrize("dim,elem,N,L", [(2, 0, 16, 3), (3, 0, 8, 3), (3, 1, 4, 2), (3, 2, 8, 3), (3, 3, 4, 2)])
def test_gs_vcycle_is_symmetric(orc, dim, elem, N, L):
    """Forward sweeps before and backward sweeps after the correction: V = V^T."""
    H = orc.Hierarchy(dim, elem, N, L, opts=orc.Options(smoother=orc.GAUSS_SEIDEL, nu_pre=2, nu_post=2))
    u = W.random_vector(H.n, seed=25)
    w = W.random_vector(H.n, seed=26)
    a, c = u @ H.vcycle(w), w @ H.vcycle(u)
    assert abs(a - c) <= 1e-12 * max(abs(a), abs(c))
    # and positive definite on these vectors
    assert u @ H.vcycle(u) > 0 and w @ H.vcycle(w) > 0


def test_gs_converges_faster_per_cycle_than_jacobi(orc):
    N, L = 32, 4
    b = orc.load_vector(3, orc.Q1, N, modes=W.manufactured_modes(3))
    its = []
    for sm in (orc.JACOBI, orc.GAUSS_SEIDEL):
        H = orc.Hierarchy(3, orc.Q1, N, L, opts=orc.Options(smoother=sm, omega=0.8))
        x, hist, it, conv = H.solve(b, 1e-10)
        assert conv
        its.append(it)
    assert its[1] < its[0]


# ---------------------------------------------------------------------------------
# Conjugate gradients preconditioned by one V-cycle (Sec. 1: MG as a preconditioner)
# ---------------------------------------------------------------------------------
def _textbook_pcg(A, Minv, b, tol, maxit=100):
    """Preconditioned CG written from the textbook with dense numpy operators."""
    x = np.zeros_like(b)
    r = b - A @ x
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    p = None
    rz_old = None
    for _ in range(maxit):
        if hist[-1] <= tol:
            break
        z = Minv @ r
        rz = r @ z
        p = z if p is None else z + (rz / rz_old) * p
        q = A @ p
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rz_old = rz
        hist.append(np.linalg.norm(r) / nb)
    return x, np.array(hist)


@pytest.mark.parametrize("dim,elem,N,L,smoother", [(2, 0, 16, 3, 0), (2, 0, 16, 3, 1), (3, 0, 8, 3, 2),
                                                    (3, 1, 4, 2, 0), (3, 1, 4, 2, 2)])
def test_pcg_matches_textbook_pcg_with_closed_form_vcycle(orc, dim, elem, N, L, smoother):
    opts = orc.Options(smoother=smoother, omega=0.7, nu_pre=2, nu_post=2)
    H = orc.Hierarchy(dim, elem, N, L, opts=opts)
    b = W.random_vector(H.n, seed=41)
    x, hist, it, conv = H.pcg(b, 1e-11)
    A = H.A(L - 1).dense()
    xt, ht = _textbook_pcg(A, _vcycle_operator(H, opts, L - 1), b, 1e-11)
    assert conv and it == len(ht) - 1
    np.testing.assert_allclose(hist, ht, rtol=1e-8, atol=0)
    assert np.linalg.norm(x - xt) <= 1e-10 * np.linalg.norm(xt)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_pcg_with_exact_preconditioner_converges_in_one_step(orc):
    """One level: the V-cycle is the LU solve, M^-1 = A^-1, so x_1 is the solution."""
    H = orc.Hierarchy(3, orc.Q1, 8, 1)
    b = W.random_vector(H.n, seed=42)
    x, hist, it, conv = H.pcg(b, 1e-13)
    assert conv and it == 1 and hist[1] <= 1e-14


@pytest.mark.parametrize("smoother", [0, 1, 2])
def test_pcg_needs_no_more_cycles_than_defect_correction(orc, smoother):
    N, L = 32, 4
    b = orc.load_vector(3, orc.Q1, N, modes=W.manufactured_modes(3))
    H = orc.Hierarchy(3, orc.Q1, N, L, opts=orc.Options(smoother=smoother, omega=0.8, nu_pre=1, nu_post=1))
    x1, h1, it1, c1 = H.solve(b, 1e-10)
    x2, h2, it2, c2 = H.pcg(b, 1e-10)
    assert c1 and c2 and it2 <= it1
    r = b - orc.spmv(H.A(L - 1), x2)  # the recursive residual tracks the true one
    assert abs(np.linalg.norm(r) / np.linalg.norm(b) - h2[-1]) <= 1e-3 * h2[-1]


# ---------------------------------------------------------------------------------
# Crank-Nicolson heat equation (Sec. 6 "Model Problem"): mass matrix, shifted operator
# ---------------------------------------------------------------------------------
def test_q1_mass_element_textbook_values(orc):
    from fractions import Fraction as Fr

    from oracle import elements
    for dim in (2, 3):
        M = elements.q1_mass_exact(dim)
        for a in range(2 ** dim):
            for b in range(2 ** dim):
                want = Fr(1)
                for d in range(dim):
                    want *= Fr(1, 3) if ((a >> d) & 1) == ((b >> d) & 1) else Fr(1, 6)
                assert M[a][b] == want
        assert sum(sum(r) for r in M) == 1  # the unit cell's volume


@pytest.mark.parametrize("dim,N", [(2, 8), (2, 12), (3, 6)])
def test_q1_mass_is_kronecker_product(orc, dim, N):
    h = 1.0 / N
    n1 = N - 1
    M1 = (h / 6) * (4 * np.eye(n1) + np.eye(n1, k=1) + np.eye(n1, k=-1))
    want = M1
    for _ in range(dim - 1):
        want = np.kron(want, M1)
    M = orc.assemble_mass(dim, orc.Q1, N).dense()
    assert np.max(np.abs(M - want)) <= 1e-15 * np.max(np.abs(want))


def _mode_vector(dim, N, ks):
    x = np.arange(1, N) / N
    v = np.ones(1)
    for d in reversed(range(dim)):
        v = np.multiply.outer(v, np.sin(ks[d] * np.pi * x))
    return v.reshape(-1)


@pytest.mark.parametrize("dim,N,L,ks", [(2, 16, 3, (1, 2)), (2, 16, 3, (5, 3)), (3, 8, 2, (1, 2, 3))])
def test_cn_step_damps_a_discrete_mode_by_the_closed_form_factor(orc, dim, N, L, ks):
    """With f = 0 a DST mode is an eigenvector of A and M: u^n = rho^n u^0 with
    rho = (sigma - lam) / (sigma + lam), lam = sum_d kappa_k / mu_k (1D eigenvalues)."""
    h = 1.0 / N
    sigma = 2.0 / 0.01
    lam = 0.0
    for k in ks:
        kap = (2.0 / h) * (1 - np.cos(k * np.pi / N))
        mu = (h / 6.0) * (4 + 2 * np.cos(k * np.pi / N))
        lam += kap / mu
    rho = (sigma - lam) / (sigma + lam)
    H = orc.Hierarchy(dim, orc.Q1, N, L, opts=orc.Options(omega=0.8), mass=sigma)
    B = orc.heat_B(dim, orc.Q1, N, sigma)
    u0 = _mode_vector(dim, N, ks)
    n_steps = 5
    u, its = orc.heat(H, B, np.zeros_like(u0), np.zeros(n_steps + 1), u0, 1e-14)
    assert np.linalg.norm(u - rho ** n_steps * u0) <= 1e-11 * np.linalg.norm(u0)


def test_cn_matches_dense_direct_time_stepping(orc):
    dim, N, L = 2, 12, 2
    wl = W.heat_workload(dim=dim, n_cells=N, n_levels=L, dt=0.02, t_end=0.2)
    sigma = wl["sigma"]
    H = orc.Hierarchy(dim, orc.Q1, N, L, opts=orc.Options(omega=0.8), mass=sigma)
    B = orc.heat_B(dim, orc.Q1, N, sigma)
    bF = orc.load_vector(dim, orc.Q1, N, modes=wl["source_modes"])
    u, its = orc.heat(H, B, bF, wl["g"], wl["u0"], 1e-13)
    A = orc.assemble(dim, orc.Q1, N).dense()
    M = orc.assemble_mass(dim, orc.Q1, N).dense()
    dt = wl["dt"]
    ud = wl["u0"].copy()
    for k in range(wl["n_steps"]):  # the unscaled textbook step
        rhs = (M - dt / 2 * A) @ ud + dt / 2 * (wl["g"][k] + wl["g"][k + 1]) * bF
        ud = np.linalg.solve(M + dt / 2 * A, rhs)
    assert np.linalg.norm(u - ud) <= 1e-10 * np.linalg.norm(ud)
    # and the shifted operator of every level is A_l + sigma M_l
    for l in range(L):
        Nl = H.level_N(l)
        want = orc.assemble(dim, orc.Q1, Nl).dense() + sigma * orc.assemble_mass(dim, orc.Q1, Nl).dense()
        assert np.max(np.abs(H.A(l).dense() - want)) <= 1e-15 * np.max(np.abs(want))


@pytest.mark.slow
def test_heat_manufactured_solution_is_second_order(orc):
    """dt proportional to h: the L2 error at t_end falls by about 4 per refinement."""
    errs = []
    for N in (8, 16, 32):
        wl = W.heat_workload(dim=3, n_cells=N, n_levels=2, dt=0.5 / N, t_end=0.5)
        H = orc.Hierarchy(3, orc.Q1, N, 2 if N == 8 else 3, opts=orc.Options(omega=0.8), mass=wl["sigma"])
        B = orc.heat_B(3, orc.Q1, N, wl["sigma"])
        bF = orc.load_vector(3, orc.Q1, N, modes=wl["source_modes"])
        u, its = orc.heat(H, B, bF, wl["g"], wl["u0"], 1e-12)
        errs.append(orc.l2_error(3, orc.Q1, N, [(wl["exact_amp"], (1, 1, 1))], u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 1.8) & (rates < 2.2)), (errs, rates)


# ---------------------------------------------------------------------------------
# P1 / P2 on the Kuhn tetrahedra of the cube grid (the paper's elements, Sec. 6)
# ---------------------------------------------------------------------------------
def _kuhn_vertices(perm):
    v = [np.zeros(3)]
    for d in perm:
        w = v[-1].copy()
        w[d] += 1
        v.append(w)
    return np.array(v)


def _tet_quadrature(V, order=6):
    """Conical-product Gauss rule on the tetrahedron with vertices V (Stroud): points, weights."""
    from scipy.special import roots_jacobi
    from numpy.polynomial.legendre import leggauss
    x1, w1 = roots_jacobi(order, 2, 0)   # (1-t)^2 weight
    x2, w2 = roots_jacobi(order, 1, 0)   # (1-t) weight
    x3, w3 = leggauss(order)
    pts, wts = [], []
    for a, wa in zip(x1, w1):
        for b, wb in zip(x2, w2):
            for c, wc in zip(x3, w3):
                u, v, w = (1 + a) / 2, (1 + b) / 2, (1 + c) / 2
                # collapsed coordinates: barycentric (l1, l2, l3) of the tetrahedron
                l1 = u
                l2 = (1 - u) * v
                l3 = (1 - u) * (1 - v) * w
                lam = np.array([1 - l1 - l2 - l3, l1, l2, l3])
                pts.append(lam @ V)
                wts.append(wa * wb * wc / 8.0 / 8.0 * 6.0)
    vol = abs(np.linalg.det((V[1:] - V[0]).T)) / 6.0
    w = np.array(wts)
    return np.array(pts), w * vol / w.sum()


def _p2_basis_numeric(V, x):
    """P2 basis values and gradients at x on the tetrahedron V, from the affine barycentric map."""
    T = np.vstack([V.T, np.ones(4)])
    Ti = np.linalg.inv(T)
    lam = Ti @ np.append(x, 1.0)
    g = Ti[:, :3]  # gradients of lambda_a
    vals, grads = [], []
    for a in range(4):
        vals.append(lam[a] * (2 * lam[a] - 1))
        grads.append((4 * lam[a] - 1) * g[a])
    for a, b in [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]:
        vals.append(4 * lam[a] * lam[b])
        grads.append(4 * (lam[b] * g[a] + lam[a] * g[b]))
    return np.array(vals), np.array(grads)


def test_tet_elements_match_numeric_quadrature(orc):
    from oracle import elements as E
    for perm in E.KUHN_PERMS:
        V = _kuhn_vertices(perm)
        X, Wq = _tet_quadrature(V)
        K = np.zeros((10, 10))
        M = np.zeros((10, 10))
        for x, w in zip(X, Wq):
            v, g = _p2_basis_numeric(V, x)
            K += w * g @ g.T
            M += w * np.outer(v, v)
        assert np.max(np.abs(np.array(E.tet_stiffness_exact(2, perm), dtype=float) - K)) <= 1e-13
        assert np.max(np.abs(np.array(E.tet_mass_exact(2), dtype=float) - M)) <= 1e-14
    # P1: the path-graph Laplacian over 6 and the textbook mass |T| (1 + delta_ab) / 20
    G = np.array([[1, -1, 0, 0], [-1, 2, -1, 0], [0, -1, 2, -1], [0, 0, -1, 1]]) / 6
    assert np.array_equal(np.array(E.tet_stiffness_exact(1), dtype=float), G)
    assert np.array_equal(np.array(E.tet_mass_exact(1), dtype=float), (np.ones((4, 4)) + np.eye(4)) / 120)


@pytest.mark.parametrize("N", [4, 7])
def test_p1_stiffness_is_the_seven_point_laplacian(orc, N):
    """P1 on the Kuhn triangulation gives h (T x I x I + I x T x I + I x I x T), T = tridiag(-1, 2, -1)."""
    h = 1.0 / N
    n1 = N - 1
    T = 2 * np.eye(n1) - np.eye(n1, k=1) - np.eye(n1, k=-1)
    I = np.eye(n1)
    want = h * (np.kron(np.kron(I, I), T) + np.kron(np.kron(I, T), I) + np.kron(np.kron(T, I), I))
    A = orc.assemble(3, orc.P1, N).dense()
    assert np.max(np.abs(A - want)) <= 1e-15 * np.max(np.abs(want))


@pytest.mark.parametrize("elem,Nc", [(2, 4), (3, 3), (3, 4)])
def test_tet_prolongation_interpolates_the_element_exactly(orc, elem, Nc):
    """Away from the boundary a row of P applied to the coarse nodal values of a linear (P1)
    or quadratic (P2) function gives its value at the fine node."""
    P = orc.prolongation(3, elem, Nc).dense()
    xc, xf = orc.node_coords(elem, Nc), orc.node_coords(elem, 2 * Nc)
    rng = np.random.Generator(np.random.PCG64(5))
    c = rng.standard_normal(10)

    def q(x):
        x0, x1, x2 = x[:, 0], x[:, 1], x[:, 2]
        v = c[0] + c[1] * x0 + c[2] * x1 + c[3] * x2
        if elem == orc.P2:
            v = v + c[4] * x0 * x0 + c[5] * x1 * x1 + c[6] * x2 * x2 + c[7] * x0 * x1 + c[8] * x1 * x2 + c[9] * x0 * x2
        return v
    y = P @ q(xc)
    hc = 1.0 / Nc
    inner = np.all((xf >= hc - 1e-12) & (xf <= 1 - hc + 1e-12), axis=1)  # no Dirichlet node in its cell
    assert inner.any()
    assert np.max(np.abs(y[inner] - q(xf)[inner])) <= 1e-13
    # and every row's weights sum to one there (partition of unity)
    assert np.allclose(P[inner].sum(axis=1), 1.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("elem,N,L,sm", [(2, 8, 3, 0), (2, 8, 3, 2), (3, 4, 2, 0), (3, 4, 2, 1), (3, 4, 2, 2)])
def test_tet_mg_matches_dense_solve(orc, elem, N, L, sm):
    H = orc.Hierarchy(3, elem, N, L, opts=orc.Options(smoother=sm, omega=0.7, nu_pre=2, nu_post=2))
    b = W.random_vector(H.n, seed=61)
    x, hist, it, conv = H.solve(b, 1e-12)
    assert conv
    xd = np.linalg.solve(H.A(L - 1).dense(), b)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


@pytest.mark.parametrize("elem,N,ncol", [(2, 6, 4), (2, 9, 4), (3, 3, 15), (3, 5, 15)])
def test_tet_gs_colouring_is_valid(orc, elem, N, ncol):
    """P1: (vx+vy+vz) mod 4; P2: (wx+2wy+4wz) mod 15 on the 2N grid; with and without a mass shift."""
    assert orc.n_colours(3, elem) == ncol
    col = orc.colours(3, elem, N)
    assert set(np.unique(col)) == set(range(ncol))
    for mass in (0.0, 200.0):
        A = orc.assemble(3, elem, N).to_scipy() + mass * orc.assemble_mass(3, elem, N).to_scipy()
        A = A.tocoo()
        off = A.row != A.col
        assert not np.any(col[A.row[off]] == col[A.col[off]])


@pytest.mark.slow
@pytest.mark.parametrize("elem,Ns,order", [(2, (8, 16, 32), 2), (3, (4, 8, 16), 3)])
def test_tet_nodal_error_has_the_element_order(orc, elem, Ns, order):
    """Manufactured u = prod sin(pi x_d): the nodal error falls at least as h^order."""
    errs = []
    for N in Ns:
        L = 2 if N <= 8 else 3
        H = orc.Hierarchy(3, elem, N, L, opts=orc.Options(omega=0.7))
        b = orc.load_vector(3, elem, N, modes=W.manufactured_modes(3))
        x, hist, it, conv = H.solve(b, 1e-13)
        X = orc.node_coords(elem, N)
        u = np.prod(np.sin(np.pi * X), axis=1)
        errs.append(np.max(np.abs(x - u)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > order - 0.1), (errs, rates)


def test_tet_dof_counts_match_the_paper(orc):
    """The paper's Sec. 6 counts: its six-level P1 hierarchy (512 -> 16 cells per axis) has
    6 N^3 tetrahedra and (N+1)^3 nodes per level, and P2 on N cells has the (2N+1)^3 nodes of
    the grid of 2N cells; the oracle's interior numbering plus the boundary nodes gives them."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_sec6_dof_counts.txt")
    rows = [l.split(None, 5) for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for elem_name, n_cells, cells, dofs, kind, _src in rows:
        N, cells, dofs = int(n_cells), int(cells), int(dofs)
        elem = orc.P1 if elem_name == "P1" else orc.P2
        M = N if elem == orc.P1 else 2 * N  # node grid
        boundary = (M + 1) ** 3 - (M - 1) ** 3
        assert orc.ndofs(3, elem, N) + boundary == dofs
        assert cells == (6 * N ** 3 if kind == "tet" else N ** 3)
    # the hierarchy: 512 and 16 cells per axis are six levels apart
    assert 512 >> 5 == 16
