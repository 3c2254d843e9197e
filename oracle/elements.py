"""Exact reference-element tables for the FP64 multigrid oracle.

TEST INFRASTRUCTURE. This module is part of the oracle: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may use it.
It shares no code with the CUDA library.

Everything here is computed in exact rational arithmetic (``fractions.Fraction``) from
the definitions of the elements, and converted to the nearest double only at the end.

* Conforming Q1 on the unit square / cube: the local basis is the tensor product of
  the 1D hat functions, the element stiffness is the integral of grad(phi_a).grad(phi_b)
  over the unit cell (the Galerkin matrix of the sparse FE system, Sec. 2 "FEM and
  iterative methods" and Sec. 3 of the paper: the assembled system matrix).
* Nonconforming rotated Q1 (Rannacher-Turek, face-mean degrees of freedom) on the unit
  cube: local space span{1, x, y, z, x^2-y^2, y^2-z^2}; the DOFs are the six face
  means, ordered x0, x1, y0, y1, z0, z1. The paper only names "nonconforming" finite
  elements (Sec. 1, Sec. 4.2); the element itself is the standard Rannacher-Turek one.
* The rotated-Q1 prolongation by face averaging (Sec. 5.4 "Restriction and prolongation
  operators" only names general transfer operators; the face-mean form is used here):
  a fine face receives the mean over that fine face of the coarse cell's local function,
  averaged over the coarse cells that contain the fine face.
"""
from fractions import Fraction as Fr
from itertools import product

# ---------------------------------------------------------------------------------
# A tiny exact polynomial algebra in (x, y, z): dict {(ex, ey, ez): Fraction}
# ---------------------------------------------------------------------------------


def _padd(p, q, s=Fr(1)):
    r = dict(p)
    for k, v in q.items():
        r[k] = r.get(k, Fr(0)) + s * v
    return {k: v for k, v in r.items() if v != 0}


def _pmul(p, q):
    r = {}
    for (a, av), (b, bv) in product(p.items(), q.items()):
        k = (a[0] + b[0], a[1] + b[1], a[2] + b[2])
        r[k] = r.get(k, Fr(0)) + av * bv
    return {k: v for k, v in r.items() if v != 0}


def _pdiff(p, axis):
    r = {}
    for k, v in p.items():
        if k[axis] > 0:
            kk = list(k)
            kk[axis] -= 1
            r[tuple(kk)] = r.get(tuple(kk), Fr(0)) + v * k[axis]
    return {k: v for k, v in r.items() if v != 0}


def _mono_int(e, lo, hi):
    """Exact integral of t^e over [lo, hi]."""
    return (Fr(hi) ** (e + 1) - Fr(lo) ** (e + 1)) / (e + 1)


def _pint_box(p, box):
    """Exact integral of p over the box [(lo_x,hi_x), (lo_y,hi_y), (lo_z,hi_z)]."""
    tot = Fr(0)
    for k, v in p.items():
        t = v
        for d in range(3):
            t *= _mono_int(k[d], *box[d])
        tot += t
    return tot


def _pmean_face(p, axis, value, ranges):
    """Exact mean of p over the axis-aligned square {x_axis = value} x ranges (two others)."""
    others = [d for d in range(3) if d != axis]
    tot = Fr(0)
    for k, v in p.items():
        t = v * Fr(value) ** k[axis]
        for d, (lo, hi) in zip(others, ranges):
            t *= _mono_int(k[d], lo, hi)
        tot += t
    area = (Fr(ranges[0][1]) - Fr(ranges[0][0])) * (Fr(ranges[1][1]) - Fr(ranges[1][0]))
    return tot / area


def _var(axis):
    e = [0, 0, 0]
    e[axis] = 1
    return {tuple(e): Fr(1)}


_ONE = {(0, 0, 0): Fr(1)}

# ---------------------------------------------------------------------------------
# Conforming Q1
# ---------------------------------------------------------------------------------


def q1_basis(dim):
    """Local Q1 basis on the unit cell; vertex a has coordinates (a&1, (a>>1)&1, (a>>2)&1)."""
    basis = []
    for a in range(2 ** dim):
        p = dict(_ONE)
        for d in range(dim):
            xd = _var(d)
            f = xd if (a >> d) & 1 else _padd(_ONE, xd, Fr(-1))
            p = _pmul(p, f)
        basis.append(p)
    return basis


def q1_stiffness_exact(dim):
    """K[a][b] = int_{unit cell} grad phi_a . grad phi_b, exact rationals (dim = 2 or 3)."""
    basis = q1_basis(dim)
    box = [(0, 1)] * dim + [(0, 0)] * (3 - dim)
    nl = len(basis)
    K = [[Fr(0)] * nl for _ in range(nl)]
    for a in range(nl):
        for b in range(nl):
            g = {}
            for d in range(dim):
                g = _padd(g, _pmul(_pdiff(basis[a], d), _pdiff(basis[b], d)))
            if dim == 2:
                # integrate over the unit square: drop the z factor (z-degree is 0)
                K[a][b] = sum((v * _mono_int(k[0], 0, 1) * _mono_int(k[1], 0, 1)
                               for k, v in g.items()), Fr(0))
            else:
                K[a][b] = _pint_box(g, box)
    return K


def q1_mass_exact(dim):
    """M[a][b] = int_{unit cell} phi_a phi_b, exact rationals (dim = 2 or 3)."""
    basis = q1_basis(dim)
    box = [(0, 1)] * dim + [(0, 0)] * (3 - dim)
    nl = len(basis)
    M = [[Fr(0)] * nl for _ in range(nl)]
    for a in range(nl):
        for b in range(nl):
            g = _pmul(basis[a], basis[b])
            if dim == 2:
                M[a][b] = sum((v * _mono_int(k[0], 0, 1) * _mono_int(k[1], 0, 1)
                               for k, v in g.items()), Fr(0))
            else:
                M[a][b] = _pint_box(g, box)
    return M


# ---------------------------------------------------------------------------------
# Rotated Q1 (Rannacher-Turek, face means), 3D only
# ---------------------------------------------------------------------------------

RQ1_FACES = [(0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]  # (normal axis, side)


def rq1_monomials():
    x, y, z = _var(0), _var(1), _var(2)
    return [dict(_ONE), x, y, z, _padd(_pmul(x, x), _pmul(y, y), Fr(-1)),
            _padd(_pmul(y, y), _pmul(z, z), Fr(-1))]


def _solve_exact(M, rhs_cols):
    """Gauss-Jordan elimination in exact rationals: returns X with M X = rhs."""
    n = len(M)
    A = [list(M[i]) + list(rhs_cols[i]) for i in range(n)]
    for c in range(n):
        p = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[p] = A[p], A[c]
        piv = A[c][c]
        A[c] = [v / piv for v in A[c]]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c]
                A[r] = [vr - f * vc for vr, vc in zip(A[r], A[c])]
    return [row[n:] for row in A]


def rq1_basis_coefficients():
    """C[m][a]: phi_a = sum_m C[m][a] * monomial_m, with face-mean DOFs (delta property)."""
    mons = rq1_monomials()
    full = [(0, 1), (0, 1)]
    M = [[_pmean_face(mons[m], ax, side, full) for m in range(6)] for (ax, side) in RQ1_FACES]
    ident = [[Fr(int(i == j)) for j in range(6)] for i in range(6)]
    return _solve_exact(M, ident)  # rows: monomials, columns: basis functions


def rq1_basis():
    C = rq1_basis_coefficients()
    mons = rq1_monomials()
    basis = []
    for a in range(6):
        p = {}
        for m in range(6):
            p = _padd(p, mons[m], C[m][a])
        basis.append(p)
    return basis


def rq1_stiffness_exact():
    basis = rq1_basis()
    box = [(0, 1)] * 3
    K = [[Fr(0)] * 6 for _ in range(6)]
    for a in range(6):
        for b in range(6):
            g = {}
            for d in range(3):
                g = _padd(g, _pmul(_pdiff(basis[a], d), _pdiff(basis[b], d)))
            K[a][b] = _pint_box(g, box)
    return K


def rq1_fine_face_weights_exact():
    """W[axis][v][s1][s2][a]: mean over a fine face of the coarse cell's basis function a.

    The coarse cell is the unit cube. The fine face is normal to ``axis`` at position
    v in {0: 0, 1: 1/2, 2: 1}, and covers the sub-square (s1, s2) in {0,1}^2 of the two
    other axes, taken in increasing axis order (s = 0: [0, 1/2], s = 1: [1/2, 1]).
    """
    basis = rq1_basis()
    half = Fr(1, 2)
    pos = [Fr(0), half, Fr(1)]
    sub = [(Fr(0), half), (half, Fr(1))]
    W = [[[[None] * 2 for _ in range(2)] for _ in range(3)] for _ in range(3)]
    for ax in range(3):
        for v in range(3):
            for s1 in range(2):
                for s2 in range(2):
                    W[ax][v][s1][s2] = [_pmean_face(basis[a], ax, pos[v], [sub[s1], sub[s2]])
                                        for a in range(6)]
    return W


# ---------------------------------------------------------------------------------
# P1 / P2 on tetrahedra: the Kuhn (Freudenthal) triangulation of the cube grid
# ---------------------------------------------------------------------------------
# A cell is split into 6 tetrahedra, one per permutation pi of the axes: the path
# 0 -> e_pi0 -> e_pi0 + e_pi1 -> (1,1,1) through the unit cell. Its barycentric
# coordinates are lambda_0 = 1 - s_pi0, lambda_1 = s_pi0 - s_pi1, lambda_2 = s_pi1 - s_pi2,
# lambda_3 = s_pi2 (s the local coordinate), with constant gradients g_0 = -e_pi0,
# g_1 = e_pi0 - e_pi1, g_2 = e_pi1 - e_pi2, g_3 = e_pi2. Halving the grid splits each of
# these tetrahedra into 8 of the finer grid's, so the P1 and P2 spaces are nested.

KUHN_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
P2_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]  # local nodes 4..9


def kuhn_grads(perm):
    """Gradients of the barycentric coordinates of the Kuhn tetrahedron `perm` (unit cell)."""
    e = [[1 if d == a else 0 for d in range(3)] for a in range(3)]
    g0 = [-v for v in e[perm[0]]]
    g1 = [e[perm[0]][d] - e[perm[1]][d] for d in range(3)]
    g2 = [e[perm[1]][d] - e[perm[2]][d] for d in range(3)]
    g3 = list(e[perm[2]])
    return [g0, g1, g2, g3]


def _bmul(p, q):
    """Product of polynomials in the barycentric coordinates {(a0,a1,a2,a3): coeff}."""
    r = {}
    for k1, v1 in p.items():
        for k2, v2 in q.items():
            k = tuple(a + b for a, b in zip(k1, k2))
            r[k] = r.get(k, Fr(0)) + v1 * v2
    return r


def _bint(p):
    """Integral over the unit cell's Kuhn tetrahedron (volume 1/6):
    int lambda^alpha = alpha! 3! |T| / (|alpha| + 3)!."""
    from math import factorial
    tot = Fr(0)
    for k, v in p.items():
        num = 1
        for a in k:
            num *= factorial(a)
        tot += v * Fr(num * factorial(3), factorial(sum(k) + 3)) * Fr(1, 6)
    return tot


def _lam(a, c=Fr(1)):
    k = [0, 0, 0, 0]
    k[a] = 1
    return {tuple(k): c}


def tet_basis(order):
    """P1 or P2 basis on a tetrahedron as polynomials in lambda, and their gradients as
    lists of (polynomial coefficient of g_a) for a = 0..3."""
    one = {(0, 0, 0, 0): Fr(1)}
    if order == 1:
        basis = [_lam(a) for a in range(4)]
        grads = [[one if b == a else {} for b in range(4)] for a in range(4)]
        return basis, grads
    basis, grads = [], []
    for a in range(4):  # vertex: lambda_a (2 lambda_a - 1), gradient (4 lambda_a - 1) g_a
        basis.append(_bmul(_lam(a), {**_lam(a, Fr(2)), (0, 0, 0, 0): Fr(-1)}))
        grads.append([{**_lam(a, Fr(4)), (0, 0, 0, 0): Fr(-1)} if b == a else {} for b in range(4)])
    for a, b in P2_EDGES:  # edge: 4 lambda_a lambda_b, gradient 4 (lambda_b g_a + lambda_a g_b)
        basis.append(_bmul(_lam(a, Fr(4)), _lam(b)))
        grads.append([_lam(b, Fr(4)) if c == a else (_lam(a, Fr(4)) if c == b else {}) for c in range(4)])
    return basis, grads


def tet_stiffness_exact(order, perm=(0, 1, 2)):
    """K[i][j] = int_T grad N_i . grad N_j on the unit cell's Kuhn tetrahedron `perm`."""
    basis, grads = tet_basis(order)
    g = kuhn_grads(perm)
    G = [[sum(g[a][d] * g[b][d] for d in range(3)) for b in range(4)] for a in range(4)]
    n = len(basis)
    K = [[Fr(0)] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            acc = {}
            for a in range(4):
                for b in range(4):
                    if G[a][b] == 0 or not grads[i][a] or not grads[j][b]:
                        continue
                    t = _bmul(grads[i][a], grads[j][b])
                    for k, v in t.items():
                        acc[k] = acc.get(k, Fr(0)) + v * G[a][b]
            K[i][j] = _bint(acc)
    return K


def tet_mass_exact(order):
    """M[i][j] = int_T N_i N_j on a Kuhn tetrahedron of the unit cell (volume 1/6)."""
    basis, _ = tet_basis(order)
    n = len(basis)
    return [[_bint(_bmul(basis[i], basis[j])) for j in range(n)] for i in range(n)]


# ---------------------------------------------------------------------------------
# Double-precision tables handed to the C oracle (nearest double of each rational)
# ---------------------------------------------------------------------------------


def q1_stiffness(dim):
    """Row-major flat list of the unit-cell Q1 stiffness, nearest doubles."""
    return [float(v) for row in q1_stiffness_exact(dim) for v in row]


def q1_mass(dim):
    """Row-major flat list of the unit-cell Q1 mass matrix, nearest doubles."""
    return [float(v) for row in q1_mass_exact(dim) for v in row]


def tet_stiffness(order):
    """Row-major flat P1 (4x4) or P2 (10x10) Kuhn-tetrahedron stiffness, nearest doubles."""
    return [float(v) for row in tet_stiffness_exact(order) for v in row]


def tet_mass(order):
    return [float(v) for row in tet_mass_exact(order) for v in row]


def rq1_stiffness():
    return [float(v) for row in rq1_stiffness_exact() for v in row]


def rq1_basis_table():
    """Flat C[m][a] (m-major), nearest doubles."""
    return [float(v) for row in rq1_basis_coefficients() for v in row]


def rq1_prolong_table():
    """Flat W[axis][v][s1][s2][a] (3*3*2*2*6 = 216 entries), nearest doubles (all dyadic)."""
    W = rq1_fine_face_weights_exact()
    out = []
    for ax in range(3):
        for v in range(3):
            for s1 in range(2):
                for s2 in range(2):
                    out.extend(float(w) for w in W[ax][v][s1][s2])
    return out
