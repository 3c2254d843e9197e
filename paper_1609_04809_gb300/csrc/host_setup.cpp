// host_setup.cpp -- host-side construction of the multigrid hierarchy.
//
// Compiled with -ffp-contract=off: every product and sum below is rounded on its own,
// in the order written, on x86 and Arm alike.
//
// Assembly is row-wise (one row per OpenMP iteration, no shared writes): for the DOF of
// row i, the cells that contain it are visited in increasing lexicographic cell order
// and each adds (k_e h^(d-2)) K_ref[a][b] to entry (i, j). Every entry therefore
// receives its element contributions in increasing cell order, starting from 0.0.
#include "host_setup.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace mgh {

static const double kPi = 3.14159265358979323846;  // nearest double to pi

int64_t ndofs(int dim, int elem, int N)
{
    int64_t n1 = N - 1, NN = N;
    if (elem == MG_Q1) return dim == 2 ? n1 * n1 : n1 * n1 * n1;
    if (elem == MG_P1) return n1 * n1 * n1;
    if (elem == MG_P2) return (2 * NN - 1) * (2 * NN - 1) * (2 * NN - 1);
    return 3 * n1 * NN * NN;
}

// ---------------------------------------------------------------------------------
// Reference element matrices on the unit cell
// ---------------------------------------------------------------------------------
// Q1: the tensor-product basis gives K_ref = sum_d K1(a_d,b_d) prod_{e!=d} M1(a_e,b_e)
// with the 1D stiffness K1 = [[1,-1],[-1,1]] and mass M1 = [[2,1],[1,2]]/6. The integer
// numerator over 6^(d-1) is exact; one division rounds it.
static void q1_kref(int dim, double *K)
{
    static const int K1[2][2] = {{1, -1}, {-1, 1}};
    static const int M1[2][2] = {{2, 1}, {1, 2}};
    int nl = 1 << dim;
    double den = dim == 2 ? 6.0 : 36.0;
    for (int a = 0; a < nl; a++)
        for (int b = 0; b < nl; b++) {
            int num = 0;
            for (int d = 0; d < dim; d++) {
                int t = K1[(a >> d) & 1][(b >> d) & 1];
                for (int e = 0; e < dim; e++)
                    if (e != d) t *= M1[(a >> e) & 1][(b >> e) & 1];
                num += t;
            }
            K[a * nl + b] = (double)num / den;
        }
}

// Q1 mass on the unit cell: M_ref = prod_d M1(a_d, b_d), the integer numerator over 6^d
// rounded by one division.
static void q1_mref(int dim, double *M)
{
    static const int M1[2][2] = {{2, 1}, {1, 2}};
    int nl = 1 << dim;
    double den = dim == 2 ? 36.0 : 216.0;
    for (int a = 0; a < nl; a++)
        for (int b = 0; b < nl; b++) {
            int num = 1;
            for (int d = 0; d < dim; d++) num *= M1[(a >> d) & 1][(b >> d) & 1];
            M[a * nl + b] = (double)num / den;
        }
}

// Rotated Q1 on the unit cube, faces x0,x1,y0,y1,z0,z1: 3 on the diagonal, 1 for the
// opposite face, -1 for the four other faces.
static void rq1_kref(double *K)
{
    for (int a = 0; a < 6; a++)
        for (int b = 0; b < 6; b++) K[a * 6 + b] = a == b ? 3.0 : ((a ^ 1) == b ? 1.0 : -1.0);
}

// Rotated-Q1 basis: phi_a = sum_m C[m][a] mon_m, mon = (1, x, y, z, x^2-y^2, y^2-z^2),
// the dual basis of the six face means on the unit cube.
static const double kRq1C[6][6] = {
    {2.0 / 3.0, -1.0 / 3.0, 2.0 / 3.0, -1.0 / 3.0, 2.0 / 3.0, -1.0 / 3.0},
    {-3.0, -1.0, 1.0, 1.0, 1.0, 1.0},
    {1.0, 1.0, -3.0, -1.0, 1.0, 1.0},
    {1.0, 1.0, 1.0, 1.0, -3.0, -1.0},
    {2.0, 2.0, -1.0, -1.0, -1.0, -1.0},
    {1.0, 1.0, 1.0, 1.0, -2.0, -2.0},
};

// ---------------------------------------------------------------------------------
// Local-to-global maps
// ---------------------------------------------------------------------------------
static inline int64_t q1_vertex(int dim, int N, int vx, int vy, int vz)
{
    if (vx <= 0 || vx >= N || vy <= 0 || vy >= N) return -1;
    if (dim == 3 && (vz <= 0 || vz >= N)) return -1;
    int64_t n1 = N - 1;
    int64_t idx = (vx - 1) + n1 * (vy - 1);
    if (dim == 3) idx += n1 * n1 * (vz - 1);
    return idx;
}

// face normal to axis f at normal position p; (q1, q2): cells of the two other axes in
// increasing axis order
static inline int64_t rq1_face(int N, int f, int p, int q1, int q2)
{
    if (p <= 0 || p >= N) return -1;
    int64_t n1 = N - 1, NN = N, fam = n1 * NN * NN;
    switch (f) {
    case 0: return (p - 1) + n1 * (q1 + NN * q2);
    case 1: return fam + q1 + NN * ((p - 1) + n1 * q2);
    default: return 2 * fam + q1 + NN * (q2 + NN * (p - 1));
    }
}

static inline int cell_dofs(int dim, int elem, int N, int cx, int cy, int cz, int64_t *g)
{
    if (elem == MG_Q1) {
        int nl = 1 << dim;
        for (int a = 0; a < nl; a++) g[a] = q1_vertex(dim, N, cx + (a & 1), cy + ((a >> 1) & 1), cz + ((a >> 2) & 1));
        return nl;
    }
    g[0] = rq1_face(N, 0, cx, cy, cz);
    g[1] = rq1_face(N, 0, cx + 1, cy, cz);
    g[2] = rq1_face(N, 1, cy, cx, cz);
    g[3] = rq1_face(N, 1, cy + 1, cx, cz);
    g[4] = rq1_face(N, 2, cz, cx, cy);
    g[5] = rq1_face(N, 2, cz + 1, cx, cy);
    return 6;
}

// decode a rotated-Q1 face: family f, normal position p, cells (q1, q2) of the other axes
static inline void rq1_decode(int N, int64_t i, int &f, int &p, int &q1, int &q2)
{
    int64_t NN = N, fam = (int64_t)(N - 1) * NN * NN;
    f = (int)(i / fam);
    int64_t r = i % fam;
    if (f == 0) {
        p = (int)(r % (N - 1)) + 1;
        q1 = (int)((r / (N - 1)) % NN);
        q2 = (int)(r / ((N - 1) * NN));
    } else if (f == 1) {
        q1 = (int)(r % NN);
        p = (int)((r / NN) % (N - 1)) + 1;
        q2 = (int)(r / (NN * (N - 1)));
    } else {
        q1 = (int)(r % NN);
        q2 = (int)((r / NN) % NN);
        p = (int)(r / (NN * NN)) + 1;
    }
}

// cells containing DOF i, as (cx, cy, cz) in increasing lexicographic order; the local
// index of the DOF in each cell goes to loc[]
static inline int dof_cells(int dim, int elem, int N, int64_t i, int (*c)[3], int *loc)
{
    int m = 0;
    if (elem == MG_Q1) {
        int v[3];
        q1_coords(dim, N, i, v);
        int zlo = dim == 3 ? v[2] - 1 : 0, zhi = dim == 3 ? v[2] : 0;
        for (int cz = zlo; cz <= zhi; cz++)
            for (int cy = v[1] - 1; cy <= v[1]; cy++)
                for (int cx = v[0] - 1; cx <= v[0]; cx++) {
                    c[m][0] = cx;
                    c[m][1] = cy;
                    c[m][2] = cz;
                    loc[m] = (v[0] - cx) + 2 * (v[1] - cy) + (dim == 3 ? 4 * (v[2] - cz) : 0);
                    m++;
                }
        return m;
    }
    int f, p, q1, q2;
    rq1_decode(N, i, f, p, q1, q2);
    int o1 = f == 0 ? 1 : 0, o2 = f == 2 ? 1 : 2;
    for (int s = 0; s < 2; s++) {  // the cell below the face first (lower lexicographic index)
        c[m][f] = p - 1 + s;
        c[m][o1] = q1;
        c[m][o2] = q2;
        loc[m] = 2 * f + (s == 0 ? 1 : 0);  // the face is the upper face of the lower cell
        m++;
    }
    return m;
}

// ---------------------------------------------------------------------------------
// Row-wise assembly
// ---------------------------------------------------------------------------------
struct RowAcc {
    int m = 0;
    int64_t col[96];  // P2 rows hold up to 65 entries
    double val[96];
    void add(int64_t j, double v)
    {
        for (int k = 0; k < m; k++)
            if (col[k] == j) {
                val[k] = val[k] + v;
                return;
            }
        col[m] = j;
        val[m] = 0.0 + v;
        m++;
    }
    void sort()
    {
        for (int a = 1; a < m; a++) {  // insertion sort by column
            int64_t cj = col[a];
            double vj = val[a];
            int b = a - 1;
            while (b >= 0 && col[b] > cj) {
                col[b + 1] = col[b];
                val[b + 1] = val[b];
                b--;
            }
            col[b + 1] = cj;
            val[b + 1] = vj;
        }
    }
};

static void assemble_row(int dim, int elem, int N, const double *k, const double *kref, double hfac, int64_t i,
                         RowAcc &acc)
{
    int c[8][3], loc[8];
    int64_t g[8];
    int nl = elem == MG_Q1 ? (1 << dim) : 6;
    int64_t NN = N;
    int mc = dof_cells(dim, elem, N, i, c, loc);
    acc.m = 0;
    for (int q = 0; q < mc; q++) {
        int64_t e = c[q][0] + NN * (c[q][1] + NN * c[q][2]);
        double ke = k ? k[e] : 1.0;
        double s = ke * hfac;
        cell_dofs(dim, elem, N, c[q][0], c[q][1], c[q][2], g);
        int a = loc[q];
        for (int b = 0; b < nl; b++)
            if (g[b] >= 0) acc.add(g[b], s * kref[a * nl + b]);
    }
    acc.sort();
}

// ---------------------------------------------------------------------------------
// P1 / P2 on the Kuhn tetrahedra of the cube grid (3D)
// ---------------------------------------------------------------------------------
// Cell (cx,cy,cz) holds six tetrahedra, one per permutation pi of the axes (in the order
// of kKuhn): the path v0 = (cx,cy,cz), v1 = v0 + e_pi0, v2 = v1 + e_pi1, v3 = v0 + (1,1,1).
// Their barycentric coordinates at local point s are 1 - s_pi0, s_pi0 - s_pi1,
// s_pi1 - s_pi2, s_pi2. Halving the grid splits each into 8 tetrahedra of the finer one.
// P1 DOFs are the interior vertices (numbered like Q1); P2 DOFs are the interior points
// of the grid of 2N cells (vertices and edge midpoints), local nodes 0..3 the vertices
// and 4..9 the midpoints of edges (01) (02) (03) (12) (13) (23).
static const int kKuhn[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
static const int kTetEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

static inline int64_t grid_point(int M, const int *w)  // interior point of the M-cell grid, or -1
{
    for (int d = 0; d < 3; d++)
        if (w[d] <= 0 || w[d] >= M) return -1;
    int64_t m1 = M - 1;
    return (w[0] - 1) + m1 * ((w[1] - 1) + m1 * (int64_t)(w[2] - 1));
}

static int tet_nodes(int elem, int N, int cx, int cy, int cz, int t, int64_t *g)
{
    int v[4][3] = {{cx, cy, cz}};
    for (int a = 1; a < 4; a++) {
        for (int d = 0; d < 3; d++) v[a][d] = v[a - 1][d];
        v[a][kKuhn[t][a - 1]] += 1;
    }
    if (elem == MG_P1) {
        for (int a = 0; a < 4; a++) g[a] = grid_point(N, v[a]);
        return 4;
    }
    for (int a = 0; a < 4; a++) {
        int w[3] = {2 * v[a][0], 2 * v[a][1], 2 * v[a][2]};
        g[a] = grid_point(2 * N, w);
    }
    for (int e = 0; e < 6; e++) {
        const int *A = v[kTetEdge[e][0]], *B = v[kTetEdge[e][1]];
        int w[3] = {A[0] + B[0], A[1] + B[1], A[2] + B[2]};
        g[4 + e] = grid_point(2 * N, w);
    }
    return 10;
}

// exact rationals for the element tables
struct Rat {
    int64_t p = 0, q = 1;
};
static int64_t gcd64(int64_t a, int64_t b)
{
    if (a < 0) a = -a;
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a ? a : 1;
}
static Rat rat(int64_t p, int64_t q)
{
    int64_t g = gcd64(p, q);
    return Rat{p / g, q / g};
}
static Rat radd(Rat a, Rat b) { return rat(a.p * b.q + b.p * a.q, a.q * b.q); }
static Rat rmul(Rat a, Rat b) { return rat(a.p * b.p, a.q * b.q); }

// polynomial in the four barycentric coordinates: terms (exponents, coefficient)
struct Term {
    int e[4];
    Rat c;
};
using Poly = std::vector<Term>;
static Poly pmul(const Poly &a, const Poly &b)
{
    Poly r;
    for (const Term &x : a)
        for (const Term &y : b) {
            Term t;
            for (int k = 0; k < 4; k++) t.e[k] = x.e[k] + y.e[k];
            t.c = rmul(x.c, y.c);
            r.push_back(t);
        }
    return r;
}
// integral over a Kuhn tetrahedron of the unit cell (volume 1/6):
// int lambda^alpha = alpha! 3! |T| / (|alpha| + 3)! = alpha! / (|alpha| + 3)!
static Rat pint(const Poly &a)
{
    static const int64_t fact[12] = {1, 1, 2, 6, 24, 120, 720, 5040, 40320, 362880, 3628800, 39916800};
    Rat s;
    for (const Term &t : a) {
        int64_t num = 1;
        int deg = 0;
        for (int k = 0; k < 4; k++) {
            num *= fact[t.e[k]];
            deg += t.e[k];
        }
        s = radd(s, rmul(t.c, rat(num, fact[deg + 3])));
    }
    return s;
}
static Poly lam(int a, int64_t c = 1)
{
    Term t{{0, 0, 0, 0}, rat(c, 1)};
    t.e[a] = 1;
    return Poly{t};
}
static Poly konst(int64_t c) { return Poly{Term{{0, 0, 0, 0}, rat(c, 1)}}; }
static Poly padd(Poly a, const Poly &b)
{
    a.insert(a.end(), b.begin(), b.end());
    return a;
}

// unit-cell element stiffness and mass of P1 (4 x 4) or P2 (10 x 10), nearest doubles of
// the exact rationals (the same for all six tetrahedra: congruent with the same order)
static void tet_tables(int elem, double *K, double *M)
{
    int nl = elem == MG_P1 ? 4 : 10;
    // gradients of lambda for the path (0,1,2): -e0, e0 - e1, e1 - e2, e2
    static const int g[4][3] = {{-1, 0, 0}, {1, -1, 0}, {0, 1, -1}, {0, 0, 1}};
    int G[4][4];
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) G[a][b] = g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2];
    std::vector<Poly> N((size_t)nl);
    std::vector<std::vector<Poly>> dN((size_t)nl, std::vector<Poly>(4));  // grad N_i = sum_a dN[i][a] g_a
    if (elem == MG_P1) {
        for (int a = 0; a < 4; a++) {
            N[a] = lam(a);
            dN[a][a] = konst(1);
        }
    } else {
        for (int a = 0; a < 4; a++) {  // lambda_a (2 lambda_a - 1)
            N[a] = pmul(lam(a), padd(lam(a, 2), konst(-1)));
            dN[a][a] = padd(lam(a, 4), konst(-1));
        }
        for (int e = 0; e < 6; e++) {  // 4 lambda_a lambda_b
            int a = kTetEdge[e][0], b = kTetEdge[e][1];
            N[4 + e] = pmul(lam(a, 4), lam(b));
            dN[4 + e][a] = lam(b, 4);
            dN[4 + e][b] = lam(a, 4);
        }
    }
    for (int i = 0; i < nl; i++)
        for (int j = 0; j < nl; j++) {
            Rat k;
            for (int a = 0; a < 4; a++)
                for (int b = 0; b < 4; b++)
                    if (G[a][b] && !dN[i][a].empty() && !dN[j][b].empty())
                        k = radd(k, rmul(rat(G[a][b], 1), pint(pmul(dN[i][a], dN[j][b]))));
            Rat m = pint(pmul(N[i], N[j]));
            K[i * nl + j] = (double)k.p / (double)k.q;
            M[i * nl + j] = (double)m.p / (double)m.q;
        }
}

// the tetrahedra (cell * 6 + t, increasing) that contain DOF i, and i's local index
static int node_tets(int elem, int N, int64_t i, int64_t *et, int *loc)
{
    int M = elem == MG_P1 ? N : 2 * N;
    int64_t m1 = M - 1, NN = N;
    int w[3] = {(int)(i % m1) + 1, (int)((i / m1) % m1) + 1, (int)(i / (m1 * m1)) + 1};
    int lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
        lo[d] = elem == MG_P1 ? w[d] - 1 : (w[d] - 1) >> 1;
        hi[d] = elem == MG_P1 ? w[d] : w[d] >> 1;
        lo[d] = std::max(lo[d], 0);
        hi[d] = std::min(hi[d], N - 1);
    }
    int m = 0;
    int64_t g[10];
    for (int cz = lo[2]; cz <= hi[2]; cz++)
        for (int cy = lo[1]; cy <= hi[1]; cy++)
            for (int cx = lo[0]; cx <= hi[0]; cx++)
                for (int t = 0; t < 6; t++) {
                    int nl = tet_nodes(elem, N, cx, cy, cz, t, g);
                    for (int a = 0; a < nl; a++)
                        if (g[a] == i) {
                            et[m] = (cx + NN * (cy + NN * (int64_t)cz)) * 6 + t;
                            loc[m] = a;
                            m++;
                            break;
                        }
                }
    return m;
}

static void assemble_row_tet(int elem, int N, const double *k, const double *kref, double hfac, int64_t i,
                             RowAcc &acc)
{
    int64_t et[64], g[10], NN = N;
    int loc[64];
    int nl = elem == MG_P1 ? 4 : 10;
    int mt = node_tets(elem, N, i, et, loc);
    acc.m = 0;
    for (int q = 0; q < mt; q++) {
        int64_t c = et[q] / 6;
        double s = (k ? k[c] : 1.0) * hfac;
        tet_nodes(elem, N, (int)(c % NN), (int)((c / NN) % NN), (int)(c / (NN * NN)), (int)(et[q] % 6), g);
        for (int b = 0; b < nl; b++)
            if (g[b] >= 0) acc.add(g[b], s * kref[loc[q] * nl + b]);
    }
    acc.sort();
}

// Interpolation of the coarse function at the fine nodes (nested spaces): a fine node at
// coarse-cell coordinates c + s lies in the tetrahedron whose permutation sorts s
// decreasing (ties by axis); the weights are the coarse basis values there (dyadic).
static int prolong_row_tet(int elem, int Nc, int64_t i, int64_t *cols, double *vals)
{
    int Nf = 2 * Nc;
    int Mf = elem == MG_P1 ? Nf : 2 * Nf, r = elem == MG_P1 ? 2 : 4;
    int64_t m1 = Mf - 1;
    int w[3] = {(int)(i % m1) + 1, (int)((i / m1) % m1) + 1, (int)(i / (m1 * m1)) + 1};
    int c[3];
    double sv[3];
    for (int d = 0; d < 3; d++) {
        c[d] = std::min(w[d] / r, Nc - 1);
        sv[d] = (double)(w[d] - r * c[d]) / (double)r;
    }
    int pi[3] = {0, 1, 2};
    for (int a = 1; a < 3; a++)
        for (int b = a; b > 0 && sv[pi[b]] > sv[pi[b - 1]]; b--) std::swap(pi[b], pi[b - 1]);
    int t = 0;
    while (kKuhn[t][0] != pi[0] || kKuhn[t][1] != pi[1] || kKuhn[t][2] != pi[2]) t++;
    double l[4] = {1.0 - sv[pi[0]], sv[pi[0]] - sv[pi[1]], sv[pi[1]] - sv[pi[2]], sv[pi[2]]};
    int64_t g[10];
    int nl = tet_nodes(elem, Nc, c[0], c[1], c[2], t, g);
    double wt[10];
    if (elem == MG_P1) {
        for (int a = 0; a < 4; a++) wt[a] = l[a];
    } else {
        for (int a = 0; a < 4; a++) wt[a] = l[a] * (2.0 * l[a] - 1.0);
        for (int e = 0; e < 6; e++) wt[4 + e] = (4.0 * l[kTetEdge[e][0]]) * l[kTetEdge[e][1]];
    }
    int m = 0;
    for (int a = 0; a < nl; a++)
        if (g[a] >= 0 && wt[a] != 0.0) {
            cols[m] = g[a];
            vals[m] = wt[a];
            m++;
        }
    for (int a = 1; a < m; a++)  // columns ascending
        for (int b = a; b > 0 && cols[b] < cols[b - 1]; b--) {
            std::swap(cols[b], cols[b - 1]);
            std::swap(vals[b], vals[b - 1]);
        }
    return m;
}

static void assemble_with(int dim, int elem, int N, const double *k, const double *kref, double hfac, Csr &A);

void assemble(int dim, int elem, int N, const double *k, Csr &A)
{
    double kref[100], mref[100];
    if (elem == MG_P1 || elem == MG_P2) {
        tet_tables(elem, kref, mref);
        assemble_with(3, elem, N, k, kref, 1.0 / (double)N, A);
        return;
    }
    if (elem == MG_Q1)
        q1_kref(dim, kref);
    else
        rq1_kref(kref);
    double h = 1.0 / (double)N;
    assemble_with(dim, elem, N, k, kref, dim == 2 ? 1.0 : h, A);
}

void assemble_mass(int dim, int elem, int N, Csr &M)
{
    double kref[100], mref[100];
    if (elem == MG_P1 || elem == MG_P2)
        tet_tables(elem, kref, mref);
    else
        q1_mref(dim, mref);
    double h = 1.0 / (double)N;
    assemble_with(dim, elem, N, nullptr, mref, dim == 2 ? h * h : (h * h) * h, M);
}

// element matrices (k_e * hfac) * kref, added row by row in increasing cell order
static void assemble_with(int dim, int elem, int N, const double *k, const double *kref, double hfac, Csr &A)
{
    int64_t n = ndofs(dim, elem, N);
    A.nrows = A.ncols = n;
    A.rowptr.assign((size_t)n + 1, 0);
    const bool tet = elem == MG_P1 || elem == MG_P2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        RowAcc acc;
        if (tet)
            assemble_row_tet(elem, N, k, kref, hfac, i, acc);
        else
            assemble_row(dim, elem, N, k, kref, hfac, i, acc);
        A.rowptr[i + 1] = acc.m;
    }
    for (int64_t i = 0; i < n; i++) A.rowptr[i + 1] += A.rowptr[i];
    A.col.resize((size_t)A.rowptr[n]);
    A.val.resize((size_t)A.rowptr[n]);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        RowAcc acc;
        if (tet)
            assemble_row_tet(elem, N, k, kref, hfac, i, acc);
        else
            assemble_row(dim, elem, N, k, kref, hfac, i, acc);
        int64_t p = A.rowptr[i];
        for (int q = 0; q < acc.m; q++) {
            A.col[p + q] = (int32_t)acc.col[q];
            A.val[p + q] = acc.val[q];
        }
    }
}

// ---------------------------------------------------------------------------------
// Grid transfers
// ---------------------------------------------------------------------------------
// Rotated Q1 face averaging. The mean over a fine face of a coarse cell's basis
// function: a fine face in the mid-plane of the coarse cell (normal axis f, sub-square
// s1, s2 of the other axes o1 < o2) takes 1/2 from face (o1, side s1) and 1/2 from face
// (o2, side s2); a fine face on the coarse face (f, side v) takes 1 from that face,
// +1/4 from faces (o1, s1) and (o2, s2) and -1/4 from (o1, 1-s1) and (o2, 1-s2).
// Faces on a coarse face shared by two coarse cells average the two cells.
static inline void rq1_fine_weights(int f, int v /*0 lower face, 1 mid-plane, 2 upper face*/, int s1, int s2,
                                    double *w)
{
    int o1 = f == 0 ? 1 : 0, o2 = f == 2 ? 1 : 2;
    for (int a = 0; a < 6; a++) w[a] = 0.0;
    if (v == 1) {
        w[2 * o1 + s1] = 0.5;
        w[2 * o2 + s2] = 0.5;
        return;
    }
    w[2 * f + (v == 2 ? 1 : 0)] = 1.0;
    w[2 * o1 + s1] = 0.25;
    w[2 * o1 + (1 - s1)] = -0.25;
    w[2 * o2 + s2] = 0.25;
    w[2 * o2 + (1 - s2)] = -0.25;
}

static int prolong_row(int dim, int elem, int Nc, int64_t i, int64_t *cols, double *vals)
{
    int Nf = 2 * Nc, m = 0;
    if (elem == MG_Q1) {
        int v[3];
        q1_coords(dim, Nf, i, v);
        int lo[3] = {v[0] / 2, v[1] / 2, dim == 3 ? v[2] / 2 : 0};
        int hi[3] = {(v[0] + 1) / 2, (v[1] + 1) / 2, dim == 3 ? (v[2] + 1) / 2 : 0};
        for (int Z = lo[2]; Z <= hi[2]; Z++)
            for (int Y = lo[1]; Y <= hi[1]; Y++)
                for (int X = lo[0]; X <= hi[0]; X++) {
                    int64_t J = q1_vertex(dim, Nc, X, Y, dim == 3 ? Z : 1);
                    if (J < 0) continue;
                    int V[3] = {X, Y, Z};
                    double w = 1.0;
                    for (int d = 0; d < dim; d++) w = w * (v[d] == 2 * V[d] ? 1.0 : 0.5);
                    cols[m] = J;
                    vals[m] = w;
                    m++;
                }
        return m;  // ascending J already
    }
    int f, p, q1, q2;
    rq1_decode(Nf, i, f, p, q1, q2);
    int o1 = f == 0 ? 1 : 0, o2 = f == 2 ? 1 : 2;
    int ncell = p % 2 == 0 ? 2 : 1;
    double scale = ncell == 2 ? 0.5 : 1.0;
    RowAcc acc;
    for (int c = 0; c < ncell; c++) {
        int cell[3], v;
        if (ncell == 2) {
            cell[f] = p / 2 - 1 + c;
            v = c == 0 ? 2 : 0;
        } else {
            cell[f] = (p - 1) / 2;
            v = 1;
        }
        cell[o1] = q1 / 2;
        cell[o2] = q2 / 2;
        double w[6];
        rq1_fine_weights(f, v, q1 % 2, q2 % 2, w);
        int64_t g[6];
        cell_dofs(3, MG_RQ1, Nc, cell[0], cell[1], cell[2], g);
        for (int a = 0; a < 6; a++)
            if (g[a] >= 0 && w[a] != 0.0) acc.add(g[a], scale * w[a]);
    }
    acc.sort();
    for (int q = 0; q < acc.m; q++) {
        cols[q] = acc.col[q];
        vals[q] = acc.val[q];
    }
    return acc.m;
}

void prolongation(int dim, int elem, int Nc, Csr &P)
{
    int Nf = 2 * Nc;
    int64_t nf = ndofs(dim, elem, Nf), nc = ndofs(dim, elem, Nc);
    P.nrows = nf;
    P.ncols = nc;
    P.rowptr.assign((size_t)nf + 1, 0);
    const bool tet = elem == MG_P1 || elem == MG_P2;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nf; i++) {
        int64_t cols[16];
        double vals[16];
        P.rowptr[i + 1] = tet ? prolong_row_tet(elem, Nc, i, cols, vals) : prolong_row(dim, elem, Nc, i, cols, vals);
    }
    for (int64_t i = 0; i < nf; i++) P.rowptr[i + 1] += P.rowptr[i];
    P.col.resize((size_t)P.rowptr[nf]);
    P.val.resize((size_t)P.rowptr[nf]);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nf; i++) {
        int64_t cols[16];
        double vals[16];
        int m = tet ? prolong_row_tet(elem, Nc, i, cols, vals) : prolong_row(dim, elem, Nc, i, cols, vals);
        for (int q = 0; q < m; q++) {
            P.col[P.rowptr[i] + q] = (int32_t)cols[q];
            P.val[P.rowptr[i] + q] = vals[q];
        }
    }
}

void transpose(const Csr &M, Csr &T)
{
    T.nrows = M.ncols;
    T.ncols = M.nrows;
    T.rowptr.assign((size_t)T.nrows + 1, 0);
    for (int64_t k = 0; k < M.nnz(); k++) T.rowptr[M.col[k] + 1]++;
    for (int64_t j = 0; j < T.nrows; j++) T.rowptr[j + 1] += T.rowptr[j];
    T.col.resize(M.col.size());
    T.val.resize(M.val.size());
    std::vector<int64_t> next(T.rowptr.begin(), T.rowptr.end() - 1);
    for (int64_t i = 0; i < M.nrows; i++)
        for (int64_t k = M.rowptr[i]; k < M.rowptr[i + 1]; k++) {
            int64_t q = next[M.col[k]]++;
            T.col[q] = (int32_t)i;
            T.val[q] = M.val[k];
        }
}

void galerkin(const Csr &R, const Csr &A, const Csr &P, Csr &Ac)
{
    int64_t nc = R.nrows;
    Ac.nrows = Ac.ncols = nc;
    Ac.rowptr.assign((size_t)nc + 1, 0);
    std::vector<std::vector<int32_t>> rc((size_t)nc);
    std::vector<std::vector<double>> rv((size_t)nc);
#pragma omp parallel
    {
        std::vector<double> acc((size_t)nc, 0.0);
        std::vector<char> mark((size_t)nc, 0);
        std::vector<int64_t> list;
#pragma omp for schedule(dynamic, 64)
        for (int64_t I = 0; I < nc; I++) {
            list.clear();
            for (int64_t ki = R.rowptr[I]; ki < R.rowptr[I + 1]; ki++) {
                int64_t i = R.col[ki];
                for (int64_t kj = A.rowptr[i]; kj < A.rowptr[i + 1]; kj++) {
                    int64_t j = A.col[kj];
                    double ra = R.val[ki] * A.val[kj];
                    for (int64_t kJ = P.rowptr[j]; kJ < P.rowptr[j + 1]; kJ++) {
                        int64_t J = P.col[kJ];
                        if (!mark[J]) {
                            mark[J] = 1;
                            list.push_back(J);
                        }
                        acc[J] = acc[J] + ra * P.val[kJ];
                    }
                }
            }
            std::sort(list.begin(), list.end());
            rc[I].resize(list.size());
            rv[I].resize(list.size());
            for (size_t a = 0; a < list.size(); a++) {
                rc[I][a] = (int32_t)list[a];
                rv[I][a] = acc[list[a]];
                acc[list[a]] = 0.0;
                mark[list[a]] = 0;
            }
        }
    }
    for (int64_t I = 0; I < nc; I++) Ac.rowptr[I + 1] = Ac.rowptr[I] + (int64_t)rc[I].size();
    Ac.col.resize((size_t)Ac.rowptr[nc]);
    Ac.val.resize((size_t)Ac.rowptr[nc]);
    for (int64_t I = 0; I < nc; I++) {
        std::copy(rc[I].begin(), rc[I].end(), Ac.col.begin() + Ac.rowptr[I]);
        std::copy(rv[I].begin(), rv[I].end(), Ac.val.begin() + Ac.rowptr[I]);
    }
}

bool coarse_coefficient(int dim, int NL, const double *kL, int Nl, std::vector<double> &kl)
{
    int r = NL / Nl;
    int64_t NNl = Nl, NNL = NL;
    int64_t ncl = dim == 2 ? NNl * NNl : NNl * NNl * NNl;
    kl.assign((size_t)ncl, 0.0);
    for (int64_t c = 0; c < ncl; c++) {
        int64_t cx = c % NNl, cy = (c / NNl) % NNl, cz = dim == 3 ? c / (NNl * NNl) : 0;
        double k0 = kL[cx * r + NNL * (cy * r + NNL * cz * r)];
        for (int dz = 0; dz < (dim == 3 ? r : 1); dz++)
            for (int dy = 0; dy < r; dy++)
                for (int dx = 0; dx < r; dx++)
                    if (kL[(cx * r + dx) + NNL * ((cy * r + dy) + NNL * (cz * r + dz))] != k0) return false;
        kl[c] = k0;
    }
    return true;
}

// ---------------------------------------------------------------------------------
// Load vector: per-cell element vectors (3-point Gauss per axis), then row-wise sums in
// increasing cell order
// ---------------------------------------------------------------------------------
static inline double eval_f(int dim, const mg_rhs *f, const double *p)
{
    if (f->n_modes == 0) return f->f_const;
    double s_f = 0.0;
    for (int m = 0; m < f->n_modes; m++) {
        const int *k = f->freq + 3 * m;
        int ksq = 0;
        for (int d = 0; d < dim; d++) ksq += k[d] * k[d];
        double c = (f->amp[m] * (kPi * kPi)) * (double)ksq;
        double s = std::sin(((double)k[0] * kPi) * p[0]);
        s = s * std::sin(((double)k[1] * kPi) * p[1]);
        if (dim == 3) s = s * std::sin(((double)k[2] * kPi) * p[2]);
        s_f = s_f + c * s;
    }
    return s_f;
}

static inline double basis_value(int dim, int elem, int a, const double *xi)
{
    if (elem == MG_Q1) {
        double t = 1.0;
        for (int d = 0; d < dim; d++) t = t * (((a >> d) & 1) ? xi[d] : (1.0 - xi[d]));
        return t;
    }
    double mon[6] = {1.0, xi[0], xi[1], xi[2], xi[0] * xi[0] - xi[1] * xi[1], xi[1] * xi[1] - xi[2] * xi[2]};
    double s = 0.0;
    for (int m = 0; m < 6; m++) s = s + kRq1C[m][a] * mon[m];
    return s;
}

void load_vector(int dim, int elem, int N, const mg_rhs *f, double *b)
{
    if (elem == MG_P1 || elem == MG_P2) {
        // b = M f_I: the mass matrix times f at the nodes (column-ascending fused sums)
        Csr M;
        assemble_mass(3, elem, N, M);
        int Mg = elem == MG_P1 ? N : 2 * N;
        int64_t m1 = Mg - 1;
        std::vector<double> fi((size_t)M.nrows);
        for (int64_t i = 0; i < M.nrows; i++) {
            double x[3] = {(double)((int)(i % m1) + 1) / (double)Mg, (double)((int)((i / m1) % m1) + 1) / (double)Mg,
                           (double)((int)(i / (m1 * m1)) + 1) / (double)Mg};
            fi[i] = eval_f(3, f, x);
        }
        for (int64_t i = 0; i < M.nrows; i++) {
            double acc = 0.0;
            for (int64_t k = M.rowptr[i]; k < M.rowptr[i + 1]; k++) acc = std::fma(M.val[k], fi[M.col[k]], acc);
            b[i] = acc;
        }
        return;
    }
    int64_t n = ndofs(dim, elem, N), NN = N;
    int64_t ncells = dim == 2 ? NN * NN : NN * NN * NN;
    int nl = elem == MG_Q1 ? (1 << dim) : 6;
    double h = 1.0 / (double)N;
    double hd = dim == 2 ? h * h : (h * h) * h;
    double sq = std::sqrt(0.6);
    const double gx[3] = {0.5 - 0.5 * sq, 0.5, 0.5 + 0.5 * sq};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    int nqz = dim == 3 ? 3 : 1;
    // basis values at the quadrature points do not depend on the cell
    double phi[27][8];
    for (int qz = 0; qz < nqz; qz++)
        for (int qy = 0; qy < 3; qy++)
            for (int qx = 0; qx < 3; qx++) {
                double xi[3] = {gx[qx], gx[qy], dim == 3 ? gx[qz] : 0.0};
                for (int a = 0; a < nl; a++) phi[(qz * 3 + qy) * 3 + qx][a] = basis_value(dim, elem, a, xi);
            }
    std::vector<double> be((size_t)ncells * nl);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ncells; e++) {
        int c[3] = {(int)(e % NN), (int)((e / NN) % NN), dim == 3 ? (int)(e / (NN * NN)) : 0};
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int qz = 0; qz < nqz; qz++)
            for (int qy = 0; qy < 3; qy++)
                for (int qx = 0; qx < 3; qx++) {
                    double xi[3] = {gx[qx], gx[qy], dim == 3 ? gx[qz] : 0.0};
                    double p[3];
                    for (int d = 0; d < 3; d++) p[d] = ((double)c[d] + xi[d]) * h;
                    double wq = gw[qx] * gw[qy];
                    if (dim == 3) wq = wq * gw[qz];
                    double fw = eval_f(dim, f, p) * (wq * hd);
                    const double *ph = phi[(qz * 3 + qy) * 3 + qx];
                    for (int a = 0; a < nl; a++) acc[a] = acc[a] + fw * ph[a];
                }
        for (int a = 0; a < nl; a++) be[(size_t)e * nl + a] = acc[a];
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int c[8][3], loc[8];
        int mc = dof_cells(dim, elem, N, i, c, loc);
        double s = 0.0;
        for (int q = 0; q < mc; q++) {
            int64_t e = c[q][0] + NN * (c[q][1] + NN * c[q][2]);
            s = s + be[(size_t)e * nl + loc[q]];
        }
        b[i] = s;
    }
}

// Q1 load vector by the same tensor 3-point Gauss rule, factorised: for f a sum of
// products of sines (or a constant) the rule splits into one-dimensional sums per mode
// and axis, b = sum_m c_m X_m (x) Y_m [(x) Z_m], at O(modes * n) cost. Equal to
// load_vector up to rounding (the sums are grouped differently).
void load_vector_factors(int dim, int N, const mg_rhs *f, std::vector<double> &v, std::vector<double> &c)
{
    int64_t n1 = N - 1;
    double h = 1.0 / (double)N;
    double sq = std::sqrt(0.6);
    const double gx[3] = {0.5 - 0.5 * sq, 0.5, 0.5 + 0.5 * sq};
    const double gw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    int nm = f->n_modes == 0 ? 1 : f->n_modes;
    // v[m][d][i-1]: integral of (sin or 1) times the hat of node i along axis d
    v.assign((size_t)nm * 3 * n1, 0.0);
    c.assign(nm, 0.0);
    for (int m = 0; m < nm; m++) {
        int ksq = 0;
        if (f->n_modes)
            for (int d = 0; d < dim; d++) ksq += f->freq[3 * m + d] * f->freq[3 * m + d];
        c[m] = f->n_modes ? (f->amp[m] * (kPi * kPi)) * (double)ksq : f->f_const;
        for (int d = 0; d < dim; d++) {
            double kd = f->n_modes ? (double)f->freq[3 * m + d] * kPi : 0.0;
            double *vv = v.data() + ((size_t)m * 3 + d) * n1;
            for (int64_t i = 1; i <= n1; i++) {
                double s = 0.0;
                for (int side = 0; side < 2; side++) {  // cell i-1 (node at its upper end), cell i
                    int64_t cell = i - 1 + side;
                    for (int q = 0; q < 3; q++) {
                        double x = ((double)cell + gx[q]) * h;
                        double g = f->n_modes ? std::sin(kd * x) : 1.0;
                        double phi = side == 0 ? gx[q] : 1.0 - gx[q];
                        s = s + (gw[q] * h) * g * phi;
                    }
                }
                vv[i - 1] = s;
            }
        }
    }
}

void load_vector_separable(int dim, int N, const mg_rhs *f, double *b)
{
    int64_t n1 = N - 1, n = dim == 2 ? n1 * n1 : n1 * n1 * n1;
    std::vector<double> v, c;
    load_vector_factors(dim, N, f, v, c);
    int nm = (int)c.size();
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t ix = i % n1, iy = (i / n1) % n1, iz = dim == 3 ? i / (n1 * n1) : 0;
        double s = 0.0;
        for (int m = 0; m < nm; m++) {
            const double *vm = v.data() + (size_t)m * 3 * n1;
            double t = vm[ix] * vm[n1 + iy];
            if (dim == 3) t = t * vm[2 * n1 + iz];
            s = s + c[m] * t;
        }
        b[i] = s;
    }
}

// ---------------------------------------------------------------------------------
// Power method on D^-1 A (start vector from SplitMix64)
// ---------------------------------------------------------------------------------
static inline uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static double seq_norm(const std::vector<double> &v)
{
    double s = 0.0;
    for (double x : v) s = s + x * x;
    return std::sqrt(s);
}

double power_lambda(const Csr &A, const std::vector<double> &dinv, int iters, uint64_t seed)
{
    int64_t n = A.nrows;
    std::vector<double> v((size_t)n), w((size_t)n);
    for (int64_t i = 0; i < n; i++) {
        double u = (double)(splitmix64(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
        v[i] = 1.0 + 0.2 * (u - 0.5);
    }
    double nv = seq_norm(v);
    for (int64_t i = 0; i < n; i++) v[i] = v[i] / nv;
    double lam = 0.0;
    for (int it = 0; it < iters; it++) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            double s = 0.0;
            for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) s = std::fma(A.val[k], v[A.col[k]], s);
            w[i] = dinv[i] * s;
        }
        lam = seq_norm(w);
        for (int64_t i = 0; i < n; i++) v[i] = w[i] / lam;
    }
    return lam;
}

void build_hierarchy(int dim, int elem, int N_finest, int n_levels, const double *k_finest, int stop,
                     HostHierarchy &H, double mass)
{
    int Lf = n_levels - 1;
    H.N.assign((size_t)n_levels, 0);
    H.galerkin.assign((size_t)n_levels, 0);
    H.A.assign((size_t)n_levels, Csr());
    H.P.assign((size_t)n_levels, Csr());
    H.R.assign((size_t)n_levels, Csr());
    bool use_galerkin = false;
    for (int l = Lf; l >= stop; l--) {
        int Nl = N_finest >> (Lf - l);
        H.N[l] = Nl;
        if (l < Lf) {
            prolongation(dim, elem, Nl, H.P[l + 1]);
            transpose(H.P[l + 1], H.R[l + 1]);
        }
        std::vector<double> kl;
        const double *kp = nullptr;
        if (k_finest && !use_galerkin) {
            if (l == Lf)
                kp = k_finest;
            else if (coarse_coefficient(dim, N_finest, k_finest, Nl, kl))
                kp = kl.data();
            else
                use_galerkin = true;
        }
        if (use_galerkin) {
            galerkin(H.R[l + 1], H.A[l + 1], H.P[l + 1], H.A[l]);
            H.galerkin[l] = 1;
        } else {
            assemble(dim, elem, Nl, kp, H.A[l]);
            if (mass != 0.0) {  // the shifted operator A + mass * M (same pattern)
                Csr M;
                assemble_mass(dim, elem, Nl, M);
                for (size_t q = 0; q < M.val.size(); q++) H.A[l].val[q] = H.A[l].val[q] + mass * M.val[q];
            }
        }
    }
}

double level_lambda(const Csr &A, int iters, uint64_t seed)
{
    std::vector<double> dinv((size_t)A.nrows);
    for (int64_t i = 0; i < A.nrows; i++) {
        double dg = 0.0;
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++)
            if (A.col[k] == i) dg = A.val[k];
        dinv[i] = 1.0 / dg;
    }
    return power_lambda(A, dinv, iters, seed);
}

void round_fp32(const Csr &A, std::vector<float> &val32)
{
    val32.resize(A.val.size());
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A.nrows; i++) {
        double rowsum = 0.0, off32 = 0.0;
        int64_t dpos = -1;
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) {
            rowsum = rowsum + A.val[k];
            if (A.col[k] == i) {
                dpos = k;
            } else {
                val32[k] = (float)A.val[k];
                off32 = off32 + (double)val32[k];
            }
        }
        if (dpos >= 0) val32[dpos] = (float)(rowsum - off32);
    }
}


// ------------------------------------------------------------------------------------
// Multicolour Gauss-Seidel ordering (DOFs numbered colour-wise, Sec. 4 "DOF Reordering")
// ------------------------------------------------------------------------------------
int n_colours(int dim, int elem)
{
    if (elem == MG_Q1) return 1 << dim;
    if (elem == MG_P1) return 4;
    return elem == MG_RQ1 ? 6 : 15;
}

int dof_colour(int dim, int elem, int N, int64_t i)
{
    if (elem == MG_P1 || elem == MG_P2) {
        // P1: vertex coordinate sum mod 4 (Kuhn-edge offsets sum to 1..3 in absolute value);
        // P2: (wx + 2 wy + 4 wz) mod 15 on the grid of 2N cells (no offset between two
        // nodes of a Kuhn tetrahedron is 0 mod 15)
        int M = elem == MG_P1 ? N : 2 * N;
        int64_t m1 = M - 1;
        int w[3] = {(int)(i % m1) + 1, (int)((i / m1) % m1) + 1, (int)(i / (m1 * m1)) + 1};
        return elem == MG_P1 ? (w[0] + w[1] + w[2]) % 4 : (w[0] + 2 * w[1] + 4 * w[2]) % 15;
    }
    if (elem == MG_Q1) {
        int v[3];
        q1_coords(dim, N, i, v);
        return (v[0] & 1) | (v[1] & 1) << 1 | (dim == 3 ? (v[2] & 1) << 2 : 0);
    }
    int f, p, q1, q2;
    rq1_decode(N, i, f, p, q1, q2);
    return 2 * f + (p & 1);
}

void colour_order(int dim, int elem, int N, std::vector<int32_t> &perm, std::vector<int64_t> &coff)
{
    int64_t n = ndofs(dim, elem, N);
    int nc = n_colours(dim, elem);
    coff.assign((size_t)nc + 1, 0);
    std::vector<uint8_t> col((size_t)n);
    for (int64_t i = 0; i < n; i++) {
        col[i] = (uint8_t)dof_colour(dim, elem, N, i);
        coff[col[i] + 1]++;
    }
    for (int c = 0; c < nc; c++) coff[c + 1] += coff[c];
    std::vector<int64_t> next(coff.begin(), coff.end() - 1);
    perm.resize((size_t)n);
    for (int64_t i = 0; i < n; i++) perm[next[col[i]]++] = (int32_t)i;
}

std::vector<std::pair<int64_t, int64_t>> colour_launch_groups(const Csr &A, int dim, int elem, int N,
                                                              const std::vector<int64_t> &coff)
{
    int nc = (int)coff.size() - 1;
    std::vector<bool> coupled((size_t)nc * nc, false);
    for (int64_t i = 0; i < A.nrows; i++) {
        int ci = dof_colour(dim, elem, N, i);
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++)
            if (A.val[k] != 0.0) coupled[(size_t)ci * nc + dof_colour(dim, elem, N, A.col[k])] = true;
    }
    std::vector<std::pair<int64_t, int64_t>> g;
    for (int c = 0; c < nc;) {
        if (c + 1 < nc && !coupled[(size_t)c * nc + c + 1] && !coupled[(size_t)(c + 1) * nc + c]) {
            g.push_back({coff[c], coff[c + 2]});
            c += 2;
        } else {
            g.push_back({coff[c], coff[c + 1]});
            c += 1;
        }
    }
    return g;
}

bool colouring_valid(const Csr &A, int dim, int elem, int N)
{
    for (int64_t i = 0; i < A.nrows; i++) {
        int ci = dof_colour(dim, elem, N, i);
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++)
            if (A.col[k] != i && dof_colour(dim, elem, N, A.col[k]) == ci) return false;
    }
    return true;
}

}  // namespace mgh
