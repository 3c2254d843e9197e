/*
 * mg_oracle.c -- plain FP64 CPU oracle for the geometric multigrid solve.
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline / reference leg may build, load or call this file. It shares no code,
 * header, table or helper with the CUDA library; the two meet only through the
 * seeded inputs (right-hand sides, coefficient fields) that both receive.
 *
 * It is deliberately slow and literal: compressed sparse rows (CSR) built by an
 * element loop, one sequential sum per row, a dense LU on the coarsest level, and the
 * V-cycle written as a recursion in the order of the paper's V-cycle algorithm
 * (Sec. 5.3 "Parallel Multigrid Cycle", Algorithm "Parallel Multigrid Solver
 * (V-Cycle)"): pre-smoothing, restriction of the residual, recursion down to an exact
 * coarsest solve, prolongation and correction, post-smoothing.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared mg_oracle.c -lm
 * (-ffp-contract=off keeps every a*b+c as a rounded product followed by a rounded
 * sum, on x86 and on Arm alike.)
 *
 * Threads: the row loops of the sparse products, the residual, the smoother updates and
 * the prolongation may run on several OpenMP threads (orc_set_threads). Each row is
 * still one sequential sum computed by one thread, so the results do not depend on the
 * thread count; norms, inner products and everything else stay sequential.
 *
 * Floating-point conventions (the reading of every step, in the order evaluated):
 *   y_i = sum_j a_ij x_j           column-ascending, starting from 0.0, each term
 *                                  added by a fused multiply-add s <- fma(a_ij, x_j, s)
 *                                  (IEEE 754 fusedMultiplyAdd: one rounding per term)
 *   residual r_i = b_i - y_i
 *   damped Jacobi x_i <- x_i + omega*(dinv_i*r_i),    dinv_i = 1.0/a_ii
 *   Gauss-Seidel  x_i <- x_i + dinv_i*(b_i - sum_j a_ij x_j), rows one at a time in
 *                 colour order (the latest value of every x_j is used)
 *   Chebyshev step  d_i <- c1*d_i + c2*(dinv_i*r_i),  x_i <- x_i + d_i
 *   restriction b_c = R r with R = P^T stored by rows (fine index ascending)
 *   prolongation x_i <- x_i + t_i,  t_i = sum_J p_iJ c_J   (coarse index ascending, fused)
 *   coarsest solve: LU with partial pivoting; forward substitution sums column-
 *   ascending, back substitution sums column-descending, both fused like the row sums;
 *   back substitution multiplies by the pivot's reciprocal, 1.0/u_ii.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q1 0
#define ORC_RQ1 1
#define ORC_P1 2 /* conforming P1 on the Kuhn tetrahedra of the cube grid (3D) */
#define ORC_P2 3 /* conforming P2 on the same tetrahedra (3D) */
#define ORC_PI 3.14159265358979323846 /* nearest double to pi */

typedef struct {
    int64_t nrows, ncols, nnz;
    int64_t *rowptr; /* nrows + 1 */
    int32_t *col;    /* nnz, ascending within each row */
    double *val;     /* nnz */
} orc_csr;

void orc_csr_free(orc_csr *m)
{
    free(m->rowptr);
    free(m->col);
    free(m->val);
    memset(m, 0, sizeof(*m));
}

/* ------------------------------------------------------------------------------ */
/* Degree-of-freedom numbering on a uniform grid of N cells per axis (h = 1/N).      */
/* Dirichlet boundary DOFs are eliminated: only interior DOFs are numbered.          */
/*   Q1:  interior vertex (ix,iy[,iz]) in [1,N-1]^d,                                 */
/*        index (ix-1) + (N-1)*((iy-1) + (N-1)*(iz-1)).                              */
/*   RQ1: faces, family x (normal x): position i in [1,N-1], cells j,k in [0,N):      */
/*        (i-1) + (N-1)*(j + N*k); family y: i + N*((j-1) + (N-1)*k);                */
/*        family z: i + N*(j + N*(k-1)); families stored x, then y, then z.          */
/* ------------------------------------------------------------------------------ */

int orc_colour(int dim, int elem, int N, int64_t i);
int orc_n_colours(int dim, int elem);
void orc_tet_node_coords(int elem, int N, int64_t i, double *x);

int64_t orc_ndofs(int dim, int elem, int N)
{
    int64_t n1 = N - 1;
    if (elem == ORC_Q1)
        return dim == 2 ? n1 * n1 : n1 * n1 * n1;
    if (elem == ORC_P1)
        return n1 * n1 * n1;
    if (elem == ORC_P2)
        return (int64_t)(2 * N - 1) * (2 * N - 1) * (2 * N - 1);
    return 3 * n1 * (int64_t)N * N;
}

static int64_t q1_vertex(int dim, int N, int vx, int vy, int vz)
{
    if (vx <= 0 || vx >= N || vy <= 0 || vy >= N)
        return -1;
    if (dim == 3 && (vz <= 0 || vz >= N))
        return -1;
    int64_t n1 = N - 1;
    int64_t idx = (vx - 1) + n1 * (vy - 1);
    if (dim == 3)
        idx += n1 * n1 * (vz - 1);
    return idx;
}

/* face of family f at normal position p; (q1,q2) = cell indices of the other two axes
 * in increasing axis order */
static int64_t rq1_face(int N, int f, int p, int q1, int q2)
{
    if (p <= 0 || p >= N)
        return -1;
    int64_t n1 = N - 1, NN = N;
    int64_t fam = n1 * NN * NN;
    if (f == 0) /* x-face: p = i, q1 = j, q2 = k */
        return (p - 1) + n1 * (q1 + NN * q2);
    if (f == 1) /* y-face: q1 = i, p = j, q2 = k */
        return fam + q1 + NN * ((p - 1) + n1 * q2);
    /* z-face: q1 = i, q2 = j, p = k */
    return 2 * fam + q1 + NN * (q2 + NN * (p - 1));
}

/* global DOFs of cell (cx,cy,cz), -1 for a Dirichlet DOF; returns local count */
static int cell_dofs(int dim, int elem, int N, int cx, int cy, int cz, int64_t *g)
{
    if (elem == ORC_Q1) {
        int nl = 1 << dim;
        for (int a = 0; a < nl; a++)
            g[a] = q1_vertex(dim, N, cx + (a & 1), cy + ((a >> 1) & 1), cz + ((a >> 2) & 1));
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

/* cells (as lexicographic cell indices, ascending) that contain DOF i */
static int dof_cells(int dim, int elem, int N, int64_t i, int64_t *cells)
{
    int64_t NN = N;
    int m = 0;
    if (elem == ORC_Q1) {
        int64_t n1 = N - 1;
        int vx = (int)(i % n1) + 1;
        int vy = (int)((i / n1) % n1) + 1;
        int vz = dim == 3 ? (int)(i / (n1 * n1)) + 1 : 0;
        int zlo = dim == 3 ? vz - 1 : 0, zhi = dim == 3 ? vz : 0;
        for (int cz = zlo; cz <= zhi; cz++)
            for (int cy = vy - 1; cy <= vy; cy++)
                for (int cx = vx - 1; cx <= vx; cx++)
                    cells[m++] = cx + NN * (cy + NN * cz);
        return m;
    }
    int64_t fam = (int64_t)(N - 1) * NN * NN;
    int f = (int)(i / fam);
    int64_t r = i % fam;
    int cx, cy, cz;
    if (f == 0) {
        cx = (int)(r % (N - 1)) + 1;
        cy = (int)((r / (N - 1)) % NN);
        cz = (int)(r / ((N - 1) * NN));
        cells[m++] = (cx - 1) + NN * (cy + NN * cz);
        cells[m++] = cx + NN * (cy + NN * cz);
    } else if (f == 1) {
        cx = (int)(r % NN);
        cy = (int)((r / NN) % (N - 1)) + 1;
        cz = (int)(r / (NN * (N - 1)));
        cells[m++] = cx + NN * ((cy - 1) + NN * cz);
        cells[m++] = cx + NN * (cy + NN * cz);
    } else {
        cx = (int)(r % NN);
        cy = (int)((r / NN) % NN);
        cz = (int)(r / (NN * NN)) + 1;
        cells[m++] = cx + NN * (cy + NN * (cz - 1));
        cells[m++] = cx + NN * (cy + NN * cz);
    }
    return m;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

static int64_t find_col(const orc_csr *A, int64_t row, int64_t col)
{
    int64_t lo = A->rowptr[row], hi = A->rowptr[row + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (A->col[mid] == col)
            return mid;
        if (A->col[mid] < col)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

/* ------------------------------------------------------------------------------ */
/* Assembly of the stiffness matrix, a_ij = sum_e k_e * int_e grad phi_i . grad phi_j */
/* ------------------------------------------------------------------------------ */

/*
 * kref: unit-cell element stiffness (nloc x nloc, row-major). The physical element
 * matrix of a cube of side h in d dimensions is h^(d-2) * kref, times the cell's
 * coefficient k_e. Each contribution is evaluated as (k_e*h^(d-2))*kref[a][b] and added
 * to a_ij in increasing lexicographic cell order, starting from 0.0.
 * k_cell: per-cell coefficient on this grid (lexicographic, x fastest) or NULL (k=1).
 */
static int assemble_ref(int dim, int elem, int N, const double *kref, const double *k_cell, double hfac,
                        orc_csr *A);

int orc_assemble(int dim, int elem, int N, const double *kref, const double *k_cell, orc_csr *A)
{
    double h = 1.0 / (double)N;
    return assemble_ref(dim, elem, N, kref, k_cell, dim == 2 ? 1.0 : h, A);
}

/*
 * Consistent mass matrix m_ij = sum_e int_e phi_i phi_j (the time derivative of the heat
 * equation, Sec. 6 "Model Problem"): the element matrix of a cell of side h is h^d mref
 * (mref on the unit cell), added in increasing lexicographic cell order like the
 * stiffness; same pattern as orc_assemble.
 */
int orc_assemble_mass(int dim, int elem, int N, const double *mref, orc_csr *M)
{
    double h = 1.0 / (double)N;
    return assemble_ref(dim, elem, N, mref, NULL, dim == 2 ? h * h : (h * h) * h, M);
}

/* element loop shared by the stiffness and the mass matrix: element matrix
 * (k_e * hfac) * kref[a][b] */
static int assemble_tet(int elem, int N, const double *kref, const double *k_cell, double hfac, orc_csr *A);

static int assemble_ref(int dim, int elem, int N, const double *kref, const double *k_cell, double hfac,
                        orc_csr *A)
{
    if (elem == ORC_P1 || elem == ORC_P2)
        return assemble_tet(elem, N, kref, k_cell, hfac, A);
    int64_t n = orc_ndofs(dim, elem, N);
    int64_t NN = N, ncells = dim == 2 ? NN * NN : NN * NN * NN;
    memset(A, 0, sizeof(*A));
    A->nrows = A->ncols = n;
    A->rowptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!A->rowptr)
        return -1;

    /* pattern: row i couples to every interior DOF of every cell that contains i */
    for (int pass = 0; pass < 2; pass++) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            int64_t cells[8], g[8], cand[64];
            int mc = dof_cells(dim, elem, N, i, cells);
            int m = 0;
            for (int c = 0; c < mc; c++) {
                int64_t e = cells[c];
                int cx = (int)(e % NN), cy = (int)((e / NN) % NN), cz = (int)(e / (NN * NN));
                int nl = cell_dofs(dim, elem, N, cx, cy, cz, g);
                for (int a = 0; a < nl; a++)
                    if (g[a] >= 0)
                        cand[m++] = g[a];
            }
            qsort(cand, (size_t)m, sizeof(int64_t), cmp_i64);
            int u = 0;
            for (int a = 0; a < m; a++)
                if (u == 0 || cand[a] != cand[u - 1])
                    cand[u++] = cand[a];
            if (pass == 0) {
                A->rowptr[i + 1] = u;
            } else {
                int64_t p = A->rowptr[i];
                for (int a = 0; a < u; a++)
                    A->col[p + a] = (int32_t)cand[a];
            }
        }
        if (pass == 0) {
            for (int64_t i = 0; i < n; i++)
                A->rowptr[i + 1] += A->rowptr[i];
            A->nnz = A->rowptr[n];
            A->col = (int32_t *)malloc((size_t)A->nnz * sizeof(int32_t));
            A->val = (double *)calloc((size_t)A->nnz, sizeof(double));
            if (!A->col || !A->val)
                return -1;
        }
    }

    /* values: a_ij = sum over the cells e that contain DOFs i and j, in lexicographic
     * (ascending) cell order, of (k_e * hfac) * kref[a][b], a and b the local numbers of i
     * and j in e. Row i is filled by visiting its cells in ascending order, so every entry
     * receives its terms in the order of a loop over all cells; rows are independent. */
    (void)ncells;
    int nloc = elem == ORC_Q1 ? (1 << dim) : 6;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t cells[8], g[8];
        int mc = dof_cells(dim, elem, N, i, cells);
        for (int c = 0; c < mc; c++) {
            int64_t e = cells[c];
            int cx = (int)(e % NN), cy = (int)((e / NN) % NN), cz = dim == 3 ? (int)(e / (NN * NN)) : 0;
            double ke = k_cell ? k_cell[e] : 1.0;
            double s = ke * hfac;
            cell_dofs(dim, elem, N, cx, cy, cz, g);
            int a = 0;
            while (g[a] != i)
                a++;
            for (int b = 0; b < nloc; b++) {
                if (g[b] < 0)
                    continue;
                int64_t p = find_col(A, i, g[b]);
                A->val[p] = A->val[p] + s * kref[a * nloc + b];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Grid transfer operators between level l-1 (Nc cells per axis) and l (Nf = 2 Nc).  */
/* P has fine rows and coarse columns; the restriction is R = P^T (Sec. 5.4).        */
/* ------------------------------------------------------------------------------ */

typedef struct {
    int64_t col;
    double w;
} orc_entry;

static int cmp_entry(const void *a, const void *b)
{
    int64_t x = ((const orc_entry *)a)->col, y = ((const orc_entry *)b)->col;
    return (x > y) - (x < y);
}

/* fine row -> list of (coarse column, weight), unsorted, may repeat a column */
static int prolong_row(int dim, int elem, int Nc, int64_t i, const double *rq1_w, orc_entry *out)
{
    int Nf = 2 * Nc;
    int m = 0;
    if (elem == ORC_Q1) {
        /* nodal interpolation: p_iJ = phi_J^coarse(x_i), a product of 1D hats */
        int64_t n1 = Nf - 1;
        int v[3] = {(int)(i % n1) + 1, (int)((i / n1) % n1) + 1, dim == 3 ? (int)(i / (n1 * n1)) + 1 : 0};
        int lo[3], hi[3];
        for (int d = 0; d < 3; d++) {
            if (d >= dim) {
                lo[d] = hi[d] = 0;
                continue;
            }
            lo[d] = v[d] / 2;             /* coarse vertices with |v - 2V| <= 1 */
            hi[d] = (v[d] + 1) / 2;
        }
        for (int Z = lo[2]; Z <= hi[2]; Z++)
            for (int Y = lo[1]; Y <= hi[1]; Y++)
                for (int X = lo[0]; X <= hi[0]; X++) {
                    int64_t J = q1_vertex(dim, Nc, X, Y, dim == 3 ? Z : 1);
                    if (J < 0)
                        continue;
                    int V[3] = {X, Y, Z};
                    double w = 1.0;
                    for (int d = 0; d < dim; d++) {
                        int dist = abs(v[d] - 2 * V[d]); /* in fine mesh widths */
                        w = w * (1.0 - 0.5 * (double)dist);
                    }
                    out[m].col = J;
                    out[m].w = w;
                    m++;
                }
        return m;
    }
    /* rotated Q1: face averaging. Decode the fine face. */
    int64_t NN = Nf, fam = (int64_t)(Nf - 1) * NN * NN;
    int f = (int)(i / fam);
    int64_t r = i % fam;
    int p, q1, q2; /* normal position, cells along the two other axes (increasing axis) */
    if (f == 0) {
        p = (int)(r % (Nf - 1)) + 1;
        q1 = (int)((r / (Nf - 1)) % NN);
        q2 = (int)(r / ((Nf - 1) * NN));
    } else if (f == 1) {
        q1 = (int)(r % NN);
        p = (int)((r / NN) % (Nf - 1)) + 1;
        q2 = (int)(r / (NN * (Nf - 1)));
    } else {
        q1 = (int)(r % NN);
        q2 = (int)((r / NN) % NN);
        p = (int)(r / (NN * NN)) + 1;
    }
    int Q1 = q1 / 2, Q2 = q2 / 2, s1 = q1 % 2, s2 = q2 % 2;
    int cellpos[2], vpos[2], ncell;
    if (p % 2 == 0) { /* on a coarse face: the two coarse cells that share it */
        ncell = 2;
        cellpos[0] = p / 2 - 1;
        vpos[0] = 2; /* the face is this cell's upper face */
        cellpos[1] = p / 2;
        vpos[1] = 0; /* lower face */
    } else {          /* inside one coarse cell, at its mid-plane */
        ncell = 1;
        cellpos[0] = (p - 1) / 2;
        vpos[0] = 1;
    }
    double inv = ncell == 2 ? 0.5 : 1.0;
    for (int c = 0; c < ncell; c++) {
        int cxyz[3];
        cxyz[f] = cellpos[c];
        int o1 = f == 0 ? 1 : 0, o2 = f == 2 ? 1 : 2;
        cxyz[o1] = Q1;
        cxyz[o2] = Q2;
        int64_t g[6];
        cell_dofs(3, ORC_RQ1, Nc, cxyz[0], cxyz[1], cxyz[2], g);
        const double *w = rq1_w + ((((f * 3 + vpos[c]) * 2 + s1) * 2 + s2) * 6);
        for (int a = 0; a < 6; a++) {
            if (g[a] < 0 || w[a] == 0.0)
                continue;
            out[m].col = g[a];
            out[m].w = inv * w[a];
            m++;
        }
    }
    return m;
}

/* rq1_w: W[axis][v][s1][s2][a] mean of coarse basis a over the fine face (elements.py) */
static int prolong_tet(int elem, int Nc, orc_csr *P);

int orc_prolongation(int dim, int elem, int Nc, const double *rq1_w, orc_csr *P)
{
    if (elem == ORC_P1 || elem == ORC_P2)
        return prolong_tet(elem, Nc, P);
    int Nf = 2 * Nc;
    int64_t nf = orc_ndofs(dim, elem, Nf), nc = orc_ndofs(dim, elem, Nc);
    orc_entry ent[16];
    memset(P, 0, sizeof(*P));
    P->nrows = nf;
    P->ncols = nc;
    P->rowptr = (int64_t *)calloc((size_t)nf + 1, sizeof(int64_t));
    if (!P->rowptr)
        return -1;
    for (int pass = 0; pass < 2; pass++) {
        for (int64_t i = 0; i < nf; i++) {
            int m = prolong_row(dim, elem, Nc, i, rq1_w, ent);
            qsort(ent, (size_t)m, sizeof(orc_entry), cmp_entry);
            /* merge repeated columns in ascending order of appearance after the sort */
            int u = 0;
            for (int a = 0; a < m; a++) {
                if (u > 0 && ent[u - 1].col == ent[a].col)
                    ent[u - 1].w = ent[u - 1].w + ent[a].w;
                else
                    ent[u++] = ent[a];
            }
            if (pass == 0) {
                P->rowptr[i + 1] = u;
            } else {
                int64_t q = P->rowptr[i];
                for (int a = 0; a < u; a++) {
                    P->col[q + a] = (int32_t)ent[a].col;
                    P->val[q + a] = ent[a].w;
                }
            }
        }
        if (pass == 0) {
            for (int64_t i = 0; i < nf; i++)
                P->rowptr[i + 1] += P->rowptr[i];
            P->nnz = P->rowptr[nf];
            P->col = (int32_t *)malloc((size_t)P->nnz * sizeof(int32_t));
            P->val = (double *)malloc((size_t)P->nnz * sizeof(double));
            if (!P->col || !P->val)
                return -1;
        }
    }
    return 0;
}

/* T = M^T by a counting sort over columns: rows of T list M's rows in ascending order */
int orc_transpose(const orc_csr *M, orc_csr *T)
{
    memset(T, 0, sizeof(*T));
    T->nrows = M->ncols;
    T->ncols = M->nrows;
    T->nnz = M->nnz;
    T->rowptr = (int64_t *)calloc((size_t)T->nrows + 1, sizeof(int64_t));
    T->col = (int32_t *)malloc((size_t)T->nnz * sizeof(int32_t));
    T->val = (double *)malloc((size_t)T->nnz * sizeof(double));
    if (!T->rowptr || !T->col || !T->val)
        return -1;
    for (int64_t k = 0; k < M->nnz; k++)
        T->rowptr[M->col[k] + 1]++;
    for (int64_t j = 0; j < T->nrows; j++)
        T->rowptr[j + 1] += T->rowptr[j];
    int64_t *next = (int64_t *)malloc((size_t)T->nrows * sizeof(int64_t));
    if (!next)
        return -1;
    memcpy(next, T->rowptr, (size_t)T->nrows * sizeof(int64_t));
    for (int64_t i = 0; i < M->nrows; i++)
        for (int64_t k = M->rowptr[i]; k < M->rowptr[i + 1]; k++) {
            int64_t q = next[M->col[k]]++;
            T->col[q] = (int32_t)i;
            T->val[q] = M->val[k];
        }
    free(next);
    return 0;
}

/* Galerkin coarse operator A_c = R A P, entries accumulated as (r_Ii*a_ij)*p_jJ over
 * i ascending in R's row, j ascending in A's row, J ascending in P's row. */
int orc_galerkin(const orc_csr *R, const orc_csr *A, const orc_csr *P, orc_csr *Ac)
{
    int64_t nc = R->nrows;
    memset(Ac, 0, sizeof(*Ac));
    Ac->nrows = Ac->ncols = nc;
    Ac->rowptr = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    double *acc = (double *)calloc((size_t)nc, sizeof(double));
    char *mark = (char *)calloc((size_t)nc, 1);
    int64_t *list = (int64_t *)malloc((size_t)nc * sizeof(int64_t));
    if (!Ac->rowptr || !acc || !mark || !list)
        return -1;
    int64_t cap = 0;
    for (int pass = 0; pass < 2; pass++) {
        for (int64_t I = 0; I < nc; I++) {
            int64_t m = 0;
            for (int64_t ki = R->rowptr[I]; ki < R->rowptr[I + 1]; ki++) {
                int64_t i = R->col[ki];
                for (int64_t kj = A->rowptr[i]; kj < A->rowptr[i + 1]; kj++) {
                    int64_t j = A->col[kj];
                    double ra = R->val[ki] * A->val[kj];
                    for (int64_t kJ = P->rowptr[j]; kJ < P->rowptr[j + 1]; kJ++) {
                        int64_t J = P->col[kJ];
                        if (!mark[J]) {
                            mark[J] = 1;
                            list[m++] = J;
                        }
                        acc[J] = acc[J] + ra * P->val[kJ];
                    }
                }
            }
            qsort(list, (size_t)m, sizeof(int64_t), cmp_i64);
            if (pass == 0) {
                Ac->rowptr[I + 1] = m;
            } else {
                int64_t q = Ac->rowptr[I];
                for (int64_t a = 0; a < m; a++) {
                    Ac->col[q + a] = (int32_t)list[a];
                    Ac->val[q + a] = acc[list[a]];
                }
            }
            for (int64_t a = 0; a < m; a++) {
                acc[list[a]] = 0.0;
                mark[list[a]] = 0;
            }
        }
        if (pass == 0) {
            for (int64_t I = 0; I < nc; I++)
                Ac->rowptr[I + 1] += Ac->rowptr[I];
            Ac->nnz = Ac->rowptr[nc];
            cap = Ac->nnz;
            Ac->col = (int32_t *)malloc((size_t)cap * sizeof(int32_t));
            Ac->val = (double *)malloc((size_t)cap * sizeof(double));
            if (!Ac->col || !Ac->val)
                return -1;
        }
    }
    free(acc);
    free(mark);
    free(list);
    return 0;
}

/* ------------------------------------------------------------------------------ */
/* Load vector b_i = int f phi_i, 3-point Gauss per axis per cell                     */
/* ------------------------------------------------------------------------------ */

/*
 * f is either a constant (nmodes == 0: f = fconst) or the right-hand side of the
 * manufactured solution u = sum_m amp_m prod_d sin(k_md pi x_d):
 *   f = sum_m c_m * (sin(k_m1 pi x) * sin(k_m2 pi y) [* sin(k_m3 pi z)]),
 *   c_m = (amp_m * (pi*pi)) * |k_m|^2.
 * rq1_basis: C[m][a] monomial coefficients of the rotated-Q1 basis (elements.py).
 */
static double eval_f(int dim, int nmodes, const double *amp, const int *kf, double fconst, const double *p)
{
    if (nmodes == 0)
        return fconst;
    double f = 0.0;
    for (int m = 0; m < nmodes; m++) {
        int ksq = 0;
        for (int d = 0; d < dim; d++)
            ksq += kf[3 * m + d] * kf[3 * m + d];
        double c = (amp[m] * (ORC_PI * ORC_PI)) * (double)ksq;
        double s = sin(((double)kf[3 * m + 0] * ORC_PI) * p[0]);
        s = s * sin(((double)kf[3 * m + 1] * ORC_PI) * p[1]);
        if (dim == 3)
            s = s * sin(((double)kf[3 * m + 2] * ORC_PI) * p[2]);
        f = f + c * s;
    }
    return f;
}

static double eval_u(int dim, int nmodes, const double *amp, const int *kf, const double *p)
{
    double u = 0.0;
    for (int m = 0; m < nmodes; m++) {
        double s = sin(((double)kf[3 * m + 0] * ORC_PI) * p[0]);
        s = s * sin(((double)kf[3 * m + 1] * ORC_PI) * p[1]);
        if (dim == 3)
            s = s * sin(((double)kf[3 * m + 2] * ORC_PI) * p[2]);
        u = u + amp[m] * s;
    }
    return u;
}

static double basis_at(int dim, int elem, int a, const double *xi, const double *rq1_basis)
{
    if (elem == ORC_Q1) {
        double t = 1.0;
        for (int d = 0; d < dim; d++)
            t = t * (((a >> d) & 1) ? xi[d] : (1.0 - xi[d]));
        return t;
    }
    double mon[6] = {1.0, xi[0], xi[1], xi[2], xi[0] * xi[0] - xi[1] * xi[1], xi[1] * xi[1] - xi[2] * xi[2]};
    double s = 0.0;
    for (int m = 0; m < 6; m++)
        s = s + rq1_basis[m * 6 + a] * mon[m];
    return s;
}

static void gauss3(double *xi, double *w)
{
    double s = sqrt(0.6);
    xi[0] = 0.5 - 0.5 * s;
    xi[1] = 0.5;
    xi[2] = 0.5 + 0.5 * s;
    w[0] = 5.0 / 18.0;
    w[1] = 8.0 / 18.0;
    w[2] = 5.0 / 18.0;
}

int orc_load_vector(int dim, int elem, int N, int nmodes, const double *amp, const int *kf, double fconst,
                    const double *rq1_basis, double *b)
{
    int64_t n = orc_ndofs(dim, elem, N), NN = N;
    int64_t ncells = dim == 2 ? NN * NN : NN * NN * NN;
    double h = 1.0 / (double)N;
    double hd = dim == 2 ? h * h : (h * h) * h;
    double gx[3], gw[3];
    gauss3(gx, gw);
    int nloc = elem == ORC_Q1 ? (1 << dim) : 6;
    int nqz = dim == 3 ? 3 : 1;
    /* cell contributions be[e][a] (cells independent), then b_i = the sum of its cells'
     * contributions in ascending cell order from 0.0 (rows independent): the order of a
     * loop over the cells adding into b */
    double *bec = (double *)malloc((size_t)ncells * nloc * sizeof(double));
    if (!bec)
        return -1;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ncells; e++) {
        int c[3] = {(int)(e % NN), (int)((e / NN) % NN), dim == 3 ? (int)(e / (NN * NN)) : 0};
        double be[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int qz = 0; qz < nqz; qz++)
            for (int qy = 0; qy < 3; qy++)
                for (int qx = 0; qx < 3; qx++) {
                    double xi[3] = {gx[qx], gx[qy], dim == 3 ? gx[qz] : 0.0};
                    double p[3];
                    for (int d = 0; d < 3; d++)
                        p[d] = ((double)c[d] + xi[d]) * h;
                    double wq = gw[qx] * gw[qy];
                    if (dim == 3)
                        wq = wq * gw[qz];
                    double fw = eval_f(dim, nmodes, amp, kf, fconst, p) * (wq * hd);
                    for (int a = 0; a < nloc; a++)
                        be[a] = be[a] + fw * basis_at(dim, elem, a, xi, rq1_basis);
                }
        for (int a = 0; a < nloc; a++)
            bec[e * nloc + a] = be[a];
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        int64_t cells[8], g[8];
        int mc = dof_cells(dim, elem, N, i, cells);
        double bi = 0.0;
        for (int c = 0; c < mc; c++) {
            int64_t e = cells[c];
            cell_dofs(dim, elem, N, (int)(e % NN), (int)((e / NN) % NN), dim == 3 ? (int)(e / (NN * NN)) : 0, g);
            int a = 0;
            while (g[a] != i)
                a++;
            bi = bi + bec[e * nloc + a];
        }
        b[i] = bi;
    }
    free(bec);
    return 0;
}

/* L2 error ||u - u_h|| of the discrete function with DOF vector x, 3-point Gauss/cell */
double orc_l2_error(int dim, int elem, int N, int nmodes, const double *amp, const int *kf,
                    const double *rq1_basis, const double *x)
{
    int64_t NN = N, ncells = dim == 2 ? NN * NN : NN * NN * NN;
    double h = 1.0 / (double)N, hd = dim == 2 ? h * h : h * h * h;
    double gx[3], gw[3];
    gauss3(gx, gw);
    int nloc = elem == ORC_Q1 ? (1 << dim) : 6;
    int nqz = dim == 3 ? 3 : 1;
    double err = 0.0;
    int64_t g[8];
    for (int64_t e = 0; e < ncells; e++) {
        int c[3] = {(int)(e % NN), (int)((e / NN) % NN), dim == 3 ? (int)(e / (NN * NN)) : 0};
        cell_dofs(dim, elem, N, c[0], c[1], c[2], g);
        for (int qz = 0; qz < nqz; qz++)
            for (int qy = 0; qy < 3; qy++)
                for (int qx = 0; qx < 3; qx++) {
                    double xi[3] = {gx[qx], gx[qy], dim == 3 ? gx[qz] : 0.0};
                    double p[3];
                    for (int d = 0; d < 3; d++)
                        p[d] = ((double)c[d] + xi[d]) * h;
                    double wq = gw[qx] * gw[qy] * (dim == 3 ? gw[qz] : 1.0);
                    double uh = 0.0;
                    for (int a = 0; a < nloc; a++)
                        if (g[a] >= 0)
                            uh += x[g[a]] * basis_at(dim, elem, a, xi, rq1_basis);
                    double d = uh - eval_u(dim, nmodes, amp, kf, p);
                    err += wq * hd * d * d;
                }
    }
    return sqrt(err);
}

/* ------------------------------------------------------------------------------ */
/* Sparse kernels                                                                    */
/* ------------------------------------------------------------------------------ */

/* threads for the row loops below (results are the same for every count) */
void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int orc_get_threads(void) { return omp_get_max_threads(); }

void orc_spmv(const orc_csr *A, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->nrows; i++) {
        double s = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
            s = fma(A->val[k], x[A->col[k]], s);
        y[i] = s;
    }
}

static void residual(const orc_csr *A, const double *b, const double *x, double *r)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < A->nrows; i++) {
        double s = 0.0;
        for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
            s = fma(A->val[k], x[A->col[k]], s);
        r[i] = b[i] - s;
    }
}

static double diag_of(const orc_csr *A, int64_t i)
{
    int64_t p = find_col(A, i, i);
    return p >= 0 ? A->val[p] : 0.0;
}

static double norm2(const double *v, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++)
        s = s + v[i] * v[i];
    return sqrt(s);
}

/* ||v||_2 for the residual history and the stopping test: the sum of squares is
 * accumulated with Neumaier's compensated summation (Neumaier 1974), so the reported
 * norm is within a few ulps of the exact one for any length, unlike the plain
 * sequential sum whose relative error grows with n. */
static double norm2_accurate(const double *v, int64_t n)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double t = v[i] * v[i];
        double u = s + t;
        if (fabs(s) >= fabs(t))
            c = c + ((s - u) + t);
        else
            c = c + ((t - u) + s);
        s = u;
    }
    return sqrt(s + c);
}

/* ------------------------------------------------------------------------------ */
/* Coarsest level: dense LU with partial pivoting (first row of maximal |a| wins)    */
/* ------------------------------------------------------------------------------ */

int orc_lu_factor(double *a, int n, int *piv)
{
    for (int k = 0; k < n; k++) {
        int p = k;
        double best = fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; i++)
            if (fabs(a[(size_t)i * n + k]) > best) {
                best = fabs(a[(size_t)i * n + k]);
                p = i;
            }
        piv[k] = p;
        if (best == 0.0)
            return -1;
        if (p != k)
            for (int j = 0; j < n; j++) {
                double t = a[(size_t)k * n + j];
                a[(size_t)k * n + j] = a[(size_t)p * n + j];
                a[(size_t)p * n + j] = t;
            }
        for (int i = k + 1; i < n; i++) {
            double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
            a[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; j++)
                a[(size_t)i * n + j] = a[(size_t)i * n + j] - l * a[(size_t)k * n + j];
        }
    }
    return 0;
}

void orc_lu_solve(const double *lu, int n, const int *piv, const double *b, double *x)
{
    for (int i = 0; i < n; i++)
        x[i] = b[i];
    for (int k = 0; k < n; k++)
        if (piv[k] != k) {
            double t = x[k];
            x[k] = x[piv[k]];
            x[piv[k]] = t;
        }
    for (int i = 0; i < n; i++) { /* L y = Pb, unit diagonal */
        double s = 0.0;
        for (int j = 0; j < i; j++)
            s = fma(lu[(size_t)i * n + j], x[j], s);
        x[i] = x[i] - s;
    }
    for (int i = n - 1; i >= 0; i--) { /* U x = y; the sum runs from j = n-1 down to i+1,
                                          * the order in which the x_j become known; the
                                          * result is multiplied by the pivot's reciprocal */
        double s = 0.0;
        for (int j = n - 1; j > i; j--)
            s = fma(lu[(size_t)i * n + j], x[j], s);
        double inv = 1.0 / lu[(size_t)i * n + i];
        x[i] = (x[i] - s) * inv;
    }
}


/* ------------------------------------------------------------------------------ */
/* P1 / P2 on tetrahedra (3D): the Kuhn (Freudenthal) triangulation of the grid.     */
/* Cell (cx,cy,cz) holds one tetrahedron per permutation pi of the axes, in the      */
/* order (012) (021) (102) (120) (201) (210): vertices v0 = (cx,cy,cz), v1 = v0 +    */
/* e_pi0, v2 = v1 + e_pi1, v3 = v0 + (1,1,1). Refinement by halving splits each into */
/* 8 tetrahedra of the finer grid (Freudenthal), so the spaces are nested.           */
/*   P1 DOFs: interior vertices, numbered like Q1.                                   */
/*   P2 DOFs: vertices and edge midpoints = the interior points of the grid of 2N    */
/*   cells per axis, numbered like Q1 there; local nodes 0..3 are the vertices,      */
/*   4..9 the midpoints of edges (01) (02) (03) (12) (13) (23).                      */
/* The element matrix of a tetrahedron of a cell of side h is (k_e * hfac) * kref    */
/* (the same table for all six: they are congruent with the same local order).       */
/* ------------------------------------------------------------------------------ */
static const int KUHN[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
static const int TET_EDGE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

/* global DOFs of tetrahedron t of cell (cx,cy,cz) (-1: Dirichlet); returns the count */
static int tet_dofs(int elem, int N, int cx, int cy, int cz, int t, int64_t *g)
{
    int v[4][3];
    v[0][0] = cx;
    v[0][1] = cy;
    v[0][2] = cz;
    for (int a = 1; a < 4; a++) {
        for (int d = 0; d < 3; d++)
            v[a][d] = v[a - 1][d];
        if (a < 3)
            v[a][KUHN[t][a - 1]] += 1;
        else
            v[a][KUHN[t][2]] += 1;
    }
    if (elem == ORC_P1) {
        for (int a = 0; a < 4; a++)
            g[a] = q1_vertex(3, N, v[a][0], v[a][1], v[a][2]);
        return 4;
    }
    for (int a = 0; a < 4; a++)
        g[a] = q1_vertex(3, 2 * N, 2 * v[a][0], 2 * v[a][1], 2 * v[a][2]);
    for (int e = 0; e < 6; e++) {
        int a = TET_EDGE[e][0], b = TET_EDGE[e][1];
        g[4 + e] = q1_vertex(3, 2 * N, v[a][0] + v[b][0], v[a][1] + v[b][1], v[a][2] + v[b][2]);
    }
    return 10;
}

/* the tetrahedra containing DOF i, as cell * 6 + t in increasing order */
static int node_tets(int elem, int N, int64_t i, int64_t *out)
{
    int M = elem == ORC_P1 ? N : 2 * N; /* grid of the DOFs */
    int64_t m1 = M - 1, NN = N;
    int w[3] = {(int)(i % m1) + 1, (int)((i / m1) % m1) + 1, (int)(i / (m1 * m1)) + 1};
    int lo[3], hi[3];
    for (int d = 0; d < 3; d++) {
        if (elem == ORC_P1) {
            lo[d] = w[d] - 1;
            hi[d] = w[d];
        } else {
            lo[d] = (w[d] - 1) >> 1;
            hi[d] = w[d] >> 1;
        }
        if (lo[d] < 0)
            lo[d] = 0;
        if (hi[d] > N - 1)
            hi[d] = N - 1;
    }
    int m = 0;
    int64_t g[10];
    for (int cz = lo[2]; cz <= hi[2]; cz++)
        for (int cy = lo[1]; cy <= hi[1]; cy++)
            for (int cx = lo[0]; cx <= hi[0]; cx++)
                for (int t = 0; t < 6; t++) {
                    int nl = tet_dofs(elem, N, cx, cy, cz, t, g);
                    for (int a = 0; a < nl; a++)
                        if (g[a] == i) {
                            out[m++] = (cx + NN * (cy + NN * (int64_t)cz)) * 6 + t;
                            break;
                        }
                }
    return m;
}

static int assemble_tet(int elem, int N, const double *kref, const double *k_cell, double hfac, orc_csr *A)
{
    int64_t n = orc_ndofs(3, elem, N), NN = N;
    int nl = elem == ORC_P1 ? 4 : 10;
    memset(A, 0, sizeof(*A));
    A->nrows = A->ncols = n;
    A->rowptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!A->rowptr)
        return -1;
    int64_t tets[256], g[10], cand[2560];
    for (int pass = 0; pass < 2; pass++) {
        for (int64_t i = 0; i < n; i++) {
            int mt = node_tets(elem, N, i, tets);
            int m = 0;
            for (int q = 0; q < mt; q++) {
                int64_t c = tets[q] / 6;
                int t = (int)(tets[q] % 6);
                tet_dofs(elem, N, (int)(c % NN), (int)((c / NN) % NN), (int)(c / (NN * NN)), t, g);
                for (int a = 0; a < nl; a++)
                    if (g[a] >= 0)
                        cand[m++] = g[a];
            }
            qsort(cand, (size_t)m, sizeof(int64_t), cmp_i64);
            int u = 0;
            for (int a = 0; a < m; a++)
                if (u == 0 || cand[a] != cand[u - 1])
                    cand[u++] = cand[a];
            if (pass == 0) {
                A->rowptr[i + 1] = u;
            } else {
                int64_t p = A->rowptr[i];
                for (int a = 0; a < u; a++)
                    A->col[p + a] = (int32_t)cand[a];
            }
        }
        if (pass == 0) {
            for (int64_t i = 0; i < n; i++)
                A->rowptr[i + 1] += A->rowptr[i];
            A->nnz = A->rowptr[n];
            A->col = (int32_t *)malloc((size_t)A->nnz * sizeof(int32_t));
            A->val = (double *)calloc((size_t)A->nnz, sizeof(double));
            if (!A->col || !A->val)
                return -1;
        }
    }
    /* values: element loop, cells in lexicographic order, tetrahedra in KUHN order */
    int64_t ncells = NN * NN * NN;
    for (int64_t e = 0; e < ncells; e++) {
        int cx = (int)(e % NN), cy = (int)((e / NN) % NN), cz = (int)(e / (NN * NN));
        double ke = k_cell ? k_cell[e] : 1.0;
        double sc = ke * hfac;
        for (int t = 0; t < 6; t++) {
            tet_dofs(elem, N, cx, cy, cz, t, g);
            for (int a = 0; a < nl; a++) {
                if (g[a] < 0)
                    continue;
                for (int b = 0; b < nl; b++) {
                    if (g[b] < 0)
                        continue;
                    int64_t p = find_col(A, g[a], g[b]);
                    A->val[p] = A->val[p] + sc * kref[a * nl + b];
                }
            }
        }
    }
    return 0;
}

/*
 * Prolongation = interpolation of the coarse function at the fine nodes (the spaces
 * are nested; the paper's general transfer of Sec. 5.4 reduces to this for conforming
 * elements). A fine node at coarse-cell coordinates c + s, s in [0,1]^3 (c the cell
 * of the node, the last cell on the upper boundary), lies in the Kuhn tetrahedron
 * whose permutation sorts s in decreasing order (ties by axis); there
 * lambda = (1 - s_pi0, s_pi0 - s_pi1, s_pi1 - s_pi2, s_pi2) and the weights are the
 * coarse basis values (P1: lambda_a; P2: lambda_a (2 lambda_a - 1), 4 lambda_a lambda_b).
 * All are dyadic, so exact. Zero weights and Dirichlet coarse DOFs are dropped.
 */
static int prolong_tet(int elem, int Nc, orc_csr *P)
{
    int Nf = 2 * Nc;
    int64_t nf = orc_ndofs(3, elem, Nf), nc = orc_ndofs(3, elem, Nc);
    int Mf = elem == ORC_P1 ? Nf : 2 * Nf; /* fine node grid */
    int r = elem == ORC_P1 ? 2 : 4;        /* fine node spacings per coarse cell */
    int64_t m1 = Mf - 1;
    memset(P, 0, sizeof(*P));
    P->nrows = nf;
    P->ncols = nc;
    P->rowptr = (int64_t *)calloc((size_t)nf + 1, sizeof(int64_t));
    if (!P->rowptr)
        return -1;
    orc_entry ent[10];
    for (int pass = 0; pass < 2; pass++) {
        for (int64_t i = 0; i < nf; i++) {
            int w[3] = {(int)(i % m1) + 1, (int)((i / m1) % m1) + 1, (int)(i / (m1 * m1)) + 1};
            int c[3];
            double sv[3];
            for (int d = 0; d < 3; d++) {
                c[d] = w[d] / r;
                if (c[d] > Nc - 1)
                    c[d] = Nc - 1;
                sv[d] = (double)(w[d] - r * c[d]) / (double)r;
            }
            int pi[3] = {0, 1, 2};
            for (int a = 1; a < 3; a++) /* stable insertion sort, decreasing s */
                for (int b = a; b > 0 && sv[pi[b]] > sv[pi[b - 1]]; b--) {
                    int tmp = pi[b];
                    pi[b] = pi[b - 1];
                    pi[b - 1] = tmp;
                }
            int t = 0;
            while (!(KUHN[t][0] == pi[0] && KUHN[t][1] == pi[1] && KUHN[t][2] == pi[2]))
                t++;
            double lam[4] = {1.0 - sv[pi[0]], sv[pi[0]] - sv[pi[1]], sv[pi[1]] - sv[pi[2]], sv[pi[2]]};
            int64_t g[10];
            int nl = tet_dofs(elem, Nc, c[0], c[1], c[2], t, g);
            double wt[10];
            if (elem == ORC_P1) {
                for (int a = 0; a < 4; a++)
                    wt[a] = lam[a];
            } else {
                for (int a = 0; a < 4; a++)
                    wt[a] = lam[a] * (2.0 * lam[a] - 1.0);
                for (int e = 0; e < 6; e++)
                    wt[4 + e] = (4.0 * lam[TET_EDGE[e][0]]) * lam[TET_EDGE[e][1]];
            }
            int m = 0;
            for (int a = 0; a < nl; a++)
                if (g[a] >= 0 && wt[a] != 0.0) {
                    ent[m].col = g[a];
                    ent[m].w = wt[a];
                    m++;
                }
            qsort(ent, (size_t)m, sizeof(orc_entry), cmp_entry);
            if (pass == 0) {
                P->rowptr[i + 1] = m;
            } else {
                int64_t p = P->rowptr[i];
                for (int a = 0; a < m; a++) {
                    P->col[p + a] = (int32_t)ent[a].col;
                    P->val[p + a] = ent[a].w;
                }
            }
        }
        if (pass == 0) {
            for (int64_t i = 0; i < nf; i++)
                P->rowptr[i + 1] += P->rowptr[i];
            P->nnz = P->rowptr[nf];
            P->col = (int32_t *)malloc((size_t)(P->nnz ? P->nnz : 1) * sizeof(int32_t));
            P->val = (double *)malloc((size_t)(P->nnz ? P->nnz : 1) * sizeof(double));
            if (!P->col || !P->val)
                return -1;
        }
    }
    return 0;
}

/*
 * Load vector of the tetrahedral elements: b = M f_I, the consistent mass matrix times
 * the nodal values of f (the quadrature is not given by the paper; interpolating f
 * keeps the order of the element, 2 for P1 and 3 for P2). mref: the element mass table;
 * the row sums are column-ascending fused multiply-adds as in orc_spmv.
 */
int orc_load_vector_tet(int elem, int N, int nmodes, const double *amp, const int *kf, double fconst,
                        const double *mref, double *b)
{
    orc_csr M;
    double h = 1.0 / (double)N;
    if (assemble_tet(elem, N, mref, NULL, (h * h) * h, &M))
        return -1;
    int64_t n = M.nrows;
    double *f = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; i++) {
        double x[3];
        orc_tet_node_coords(elem, N, i, x);
        f[i] = eval_f(3, nmodes, amp, kf, fconst, x);
    }
    orc_spmv(&M, f, b);
    free(f);
    orc_csr_free(&M);
    return 0;
}

/* coordinate of DOF i of a tetrahedral element on N cells (node grid: N for P1, 2N for P2) */
void orc_tet_node_coords(int elem, int N, int64_t i, double *x)
{
    int M = elem == ORC_P1 ? N : 2 * N;
    int64_t m1 = M - 1;
    int w[3] = {(int)(i % m1) + 1, (int)((i / m1) % m1) + 1, (int)(i / (m1 * m1)) + 1};
    for (int d = 0; d < 3; d++)
        x[d] = (double)w[d] / (double)M;
}

/* ------------------------------------------------------------------------------ */
/* Hierarchy and V-cycle                                                             */
/* ------------------------------------------------------------------------------ */

#define ORC_MAXLEV 16

typedef struct {
    int dim, elem, n_levels;
    int N[ORC_MAXLEV];          /* cells per axis, level 0 = coarsest */
    int galerkin[ORC_MAXLEV];   /* 1 if A_l = R A_{l+1} P */
    orc_csr A[ORC_MAXLEV], P[ORC_MAXLEV], R[ORC_MAXLEV]; /* P[l], R[l] for l >= 1 */
    double *dinv[ORC_MAXLEV];
    double lam[ORC_MAXLEV];     /* power-iteration estimate of lambda_max(D^-1 A_l) */
    double *lu;
    int *piv;
    int n0;
    double *b[ORC_MAXLEV], *x[ORC_MAXLEV], *r[ORC_MAXLEV], *t[ORC_MAXLEV], *d[ORC_MAXLEV];
    int *colour[ORC_MAXLEV];    /* Gauss-Seidel colour of every DOF */
} orc_hier;

typedef struct {
    int smoother;       /* 0: damped Jacobi, 1: Chebyshev, 2: multicolour Gauss-Seidel */
    double omega;       /* Jacobi damping */
    int cheb_degree;    /* matrix-vector products per Chebyshev application */
    int nu_pre, nu_post;/* smoother applications before / after the coarse correction */
    double cheb_hi;     /* lambda_u = cheb_hi * lambda_hat */
    double cheb_ratio;  /* lambda_l = lambda_u / cheb_ratio */
    int max_iters;
} orc_opts;

static uint64_t splitmix64(uint64_t seed, uint64_t i)
{
    /* SplitMix64 (Steele, Lea, Flood 2014) in counter form: output i of the sequence
     * started at `seed` */
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* lambda_hat: `iters` steps of the power method on D^-1 A, start vector
 * v_i = 1 + 0.2*(u_i - 0.5), u_i = splitmix64(seed, i) / 2^64 (53-bit), normalised */
double orc_power_lambda(const orc_csr *A, const double *dinv, int iters, uint64_t seed)
{
    int64_t n = A->nrows;
    double *v = (double *)malloc((size_t)n * sizeof(double));
    double *w = (double *)malloc((size_t)n * sizeof(double));
    for (int64_t i = 0; i < n; i++) {
        double u = (double)(splitmix64(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
        v[i] = 1.0 + 0.2 * (u - 0.5);
    }
    double nv = norm2(v, n);
    for (int64_t i = 0; i < n; i++)
        v[i] = v[i] / nv;
    double lam = 0.0;
    for (int it = 0; it < iters; it++) {
        orc_spmv(A, v, w);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            w[i] = dinv[i] * w[i];
        lam = norm2(w, n);
        for (int64_t i = 0; i < n; i++)
            v[i] = w[i] / lam;
    }
    free(v);
    free(w);
    return lam;
}

void orc_free(orc_hier *H)
{
    if (!H)
        return;
    for (int l = 0; l < H->n_levels; l++) {
        orc_csr_free(&H->A[l]);
        orc_csr_free(&H->P[l]);
        orc_csr_free(&H->R[l]);
        free(H->dinv[l]);
        free(H->b[l]);
        free(H->x[l]);
        free(H->r[l]);
        free(H->t[l]);
        free(H->d[l]);
        free(H->colour[l]);
    }
    free(H->lu);
    free(H->piv);
    free(H);
}

/* cells of level l are resolved by the coefficient iff every fine cell it covers has
 * the same k; then kl[c] is that value */
static int coarse_k(int dim, int NL, const double *kL, int Nl, double *kl)
{
    int r = NL / Nl;
    int64_t NNl = Nl, NNL = NL;
    int64_t ncl = dim == 2 ? NNl * NNl : NNl * NNl * NNl;
    for (int64_t c = 0; c < ncl; c++) {
        int cx = (int)(c % NNl), cy = (int)((c / NNl) % NNl), cz = dim == 3 ? (int)(c / (NNl * NNl)) : 0;
        double k0 = kL[(int64_t)cx * r + NNL * ((int64_t)cy * r + NNL * (int64_t)cz * r)];
        for (int dz = 0; dz < (dim == 3 ? r : 1); dz++)
            for (int dy = 0; dy < r; dy++)
                for (int dx = 0; dx < r; dx++) {
                    int64_t f = ((int64_t)cx * r + dx) + NNL * (((int64_t)cy * r + dy) + NNL * ((int64_t)cz * r + dz));
                    if (kL[f] != k0)
                        return 0;
                }
        kl[c] = k0;
    }
    return 1;
}

/*
 * Build the hierarchy: levels 0..n_levels-1 with N_l = N_finest / 2^(L-l).
 * Each level is rediscretised with the element tables (the paper assembles the system
 * on every level of the mesh hierarchy, Sec. 5.1); a level whose cells are not
 * resolved by the coefficient field, and every coarser one, takes the Galerkin
 * product R A P of the next finer level instead.
 */
orc_hier *orc_setup(int dim, int elem, int N_finest, int n_levels, const double *kref,
                    const double *rq1_w, const double *k_cell, int power_iters, uint64_t power_seed,
                    const double *mref, double mass)
{
    if (n_levels < 1 || n_levels > ORC_MAXLEV)
        return NULL;
    orc_hier *H = (orc_hier *)calloc(1, sizeof(orc_hier));
    H->dim = dim;
    H->elem = elem;
    H->n_levels = n_levels;
    int L = n_levels - 1;
    for (int l = 0; l <= L; l++) {
        H->N[l] = N_finest >> (L - l);
        if ((H->N[l] << (L - l)) != N_finest || H->N[l] < 2) {
            orc_free(H);
            return NULL;
        }
    }
    int use_galerkin = 0;
    for (int l = L; l >= 0; l--) {
        int Nl = H->N[l];
        if (l < L) {
            if (orc_prolongation(dim, elem, Nl, rq1_w, &H->P[l + 1]) ||
                orc_transpose(&H->P[l + 1], &H->R[l + 1])) {
                orc_free(H);
                return NULL;
            }
        }
        double *kl = NULL;
        if (k_cell && !use_galerkin) {
            int64_t NNl = Nl;
            kl = (double *)malloc((size_t)(dim == 2 ? NNl * NNl : NNl * NNl * NNl) * sizeof(double));
            if (!coarse_k(dim, N_finest, k_cell, Nl, kl))
                use_galerkin = 1;
        }
        int rc;
        if (use_galerkin) {
            rc = orc_galerkin(&H->R[l + 1], &H->A[l + 1], &H->P[l + 1], &H->A[l]);
            H->galerkin[l] = 1;
        } else {
            rc = orc_assemble(dim, elem, Nl, kref, kl, &H->A[l]);
            if (rc == 0 && mass != 0.0) { /* the shifted operator A + mass * M */
                orc_csr M;
                rc = orc_assemble_mass(dim, elem, Nl, mref, &M);
                if (rc == 0)
                    for (int64_t k = 0; k < M.nnz; k++)
                        H->A[l].val[k] = H->A[l].val[k] + mass * M.val[k];
                orc_csr_free(&M);
            }
        }
        free(kl);
        if (rc) {
            orc_free(H);
            return NULL;
        }
    }
    for (int l = 0; l <= L; l++) {
        int64_t n = H->A[l].nrows;
        H->dinv[l] = (double *)malloc((size_t)n * sizeof(double));
        for (int64_t i = 0; i < n; i++)
            H->dinv[l][i] = 1.0 / diag_of(&H->A[l], i);
        H->b[l] = (double *)calloc((size_t)n, sizeof(double));
        H->x[l] = (double *)calloc((size_t)n, sizeof(double));
        H->r[l] = (double *)calloc((size_t)n, sizeof(double));
        H->t[l] = (double *)calloc((size_t)n, sizeof(double));
        H->d[l] = (double *)calloc((size_t)n, sizeof(double));
        H->colour[l] = (int *)malloc((size_t)n * sizeof(int));
        for (int64_t i = 0; i < n; i++)
            H->colour[l][i] = orc_colour(dim, elem, H->N[l], i);
        H->lam[l] = (l > 0 && power_iters > 0) ? orc_power_lambda(&H->A[l], H->dinv[l], power_iters, power_seed) : 0.0;
    }
    /* coarsest: dense copy and LU factorisation */
    int n0 = (int)H->A[0].nrows;
    H->n0 = n0;
    H->lu = (double *)calloc((size_t)n0 * n0, sizeof(double));
    H->piv = (int *)calloc((size_t)n0, sizeof(int));
    for (int i = 0; i < n0; i++)
        for (int64_t k = H->A[0].rowptr[i]; k < H->A[0].rowptr[i + 1]; k++)
            H->lu[(size_t)i * n0 + H->A[0].col[k]] = H->A[0].val[k];
    if (orc_lu_factor(H->lu, n0, H->piv)) {
        orc_free(H);
        return NULL;
    }
    return H;
}

/*
 * Colour of DOF i for the multicolour Gauss-Seidel smoother. The paper colours the DOFs
 * of its hybrid computations and numbers them colour-wise (Sec. 4, "DOF Reordering");
 * the colouring is chosen per element such that two DOFs of one colour never share a
 * cell (or tetrahedron), hence are never coupled by A:
 *   Q1:  parity of each vertex coordinate, colour = (vx&1) + 2(vy&1) [+ 4(vz&1)]
 *        (two vertices of one cell differ by 1 in some coordinate);
 *   RQ1: face family and parity of the normal position, colour = 2f + (p&1)
 *        (the two faces of one family in a cell sit at p and p+1);
 *   P1:  colour = (vx + vy + vz) mod 4: two vertices of a Kuhn tetrahedron differ by
 *        an offset whose coordinates sum to 1, 2 or 3 in absolute value; four colours
 *        are the fewest possible (every tetrahedron is a 4-clique);
 *   P2:  colour = (wx + 2 wy + 4 wz) mod 15 on the grid of 2N cells: none of the 64
 *        offsets between two nodes of a Kuhn tetrahedron maps to 0 mod 15 (the
 *        smallest modulus of such a lattice colouring; a tetrahedron's 10 nodes need
 *        at least 10 colours).
 */
int orc_n_colours(int dim, int elem)
{
    if (elem == ORC_Q1)
        return 1 << dim;
    if (elem == ORC_P1)
        return 4;
    return elem == ORC_RQ1 ? 6 : 15;
}

int orc_colour(int dim, int elem, int N, int64_t i)
{
    int64_t n1 = N - 1, NN = N;
    if (elem == ORC_P1 || elem == ORC_P2) {
        int M = elem == ORC_P1 ? N : 2 * N; /* node grid */
        int64_t m1 = M - 1;
        int wx = (int)(i % m1) + 1, wy = (int)((i / m1) % m1) + 1, wz = (int)(i / (m1 * m1)) + 1;
        return elem == ORC_P1 ? (wx + wy + wz) % 4 : (wx + 2 * wy + 4 * wz) % 15;
    }
    if (elem == ORC_Q1) {
        int vx = (int)(i % n1) + 1;
        int vy = (int)((i / n1) % n1) + 1;
        int c = (vx & 1) + 2 * (vy & 1);
        if (dim == 3)
            c += 4 * (((int)(i / (n1 * n1)) + 1) & 1);
        return c;
    }
    int64_t fam = n1 * NN * NN;
    int f = (int)(i / fam);
    int64_t r = i % fam;
    int p;
    if (f == 0)
        p = (int)(r % n1) + 1;
    else if (f == 1)
        p = (int)((r / NN) % n1) + 1;
    else
        p = (int)(r / (NN * NN)) + 1;
    return 2 * f + (p & 1);
}

/* one Gauss-Seidel sweep over the colours in increasing order (forward) or decreasing
 * order (backward): within a colour the rows are independent, so visiting them in
 * index order is the same as updating them all at once from the current x */
void orc_gs_sweep(const orc_csr *A, const double *dinv, const int *colour, int ncol, int backward,
                  const double *b, double *x)
{
    int64_t n = A->nrows;
    for (int cc = 0; cc < ncol; cc++) {
        int c = backward ? ncol - 1 - cc : cc;
        for (int64_t i = 0; i < n; i++) {
            if (colour[i] != c)
                continue;
            double s = 0.0;
            for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; k++)
                s = fma(A->val[k], x[A->col[k]], s);
            x[i] = x[i] + dinv[i] * (b[i] - s);
        }
    }
}

/* one application of the smoother on level l: damped Jacobi sweeps, one Chebyshev
 * polynomial, or one multicolour Gauss-Seidel sweep, backward in post-smoothing so that
 * the V-cycle is a symmetric operator (the paper's smoothing step, Sec. 5.3: "a few
 * iterations" of Jacobi or Gauss-Seidel) */
static void smooth(orc_hier *H, const orc_opts *o, int l, const double *b, double *x, int post)
{
    const orc_csr *A = &H->A[l];
    int64_t n = A->nrows;
    double *r = H->r[l], *dinv = H->dinv[l], *t = H->t[l], *d = H->d[l];
    if (o->smoother == 2) {
        orc_gs_sweep(A, dinv, H->colour[l], orc_n_colours(H->dim, H->elem), post, b, x);
        return;
    }
    if (o->smoother == 0) {
        residual(A, b, x, r);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            t[i] = x[i] + o->omega * (dinv[i] * r[i]);
        memcpy(x, t, (size_t)n * sizeof(double));
        return;
    }
    /* Chebyshev acceleration of the Jacobi-preconditioned iteration on [lo, hi] */
    double hi = o->cheb_hi * H->lam[l];
    double lo = hi / o->cheb_ratio;
    double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
    double sigma = theta / delta;
    double rho0 = 1.0 / sigma;
    residual(A, b, x, r);
    double c0 = 1.0 / theta;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        d[i] = c0 * (dinv[i] * r[i]);
        x[i] = x[i] + d[i];
    }
    for (int j = 1; j < o->cheb_degree; j++) {
        residual(A, b, x, r);
        double rho1 = 1.0 / (2.0 * sigma - rho0);
        double c1 = rho1 * rho0, c2 = (2.0 * rho1) / delta;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            d[i] = c1 * d[i] + c2 * (dinv[i] * r[i]);
            x[i] = x[i] + d[i];
        }
        rho0 = rho1;
    }
}

/* V-cycle on level l for A_l x = b with x = 0 on entry */
static void vcycle(orc_hier *H, const orc_opts *o, int l, const double *b, double *x)
{
    if (l == 0) { /* exact solve on the coarsest level */
        orc_lu_solve(H->lu, H->n0, H->piv, b, x);
        return;
    }
    const orc_csr *A = &H->A[l];
    int64_t n = A->nrows;
    for (int s = 0; s < o->nu_pre; s++) /* pre-smoothing */
        smooth(H, o, l, b, x, 0);
    residual(A, b, x, H->r[l]);          /* restriction of the residual */
    double *bc = H->b[l - 1], *xc = H->x[l - 1];
    orc_spmv(&H->R[l], H->r[l], bc);
    memset(xc, 0, (size_t)H->A[l - 1].nrows * sizeof(double));
    vcycle(H, o, l - 1, bc, xc);         /* coarse-grid correction */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {    /* prolongation and correction */
        double t = 0.0;
        for (int64_t k = H->P[l].rowptr[i]; k < H->P[l].rowptr[i + 1]; k++)
            t = fma(H->P[l].val[k], xc[H->P[l].col[k]], t);
        x[i] = x[i] + t;
    }
    for (int s = 0; s < o->nu_post; s++) /* post-smoothing */
        smooth(H, o, l, b, x, 1);
}

/* one V-cycle applied to the defect: c = V(r), c starting from zero */
void orc_vcycle(orc_hier *H, const orc_opts *o, const double *r, double *c)
{
    int L = H->n_levels - 1;
    memset(c, 0, (size_t)H->A[L].nrows * sizeof(double));
    vcycle(H, o, L, r, c);
}

/*
 * Defect correction with V-cycles on the finest level:
 *   for k = 0, 1, ...: r_k = b - A x_k; hist[k] = ||r_k|| / ||b||;
 *                      stop if hist[k] <= tol; c = V(r_k); x_{k+1} = x_k + c.
 * Returns 0 on convergence (iters = k), 1 if max_iters cycles did not converge.
 * hist must hold max_iters + 1 entries.
 */
int orc_solve(orc_hier *H, const orc_opts *o, const double *b, double *x, double tol, double *hist, int *iters)
{
    int L = H->n_levels - 1;
    const orc_csr *A = &H->A[L];
    int64_t n = A->nrows;
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *c = (double *)malloc((size_t)n * sizeof(double));
    double nb = norm2_accurate(b, n);
    int status = 1;
    int k;
    for (k = 0;; k++) {
        residual(A, b, x, r);
        double nr = norm2_accurate(r, n);
        double h = nb > 0.0 ? nr / nb : nr;
        if (hist)
            hist[k] = h;
        if (h <= tol) {
            status = 0;
            break;
        }
        if (k == o->max_iters)
            break;
        orc_vcycle(H, o, r, c);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++)
            x[i] = x[i] + c[i];
    }
    *iters = k;
    free(r);
    free(c);
    return status;
}

/*
 * Right-hand side of one Crank-Nicolson step of the heat equation (Sec. 6, "Model
 * Problem": Galerkin FE in space, Crank-Nicolson in time). Multiplying the step
 *   (M + dt/2 A) u^{n+1} = (M - dt/2 A) u^n + dt/2 (b^{n+1} + b^n)
 * by sigma = 2/dt gives (A + sigma M) u^{n+1} = B u^n + (b^{n+1} + b^n) with
 * B = sigma M - A. For a separable source f(t, x) = g(t) F(x), b^n = g(t_n) b_F, so
 *   rhs_i = sum_j B_ij u_j + t * bF_i,   t = g(t_n) + g(t_{n+1}),
 * the row sum column-ascending by fused multiply-adds, then a rounded product and sum.
 */
void orc_heat_rhs(const orc_csr *B, const double *u, const double *bF, double t, double *rhs)
{
    for (int64_t i = 0; i < B->nrows; i++) {
        double s = 0.0;
        for (int64_t k = B->rowptr[i]; k < B->rowptr[i + 1]; k++)
            s = fma(B->val[k], u[B->col[k]], s);
        rhs[i] = s + t * bF[i];
    }
}

/* Euclidean inner product u.v: each product rounded, the sum by Neumaier's
 * compensated summation (as the residual norm) */
static double dot_accurate(const double *u, const double *v, int64_t n)
{
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double t = u[i] * v[i];
        double y = s + t;
        if (fabs(s) >= fabs(t))
            c += (s - y) + t;
        else
            c += (t - y) + s;
        s = y;
    }
    return s + c;
}

/*
 * Conjugate gradients preconditioned by one V-cycle (the paper's introduction, Sec. 1:
 * multigrid is often used as a preconditioner of a Krylov method such as CG or GMRES).
 * The preconditioned CG iteration (Saad, Iterative Methods for Sparse Linear Systems,
 * Alg. 9.1) with M^-1 r = V(r), the V-cycle applied to r from a zero start:
 *   r_0 = b - A x_0; hist[0] = ||r_0|| / ||b||
 *   for j = 0, 1, ...: stop if hist[j] <= tol;
 *     z_j = V(r_j); rz_j = (r_j, z_j)
 *     p_j = z_j (j = 0), p_j = z_j + (rz_j / rz_{j-1}) p_{j-1} (j > 0)
 *     q_j = A p_j; alpha_j = rz_j / (p_j, q_j)
 *     x_{j+1} = x_j + alpha_j p_j; r_{j+1} = r_j - alpha_j q_j
 *     hist[j+1] = ||r_{j+1}|| / ||b||   (the recursively updated residual)
 * The V-cycle is symmetric when nu_pre = nu_post (Gauss-Seidel: forward before the
 * correction, backward after). Returns 0 on convergence, 1 after max_iters iterations.
 */
int orc_pcg(orc_hier *H, const orc_opts *o, const double *b, double *x, double tol, double *hist, int *iters)
{
    int L = H->n_levels - 1;
    const orc_csr *A = &H->A[L];
    int64_t n = A->nrows;
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *z = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    double nb = norm2_accurate(b, n);
    residual(A, b, x, r);
    double rz_old = 0.0;
    int status = 1, j;
    for (j = 0;; j++) {
        double h = norm2_accurate(r, n);
        h = nb > 0.0 ? h / nb : h;
        if (hist)
            hist[j] = h;
        if (h <= tol) {
            status = 0;
            break;
        }
        if (j == o->max_iters)
            break;
        orc_vcycle(H, o, r, z);
        double rz = dot_accurate(r, z, n);
        if (j == 0) {
            memcpy(p, z, (size_t)n * sizeof(double));
        } else {
            double beta = rz / rz_old;
            for (int64_t i = 0; i < n; i++)
                p[i] = z[i] + beta * p[i];
        }
        orc_spmv(A, p, q);
        double alpha = rz / dot_accurate(p, q, n);
        for (int64_t i = 0; i < n; i++) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
        }
        rz_old = rz;
    }
    *iters = j;
    free(r);
    free(z);
    free(p);
    free(q);
    return status;
}

/* accessors for the test harness */
int orc_n_levels(const orc_hier *H) { return H->n_levels; }
int orc_level_N(const orc_hier *H, int l) { return H->N[l]; }
int orc_level_galerkin(const orc_hier *H, int l) { return H->galerkin[l]; }
double orc_level_lambda(const orc_hier *H, int l) { return H->lam[l]; }
const orc_csr *orc_level_A(const orc_hier *H, int l) { return &H->A[l]; }
const orc_csr *orc_level_P(const orc_hier *H, int l) { return &H->P[l]; }
const orc_csr *orc_level_R(const orc_hier *H, int l) { return &H->R[l]; }
