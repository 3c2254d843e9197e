// host_setup.h -- host-side construction of the multigrid hierarchy (internal).
//
// Mesh numbering, element matrices, grid transfers, Galerkin products, the load vector
// and the power-method eigenvalue estimate, all in FP64 on the host. The results feed
// the device formats built in solver.cu.
#pragma once

#include <cstdint>
#include <utility>
#include <vector>

#include "mg.h"

namespace mgh {

struct Csr {
    int64_t nrows = 0, ncols = 0;
    std::vector<int64_t> rowptr;  // nrows + 1
    std::vector<int32_t> col;     // ascending within a row
    std::vector<double> val;
    int64_t nnz() const { return (int64_t)col.size(); }
};

int64_t ndofs(int dim, int elem, int N);

// Stiffness matrix of the level with N cells per axis; k: per-cell coefficient on that
// grid (lexicographic, x fastest) or nullptr for k = 1.
void assemble(int dim, int elem, int N, const double *k, Csr &A);

// Consistent mass matrix m_ij = sum_e int_e phi_i phi_j (element matrix h^d M_ref, added
// in increasing cell order; Q1, P1, P2); same pattern as the stiffness matrix.
void assemble_mass(int dim, int elem, int N, Csr &M);

// Prolongation from Nc to 2 Nc cells per axis (rows: fine DOFs, columns: coarse DOFs).
void prolongation(int dim, int elem, int Nc, Csr &P);

void transpose(const Csr &M, Csr &T);

// Ac = R A P with entries summed as (r_Ii a_ij) p_jJ, i, j, J ascending.
void galerkin(const Csr &R, const Csr &A, const Csr &P, Csr &Ac);

// Per-cell coefficient of the level with Nl cells if each of its cells covers fine
// cells of one value; false otherwise.
bool coarse_coefficient(int dim, int NL, const double *kL, int Nl, std::vector<double> &kl);

void load_vector(int dim, int elem, int N, const mg_rhs *f, double *b);

// The Q1 load vector of the same rule, factorised per mode and axis (O(modes * n));
// equal to load_vector up to rounding: b_i = sum_m c[m] * ((v[m][0][ix] * v[m][1][iy])
// [* v[m][2][iz]]) in mode order, each product and sum rounded once.
void load_vector_separable(int dim, int N, const mg_rhs *f, double *b);
// Its factors: v (modes x 3 x (N-1), axis-major per mode) and c (modes).
void load_vector_factors(int dim, int N, const mg_rhs *f, std::vector<double> &v, std::vector<double> &c);

double power_lambda(const Csr &A, const std::vector<double> &dinv, int iters, uint64_t seed);

// Row-sum-preserving FP32 copy: off-diagonals rounded to nearest, the diagonal set so
// that the FP32 row sum matches the FP64 one (the Dirichlet part of the row).
void round_fp32(const Csr &A, std::vector<float> &val32);

// The host hierarchy: levels 0 (coarsest) .. n_levels-1 (finest, N_finest cells per
// axis). Level l is rediscretised with the coefficient of its cells when every cell
// covers fine cells of one value, else (and on every coarser level) it is R A P of the
// next finer level. P[l], R[l] (l >= 1) map between levels l-1 and l. Levels below
// `stop` are not built. mass != 0: every rediscretised level holds A_l + mass * M_l
// (Q1), the operator of a scaled Crank-Nicolson step; Galerkin levels take R S P.
struct HostHierarchy {
    std::vector<int> N;
    std::vector<int> galerkin;
    std::vector<Csr> A, P, R;
};
void build_hierarchy(int dim, int elem, int N_finest, int n_levels, const double *k_finest, int stop,
                     HostHierarchy &H, double mass = 0.0);

// Multicolour Gauss-Seidel ordering. Q1: the parity class of the vertex coordinates,
// colour (vx&1) + 2(vy&1) [+ 4(vz&1)]; rotated Q1: face family f and parity of the normal
// position p, colour 2f + (p&1); P1: (vx + vy + vz) mod 4; P2: (wx + 2wy + 4wz) mod 15 on
// the grid of 2N cells. DOFs of one colour never share a cell (tetrahedron).
int n_colours(int dim, int elem);
int dof_colour(int dim, int elem, int N, int64_t i);
// DOFs sorted by colour (index order within a colour): perm[coff[c] .. coff[c+1]) are
// the DOFs of colour c.
void colour_order(int dim, int elem, int N, std::vector<int32_t> &perm, std::vector<int64_t> &coff);
// true iff no stored entry (zero or not) couples two distinct DOFs of one colour
bool colouring_valid(const Csr &A, int dim, int elem, int N);
// Launch groups of a sweep: consecutive colours 2g, 2g+1 share a launch when A holds no
// nonzero between them (then updating them together gives the sequential sweep's bits;
// 3D Q1 couples no face neighbours). Returns the row ranges [start, end) in colour order.
std::vector<std::pair<int64_t, int64_t>> colour_launch_groups(const Csr &A, int dim, int elem, int N,
                                                              const std::vector<int64_t> &coff);

// Power-method estimate of lambda_max(D^-1 A) (the start vector is 1 + 0.2 (u - 1/2),
// u from SplitMix64(seed), normalised).
double level_lambda(const Csr &A, int iters, uint64_t seed);

// Lexicographic coordinates of a Q1 vertex DOF (1-based grid indices).
inline void q1_coords(int dim, int N, int64_t i, int *v)
{
    int64_t n1 = N - 1;
    v[0] = (int)(i % n1) + 1;
    v[1] = (int)((i / n1) % n1) + 1;
    v[2] = dim == 3 ? (int)(i / (n1 * n1)) + 1 : 0;
}

}  // namespace mgh
