// transfer.cuh -- grid transfers of the lattice elements (rotated Q1, P1, P2) from
// per-class offset tables (internal).
//
// The prolongation P of Sec. 5.1 (interpolation into the refined space) and the
// restriction R = P^T are translation invariant on a uniformly refined grid: the entries
// of a row depend only on where its DOF sits within a coarse cell, up to the entries that
// fall on the Dirichlet boundary. Each row is therefore generated from a small table, one
// list of (offset, target family, weight) per row class, instead of being read from a
// stored matrix: the kernel reads x and writes y, and no column indices.
//
// DOF positions are integers in the level's DOF frame (rotated Q1: half cells, the face
// centres; P1: cells, the vertices; P2: half cells, vertices and edge midpoints). One unit
// of a coarse frame is two units of the fine frame. Family g of a level holds the DOFs
// X_d = o[g][d] + s t_d (0 <= t_d < n[g][d]), numbered base[g] + t_0 + n_0 (t_1 + n_1 t_2).
// A row's class is its family and its fine-frame position modulo 4 (the coarse cell's
// size in fine units is 2 or 4).
//
// Column arithmetic. A row at fine-frame position X and an entry with fine-frame offset D
// on target family g' reach the target lattice point t'_d = (X_d + D_d - c o'_d) / q with
// c = 2 for P (coarse columns), 1 for R, and q = c s' (1, 2 or 4). Writing
// X_d - c o'_d = q a_d + r_d (0 <= r_d < q), r_d is fixed by the class, so
// t'_d = a_d + delta_d with delta_d = (D_d + r_d) / q a constant of the entry, and the
// column is anchor(g') + Delta with anchor(g') = base'(g') + a_0 + n'_0 (a_1 + n'_1 a_2)
// per row and Delta = delta_0 + n'_0 (delta_1 + n'_1 delta_2) per entry. Rows whose
// anchors lie far enough inside every target lattice skip the range test.
//
// The tables are learned on the host from the exact CSR operator and checked there
// against every row with the functions below, the kernel's own column arithmetic
// (entries in the same order, with the same weights), so the kernel's sums equal the
// CSR sums term by term.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sweep.cuh"

namespace mgk {

constexpr int XF_CLASSES = 3 * 64;  // families x (position mod 4)^3

// the lattice of one level's DOFs (host-side description)
struct LatGeom {
    int ng = 0, s = 1;
    int o[3][3] = {};
    int n[3][3] = {};
    int64_t base[4] = {};
};

// everything the kernel needs about the row and column lattices of one transfer
struct XferDev {
    int ng = 0, s = 1;          // row lattice: families, spacing
    int o[3][3] = {}, n[3][3] = {};
    int base[3] = {};
    int zb[3] = {};             // launch z of each family's first t_2 plane
    int rm = 1;                 // row frame -> fine frame factor (2: rows on the coarse level)
    int c = 1, qs = 0;          // fine frame -> column frame factor (2: coarse columns); log2 q
    int cng = 0;                // column lattice
    int co[3][3] = {}, cn[3][3] = {};
    int cbase[3] = {};
    int lo[3] = {}, hi[3] = {}; // per target family: min and max delta_d over the entries
};

// one row: its index, class and the anchors of the target families
struct XferRow {
    int r, key;
    int a[3][3];
    int anchor[3];
    bool inside;  // every entry's target lies in its lattice: no range test needed
};

__host__ __device__ __forceinline__ void xf_row_setup(const XferDev &G, int g, int t0, int t1, int t2, XferRow &R)
{
    R.r = G.base[g] + t0 + G.n[g][0] * (t1 + G.n[g][1] * t2);
    int t[3] = {t0, t1, t2}, X[3];
    for (int d = 0; d < 3; d++) X[d] = (G.o[g][d] + G.s * t[d]) * G.rm;
    R.key = g * 64 + (X[0] & 3) + 4 * (X[1] & 3) + 16 * (X[2] & 3);
    R.inside = true;
    for (int h = 0; h < 3; h++) {
        if (h >= G.cng) {
            R.anchor[h] = 0;
            for (int d = 0; d < 3; d++) R.a[h][d] = 0;
            continue;
        }
        for (int d = 0; d < 3; d++) {
            R.a[h][d] = (X[d] - G.c * G.co[h][d]) >> G.qs;  // floor division by q
            if (R.a[h][d] + G.lo[h] < 0 || R.a[h][d] + G.hi[h] >= G.cn[h][d]) R.inside = false;
        }
        R.anchor[h] = G.cbase[h] + R.a[h][0] + G.cn[h][0] * (R.a[h][1] + G.cn[h][1] * R.a[h][2]);
    }
}

// entry packing: delta_d as three signed bytes and the target family
__host__ __device__ __forceinline__ int32_t xf_pack(int d0, int d1, int d2, int g)
{
    return (int32_t)((uint32_t)(d0 & 0xff) | ((uint32_t)(d1 & 0xff) << 8) | ((uint32_t)(d2 & 0xff) << 16) |
                     ((uint32_t)g << 24));
}

__host__ __device__ __forceinline__ int xf_sel(const int *v, int h) { return h == 0 ? v[0] : (h == 1 ? v[1] : v[2]); }

// column of an entry (packed p, linear offset D) for row R, or -1 (a boundary DOF)
__host__ __device__ __forceinline__ int xf_entry_col(const XferDev &G, const XferRow &R, int32_t p, int32_t D)
{
    int h = (p >> 24) & 0xff;
    int col = xf_sel(R.anchor, h) + D;
    if (R.inside) return col;
    int dl[3] = {(int)(int8_t)(p & 0xff), (int)(int8_t)((p >> 8) & 0xff), (int)(int8_t)((p >> 16) & 0xff)};
    for (int d = 0; d < 3; d++) {
        int av = h == 0 ? R.a[0][d] : (h == 1 ? R.a[1][d] : R.a[2][d]);
        int cn = h == 0 ? G.cn[0][d] : (h == 1 ? G.cn[1][d] : G.cn[2][d]);
        int tt = av + dl[d];
        if (tt < 0 || tt >= cn) return -1;
    }
    return col;
}

// y_r = sum over the row's entries e (table order) of w_e x_col(e)  (ADD: y_r += that sum).
// Launch: x over t_0, y over t_1, z over the families' t_2 planes (G.zb). Entries are
// processed eight at a time: columns first, then the gathers, then the multiply-adds in
// order, so eight loads are in flight per thread.
template <typename T, bool ADD>
__global__ void __launch_bounds__(256) k_xfer_apply(XferDev G, const int32_t *__restrict__ cls,
                                                    const int32_t *__restrict__ ent, const int32_t *__restrict__ dlt,
                                                    const T *__restrict__ wt, const T *__restrict__ x,
                                                    T *__restrict__ y)
{
    pdl_enter();
    int z = blockIdx.z;
    int g = (G.ng > 1 && z >= G.zb[1]) + (G.ng > 2 && z >= G.zb[2]);
    int t0 = blockIdx.x * blockDim.x + threadIdx.x, t1 = blockIdx.y * blockDim.y + threadIdx.y, t2 = z - G.zb[g];
    if (t0 >= G.n[g][0] || t1 >= G.n[g][1]) return;
    XferRow R;
    xf_row_setup(G, g, t0, t1, t2, R);
    int lo = __ldg(cls + R.key), hi = __ldg(cls + R.key + 1);
    T s = T(0);
    for (int e0 = lo; e0 < hi; e0 += 8) {
        int c[8];
#pragma unroll
        for (int j = 0; j < 8; j++) c[j] = e0 + j < hi ? xf_entry_col(G, R, __ldg(ent + e0 + j), __ldg(dlt + e0 + j)) : -1;
        T v[8];
#pragma unroll
        for (int j = 0; j < 8; j++) v[j] = c[j] >= 0 ? __ldg(x + c[j]) : T(0);
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (c[j] >= 0) s = Ar<T>::mac(s, __ldg(wt + e0 + j), v[j]);
    }
    y[R.r] = ADD ? Ar<T>::add(y[R.r], s) : s;
}

}  // namespace mgk
