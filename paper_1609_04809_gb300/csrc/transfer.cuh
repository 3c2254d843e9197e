// transfer.cuh -- grid transfers of the lattice elements (rotated Q1, P1, P2) from
// per-class offset tables (internal).
//
// The prolongation P of Sec. 5.1 (interpolation into the refined space) and the
// restriction R = P^T are translation invariant on a uniformly refined grid: the entries
// of a row depend only on where its DOF sits within a coarse cell, up to the entries that
// fall on the Dirichlet boundary. Away from the boundary each row is therefore generated
// from a small table, one list of (target family, offset, weight) per row class, instead
// of being read from a stored matrix; the rows near the boundary stay explicit (SELL-32).
//
// DOF positions are integers in the level's DOF frame (rotated Q1: half cells, the face
// centres; P1: cells, the vertices; P2: half cells, vertices and edge midpoints). One unit
// of a coarse frame is two units of the fine frame. Family g of a level holds the DOFs
// X_d = o[g][d] + s t_d (0 <= t_d < n[g][d]), numbered base[g] + t_0 + n_0 (t_1 + n_1 t_2).
// A row's class is its family and its fine-frame position modulo 4 (the coarse cell's
// size in fine units is 2 or 4).
//
// Column arithmetic. A row at fine-frame position X and an entry with fine-frame offset D
// on target family h reach the target lattice point t'_d = (X_d + D_d - c o'_d) / q with
// c = 2 for P (coarse columns), 1 for R, and q = c s' (1, 2 or 4). Writing
// X_d - c o'_d = q a_d + r_d (0 <= r_d < q), r_d is fixed by the class, so
// t'_d = a_d + delta_d with delta_d = (D_d + r_d) / q a constant of the entry, and the
// column is anchor(h) + Delta with anchor(h) = base'(h) + a_0 + n'_0 (a_1 + n'_1 a_2) per
// row and Delta = delta_0 + n'_0 (delta_1 + n'_1 delta_2) per entry.
//
// The interior box of a family is the set of rows whose every entry lands inside its
// target lattice; its rows take the table with no range test. The tables are learned on
// the host from the exact CSR operator and every box row is checked there with the
// functions below, the kernel's own arithmetic, against the stored row (entries in the
// same order, with the same weights), so the kernel's sums equal the CSR sums term by
// term.
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
    int ng = 0, s = 1;           // row lattice: families, spacing
    int o[3][3] = {}, n[3][3] = {};
    int base[3] = {};
    int rm = 1;                  // row frame -> fine frame factor (2: rows on the coarse level)
    int c = 1, qs = 0;           // fine frame -> column frame factor (2: coarse columns); log2 q
    int cng = 0;                 // column lattice
    int co[3][3] = {}, cn[3][3] = {};
    int cbase[3] = {};
    int bo[3][3] = {}, bn[3][3] = {};  // interior box of each family: first t_d, extent
    int bz[4] = {};              // launch z of each family's first box plane; bz[ng] = total
    int bmax01 = 0;              // largest number of t_0 pairs in a box plane
};

// the row at lattice point t of family g: index, class, fine-frame position and the
// anchors of the target families
__host__ __device__ __forceinline__ int xf_row(const XferDev &G, int g, int t0, int t1, int t2, int &key,
                                               int anchor[3])
{
    int t[3] = {t0, t1, t2}, X[3];
    for (int d = 0; d < 3; d++) X[d] = (G.o[g][d] + G.s * t[d]) * G.rm;
    key = g * 64 + (X[0] & 3) + 4 * (X[1] & 3) + 16 * (X[2] & 3);
    for (int h = 0; h < 3; h++) {
        int a[3];
        for (int d = 0; d < 3; d++) a[d] = (X[d] - G.c * G.co[h][d]) >> G.qs;  // floor division by q
        anchor[h] = h < G.cng ? G.cbase[h] + a[0] + G.cn[h][0] * (a[1] + G.cn[h][1] * a[2]) : 0;
    }
    return G.base[g] + t0 + G.n[g][0] * (t1 + G.n[g][1] * t2);
}

// an entry: target family (top byte) and Delta (24-bit signed)
__host__ __device__ __forceinline__ int32_t xf_pack(int h, int delta)
{
    return (int32_t)(((uint32_t)h << 24) | ((uint32_t)delta & 0xffffffu));
}

__host__ __device__ __forceinline__ int xf_col(const int anchor[3], int32_t p)
{
    int h = (p >> 24) & 0xff;
    int delta = (int)((uint32_t)p << 8) >> 8;  // sign-extend the low 24 bits
    return (h == 0 ? anchor[0] : (h == 1 ? anchor[1] : anchor[2])) + delta;
}

// one table entry as the kernel reads it: packed target and offset, weight (16 bytes)
template <typename T>
struct alignas(16) XferEnt {
    int32_t p, pad;
    T w;
};

// s += the entries [lo, hi) of a row with the given anchors, in table order; four at a
// time (columns, then the gathers, then the multiply-adds), the rest one by one
template <typename T>
__device__ __forceinline__ T xf_row_sum(const XferEnt<T> *__restrict__ ent, int lo, int hi, const int anchor[3],
                                        const T *__restrict__ x)
{
    T s = T(0);
    int e = lo;
    for (; e + 4 <= hi; e += 4) {
        XferEnt<T> q[4];
        T v[4];
#pragma unroll
        for (int j = 0; j < 4; j++) q[j] = ent[e + j];
#pragma unroll
        for (int j = 0; j < 4; j++) v[j] = __ldg(x + xf_col(anchor, q[j].p));
#pragma unroll
        for (int j = 0; j < 4; j++) s = Ar<T>::mac(s, q[j].w, v[j]);
    }
    for (; e < hi; e++) {
        XferEnt<T> q = ent[e];
        s = Ar<T>::mac(s, q.w, __ldg(x + xf_col(anchor, q.p)));
    }
    return s;
}

// y_r = sum over the row's entries e (table order) of w_e x_col(e)  (ADD: y_r += that sum),
// for the rows of the interior boxes. Each thread takes two neighbouring points along
// t_0 (t_0 = bo_0 + 2k, 2k + 1), so that a warp's first rows, and its second rows, share
// one class wherever the class changes with the parity of t_0. Launch: z over the
// families' box planes (G.bz), x over the pairs of a plane.
template <typename T, bool ADD>
__global__ void __launch_bounds__(256) k_xfer_apply(XferDev G, const int32_t *__restrict__ cls,
                                                    const XferEnt<T> *__restrict__ ent, const T *__restrict__ x,
                                                    T *__restrict__ y)
{
    pdl_enter();
    int z = blockIdx.z;
    int g = (G.ng > 1 && z >= G.bz[1]) + (G.ng > 2 && z >= G.bz[2]);
    int w0 = G.bn[g][0], np = (w0 + 1) >> 1, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np * G.bn[g][1]) return;
    int t1 = i / np, k = i - t1 * np;
    int t2 = z - G.bz[g] + G.bo[g][2];
    t1 += G.bo[g][1];
    int t0 = G.bo[g][0] + 2 * k;
    int key, anchor[3];
    int r = xf_row(G, g, t0, t1, t2, key, anchor);
    T s = xf_row_sum(ent, __ldg(cls + key), __ldg(cls + key + 1), anchor, x);
    y[r] = ADD ? Ar<T>::add(y[r], s) : s;
    if (2 * k + 1 < w0) {
        r = xf_row(G, g, t0 + 1, t1, t2, key, anchor);
        s = xf_row_sum(ent, __ldg(cls + key), __ldg(cls + key + 1), anchor, x);
        y[r] = ADD ? Ar<T>::add(y[r], s) : s;
    }
}

}  // namespace mgk
