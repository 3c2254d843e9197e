// transfer.cuh -- grid transfers of the lattice elements (rotated Q1, P1, P2) from
// per-class offset tables (internal).
//
// The prolongation P of Sec. 5.1 (interpolation into the refined space) and the
// restriction R = P^T are translation invariant on a uniformly refined grid: the entries
// of a row depend only on where its DOF sits within a coarse cell, up to the entries that
// fall on the Dirichlet boundary. Each row is therefore generated from a small table, one
// list of (position offset, target family, weight) per row class, instead of being read
// from a stored matrix: the kernel reads x and writes y, and no column indices.
//
// DOF positions are integers in the level's DOF frame (rotated Q1: half cells, the face
// centres; P1: cells, the vertices; P2: half cells, vertices and edge midpoints). One unit
// of a coarse frame is two units of the fine frame. Family g of a level holds the DOFs
// X_d = o[g][d] + s t_d (0 <= t_d < n[g][d]), numbered base[g] + t_0 + n_0 (t_1 + n_1 t_2).
// A row's class is its family and its fine-frame position modulo 4 (the coarse cell's
// size in fine units is 2 or 4). The tables are learned on the host from the exact CSR
// operator and checked there against every row before a level uses them (entries in
// the same order, with the same weights), so the sums below equal the CSR sums term by
// term.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sweep.cuh"

namespace mgk {

constexpr int XF_CLASSES = 3 * 64;  // families x (position mod 4)^3

struct LatGeom {
    int ng = 0, s = 1;
    int o[3][3] = {};
    int n[3][3] = {};
    int64_t base[4] = {};
};

struct XferGeom {
    LatGeom row, col;
    int row_coarse = 0;  // 1: rows on the coarse level (R), columns on the fine level
};

__host__ __device__ __forceinline__ void lat_decode(const LatGeom &G, int64_t r, int &g, int X[3])
{
    g = 0;
    while (g + 1 < G.ng && r >= G.base[g + 1]) g++;
    int64_t t = r - G.base[g];
    int n0 = G.n[g][0], n1 = G.n[g][1];
    int64_t q = t / n0;
    X[0] = G.o[g][0] + G.s * (int)(t - q * n0);
    X[1] = G.o[g][1] + G.s * (int)(q % n1);
    X[2] = G.o[g][2] + G.s * (int)(q / n1);
}

// index of the DOF of family g at position Y, or -1 outside the family's lattice
__host__ __device__ __forceinline__ int64_t lat_encode(const LatGeom &G, int g, const int Y[3])
{
    int64_t idx = 0, mul = 1;
    for (int d = 0; d < 3; d++) {
        int u = Y[d] - G.o[g][d];
        if (u < 0 || (G.s == 2 && (u & 1))) return -1;
        int t = G.s == 2 ? u >> 1 : u;
        if (t >= G.n[g][d]) return -1;
        idx += (int64_t)t * mul;
        mul *= G.n[g][d];
    }
    return G.base[g] + idx;
}

// the row's fine-frame position and its class
__host__ __device__ __forceinline__ int xf_row(const XferGeom &S, int64_t r, int X[3])
{
    int g;
    lat_decode(S.row, r, g, X);
    if (S.row_coarse)
        for (int d = 0; d < 3; d++) X[d] *= 2;
    return g * 64 + (X[0] & 3) + 4 * (X[1] & 3) + 16 * (X[2] & 3);
}

// an entry packs the offset (three signed bytes, fine frame) and the target family
__host__ __device__ __forceinline__ int32_t xf_pack(int dx, int dy, int dz, int g)
{
    return (int32_t)((uint32_t)(dx & 0xff) | ((uint32_t)(dy & 0xff) << 8) | ((uint32_t)(dz & 0xff) << 16) |
                     ((uint32_t)g << 24));
}

// the column of entry p of a row at fine-frame position X, or -1 (a boundary DOF)
__host__ __device__ __forceinline__ int64_t xf_col(const XferGeom &S, const int X[3], int32_t p)
{
    int Y[3] = {X[0] + (int)(int8_t)(p & 0xff), X[1] + (int)(int8_t)((p >> 8) & 0xff),
                X[2] + (int)(int8_t)((p >> 16) & 0xff)};
    if (!S.row_coarse)  // columns on the coarse level: halve (even by construction)
        for (int d = 0; d < 3; d++) Y[d] = Y[d] >= 0 ? Y[d] >> 1 : -1;
    return lat_encode(S.col, (p >> 24) & 0xff, Y);
}

template <typename T>
struct XferView {
    XferGeom geo;
    const int32_t *cls;  // XF_CLASSES + 1 offsets into ent / w
    const int32_t *ent;
    const T *w;
};

// y_r = sum over the row's entries e (table order) of w_e x_col(e)  (ADD: y_r += that sum).
// Entries are processed eight at a time: their columns first, then the gathers, then the
// multiply-adds in order, so eight loads are in flight per thread.
template <typename T, bool ADD>
__global__ void __launch_bounds__(256) k_xfer_apply(XferView<T> S, int n, const T *__restrict__ x, T *__restrict__ y)
{
    pdl_enter();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int X[3];
    int key = xf_row(S.geo, r, X);
    int lo = __ldg(S.cls + key), hi = __ldg(S.cls + key + 1);
    T s = T(0);
    for (int e0 = lo; e0 < hi; e0 += 8) {
        int64_t c[8];
        T v[8], w[8];
#pragma unroll
        for (int j = 0; j < 8; j++) c[j] = e0 + j < hi ? xf_col(S.geo, X, __ldg(S.ent + e0 + j)) : -1;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            v[j] = c[j] >= 0 ? __ldg(x + c[j]) : T(0);
            w[j] = c[j] >= 0 ? __ldg(S.w + e0 + j) : T(0);
        }
#pragma unroll
        for (int j = 0; j < 8; j++)
            if (c[j] >= 0) s = Ar<T>::mac(s, w[j], v[j]);
    }
    y[r] = ADD ? Ar<T>::add(y[r], s) : s;
}

}  // namespace mgk
