// gs.cuh -- multicolour Gauss-Seidel sweeps of the multigrid smoother (internal).
//
// The paper's Gauss-Seidel step (Eq. GS) with the DOFs numbered colour-wise (Sec. 4,
// "DOF Reordering"): DOFs of one colour share no cell, so they are not coupled and a
// colour is updated by one launch, one thread per DOF, in place:
//     x_i <- x_i + dinv_i * (b_i - sum_j a_ij x_j)
// with the row sum column-ascending by fused multiply-adds (the same arithmetic as the
// level sweeps). The matrix is read from a copy whose rows are stored colour by colour
// (row r is DOF perm[r]), so a launch streams a contiguous slice of it; the vectors keep
// the lexicographic DOF order of the transfers. The x gathers use plain loads: the
// launch writes x, but only at DOFs its rows are not coupled to.
#pragma once

#include "sweep.cuh"

namespace mgk {

template <typename T>
__device__ __forceinline__ void gs_update(int i, T s, T dinv, T xi, const T *__restrict__ b, T *x)
{
    x[i] = Ar<T>::add(xi, Ar<T>::mul(dinv, Ar<T>::sub(b[i], s)));
}

// DIA copy: slot k of row r holds a(perm[r], perm[r] + offs.o[k]); x is halo-padded.
template <typename T, int K>
__global__ void __launch_bounds__(256) k_gs_dia(MatView<T> G, const int32_t *__restrict__ perm, int64_t r0, int nr,
                                                T *x, const T *__restrict__ b)
{
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nr) return;
    int64_t r = r0 + t;
    int i = __ldcs(perm + r);
    constexpr int C = K / 2;
    T a[K], xv[K];
#pragma unroll
    for (int k = 0; k < K; k++) a[k] = __ldcs(G.val + (int64_t)k * G.ld + r);
#pragma unroll
    for (int k = 0; k < K; k++) xv[k] = x[i + G.offs.o[k]];
    T s = T(0);
#pragma unroll
    for (int k = 0; k < K; k++) s = Ar<T>::mac(s, a[k], xv[k]);
    T dinv = Ar<T>::kStoredDinv ? __ldcs(G.dinv + r) : Ar<T>::rcp(a[C]);
    gs_update<T>(i, s, dinv, xv[C], b, x);
}

// ELL copy: explicit columns; padded slots hold column perm[r] and value 0.
template <typename T>
__global__ void __launch_bounds__(256) k_gs_ell(MatView<T> G, const int32_t *__restrict__ perm, int64_t r0, int nr,
                                                T *x, const T *__restrict__ b)
{
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nr) return;
    int64_t r = r0 + t;
    int i = __ldcs(perm + r);
    T s = T(0), diag = T(0);
    for (int k = 0; k < G.K; k++) {
        int c = __ldcs(G.col + (int64_t)k * G.ld + r);
        T v = __ldcs(G.val + (int64_t)k * G.ld + r);
        if (c == i && diag == T(0)) diag = v;
        s = Ar<T>::mac(s, v, x[c]);
    }
    T dinv = Ar<T>::kStoredDinv ? __ldcs(G.dinv + r) : Ar<T>::rcp(diag);
    gs_update<T>(i, s, dinv, x[i], b, x);
}

// CSR copy: the rows of A in colour order.
template <typename T>
__global__ void __launch_bounds__(256) k_gs_csr(MatView<T> G, const int32_t *__restrict__ perm, int64_t r0, int nr,
                                                T *x, const T *__restrict__ b)
{
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nr) return;
    int64_t r = r0 + t;
    int i = __ldcs(perm + r);
    T s = T(0), diag = T(0);
    int64_t k0 = G.rowptr[r], k1 = G.rowptr[r + 1];
    for (int64_t k = k0; k < k1; k++) {
        int c = G.col[k];
        T v = G.val[k];
        if (c == i) diag = v;
        s = Ar<T>::mac(s, v, x[c]);
    }
    T dinv = Ar<T>::kStoredDinv ? G.dinv[r] : Ar<T>::rcp(diag);
    gs_update<T>(i, s, dinv, x[i], b, x);
}

// dst[k*ld + r] = src[k*ld + perm[r]] for r < n, k < K: the colour-major copy of a
// slot-major (DIA / ELL) array
template <typename V>
__global__ void k_gather_rows(V *__restrict__ dst, const V *__restrict__ src, const int32_t *__restrict__ perm,
                              int64_t n, int64_t ld, int K)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * K) return;
    int64_t k = t / n, r = t % n;
    dst[k * ld + r] = src[k * ld + perm[r]];
}

}  // namespace mgk
