// sweep.cuh -- the level-operator sweeps of the multigrid V-cycle (internal).
//
// One thread per row; the row's stored entries are summed in ascending column order
// (one rounded fused multiply-add each in FP64) and the smoother update is applied in
// the same pass. See kernels.cuh for the storage formats and the FP64 rounding rules.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mgk {

// Programmatic dependent launch: wait until the preceding kernel of the stream has
// finished and its writes are visible, then let the next kernel start its launch while
// this one runs. Both are no-ops for a kernel launched without the PDL attribute.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename T>
struct Ar;
template <>
struct Ar<double> {
    static constexpr bool kStoredDinv = true;
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mac(double s, double a, double b) { return __fma_rn(a, b, s); }
    static __device__ __forceinline__ double rcp(double a) { return __ddiv_rn(1.0, a); }
};
template <>
struct Ar<float> {
    static constexpr bool kStoredDinv = false;
    static __device__ __forceinline__ float mul(float a, float b) { return a * b; }
    static __device__ __forceinline__ float add(float a, float b) { return a + b; }
    static __device__ __forceinline__ float sub(float a, float b) { return a - b; }
    static __device__ __forceinline__ float mac(float s, float a, float b) { return fmaf(a, b, s); }
    static __device__ __forceinline__ float rcp(float a) { return __fdiv_rn(1.0f, a); }
};

// Sweep modes: what a pass does with s = (A x)_i and dinv = 1 / a_ii.
enum SweepMode {
    SW_RESID = 0,    // out = b - s
    SW_JACOBI = 1,   // out = x + c1*(dinv*(b - s))                 (c1 = omega)
    SW_CHEBF = 2,    // d = c1*(dinv*(b - s)); out = x + d           (first Chebyshev step)
    SW_CHEB = 3,     // d = c1*d + c2*(dinv*(b - s)); out = x + d    (later steps)
    SW_JACOBI_Z = 4, // x = 0: out = c1*(dinv*b)
    SW_CHEBF_Z = 5,  // x = 0: d = c1*(dinv*b); out = d
};

template <int MODE>
struct IsZero {
    static constexpr bool value = MODE == SW_JACOBI_Z || MODE == SW_CHEBF_Z;
};

struct DiaOffs {
    int32_t o[27];
};

// Matrix view for the kernels (values of type T).
template <typename T>
struct MatView {
    const T *val;          // DIA/ELL: K*ld (slot-major); CSR: nnz; SELL: padded slices
    const int32_t *col;    // ELL: K*ld; CSR: nnz; SELL: padded slices
    const int64_t *rowptr; // CSR: row starts; SELL: slice starts (entries)
    const int32_t *perm;   // SELL: DOF of storage position r
    const T *dinv;         // 1 / a_ii by DOF: FP64 levels; FP32 ELL/CSR/SELL levels (read
                           // only by sweeps from x = 0, which then skip the row scan)
    int64_t ld;
    int K;
    int center;            // DIA: slot of the diagonal
    DiaOffs offs;          // DIA: column = row + offs.o[k]
};

template <typename T, int MODE>
__device__ __forceinline__ void sweep_out(int i, T s, T dinv, T xi, const T *__restrict__ b, T *__restrict__ out,
                                          T *__restrict__ d, T c1, T c2)
{
    using A = Ar<T>;
    T bi = b[i];
    if (MODE == SW_RESID) {
        out[i] = A::sub(bi, s);
    } else if (MODE == SW_JACOBI) {
        T r = A::sub(bi, s);
        out[i] = A::add(xi, A::mul(c1, A::mul(dinv, r)));
    } else if (MODE == SW_CHEBF) {
        T r = A::sub(bi, s);
        T dd = A::mul(c1, A::mul(dinv, r));
        d[i] = dd;
        out[i] = A::add(xi, dd);
    } else if (MODE == SW_CHEB) {
        T r = A::sub(bi, s);
        T dd = A::add(A::mul(c1, d[i]), A::mul(c2, A::mul(dinv, r)));
        d[i] = dd;
        out[i] = A::add(xi, dd);
    } else if (MODE == SW_JACOBI_Z) {
        out[i] = A::mul(c1, A::mul(dinv, bi));
    } else {  // SW_CHEBF_Z
        T dd = A::mul(c1, A::mul(dinv, bi));
        d[i] = dd;
        out[i] = dd;
    }
}

// DIA: column of slot k is i + offs.o[k]. x points at element 0 of a buffer padded on
// both sides by at least max|offs|, so no bounds test is needed (slots of missing
// neighbours hold 0 and read a finite padded or interior value).
template <typename T, int K, int MODE>
__global__ void __launch_bounds__(256) k_dia_sweep(MatView<T> A, int n, const T *__restrict__ x,
                                                   const T *__restrict__ b, T *__restrict__ out,
                                                   T *__restrict__ d, T c1, T c2)
{
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    constexpr int C = K / 2;  // the stored diagonals are symmetric about the main one
    if (IsZero<MODE>::value) {
        T dinv = Ar<T>::kStoredDinv ? __ldcs(A.dinv + i) : Ar<T>::rcp(__ldcs(A.val + (int64_t)C * A.ld + i));
        sweep_out<T, MODE>(i, T(0), dinv, T(0), b, out, d, c1, c2);
        return;
    }
    T a[K], xv[K];
#pragma unroll
    for (int k = 0; k < K; k++) a[k] = __ldcs(A.val + (int64_t)k * A.ld + i);
#pragma unroll
    for (int k = 0; k < K; k++) xv[k] = __ldg(x + i + A.offs.o[k]);
    T s = T(0);
#pragma unroll
    for (int k = 0; k < K; k++) s = Ar<T>::mac(s, a[k], xv[k]);
    T dinv = Ar<T>::kStoredDinv ? __ldcs(A.dinv + i) : Ar<T>::rcp(a[C]);
    sweep_out<T, MODE>(i, s, dinv, xv[C], b, out, d, c1, c2);
}

// Constant stencil: every row holds the same value a[k] at stencil position pos[k]
// ((dx+1) + 3(dy+1) + 9(dz+1), ascending, so the slots are in ascending column order),
// minus the neighbours outside the grid, which the row does not hold. One thread per
// grid point (launch: x along the grid line, y and z the other two axes); the neighbour
// masks come from the point's coordinates, and x is padded like DIA, so every load is in
// bounds and only the multiply-adds are predicated. Blocks of up to 256 threads cover
// 256 / blockDim.x neighbouring grid lines.
template <typename T>
struct StencilView {
    T a[27];
    int32_t off[27];
    int32_t pos[27];
    T dinv;  // 1 / a_ii of the stencil
    int n1;  // interior points per axis
};

template <typename T, int K, int MODE, int DIM>
__global__ void __launch_bounds__(256) k_stencil_sweep(StencilView<T> S, const T *__restrict__ x,
                                                       const T *__restrict__ b, T *__restrict__ out,
                                                       T *__restrict__ d, T c1, T c2)
{
    pdl_enter();
    int vx = blockIdx.x * blockDim.x + threadIdx.x, vy = blockIdx.y * blockDim.y + threadIdx.y;
    int vz = DIM == 3 ? blockIdx.z : 0;
    if (vx >= S.n1 || vy >= S.n1) return;
    int i = vx + S.n1 * (vy + S.n1 * vz);
    if (IsZero<MODE>::value) {
        sweep_out<T, MODE>(i, T(0), S.dinv, T(0), b, out, d, c1, c2);
        return;
    }
    constexpr int C = K / 2;
    // bit p of m: the neighbour at stencil position p lies in the grid (per axis, bit j of
    // mx, my, mz: the neighbour at offset j - 1 exists)
    unsigned mx = 2u | (vx > 0 ? 1u : 0u) | (vx < S.n1 - 1 ? 4u : 0u);
    unsigned my = 2u | (vy > 0 ? 1u : 0u) | (vy < S.n1 - 1 ? 4u : 0u);
    unsigned m = ((my & 1u) ? mx : 0u) | ((my & 2u) ? mx << 3 : 0u) | ((my & 4u) ? mx << 6 : 0u);
    if (DIM == 3) {
        unsigned mz = 2u | (vz > 0 ? 1u : 0u) | (vz < S.n1 - 1 ? 4u : 0u);
        m = ((mz & 1u) ? m : 0u) | ((mz & 2u) ? m << 9 : 0u) | ((mz & 4u) ? m << 18 : 0u);
    }
    T xv[K];
#pragma unroll
    for (int k = 0; k < K; k++) xv[k] = __ldg(x + i + S.off[k]);
    T s = T(0);
#pragma unroll
    for (int k = 0; k < K; k++)
        if ((m >> S.pos[k]) & 1u) s = Ar<T>::mac(s, S.a[k], xv[k]);
    sweep_out<T, MODE>(i, s, S.dinv, xv[C], b, out, d, c1, c2);
}

// The same sweep with the stencil's positions fixed at compile time (PM: bit p set for
// each stored position, ascending p = slot order): the offsets of a grid line become
// immediates on one row pointer per (dy, dz), and each slot's mask test a constant bit.
template <typename T, unsigned PM, int MODE, int DIM>
__global__ void __launch_bounds__(256) k_stencil_fixed(StencilView<T> S, const T *__restrict__ x,
                                                       const T *__restrict__ b, T *__restrict__ out,
                                                       T *__restrict__ d, T c1, T c2)
{
    pdl_enter();
    int vx = blockIdx.x * blockDim.x + threadIdx.x, vy = blockIdx.y * blockDim.y + threadIdx.y;
    int vz = DIM == 3 ? blockIdx.z : 0;
    if (vx >= S.n1 || vy >= S.n1) return;
    const int n1 = S.n1;
    int i = vx + n1 * (vy + n1 * vz);
    if (IsZero<MODE>::value) {
        sweep_out<T, MODE>(i, T(0), S.dinv, T(0), b, out, d, c1, c2);
        return;
    }
    unsigned mx = 2u | (vx > 0 ? 1u : 0u) | (vx < n1 - 1 ? 4u : 0u);
    unsigned my = 2u | (vy > 0 ? 1u : 0u) | (vy < n1 - 1 ? 4u : 0u);
    unsigned m = ((my & 1u) ? mx : 0u) | ((my & 2u) ? mx << 3 : 0u) | ((my & 4u) ? mx << 6 : 0u);
    if (DIM == 3) {
        unsigned mz = 2u | (vz > 0 ? 1u : 0u) | (vz < n1 - 1 ? 4u : 0u);
        m = ((mz & 1u) ? m : 0u) | ((mz & 2u) ? m << 9 : 0u) | ((mz & 4u) ? m << 18 : 0u);
    }
    constexpr int CP = DIM == 3 ? 13 : 4;  // the centre position
    const T *xi = x + i;
    T s = T(0), xc = T(0);
    int k = 0;
#pragma unroll
    for (int p = 0; p < (DIM == 3 ? 27 : 9); p++) {
        if (!((PM >> p) & 1u)) continue;
        const int dx = p % 3 - 1, dy = (p / 3) % 3 - 1, dz = DIM == 3 ? p / 9 - 1 : 0;
        T v = __ldg(xi + (dy * n1 + dz * n1 * n1) + dx);
        if (p == CP) xc = v;
        if (p == CP || ((m >> p) & 1u)) s = Ar<T>::mac(s, S.a[k], v);
        k++;
    }
    sweep_out<T, MODE>(i, s, S.dinv, xc, b, out, d, c1, c2);
}

// ELL with explicit columns; padded slots hold column i and value 0.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_ell_sweep(MatView<T> A, int n, const T *__restrict__ x,
                                                   const T *__restrict__ b, T *__restrict__ out,
                                                   T *__restrict__ d, T c1, T c2)
{
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T s = T(0), diag = T(0);
    const bool zd = IsZero<MODE>::value && (Ar<T>::kStoredDinv || A.dinv != nullptr);
    if (!zd) {
        for (int k = 0; k < A.K; k++) {
            int c = __ldcs(A.col + (int64_t)k * A.ld + i);
            T v = __ldcs(A.val + (int64_t)k * A.ld + i);
            if (c == i && diag == T(0)) diag = v;
            if (!IsZero<MODE>::value) s = Ar<T>::mac(s, v, __ldg(x + c));
        }
    }
    T dinv = Ar<T>::kStoredDinv || zd ? __ldcs(A.dinv + i) : Ar<T>::rcp(diag);
    sweep_out<T, MODE>(i, s, dinv, IsZero<MODE>::value ? T(0) : x[i], b, out, d, c1, c2);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_csr_sweep(MatView<T> A, int n, const T *__restrict__ x,
                                                   const T *__restrict__ b, T *__restrict__ out,
                                                   T *__restrict__ d, T c1, T c2)
{
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T s = T(0), diag = T(0);
    const bool zd = IsZero<MODE>::value && (Ar<T>::kStoredDinv || A.dinv != nullptr);
    if (!zd) {
        int64_t k0 = A.rowptr[i], k1 = A.rowptr[i + 1];
        for (int64_t k = k0; k < k1; k++) {
            int c = A.col[k];
            T v = A.val[k];
            if (c == i) diag = v;
            if (!IsZero<MODE>::value) s = Ar<T>::mac(s, v, __ldg(x + c));
        }
    }
    T dinv = Ar<T>::kStoredDinv || zd ? A.dinv[i] : Ar<T>::rcp(diag);
    sweep_out<T, MODE>(i, s, dinv, IsZero<MODE>::value ? T(0) : x[i], b, out, d, c1, c2);
}

// SELL-32: storage position r (rows sorted by length, slices of 32 rows) holds DOF
// perm[r]; slice s stores its rows column-major with K_s slots, K_s = its longest row,
// so slot k of position r is entry rowptr[s] + 32 k + (r mod 32). Each row keeps its CSR
// order (columns ascending); padded slots hold column perm[r] and value 0.
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_sell_sweep(MatView<T> A, int n, const T *__restrict__ x,
                                                    const T *__restrict__ b, T *__restrict__ out,
                                                    T *__restrict__ d, T c1, T c2)
{
    pdl_enter();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int i = __ldg(A.perm + r);
    T s = T(0), diag = T(0);
    const bool zd = IsZero<MODE>::value && (Ar<T>::kStoredDinv || A.dinv != nullptr);
    if (!zd) {
        int64_t base = A.rowptr[r >> 5];
        int Ks = (int)((A.rowptr[(r >> 5) + 1] - base) >> 5);
        int64_t e = base + (r & 31);
        for (int k = 0; k < Ks; k++, e += 32) {
            int c = __ldcs(A.col + e);
            T v = __ldcs(A.val + e);
            if (c == i && diag == T(0)) diag = v;
            if (!IsZero<MODE>::value) s = Ar<T>::mac(s, v, __ldg(x + c));
        }
    }
    T dinv = Ar<T>::kStoredDinv || zd ? __ldcs(A.dinv + i) : Ar<T>::rcp(diag);
    sweep_out<T, MODE>(i, s, dinv, IsZero<MODE>::value ? T(0) : x[i], b, out, d, c1, c2);
}

}  // namespace mgk
