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
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }  // 1/a correctly rounded
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
__device__ __forceinline__ T sweep_out(int i, T s, T dinv, T xi, const T *__restrict__ b, T *__restrict__ out,
                                       T *__restrict__ d, T c1, T c2)
{
    using A = Ar<T>;
    T bi = b[i], o;
    if (MODE == SW_RESID) {
        o = A::sub(bi, s);
    } else if (MODE == SW_JACOBI) {
        T r = A::sub(bi, s);
        o = A::add(xi, A::mul(c1, A::mul(dinv, r)));
    } else if (MODE == SW_CHEBF) {
        T r = A::sub(bi, s);
        T dd = A::mul(c1, A::mul(dinv, r));
        d[i] = dd;
        o = A::add(xi, dd);
    } else if (MODE == SW_CHEB) {
        T r = A::sub(bi, s);
        T dd = A::add(A::mul(c1, d[i]), A::mul(c2, A::mul(dinv, r)));
        d[i] = dd;
        o = A::add(xi, dd);
    } else if (MODE == SW_JACOBI_Z) {
        o = A::mul(c1, A::mul(dinv, bi));
    } else {  // SW_CHEBF_Z
        T dd = A::mul(c1, A::mul(dinv, bi));
        d[i] = dd;
        o = dd;
    }
    out[i] = o;
    return o;
}

// The finest level's last post-smoothing sweep of a defect-correction iteration can also
// apply the correction to the FP64 iterate, x64_i <- x64_i + c_i (upd = x64; nullptr: no
// update): the operation of k_update, one launch and one pass over c fewer.
template <typename T, int MODE>
__device__ __forceinline__ void fused_update(double *__restrict__ upd, int i, T c)
{
    if (MODE != SW_RESID && upd) upd[i] = __dadd_rn(upd[i], (double)c);
}

// sweep_out with b_i and (SW_CHEB) d_i already loaded
template <typename T, int MODE>
__device__ __forceinline__ T sweep_out_v(int i, T s, T dinv, T xi, T bi, T di, T *__restrict__ out,
                                         T *__restrict__ d, T c1, T c2)
{
    using A = Ar<T>;
    T o;
    if (MODE == SW_RESID) {
        o = A::sub(bi, s);
    } else if (MODE == SW_JACOBI) {
        T r = A::sub(bi, s);
        o = A::add(xi, A::mul(c1, A::mul(dinv, r)));
    } else if (MODE == SW_CHEBF) {
        T r = A::sub(bi, s);
        T dd = A::mul(c1, A::mul(dinv, r));
        d[i] = dd;
        o = A::add(xi, dd);
    } else if (MODE == SW_CHEB) {
        T r = A::sub(bi, s);
        T dd = A::add(A::mul(c1, di), A::mul(c2, A::mul(dinv, r)));
        d[i] = dd;
        o = A::add(xi, dd);
    } else if (MODE == SW_JACOBI_Z) {
        o = A::mul(c1, A::mul(dinv, bi));
    } else {  // SW_CHEBF_Z
        T dd = A::mul(c1, A::mul(dinv, bi));
        d[i] = dd;
        o = dd;
    }
    out[i] = o;
    return o;
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

// k_stencil_fixed in 3D with each thread marching along z through up to `zc` points of
// its grid column: the x values of the 3 x 3 neighbouring columns on planes z - 1, z,
// z + 1 stay in registers and each step loads the new plane only for the columns the
// stencil uses (9 loads per point for 3D Q1 instead of 21, 5 for P1 instead of 7). The
// row sum is the same sequence of predicated multiply-adds as k_stencil_fixed (positions
// ascending, a neighbour off the grid skipped), so both give the same bits. Planes z = -1
// and z = n1 are read from the x halo; their terms are skipped like the others off the
// grid. Launch: grid (ceil(n1 / bx), ceil(n1 / by), ceil(n1 / zc)).
template <typename T, unsigned PM, int MODE>
__global__ void __launch_bounds__(256) k_stencil_march(StencilView<T> S, int zc, const T *__restrict__ x,
                                                       const T *__restrict__ b, T *__restrict__ out,
                                                       T *__restrict__ d, T c1, T c2, double *__restrict__ upd)
{
    pdl_enter();
    const int n1 = S.n1;
    const int vx = blockIdx.x * blockDim.x + threadIdx.x, vy = blockIdx.y * blockDim.y + threadIdx.y;
    if (vx >= n1 || vy >= n1) return;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, n1);
    const int64_t plane = (int64_t)n1 * n1;
    // columns c = (dx + 1) + 3 (dy + 1) the stencil reads on any plane
    constexpr unsigned COLS = ((PM | (PM >> 9) | (PM >> 18)) & 0x1FFu);
    const unsigned mx = 2u | (vx > 0 ? 1u : 0u) | (vx < n1 - 1 ? 4u : 0u);
    const unsigned my = 2u | (vy > 0 ? 1u : 0u) | (vy < n1 - 1 ? 4u : 0u);
    const unsigned mxy = ((my & 1u) ? mx : 0u) | ((my & 2u) ? mx << 3 : 0u) | ((my & 4u) ? mx << 6 : 0u);
    const T *xr = x + vx + (int64_t)n1 * vy + plane * (z0 - 1);  // column (vx, vy), plane z0 - 1
    T A[9], B[9], C[9];
    auto load_plane = [&](T P[9]) {
        const T *rm = xr - n1, *rp = xr + n1;
#pragma unroll
        for (int c = 0; c < 9; c++) {
            if (!((COLS >> c) & 1u)) continue;
            const int dx = c % 3 - 1, dy = c / 3 - 1;
            P[c] = __ldg((dy < 0 ? rm : (dy > 0 ? rp : xr)) + dx);
        }
        xr += plane;
    };
    auto point = [&](const T Pm[9], const T P0[9], const T Pp[9], int z) {
        const int i = vx + n1 * vy + (int)(plane * z);
        if (IsZero<MODE>::value) {
            sweep_out<T, MODE>(i, T(0), S.dinv, T(0), b, out, d, c1, c2);
            return;
        }
        const unsigned mz = 2u | (z > 0 ? 1u : 0u) | (z < n1 - 1 ? 4u : 0u);
        const unsigned m = ((mz & 1u) ? mxy : 0u) | ((mz & 2u) ? mxy << 9 : 0u) | ((mz & 4u) ? mxy << 18 : 0u);
        T s = T(0);
        int k = 0;
#pragma unroll
        for (int p = 0; p < 27; p++) {
            if (!((PM >> p) & 1u)) continue;
            const int c = p % 9, dz = p / 9;
            const T v = dz == 0 ? Pm[c] : (dz == 1 ? P0[c] : Pp[c]);
            if (p == 13 || ((m >> p) & 1u)) s = Ar<T>::mac(s, S.a[k], v);
            k++;
        }
        fused_update<T, MODE>(upd, i, sweep_out<T, MODE>(i, s, S.dinv, P0[4], b, out, d, c1, c2));
    };
    if (!IsZero<MODE>::value) {
        load_plane(A);  // z0 - 1
        load_plane(B);  // z0
    }
    int z = z0;
    for (; z + 3 <= z1; z += 3) {  // planes rotate A -> B -> C by renaming
        if (!IsZero<MODE>::value) load_plane(C);
        point(A, B, C, z);
        if (!IsZero<MODE>::value) load_plane(A);
        point(B, C, A, z + 1);
        if (!IsZero<MODE>::value) load_plane(B);
        point(C, A, B, z + 2);
    }
    if (z < z1) {
        if (!IsZero<MODE>::value) load_plane(C);
        point(A, B, C, z);
        z++;
        if (z < z1) {
            if (!IsZero<MODE>::value) load_plane(A);
            point(B, C, A, z);
        }
    }
}

// Per-cell coefficient (3D Q1, FP32): the level matrix of -div(k grad u) rediscretised
// with a coefficient k_e per cell is sum_e k_e h K_ref, and the unit-cube Q1 stiffness
// K_ref has 1/3 on the diagonal, 0 between edge-adjacent corners and -1/12 between the
// other corner pairs. With kap_e = k_e h / 12 row i is therefore
//     (A x)_i = sum over the 8 cells e around vertex i of kap_e (4 x_i - s_e),
// s_e the sum of x at the four corners of e that share no edge with i (three across a
// face, one across the body): the matrix is formed from one value per cell and never
// stored. s_e is summed in pairs, (x_f1 + x_f2) + (x_f3 + x_b), so that a constant x gives
// exactly 4 x_i - s_e = 0 (the interior row sums vanish in FP32 as they do in the
// assembled matrix); a_ii = 4 sum_e kap_e. Corners on the Dirichlet boundary hold 0.
// kap: (n1 + 1)^3 cells, x fastest.
//
// A thread owns the grid column (vx, vy) over `zc` consecutive planes and marches along
// z: the x values of the 3 x 3 neighbouring columns on planes z - 1, z, z + 1 and the kap
// values of the 2 x 2 neighbouring cell columns on cell planes z, z + 1 stay in
// registers, so each step loads only the new plane (9 x and 4 kap values, gathered
// through L1 where neighbouring threads share them) instead of all 29. The three planes
// rotate by renaming (the loop is unrolled three times), loads use one row pointer per
// dy with immediate dx offsets. Columns off the grid in x or y are selected to the
// Dirichlet value 0; planes z = -1 and z = n1 fall in the zero halo of the x buffer (x is
// padded by n1^2 + n1 + 1 zeros on both sides, written at setup and never again).
struct CoefView {
    const float *kap;
    int n1;  // interior points per axis (cells per axis - 1)
    int zc;  // planes per thread
};

#ifndef MG_COEF_MIN_BLOCKS
#define MG_COEF_MIN_BLOCKS 4  // 64 registers: four 256-thread blocks per SM (measured best of 1, 4, 6)
#endif
#ifndef MG_COEF_THREADS
#define MG_COEF_THREADS 4096  // threads per SM the split into plane chunks aims at
#endif
template <int MODE>
__global__ void __launch_bounds__(256, MG_COEF_MIN_BLOCKS) k_coef_sweep(CoefView S, const float *__restrict__ x,
                                                    const float *__restrict__ b, float *__restrict__ out,
                                                    float *__restrict__ d, float c1, float c2,
                                                    double *__restrict__ upd)
{
    constexpr bool Z = IsZero<MODE>::value;
    pdl_enter();
    const int n1 = S.n1, nc = n1 + 1;
    const int vx = blockIdx.x * blockDim.x + threadIdx.x, vy = blockIdx.y * blockDim.y + threadIdx.y;
    if (vx >= n1 || vy >= n1) return;
    const int z0 = blockIdx.z * S.zc, z1 = min(z0 + S.zc, n1);
    const int64_t plane = (int64_t)n1 * n1, cplane = (int64_t)nc * nc;
    // column c = (dx + 1) + 3 (dy + 1) of the point's 3 x 3 neighbourhood lies in the grid
    const bool xlo = vx > 0, xhi = vx < n1 - 1, ylo = vy > 0, yhi = vy < n1 - 1;
    bool cin[9];
#pragma unroll
    for (int c = 0; c < 9; c++) {
        const int dx = c % 3 - 1, dy = c / 3 - 1;
        cin[c] = (dx >= 0 || xlo) && (dx <= 0 || xhi) && (dy >= 0 || ylo) && (dy <= 0 || yhi);
    }
    const float *xr = x + vx + (int64_t)n1 * vy + plane * (z0 - 1);  // column (vx, vy), plane z0 - 1
    const float *kr = S.kap + vx + (int64_t)nc * vy + cplane * z0;   // cell column (vx, vy), plane z0
    auto load_plane = [&](float P[9]) {  // the 9 columns at plane xr, then advance xr
        const float *rm = xr - n1, *rp = xr + n1;
#pragma unroll
        for (int c = 0; c < 9; c++) {
            const int dx = c % 3 - 1, dy = c / 3 - 1;
            const float v = __ldg((dy < 0 ? rm : (dy > 0 ? rp : xr)) + dx);
            P[c] = cin[c] ? v : 0.0f;
        }
        xr += plane;
    };
    auto load_cells = [&](float K[4]) {  // the 2 x 2 cells at plane kr, then advance kr
        K[0] = __ldg(kr);
        K[1] = __ldg(kr + 1);
        K[2] = __ldg(kr + nc);
        K[3] = __ldg(kr + nc + 1);
        kr += cplane;
    };
    // b_i (and d_i for the later Chebyshev steps) of the point on plane z, loaded with the
    // plane so that all of a step's loads are in flight together
    auto load_bd = [&](int z, float &bi, float &di) {
        const int i = vx + n1 * vy + (int)(plane * z);
        bi = __ldg(b + i);
        di = MODE == SW_CHEB ? d[i] : 0.0f;
    };
    // one point: planes Pm, P0, Pp (z - 1, z, z + 1), cell planes Kc, Kn (z, z + 1)
    auto point = [&](const float Pm[9], const float P0[9], const float Pp[9], const float Kc[4], const float Kn[4],
                     int z, float bi, float di) {
        const int i = vx + n1 * vy + (int)(plane * z);
        // the 8 cells around the point: cell (vx + a, vy + b, z + c), e = a + 2 b + 4 c
        float kap[8];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            kap[e] = Kc[e];
            kap[e + 4] = Kn[e];
        }
        const float ksum = ((kap[0] + kap[1]) + (kap[2] + kap[3])) + ((kap[4] + kap[5]) + (kap[6] + kap[7]));
        const float dinv = Ar<float>::rcp(4.0f * ksum);
        if (Z) {
            sweep_out_v<float, MODE>(i, 0.0f, dinv, 0.0f, bi, di, out, d, c1, c2);
            return;
        }
        // x at stencil position p = (dx+1) + 3(dy+1) + 9(dz+1): column p % 9 of plane p / 9
        auto xv = [&](int p) { return p < 9 ? Pm[p] : (p < 18 ? P0[p - 9] : Pp[p - 18]); };
        const float xc = xv(13);
        float acc = 0.0f;
#pragma unroll
        for (int e = 0; e < 8; e++) {
            // cell e lies on the side (sx, sy, sz) of the point; its corners that share no
            // edge with the point sit at (sx, sy, 0), (sx, 0, sz), (0, sy, sz), (sx, sy, sz)
            const int sx = (e & 1) ? 1 : -1, sy = ((e >> 1) & 1) ? 1 : -1, sz = (e >> 2) ? 1 : -1;
            const float fxy = xv((sx + 1) + 3 * (sy + 1) + 9);
            const float fxz = xv((sx + 1) + 3 + 9 * (sz + 1));
            const float fyz = xv(1 + 3 * (sy + 1) + 9 * (sz + 1));
            const float fb = xv((sx + 1) + 3 * (sy + 1) + 9 * (sz + 1));
            const float se = (fxy + fxz) + (fyz + fb);
            acc = fmaf(kap[e], fmaf(4.0f, xc, -se), acc);
        }
        fused_update<float, MODE>(upd, i, sweep_out_v<float, MODE>(i, acc, dinv, xc, bi, di, out, d, c1, c2));
    };
    float A[9] = {}, B[9] = {}, C[9] = {}, KA[4], KB[4];
    if (!Z) {
        load_plane(A);  // z0 - 1
        load_plane(B);  // z0
    }
    load_cells(KA);  // cell plane z0
    int z = z0;
    float bi, di;
    // roles rotate A -> B -> C (planes) and KA -> KB (cell planes) from step to step
    for (; z + 3 <= z1; z += 3) {
        if (!Z) load_plane(C);
        load_cells(KB);
        load_bd(z, bi, di);
        point(A, B, C, KA, KB, z, bi, di);
        if (!Z) load_plane(A);
        load_cells(KA);
        load_bd(z + 1, bi, di);
        point(B, C, A, KB, KA, z + 1, bi, di);
        if (!Z) load_plane(B);
        load_cells(KB);
        load_bd(z + 2, bi, di);
        point(C, A, B, KA, KB, z + 2, bi, di);
        // after three steps the planes are back in their roles (A = z + 2, B = z + 3); the
        // cell planes are swapped (KA = z + 2, KB = z + 3)
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const float t = KA[e];
            KA[e] = KB[e];
            KB[e] = t;
        }
    }
    if (z < z1) {
        if (!Z) load_plane(C);
        load_cells(KB);
        load_bd(z, bi, di);
        point(A, B, C, KA, KB, z, bi, di);
        z++;
        if (z < z1) {
            if (!Z) load_plane(A);
            load_cells(KA);
            load_bd(z, bi, di);
            point(B, C, A, KB, KA, z, bi, di);
        }
    }
}

// The residual before restriction (SW_RESID) on a per-cell-coefficient level: a second
// march over the same column ownership and launch shape, which adds each pair of s_e once
// per column and carries it from plane to plane. For the cell on the side (sx, sy, sz) of
// the point, s_e = V + U with V = x(sx, sy) on the point's plane and on plane z + sz (lower
// plane first) and U = x(sx, 0) + x(0, sy) on plane z + sz: V between planes z and z + 1
// serves the upper cells of point z and the lower cells of point z + 1; U of plane p serves
// the upper cells of point p - 1 and the lower cells of point p + 1, so it is kept for two
// steps. Per point: 8 pair additions, 8 s_e additions and 16 fused multiply-adds, and the
// boundary selects are compiled only for the warps that touch the x or y boundary (a warp
// is 32 consecutive columns of one grid line, so the test is warp-uniform). Measured, this
// is the faster march for the residual (75 against 90 us at 256^3) and the slower one for
// the smoothing steps, whose d and D^-1 need the registers the carried pairs take. Each
// 4 x_i - s_e still vanishes exactly for a constant x; the row sums the same eight terms
// as k_coef_sweep in another pairing, so the two marches agree to FP32 rounding.

// quadrant q = a + 2 b of the 3 x 3 column neighbourhood, (sx, sy) = (a ? 1 : -1, b ? 1 : -1);
// column c = (dx + 1) + 3 (dy + 1)
__device__ __forceinline__ constexpr int coef_corner(int q) { return ((q & 1) ? 2 : 0) + ((q & 2) ? 6 : 0); }
__device__ __forceinline__ constexpr int coef_edge_x(int q) { return (q & 1) ? 5 : 3; }
__device__ __forceinline__ constexpr int coef_edge_y(int q) { return (q & 2) ? 7 : 1; }

template <int MODE, bool EDGE>
__device__ __forceinline__ void coef_march(const CoefView &S, int vx, int vy, const float *__restrict__ x,
                                           const float *__restrict__ b, float *__restrict__ out,
                                           float *__restrict__ d, float c1, float c2, double *__restrict__ upd)
{
    constexpr bool Z = IsZero<MODE>::value;
    const int n1 = S.n1, nc = n1 + 1, plane = n1 * n1;
    const int z0 = blockIdx.z * S.zc, z1 = min(z0 + S.zc, n1);
    const int64_t cplane = (int64_t)nc * nc;
    bool cin[9];
#pragma unroll
    for (int c = 0; c < 9; c++) {
        const int dx = c % 3 - 1, dy = c / 3 - 1;
        cin[c] = (dx >= 0 || vx > 0) && (dx <= 0 || vx < n1 - 1) && (dy >= 0 || vy > 0) && (dy <= 0 || vy < n1 - 1);
    }
    const float *xr = x + vx + (int64_t)n1 * vy + (int64_t)plane * (z0 - 1);  // column (vx, vy), plane z0 - 1
    const float *kr = S.kap + vx + (int64_t)nc * vy + cplane * z0;            // cell column (vx, vy), plane z0
    auto load_plane = [&](float P[9]) {  // the 9 columns at plane xr, then advance xr
        const float *rm = xr - n1, *rp = xr + n1;
#pragma unroll
        for (int c = 0; c < 9; c++) {
            const int dx = c % 3 - 1, dy = c / 3 - 1;
            const float v = __ldg((dy < 0 ? rm : (dy > 0 ? rp : xr)) + dx);
            P[c] = !EDGE || cin[c] ? v : 0.0f;
        }
        xr += plane;
    };
    auto load_cells = [&](float K[4]) {  // the 2 x 2 cells at plane kr, then advance kr
        K[0] = __ldg(kr);
        K[1] = __ldg(kr + 1);
        K[2] = __ldg(kr + nc);
        K[3] = __ldg(kr + nc + 1);
        kr += cplane;
    };
    // carried state at the start of step z: the centre and corners of plane z, U of planes
    // z - 1 (Um) and z (Uc), V between planes z - 1 and z (Vm), the cell plane z (the cells
    // below) and its sum
    float xc = 0.0f, Cc[4] = {}, Um[4] = {}, Uc[4] = {}, Vm[4] = {}, Kc[4];
    if (!Z) {
        float P[9];
        load_plane(P);  // z0 - 1
#pragma unroll
        for (int q = 0; q < 4; q++) {
            Um[q] = P[coef_edge_x(q)] + P[coef_edge_y(q)];
            Cc[q] = P[coef_corner(q)];
        }
        load_plane(P);  // z0
#pragma unroll
        for (int q = 0; q < 4; q++) {
            Vm[q] = Cc[q] + P[coef_corner(q)];
            Uc[q] = P[coef_edge_x(q)] + P[coef_edge_y(q)];
            Cc[q] = P[coef_corner(q)];
        }
        xc = P[4];
    }
    load_cells(Kc);
    float kc = (Kc[0] + Kc[1]) + (Kc[2] + Kc[3]);
    int i = vx + n1 * vy + plane * z0;
    for (int z = z0; z < z1; z++, i += plane) {
        float P[9], Kn[4];
        if (!Z) load_plane(P);  // z + 1
        load_cells(Kn);         // cell plane z + 1
        const float bi = __ldg(b + i), di = MODE == SW_CHEB ? d[i] : 0.0f;
        const float kn = (Kn[0] + Kn[1]) + (Kn[2] + Kn[3]);
        const float dinv = Ar<float>::rcp(4.0f * (kc + kn));
        if (Z) {
            sweep_out_v<float, MODE>(i, 0.0f, dinv, 0.0f, bi, di, out, d, c1, c2);
        } else {
            float Up[4], Vp[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                Up[q] = P[coef_edge_x(q)] + P[coef_edge_y(q)];
                Vp[q] = Cc[q] + P[coef_corner(q)];
            }
            // the cells in the order e = a + 2 b + 4 c: below (c = 0), then above
            float acc = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; q++) acc = fmaf(Kc[q], fmaf(4.0f, xc, -(Vm[q] + Um[q])), acc);
#pragma unroll
            for (int q = 0; q < 4; q++) acc = fmaf(Kn[q], fmaf(4.0f, xc, -(Vp[q] + Up[q])), acc);
            fused_update<float, MODE>(upd, i, sweep_out_v<float, MODE>(i, acc, dinv, xc, bi, di, out, d, c1, c2));
#pragma unroll
            for (int q = 0; q < 4; q++) {
                Um[q] = Uc[q];
                Uc[q] = Up[q];
                Vm[q] = Vp[q];
                Cc[q] = P[coef_corner(q)];
            }
            xc = P[4];
        }
#pragma unroll
        for (int q = 0; q < 4; q++) Kc[q] = Kn[q];
        kc = kn;
    }
}

template <int MODE>
__global__ void __launch_bounds__(256, MG_COEF_MIN_BLOCKS) k_coef_resid(CoefView S, const float *__restrict__ x,
                                                    const float *__restrict__ b, float *__restrict__ out,
                                                    float *__restrict__ d, float c1, float c2,
                                                    double *__restrict__ upd)
{
    pdl_enter();
    const int n1 = S.n1;
    const int vx = blockIdx.x * blockDim.x + threadIdx.x, vy = blockIdx.y * blockDim.y + threadIdx.y;
    if (vx >= n1 || vy >= n1) return;
    const int wx = vx - (threadIdx.x & 31);
    if (wx >= 1 && wx + 31 <= n1 - 2 && vy >= 1 && vy <= n1 - 2)
        coef_march<MODE, false>(S, vx, vy, x, b, out, d, c1, c2, upd);
    else
        coef_march<MODE, true>(S, vx, vy, x, b, out, d, c1, c2, upd);
}

// Constant stencil of the rotated-Q1 face space (FP32 levels of a mixed hierarchy with a
// constant coefficient). The element couples each face of a cell to itself by 3h, to the
// opposite face by h and to the four other faces by -h, so the row of an interior face
// (two cells) is 6h on the diagonal, +h at the two faces opposite it and -h at the eight
// other faces of its two cells; faces on the Dirichlet boundary are absent. With hv = h
//     (A x)_i = hv ((8 x_i - S_8) - (2 x_i - (x_o1 + x_o2))),
// S_8 the sum of the eight (pairwise, so that a constant x gives exactly 0 in FP32 as the
// interior row sums do). DOF numbering as in mg.h: faces normal to x (i, j, k), i the
// face position 1..N-1 along x and (j, k) the cell, index (i-1) + (N-1)(j + N k); normal
// to y: (N-1)N^2 + i + N((j-1) + (N-1) k); normal to z: 2(N-1)N^2 + i + N(j + N(k-1)).
// Launch: grid (ceil(N / bx), ceil(N / by), 3 ceil(N / cz)), blockIdx.z = family *
// ceil(N / cz) + slab group; a thread owns the faces at (fast, line, slab) of its family
// for cz consecutive slabs. Neighbours off the grid are not loaded (predicated), so no
// padding is needed.
struct Rq1View {
    int N;       // cells per axis
    float hv;    // the coupling to an opposite face (h times the coefficient)
    float dinv;  // 1 / (6 hv)
    int cz;      // slabs per thread
};

template <int MODE>
__global__ void __launch_bounds__(256) k_stencil_rq1(Rq1View S, const float *__restrict__ x,
                                                     const float *__restrict__ b, float *__restrict__ out,
                                                     float *__restrict__ d, float c1, float c2,
                                                     double *__restrict__ upd)
{
    pdl_enter();
    // 32-bit indices: setup keeps this storage for levels of fewer than 2^31 faces
    const int N = S.N, M = N - 1;
    const int nzb = (N + S.cz - 1) / S.cz;
    const int f = blockIdx.z / nzb, c0 = (blockIdx.z - f * nzb) * S.cz;
    const int p = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y * blockDim.y + threadIdx.y;
    if (p >= N || q >= N) return;
    const int NN = N * N, ny0 = M * NN, nz0 = 2 * M * NN;
    for (int c = c0; c < min(c0 + S.cz, N); c++) {
    // the face's own index, its two opposite faces (o1 below, o2 above along the normal)
    // and the eight other faces of its two cells, with their in-grid masks
    int i, step, t0;
    int e[8];
    bool me[8];
    if (f == 0) {  // normal to x: position p + 1 (p < N - 1), cell (j, k) = (q, c)
        if (p >= M) return;  // the same for every slab
        i = p + M * (q + N * c);
        step = 1;
        t0 = p;
        // the cells on either side: x-index p (below) and p + 1 (above)
#pragma unroll
        for (int s2 = 0; s2 < 2; s2++) {
            const int cx = p + s2;
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const int jy = q + t;  // y-face position j' in 1..N-1
                e[4 * s2 + t] = ny0 + cx + N * ((jy - 1) + M * c);
                me[4 * s2 + t] = jy >= 1 && jy <= M;
                const int kz = c + t;  // z-face position k' in 1..N-1
                e[4 * s2 + 2 + t] = nz0 + cx + N * (q + N * (kz - 1));
                me[4 * s2 + 2 + t] = kz >= 1 && kz <= M;
            }
        }
    } else if (f == 1) {  // normal to y: position q + 1 (q < N - 1), cell (i, k) = (p, c)
        if (q >= M) return;  // the same for every slab
        i = ny0 + p + N * (q + M * c);
        step = N;
        t0 = q;
#pragma unroll
        for (int s2 = 0; s2 < 2; s2++) {
            const int cy = q + s2;
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const int ix = p + t;  // x-face position i' in 1..N-1
                e[4 * s2 + t] = (ix - 1) + M * (cy + N * c);
                me[4 * s2 + t] = ix >= 1 && ix <= M;
                const int kz = c + t;
                e[4 * s2 + 2 + t] = nz0 + p + N * (cy + N * (kz - 1));
                me[4 * s2 + 2 + t] = kz >= 1 && kz <= M;
            }
        }
    } else {  // normal to z: position c + 1 (c < N - 1), cell (i, j) = (p, q)
        if (c >= M) return;  // and so for every later slab
        i = nz0 + p + N * (q + N * c);
        step = NN;
        t0 = c;
#pragma unroll
        for (int s2 = 0; s2 < 2; s2++) {
            const int cz = c + s2;
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const int ix = p + t;
                e[4 * s2 + t] = (ix - 1) + M * (q + N * cz);
                me[4 * s2 + t] = ix >= 1 && ix <= M;
                const int jy = q + t;
                e[4 * s2 + 2 + t] = ny0 + p + N * ((jy - 1) + M * cz);
                me[4 * s2 + 2 + t] = jy >= 1 && jy <= M;
            }
        }
    }
    if (IsZero<MODE>::value) {
        sweep_out<float, MODE>(i, 0.0f, S.dinv, 0.0f, b, out, d, c1, c2);
        continue;
    }
    const float xc = __ldg(x + i);
    const float xo1 = t0 >= 1 ? __ldg(x + i - step) : 0.0f, xo2 = t0 + 1 <= M - 1 ? __ldg(x + i + step) : 0.0f;
    float xe[8];
#pragma unroll
    for (int k = 0; k < 8; k++) xe[k] = me[k] ? __ldg(x + e[k]) : 0.0f;
    const float s8 = ((xe[0] + xe[1]) + (xe[2] + xe[3])) + ((xe[4] + xe[5]) + (xe[6] + xe[7]));
    const float s = (8.0f * xc - s8) - (2.0f * xc - (xo1 + xo2));
    fused_update<float, MODE>(upd, i, sweep_out<float, MODE>(i, S.hv * s, S.dinv, xc, b, out, d, c1, c2));
    }
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
