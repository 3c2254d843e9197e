// kernels.cuh -- sm_103a device kernels of the multigrid V-cycle (internal).
//
// Every level operator is a sparse pass of about one multiply-add per 8 bytes, so the
// kernels are built for streaming, not tensor cores:
//   * matrices are stored column-major by slot (ELLPACK order, leading dimension ld),
//     so the 32 rows of a warp read one contiguous 128/256-byte segment per slot;
//   * DIA keeps only the diagonals that hold a nonzero (21 of the 27 for the 3D Q1
//     stiffness, whose face-neighbour couplings vanish) and needs no column indices;
//   * matrix values are read with the streaming cache hint (ld.global.cs): each value
//     is used once per pass and must not evict the gathered vector from L2;
//   * x is gathered through the read-only path and stays L2-resident across slots;
//   * one thread per row, sum over the row's slots in ascending column order.
//
// GB300 issues FP64 at a small fraction of its FP32 rate, so FP64 passes are bounded by
// the FP64 pipe before HBM: they use one fused multiply-add per stored entry and read a
// precomputed D^-1 instead of dividing. Every FP64 operation is an explicitly rounded
// intrinsic (__fma_rn, __dmul_rn, __dadd_rn) evaluated in the same order as the
// sequential definition, so FP64 results are bit-for-bit those of a CPU evaluation of
// the same formula. The FP32 inner V-cycle of the mixed-precision solve is HBM-bound
// and computes D^-1 on the fly.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sweep.cuh"

namespace mgk {

// The first pre-smoothing step on a level starts from x = 0, so it needs only the level's
// right-hand side and D^-1: the kernel that produces the right-hand side (the restriction
// from the finer level; on the finest FP32 level the outer residual) can take it
// (ZM = SW_JACOBI_Z or SW_CHEBF_Z) while it holds b_i, with the arithmetic and the stored
// values of the separate sweep (sweep_out_v). D^-1 is a stored array, 1 / a_ii of the DIA
// diagonal slot, or the constant of a constant stencil.
template <typename T>
struct ZStep {
    const T *dinv = nullptr;         // stored 1 / a_ii, or nullptr
    const T *diag = nullptr;         // a_ii (the DIA diagonal slot), or nullptr
    T cdinv = T(0);                  // 1 / a_ii of a constant stencil (dinv and diag null)
    T *out = nullptr, *d = nullptr;  // the step's x and (SW_CHEBF_Z) Chebyshev direction
    T c1 = T(0);
};

template <typename T>
__device__ __forceinline__ T zstep_dinv(const ZStep<T> &Z, int i)
{
    return Z.dinv ? __ldcs(Z.dinv + i) : (Z.diag ? Ar<T>::rcp(__ldcs(Z.diag + i)) : Z.cdinv);
}

template <typename T, int ZM>
__device__ __forceinline__ void zstep(const ZStep<T> &Z, int i, T bi)
{
    if constexpr (ZM != 0) sweep_out_v<T, ZM>(i, T(0), zstep_dinv(Z, i), T(0), bi, T(0), Z.out, Z.d, Z.c1, T(0));
}

// ------------------------------------------------------------------------------------
// Q1 grid transfers on the structured grid (no stored matrix)
// ------------------------------------------------------------------------------------
// Restriction b_c = P^T r: coarse vertex (X,Y[,Z]) gathers the 3^d fine vertices around
// (2X,2Y[,2Z]) in ascending fine index, weight prod_d (1 if on the line, 1/2 otherwise).
// ZM: the coarse level's first smoothing step as well (ZStep).
// Launch: x-lines of the coarse grid, grid (ceil(nc1/blockDim), nc1, DIM == 3 ? nc1 : 1).
template <typename T, int DIM, int ZM = 0>
__global__ void __launch_bounds__(128) k_restrict_q1(const T *__restrict__ r, T *__restrict__ bc, int Nc, ZStep<T> Zs)
{
    pdl_enter();
    int nc1 = Nc - 1, nf1 = 2 * Nc - 1;
    int X = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (X > nc1) return;
    int Y = blockIdx.y + 1, Z = DIM == 3 ? blockIdx.z + 1 : 0;
    int64_t I = (X - 1) + (int64_t)nc1 * ((Y - 1) + (DIM == 3 ? (int64_t)nc1 * (Z - 1) : 0));
    T s = T(0);
    const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
#pragma unroll
    for (int dz = zlo; dz <= zhi; dz++)
#pragma unroll
        for (int dy = -1; dy <= 1; dy++)
#pragma unroll
            for (int dx = -1; dx <= 1; dx++) {
                T w = (dx ? T(0.5) : T(1)) * (dy ? T(0.5) : T(1)) * (dz ? T(0.5) : T(1));
                int64_t j = (2 * X + dx - 1) + (int64_t)nf1 * ((2 * Y + dy - 1) + (DIM == 3 ? (int64_t)nf1 * (2 * Z + dz - 1) : 0));
                s = Ar<T>::mac(s, w, __ldg(r + j));
            }
    bc[I] = s;
    zstep<T, ZM>(Zs, (int)I, s);
}

// Prolongation and correction x_f += P x_c: fine vertex v takes the coarse vertices V
// with |v - 2V| <= 1 per axis (boundary ones are zero), ascending coarse index. Every
// such V carries the same weight prod_d (1 or 1/2) = 2^-(number of odd coordinates of v),
// so the sum is one multiply-add per term from s = 0 in the order Z, Y, X ascending.
// Thread (X, Y[, Z]), X, Y, Z = 0 .. Nc - 1, owns the 2^d fine vertices (2X + ex, 2Y + ey
// [, 2Z + ez]), e in {0, 1}, that are interior, and the 2^d coarse corners (X + dx,
// Y + dy[, Z + dz]) they draw on: all of its fine and coarse values are loaded before
// any sum, so each thread has 2^d fine values in flight instead of two. A vertex with
// e = 0 on an axis takes d = 0 only, one with e = 1 takes d = 0, 1; corners off the
// interior are read as +0, whose terms leave the sum's bits unchanged (s starts at +0,
// and s + (+0) = s), so the result is the same as summing over the interior corners only.
// Launch: grid (ceil(Nc/blockDim), Nc, DIM == 3 ? Nc : 1).
template <typename T, int DIM>
__global__ void __launch_bounds__(128) k_prolong_q1(const T *__restrict__ xc, T *__restrict__ xf, int Nc)
{
    pdl_enter();
    constexpr int NZ = DIM == 3 ? 2 : 1;
    const int nf1 = 2 * Nc - 1, nc1 = Nc - 1;
    const int X = blockIdx.x * blockDim.x + threadIdx.x;
    if (X >= Nc) return;
    const int Y = blockIdx.y, Z = DIM == 3 ? blockIdx.z : 1;
    T c[NZ][2][2], f[NZ][2][2];
    bool fin[NZ][2][2];
    // fine vertex (2X + ex, 2Y + ey, 2Z + ez) at base + ex + nf1 ey + nf1^2 ez
    const int64_t base = (2 * X - 1) + (int64_t)nf1 * ((2 * Y - 1) + (DIM == 3 ? (int64_t)nf1 * (2 * Z - 1) : 0));
#pragma unroll
    for (int dz = 0; dz < NZ; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++)
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const int cx = X + dx, cy = Y + dy, cz = Z + dz;
                const bool in = cx >= 1 && cx <= nc1 && cy >= 1 && cy <= nc1 && (DIM == 2 || (cz >= 1 && cz <= nc1));
                c[dz][dy][dx] = in ? __ldg(xc + (cx - 1) + (int64_t)nc1 * ((cy - 1) + (DIM == 3 ? (int64_t)nc1 * (cz - 1) : 0)))
                                   : T(0);
                const bool v = (2 * X + dx >= 1) && (2 * Y + dy >= 1) && (DIM == 2 || 2 * Z + dz >= 1);
                fin[dz][dy][dx] = v;
                f[dz][dy][dx] = v ? xf[base + dx + (int64_t)nf1 * (dy + (int64_t)nf1 * dz)] : T(0);
            }
#pragma unroll
    for (int ez = 0; ez < NZ; ez++)
#pragma unroll
        for (int ey = 0; ey < 2; ey++)
#pragma unroll
            for (int ex = 0; ex < 2; ex++) {
                const int odd = ex + ey + ez;
                const T w = odd == 0 ? T(1) : (odd == 1 ? T(0.5) : (odd == 2 ? T(0.25) : T(0.125)));
                T s = T(0);
#pragma unroll
                for (int dz = 0; dz <= ez; dz++)
#pragma unroll
                    for (int dy = 0; dy <= ey; dy++)
#pragma unroll
                        for (int dx = 0; dx <= ex; dx++) s = Ar<T>::mac(s, w, c[dz][dy][dx]);
                if (fin[ez][ey][ex])
                    xf[base + ex + (int64_t)nf1 * (ey + (int64_t)nf1 * ez)] = Ar<T>::add(f[ez][ey][ex], s);
            }
}

// Explicit transfer (rotated Q1, P1, P2) with the operator in SELL-32 (see k_sell_sweep):
// y_i = sum_k v_k x_col(k) in the row's CSR order (ADD: y_i += that sum); storage position
// r computes row perm[r].
template <typename T, bool ADD, int ZM = 0>
__global__ void __launch_bounds__(256) k_sell_apply(const int64_t *__restrict__ sptr, const int32_t *__restrict__ col,
                                                    const T *__restrict__ val, const int32_t *__restrict__ perm,
                                                    int n, const T *__restrict__ x, T *__restrict__ y, ZStep<T> Zs)
{
    pdl_enter();
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int i = __ldg(perm + r);
    int64_t base = sptr[r >> 5];
    int Ks = (int)((sptr[(r >> 5) + 1] - base) >> 5);
    int64_t e = base + (r & 31);
    T s = T(0);
    for (int k = 0; k < Ks; k++, e += 32) s = Ar<T>::mac(s, __ldcs(val + e), __ldg(x + __ldcs(col + e)));
    y[i] = ADD ? Ar<T>::add(y[i], s) : s;
    if (!ADD) zstep<T, ZM>(Zs, i, s);
}

// ------------------------------------------------------------------------------------
// Coarsest level: dense LU in FP64 (one CTA, n <= 1024)
// ------------------------------------------------------------------------------------
// Right-looking LU with partial pivoting; the first row of maximal |a| is the pivot.
__global__ void k_lu_factor(double *a, int n, int *piv, int *info);

// Solve with the factors: row swaps in factorisation order, then column-oriented
// substitutions so every thread owns one row and its running sum (fused multiply-adds):
// forward in ascending column order, backward in descending column order, each unknown
// of the backward pass multiplied by its pivot's reciprocal. Input and output in T.
template <typename T>
__global__ void k_coarse_solve(const double *__restrict__ lu, const int *__restrict__ piv, int n,
                               const T *__restrict__ b, T *__restrict__ x)
{
    extern __shared__ double xs[];
    pdl_enter();
    int t = threadIdx.x;
    if (t < n) xs[t] = (double)b[t];
    __syncthreads();
    if (t == 0)
        for (int k = 0; k < n; k++) {
            int p = piv[k];
            if (p != k) {
                double tmp = xs[k];
                xs[k] = xs[p];
                xs[p] = tmp;
            }
        }
    __syncthreads();
    double s = 0.0;
    double inv = t < n ? __ddiv_rn(1.0, lu[(int64_t)t * n + t]) : 0.0;  // off the dependency chain
    for (int j = 0; j < n; j++) {
        if (t == j) xs[j] = __dsub_rn(xs[j], s);
        __syncthreads();
        if (t > j && t < n) s = __fma_rn(lu[(int64_t)t * n + j], xs[j], s);
    }
    __syncthreads();
    s = 0.0;
    for (int j = n - 1; j >= 0; j--) {
        if (t == j) xs[j] = __dmul_rn(__dsub_rn(xs[j], s), inv);
        __syncthreads();
        if (t < j) s = __fma_rn(lu[(int64_t)t * n + j], xs[j], s);
    }
    __syncthreads();
    if (t < n) x[t] = (T)xs[t];
}

// Substitutions of the pivoted right-hand side xs (shared memory, n <= 64) with the LU
// factors L (shared memory, row-major) by one warp: lane l owns rows l and l + 32 and
// their running sums, one __syncwarp per column. Forward: x_i -= sum_{j<i} l_ij x_j,
// ascending j; backward: x_i = (x_i - sum_{j>i} u_ij x_j) * (1 / u_ii), descending j; sums
// by fused multiply-adds. The reciprocals are formed before the loops, so the dependent
// chain per column is one fused multiply-add, one subtraction (and one multiplication).
__device__ __forceinline__ void lu_substitute_warp(const double *L, double *xs, int n, int l)
{
    int r0 = l, r1 = l + 32;
    double inv0 = r0 < n ? __ddiv_rn(1.0, L[r0 * n + r0]) : 0.0;
    double inv1 = r1 < n ? __ddiv_rn(1.0, L[r1 * n + r1]) : 0.0;
    double s0 = 0.0, s1 = 0.0;
    for (int j = 0; j < n; j++) {
        if (j == r0) xs[j] = __dsub_rn(xs[j], s0);
        if (j == r1) xs[j] = __dsub_rn(xs[j], s1);
        __syncwarp();
        double xj = xs[j];
        if (r0 > j && r0 < n) s0 = __fma_rn(L[r0 * n + j], xj, s0);
        if (r1 > j && r1 < n) s1 = __fma_rn(L[r1 * n + j], xj, s1);
        __syncwarp();
    }
    s0 = s1 = 0.0;
    for (int j = n - 1; j >= 0; j--) {
        if (j == r0) xs[j] = __dmul_rn(__dsub_rn(xs[j], s0), inv0);
        if (j == r1) xs[j] = __dmul_rn(__dsub_rn(xs[j], s1), inv1);
        __syncwarp();
        double xj = xs[j];
        if (r0 < j) s0 = __fma_rn(L[r0 * n + j], xj, s0);
        if (r1 < j) s1 = __fma_rn(L[r1 * n + j], xj, s1);
        __syncwarp();
    }
}

// The same solve for n <= 64 by one warp with the factors in shared memory: lane l owns
// rows l and l + 32 and their running sums; one __syncwarp per column. All 256 threads
// of the block stage the factors, pivots and right-hand side first (independent loads in
// flight together), then warp 0 alone solves.
template <typename T>
__global__ void __launch_bounds__(256) k_coarse_solve_warp(const double *__restrict__ lu, const int *__restrict__ piv,
                                                           int n, const T *__restrict__ b, T *__restrict__ x)
{
    __shared__ double L[64 * 64];
    __shared__ double xs[64];
    __shared__ int ps[64];
    pdl_enter();
    int tid = threadIdx.x;
#pragma unroll 4
    for (int k = tid; k < n * n; k += 256) L[k] = lu[k];
    if (tid < n) {
        xs[tid] = (double)b[tid];
        ps[tid] = piv[tid];
    }
    __syncthreads();
    if (tid >= 32) return;
    int l = tid;
    if (l == 0)
        for (int k = 0; k < n; k++) {
            int p = ps[k];
            if (p != k) {
                double tmp = xs[k];
                xs[k] = xs[p];
                xs[p] = tmp;
            }
        }
    __syncwarp();
    lu_substitute_warp(L, xs, n, l);
    for (int k = l; k < n; k += 32) x[k] = (T)xs[k];
}

// ------------------------------------------------------------------------------------
// Coarse-level tail: the V-cycle below a small level in one thread-block-cluster launch
// ------------------------------------------------------------------------------------
// The levels with at most a few thousand rows each cost one latency-bound kernel per
// operation. The host records those operations in V-cycle order (TailOp) and one launch
// of a cluster of CTAs replays them: rows are spread over all threads of the cluster and
// a cluster barrier (release/acquire at cluster scope) separates consecutive operations.
// Each row is computed by the same arithmetic as the single-operation kernels.
enum TailOpKind { TAIL_SWEEP = 0, TAIL_RESTRICT, TAIL_COARSE, TAIL_PROLONG, TAIL_ZERO };
constexpr int TAIL_MAX_LEVELS = 8;
constexpr int TAIL_MAX_OPS = 96;

struct TailOp {
    int kind, level, mode;
    int in, out;  // x buffers 0/1; out 2 = the residual vector t
    int aux;      // RESTRICT: 1 = restrict b itself; PROLONG: coarse buffer
    double c1, c2;
};

template <typename T>
struct TailLevel {
    MatView<T> A;
    int n, N;
    T *x[2];
    T *b, *t, *d;
};

template <typename T>
struct TailProg {
    TailLevel<T> lev[TAIL_MAX_LEVELS];
    TailOp ops[TAIL_MAX_OPS];
    int nops, dim, K;
    const double *lu;
    const int *piv;
    int n0;
};

template <typename T, int K, int MODE>
__device__ __forceinline__ void tail_sweep_row(const TailLevel<T> &L, int i, const TailOp &op)
{
    constexpr int C = K / 2;
    T c1 = (T)op.c1, c2 = (T)op.c2;
    T *o = op.out == 2 ? L.t : L.x[op.out];
    if (IsZero<MODE>::value) {
        T dinv = Ar<T>::kStoredDinv ? L.A.dinv[i] : Ar<T>::rcp(L.A.val[(int64_t)C * L.A.ld + i]);
        sweep_out<T, MODE>(i, T(0), dinv, T(0), L.b, o, L.d, c1, c2);
        return;
    }
    const T *x = L.x[op.in];
    T a[K], xv[K];
#pragma unroll
    for (int k = 0; k < K; k++) a[k] = L.A.val[(int64_t)k * L.A.ld + i];
#pragma unroll
    for (int k = 0; k < K; k++) xv[k] = x[i + L.A.offs.o[k]];
    T s = T(0);
#pragma unroll
    for (int k = 0; k < K; k++) s = Ar<T>::mac(s, a[k], xv[k]);
    T dinv = Ar<T>::kStoredDinv ? L.A.dinv[i] : Ar<T>::rcp(a[C]);
    sweep_out<T, MODE>(i, s, dinv, xv[C], L.b, o, L.d, c1, c2);
}

template <typename T, int K>
__device__ __forceinline__ void tail_sweep(const TailLevel<T> &L, const TailOp &op, int g, int G)
{
    for (int i = g; i < L.n; i += G) {
        switch (op.mode) {
        case SW_RESID: tail_sweep_row<T, K, SW_RESID>(L, i, op); break;
        case SW_JACOBI: tail_sweep_row<T, K, SW_JACOBI>(L, i, op); break;
        case SW_CHEBF: tail_sweep_row<T, K, SW_CHEBF>(L, i, op); break;
        case SW_CHEB: tail_sweep_row<T, K, SW_CHEB>(L, i, op); break;
        case SW_JACOBI_Z: tail_sweep_row<T, K, SW_JACOBI_Z>(L, i, op); break;
        default: tail_sweep_row<T, K, SW_CHEBF_Z>(L, i, op); break;
        }
    }
}

template <typename T, int DIM>
__device__ __forceinline__ void tail_restrict(const TailLevel<T> &F, const TailLevel<T> &C, const TailOp &op, int g, int G)
{
    const T *r = op.aux ? F.b : F.t;
    int nc1 = C.N - 1, nf1 = F.N - 1;
    for (int I = g; I < C.n; I += G) {
        int X = I % nc1 + 1, Y = (I / nc1) % nc1 + 1, Z = DIM == 3 ? I / (nc1 * nc1) + 1 : 0;
        T s = T(0);
        const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
#pragma unroll
        for (int dz = zlo; dz <= zhi; dz++)
#pragma unroll
            for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                for (int dx = -1; dx <= 1; dx++) {
                    T w = (dx ? T(0.5) : T(1)) * (dy ? T(0.5) : T(1)) * (dz ? T(0.5) : T(1));
                    int64_t j = (2 * X + dx - 1) + (int64_t)nf1 * ((2 * Y + dy - 1) + (DIM == 3 ? (int64_t)nf1 * (2 * Z + dz - 1) : 0));
                    s = Ar<T>::mac(s, w, r[j]);
                }
        C.b[I] = s;
    }
}

template <typename T, int DIM>
__device__ __forceinline__ void tail_prolong(const TailLevel<T> &F, const TailLevel<T> &C, const TailOp &op, int g, int G)
{
    const T *xc = C.x[op.aux];
    T *xf = F.x[op.out];
    int Nc = C.N, nf1 = F.N - 1, nc1 = Nc - 1;
    for (int i = g; i < F.n; i += G) {
        int v0 = i % nf1 + 1, v1 = (i / nf1) % nf1 + 1, v2 = DIM == 3 ? i / (nf1 * nf1) + 1 : 2;
        int odd = (v0 & 1) + (v1 & 1) + (DIM == 3 ? (v2 & 1) : 0);
        const T w = odd == 0 ? T(1) : (odd == 1 ? T(0.5) : (odd == 2 ? T(0.25) : T(0.125)));
        int x0 = max(v0 >> 1, 1), x1 = min((v0 + 1) >> 1, Nc - 1);
        int y0 = max(v1 >> 1, 1), y1 = min((v1 + 1) >> 1, Nc - 1);
        int z0 = DIM == 3 ? max(v2 >> 1, 1) : 1, z1 = DIM == 3 ? min((v2 + 1) >> 1, Nc - 1) : 1;
        T t = T(0);
        for (int Z = z0; Z <= z1; Z++)
            for (int Y = y0; Y <= y1; Y++) {
                int64_t row = (int64_t)nc1 * ((Y - 1) + (DIM == 3 ? (int64_t)nc1 * (Z - 1) : 0)) - 1;
                for (int X = x0; X <= x1; X++) t = Ar<T>::mac(t, w, xc[row + X]);
            }
        xf[i] = Ar<T>::add(xf[i], t);
    }
}

// Launched as one cluster (grid = cluster size) of 512 threads per CTA.
template <typename T>
__global__ void __launch_bounds__(512) k_tail(TailProg<T> P)
{
    __shared__ double Ls[64 * 64];
    __shared__ double xs[64];
    __shared__ int ps[64];
    pdl_enter();
    int g = blockIdx.x * blockDim.x + threadIdx.x, G = gridDim.x * blockDim.x;
    for (int o = 0; o < P.nops; o++) {
        const TailOp op = P.ops[o];
        const TailLevel<T> &L = P.lev[op.level];
        if (op.kind == TAIL_SWEEP) {
            if (L.A.K == 21)
                tail_sweep<T, 21>(L, op, g, G);
            else if (L.A.K == 27)
                tail_sweep<T, 27>(L, op, g, G);
            else
                tail_sweep<T, 9>(L, op, g, G);
        } else if (op.kind == TAIL_RESTRICT) {
            if (P.dim == 3)
                tail_restrict<T, 3>(L, P.lev[op.level - 1], op, g, G);
            else
                tail_restrict<T, 2>(L, P.lev[op.level - 1], op, g, G);
        } else if (op.kind == TAIL_PROLONG) {
            if (P.dim == 3)
                tail_prolong<T, 3>(L, P.lev[op.level - 1], op, g, G);
            else
                tail_prolong<T, 2>(L, P.lev[op.level - 1], op, g, G);
        } else if (op.kind == TAIL_ZERO) {
            for (int i = g; i < L.n; i += G) L.x[op.out][i] = T(0);
        } else if (blockIdx.x == 0) {  // TAIL_COARSE: the LU solve by the first CTA
            int n = P.n0, tid = threadIdx.x;
            for (int k = tid; k < n * n; k += blockDim.x) Ls[k] = P.lu[k];
            if (tid < n) {
                xs[tid] = (double)L.b[tid];
                ps[tid] = P.piv[tid];
            }
            __syncthreads();
            if (tid < 32) {
                if (tid == 0)
                    for (int k = 0; k < n; k++) {
                        int q = ps[k];
                        if (q != k) {
                            double tmp = xs[k];
                            xs[k] = xs[q];
                            xs[q] = tmp;
                        }
                    }
                __syncwarp();
                lu_substitute_warp(Ls, xs, n, tid);
                for (int k = tid; k < n; k += 32) L.x[0][k] = (T)xs[k];
            }
        }
        // every thread of the cluster finishes op o before any starts op o + 1
        asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
    }
}

// ------------------------------------------------------------------------------------
// FP64 outer residual r = b - A64 x64 with ||r||^2, and helpers
// ------------------------------------------------------------------------------------
// Block sums of r^2 in a fixed tree order; the last block to finish (ticket) adds the
// block sums in a fixed order and writes the total, so the result does not depend on
// block scheduling.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;  // valid in thread 0
}

// Grid of the kernels that end in a reduction: a fixed number of blocks stepping through
// the rows, so that the per-block ticket of finish_norm is taken 912 times instead of
// once per 256 rows. 912 = 6 blocks on each of GB300's 152 SMs, the residency those
// kernels are compiled for (__launch_bounds__(256, 6): up to 42 registers, no spills), so
// the grid is exactly one wave; a constant keeps the summation order, hence the bits,
// independent of the device. The kernels that apply a DIA FP64 operator row by row (the
// outer residual, the CG residual and matrix product) run 3 blocks per SM with 80
// registers instead (kOuterBlocks = 456 blocks, at most kReduceBlocks partial sums); on
// the gathered formats (ELL, CSR, SELL) they keep 6 blocks per SM, which hide the latency
// of each column index's dependent load better.
constexpr int kReduceBlocks = 912;
constexpr int kOuterBlocks = 456;
constexpr int fp64_rows_blocks_per_sm(int fmt) { return fmt == 3 ? 3 : 6; }

// Sum of `part` over the grid in a fixed order: block sums to partial[], the last block
// to finish (ticket) adds them up. Returns true in the thread that wrote *out.
__device__ __forceinline__ bool finish_norm(double part, double *partial, unsigned *ticket, double *out)
{
    __shared__ double sh[32];
    __shared__ bool last;
    double s = block_sum(part, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = s;
        __threadfence();
        unsigned t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    // the block partials, read from L2 eight at a time per thread (independent loads,
    // then a fixed-order sum) so that the last block does not wait for one round trip
    // per partial
    const int G = (int)gridDim.x, B = (int)blockDim.x;
    double acc = 0.0;
    for (int k0 = threadIdx.x; k0 < G; k0 += 8 * B) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; u++) v[u] = k0 + u * B < G ? __ldcg(partial + k0 + u * B) : 0.0;
        acc += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
    }
    double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        *out = tot;
        *ticket = 0u;
        return true;
    }
    return false;
}

// Row i (at storage position r) of an FP64 operator applied to the padded vector v:
// column-ascending fused multiply-adds. FMT: 3 DIA (K slots), 2 ELL, 1 CSR, 4 SELL-32.
template <int FMT, int K>
__device__ __forceinline__ double fp64_row(const MatView<double> &A, int r, int i, const double *__restrict__ v)
{
    double s = 0.0;
    if (FMT == 3) {  // DIA
        double a[K], xv[K];
#pragma unroll
        for (int k = 0; k < K; k++) a[k] = __ldcs(A.val + (int64_t)k * A.ld + i);
#pragma unroll
        for (int k = 0; k < K; k++) xv[k] = __ldg(v + i + A.offs.o[k]);
#pragma unroll
        for (int k = 0; k < K; k++) s = __fma_rn(a[k], xv[k], s);
    } else if (FMT == 2) {  // ELL
        for (int k = 0; k < A.K; k++) {
            int c = __ldcs(A.col + (int64_t)k * A.ld + i);
            s = __fma_rn(__ldcs(A.val + (int64_t)k * A.ld + i), __ldg(v + c), s);
        }
    } else if (FMT == 4) {  // SELL-32
        int64_t base = A.rowptr[r >> 5];
        int Ks = (int)((A.rowptr[(r >> 5) + 1] - base) >> 5);
        int64_t e = base + (r & 31);
        for (int k = 0; k < Ks; k++, e += 32) s = __fma_rn(__ldcs(A.val + e), __ldg(v + __ldcs(A.col + e)), s);
    } else {  // CSR
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) s = __fma_rn(A.val[k], __ldg(v + A.col[k]), s);
    }
    return s;
}

// the DOF at storage position r (SELL permutes rows; the other formats do not)
template <int FMT>
__device__ __forceinline__ int fp64_dof(const MatView<double> &A, int r)
{
    return FMT == 4 ? __ldg(A.perm + r) : r;
}

// ZM: the finest FP32 level's first smoothing step as well (ZStep), on the defect as the
// FP32 value stored in r; its D^-1 is loaded before the row so that its latency hides
// behind the row's.
// DIA: launched on kOuterBlocks blocks (three per SM, 80 registers a thread: measured faster
// than four, five or six per SM with 64, 48 or 40 registers, where the compiler interleaves
// more of each row's 42 loads with its chain of fused multiply-adds).
template <typename Tin, int FMT, int K, int ZM = 0>
__global__ void __launch_bounds__(256, fp64_rows_blocks_per_sm(FMT)) k_outer_resid(MatView<double> A, int n, const double *__restrict__ x,
                                                     const double *__restrict__ b, Tin *__restrict__ r,
                                                     double *partial, unsigned *ticket, double *norm2,
                                                     ZStep<float> Zs)
{
    pdl_enter();
    double sq = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        int i = fp64_dof<FMT>(A, q);
        float dv = 0.0f;
        if constexpr (ZM != 0) dv = zstep_dinv(Zs, i);
        double ri = __dsub_rn(b[i], fp64_row<FMT, K>(A, q, i, x));
        const Tin rt = (Tin)ri;
        r[i] = rt;
        sq = __fma_rn(ri, ri, sq);
        if constexpr (ZM != 0)
            sweep_out_v<float, ZM>(i, 0.0f, dv, 0.0f, (float)rt, 0.0f, Zs.out, Zs.d, Zs.c1, 0.0f);
    }
    finish_norm(sq, partial, ticket, norm2);
}

// 1 / a_ii of a per-cell-coefficient level, as its sweep forms it: 4 times the sum of the
// eight cells around the vertex, the cells summed per cell plane ((k0 + k1) + (k2 + k3)),
// lower plane first. Launch: grid (ceil(n1/blockDim.x), n1, n1).
__global__ void k_coef_dinv(const float *__restrict__ kap, int n1, float *__restrict__ dinv);

__global__ void k_norm2(const double *__restrict__ v, int n, double *partial, unsigned *ticket, double *norm2);

template <typename Tin>
__global__ void __launch_bounds__(256) k_update(double *__restrict__ x, const Tin *__restrict__ c, int n)
{
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = __dadd_rn(x[i], (double)c[i]);
}

}  // namespace mgk
