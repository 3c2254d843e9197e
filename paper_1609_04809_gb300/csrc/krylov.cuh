// krylov.cuh -- conjugate gradients preconditioned by one V-cycle (internal).
//
// The paper notes that multigrid is most often used as the preconditioner of a Krylov
// method (Sec. 1). For the symmetric positive definite Q1 / rotated-Q1 systems that is
// preconditioned CG (Saad, Alg. 9.1) with M^-1 r = V(r). One iteration is one V-cycle on
// the FP64 residual (in the inner precision) followed by four FP64 kernels:
//   k_pcg_rz      rz = (r, z), beta = rz / rz_old      z: the V-cycle's correction
//   k_pcg_dir     p = z + beta p                       (beta = 0 in the first iteration)
//   k_pcg_apply   q = A p, pq = (p, q), alpha = rz / pq   A: the FP64 finest operator
//   k_pcg_update  x += alpha p, r -= alpha q, ||r||^2; rz_old = rz
// The scalars live in device memory (scal[]), so the iteration needs no host round trip
// except for the residual norm of the stopping test. Each division is done once, by the
// thread that finishes the reduction it needs. Inner products are reduced in a
// fixed order (block sums, then the last block), so a solve is deterministic.
#pragma once

#include "kernels.cuh"

namespace mgk {

enum PcgScalar { PCG_RZ = 0, PCG_RZ_OLD = 1, PCG_PQ = 2, PCG_ALPHA = 3, PCG_BETA = 4, PCG_NSCAL = 8 };

// r = b - A x in FP64 (kept in r64 and, in the inner precision, in rin: the V-cycle's
// right-hand side); p = 0, rz_old = 0; ||r||^2 -> norm2. ZM: also the finest FP32 level's
// first smoothing step on rin (ZStep, as in k_outer_resid).
template <typename Tin, int FMT, int K, int ZM = 0>
__global__ void __launch_bounds__(256, fp64_rows_blocks_per_sm(FMT)) k_pcg_init(MatView<double> A, int n, const double *__restrict__ x,
                                                  const double *__restrict__ b, double *__restrict__ r64,
                                                  Tin *__restrict__ rin, double *__restrict__ p, double *scal,
                                                  double *partial, unsigned *ticket, double *norm2, ZStep<float> Zs)
{
    pdl_enter();
    double sq = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        int i = fp64_dof<FMT>(A, q);
        float dv = 0.0f;
        if constexpr (ZM != 0) dv = zstep_dinv(Zs, i);
        double ri = __dsub_rn(b[i], fp64_row<FMT, K>(A, q, i, x));
        r64[i] = ri;
        rin[i] = (Tin)ri;
        if constexpr (ZM != 0)
            sweep_out_v<float, ZM>(i, 0.0f, dv, 0.0f, (float)(Tin)ri, 0.0f, Zs.out, Zs.d, Zs.c1, 0.0f);
        p[i] = 0.0;
        sq = __fma_rn(ri, ri, sq);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) scal[PCG_RZ_OLD] = 0.0;
    finish_norm(sq, partial, ticket, norm2);
}

template <typename Tin>
__global__ void __launch_bounds__(256, 6) k_pcg_rz(const double *__restrict__ r, const Tin *__restrict__ z, int n,
                                                double *partial, unsigned *ticket, double *scal)
{
    pdl_enter();
    double part = 0.0;
    const int st = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    // four rows' loads in flight per thread; the sum runs in the same row order as a
    // plain grid-stride loop
    for (; i + 3 * st < n; i += 4 * st) {
        double r0 = r[i], r1 = r[i + st], r2 = r[i + 2 * st], r3 = r[i + 3 * st];
        double z0 = (double)z[i], z1 = (double)z[i + st], z2 = (double)z[i + 2 * st], z3 = (double)z[i + 3 * st];
        part = __fma_rn(r0, z0, part);
        part = __fma_rn(r1, z1, part);
        part = __fma_rn(r2, z2, part);
        part = __fma_rn(r3, z3, part);
    }
    for (; i < n; i += st) part = __fma_rn(r[i], (double)z[i], part);
    if (finish_norm(part, partial, ticket, scal + PCG_RZ)) {
        double ro = scal[PCG_RZ_OLD];
        scal[PCG_BETA] = ro == 0.0 ? 0.0 : __ddiv_rn(scal[PCG_RZ], ro);
    }
}

template <typename Tin>
__global__ void __launch_bounds__(256) k_pcg_dir(const Tin *__restrict__ z, double *__restrict__ p, int n,
                                                 const double *__restrict__ scal)
{
    pdl_enter();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = __dadd_rn((double)z[i], __dmul_rn(scal[PCG_BETA], p[i]));
}

template <int FMT, int K>
__global__ void __launch_bounds__(256, fp64_rows_blocks_per_sm(FMT)) k_pcg_apply(MatView<double> A, int n, const double *__restrict__ p,
                                                   double *__restrict__ q, double *partial, unsigned *ticket,
                                                   double *scal)
{
    pdl_enter();
    double part = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int i = fp64_dof<FMT>(A, t);
        double s = fp64_row<FMT, K>(A, t, i, p);
        q[i] = s;
        part = __fma_rn(p[i], s, part);
    }
    if (finish_norm(part, partial, ticket, scal + PCG_PQ)) scal[PCG_ALPHA] = __ddiv_rn(scal[PCG_RZ], scal[PCG_PQ]);
}

// ZM: also the finest FP32 level's first smoothing step on rin (ZStep, as in k_outer_resid)
template <typename Tin, int ZM = 0>
__global__ void __launch_bounds__(256, 6) k_pcg_update(double *__restrict__ x, double *__restrict__ r,
                                                    Tin *__restrict__ rin, const double *__restrict__ p,
                                                    const double *__restrict__ q, int n, double *scal,
                                                    double *partial, unsigned *ticket, double *norm2,
                                                    ZStep<float> Zs)
{
    pdl_enter();
    double alpha = scal[PCG_ALPHA];
    double sq = 0.0;
    const int st = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + st < n; i += 2 * st) {  // two rows' loads in flight (eight loads), rows in order
        double xv[2], pv[2], rv[2], qv[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            int j = i + u * st;
            xv[u] = x[j];
            pv[u] = p[j];
            rv[u] = r[j];
            qv[u] = q[j];
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
            int j = i + u * st;
            x[j] = __dadd_rn(xv[u], __dmul_rn(alpha, pv[u]));
            double ri = __dsub_rn(rv[u], __dmul_rn(alpha, qv[u]));
            r[j] = ri;
            rin[j] = (Tin)ri;
            sq = __fma_rn(ri, ri, sq);
            zstep<float, ZM>(Zs, j, (float)(Tin)ri);
        }
    }
    for (; i < n; i += st) {
        x[i] = __dadd_rn(x[i], __dmul_rn(alpha, p[i]));
        double ri = __dsub_rn(r[i], __dmul_rn(alpha, q[i]));
        r[i] = ri;
        rin[i] = (Tin)ri;
        sq = __fma_rn(ri, ri, sq);
        zstep<float, ZM>(Zs, i, (float)(Tin)ri);
    }
    if (finish_norm(sq, partial, ticket, norm2)) scal[PCG_RZ_OLD] = scal[PCG_RZ];
}

}  // namespace mgk
