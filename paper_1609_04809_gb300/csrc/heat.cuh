// heat.cuh -- right-hand side of a Crank-Nicolson step of the heat equation (internal).
//
// The paper's model problem (Sec. 6) is the heat equation, Galerkin FE in space and
// Crank-Nicolson in time. With sigma = 2/dt a step is (A + sigma M) u' = B u + t bF,
// B = sigma M - A, t = g(t_k) + g(t_{k+1}) for a separable source g(t) F(x). The
// system is solved by the multigrid hierarchy built on A + sigma M; this kernel forms
// its right-hand side from the current solution in one pass over B.
#pragma once

#include "krylov.cuh"

namespace mgk {

template <int FMT, int K>
__global__ void __launch_bounds__(256) k_heat_rhs(MatView<double> B, int n, const double *__restrict__ u,
                                                  const double *__restrict__ bF, double t, double *__restrict__ rhs)
{
    pdl_enter();
    int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    int i = fp64_dof<FMT>(B, q);
    rhs[i] = __dadd_rn(fp64_row<FMT, K>(B, q, i, u), __dmul_rn(t, bF[i]));
}

}  // namespace mgk
