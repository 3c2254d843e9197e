"""Seeded synthetic inputs for the multigrid solve.

This module only draws random numbers and describes problem shapes: it holds none of
the method's arithmetic (no assembly, no quadrature, no smoothing). Both the CUDA path
and the CPU oracle receive what it produces: coefficient fields, manufactured-solution
modes, right-hand-side vectors and serving traces. It imports nothing from the rest of
the package.

The paper's workloads are manufactured-solution PDEs on the unit cube (Sec. 6.2, the
heat-equation model problem with a product-of-sines solution); the workloads below keep
that structure for the steady Poisson / diffusion problems solved here.
"""
import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count, start=0):
    """Outputs start..start+count-1 of SplitMix64 (Steele, Lea, Flood 2014) from `seed`.

    Counter form: z_i = seed + (i+1)*0x9E3779B97F4A7C15, then the published mixing
    steps. Returns uint64 values.
    """
    with np.errstate(over="ignore"):
        i = np.arange(start, start + count, dtype=np.uint64)
        z = np.uint64(seed) + (i + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed, count, start=0):
    """Doubles in [0, 1): the top 53 bits of each SplitMix64 output times 2^-53."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def k_blocks(n_cells, dim=3, blocks_per_axis=16, log10_lo=-2.0, log10_hi=2.0, seed=20260101):
    """Piecewise-constant diffusion coefficient on blocks_per_axis^dim equal blocks.

    Block b (lexicographic, x fastest) gets k_b = 10^(lo + (hi - lo) * U_b), U_b the b-th
    uniform draw of SplitMix64(seed). Returns the per-cell field on n_cells^dim cells,
    lexicographic with x fastest, as float64.
    """
    assert n_cells % blocks_per_axis == 0
    nb = blocks_per_axis ** dim
    u = uniform01(seed, nb)
    kb = 10.0 ** (log10_lo + (log10_hi - log10_lo) * u)
    r = n_cells // blocks_per_axis
    kb = kb.reshape((blocks_per_axis,) * dim)  # index order (z,) y, x
    k = kb
    for ax in range(dim):
        k = np.repeat(k, r, axis=ax)
    return np.ascontiguousarray(k.reshape(-1))


def manufactured_modes(dim):
    """u = prod_d sin(pi x_d): one mode of amplitude 1 with unit frequencies."""
    return [(1.0, (1,) * dim)]


def q1_nodal_sine(dim, n_cells, freqs=None, amp=1.0):
    """amp * prod_d sin(k_d pi x_d) at the interior Q1 vertices (lexicographic, x fastest)."""
    freqs = freqs or (1,) * dim
    x = np.arange(1, n_cells) / n_cells
    v = amp * np.ones(1)
    for d in reversed(range(dim)):  # x fastest: the last axis outermost
        v = np.multiply.outer(v, np.sin(freqs[d] * np.pi * x))
    return v.reshape(-1).copy()


def heat_workload(dim=3, n_cells=128, n_levels=6, dt=0.01, t_end=5.0, decay=0.1):
    """The heat-equation workload (the paper's model problem, Sec. 6, on hexahedra with
    homogeneous Dirichlet data): u = exp(-decay t) prod_d sin(pi x_d) solves
    u_t - Lap u = f with f = (d pi^2 - decay) exp(-decay t) prod_d sin(pi x_d), i.e.
    f(t, x) = g(t) F(x) with g(t) = exp(-decay t).

    Returns a dict: sigma = 2 / dt (the operator A + sigma M of the scaled Crank-Nicolson
    step), n_steps, g (g(t_k), k = 0..n_steps), the sine mode of F for the load-vector
    routines (amplitude (d pi^2 - decay) / (d pi^2): they build f = amp pi^2 |k|^2 sin),
    u0 (nodal values of u at t = 0) and the exact solution's amplitude at t_end."""
    n_steps = int(round(t_end / dt))
    g = np.exp(-decay * dt * np.arange(n_steps + 1))
    dpi2 = dim * np.pi ** 2
    return dict(dim=dim, n_cells=n_cells, n_levels=n_levels, dt=dt, sigma=2.0 / dt, n_steps=n_steps, g=g,
                source_modes=[((dpi2 - decay) / dpi2, (1,) * dim)], u0=q1_nodal_sine(dim, n_cells),
                exact_amp=float(np.exp(-decay * dt * n_steps)))


def random_modes(dim, n_modes=4, kmax=8, seed=0):
    """n_modes sine modes with integer frequencies U{1..kmax} per axis and N(0,1) amplitudes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    freq = rng.integers(1, kmax + 1, size=(n_modes, dim))
    amp = rng.standard_normal(n_modes)
    return [(float(amp[m]), tuple(int(v) for v in freq[m])) for m in range(n_modes)]


def random_vector(n, seed=0):
    """A seeded N(0,1) vector of length n (a rough right-hand side: every frequency)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n)


def ndofs(dim, element, n_cells):
    """Interior DOF count: Q1 (element 0) and P1 (2) vertices, rotated Q1 (1) faces, P2 (3)
    the points of the grid of 2 n_cells cells."""
    n1 = n_cells - 1
    if element in (0, 2):
        return n1 ** dim
    if element == 3:
        return (2 * n_cells - 1) ** dim
    return 3 * n1 * n_cells * n_cells


# The five workloads, as concrete problem descriptions.
#   smoother 0: damped Jacobi, 1: Chebyshev; element 0: Q1, 1: rotated Q1;
#   precision "fp64" / "mixed"; nu counts smoother applications (a Chebyshev
#   application of degree 2 is two matrix-vector products).
CONFIGS = {
    "q1_2d_64": dict(dim=2, element=0, n_cells=64, n_levels=5, smoother=0, omega=0.8,
                     cheb_degree=2, nu_pre=2, nu_post=2, tol=1e-10, rhs="manufactured",
                     precision="fp64"),
    "q1_3d_128_cheb": dict(dim=3, element=0, n_cells=128, n_levels=6, smoother=1, omega=0.8,
                           cheb_degree=2, nu_pre=1, nu_post=1, tol=1e-10, rhs="manufactured",
                           precision="fp64"),
    "rq1_3d_96": dict(dim=3, element=1, n_cells=96, n_levels=6, smoother=0, omega=0.7,
                      cheb_degree=2, nu_pre=2, nu_post=2, tol=1e-10, rhs="manufactured",
                      precision="fp64"),
    "q1_3d_256_vark": dict(dim=3, element=0, n_cells=256, n_levels=7, smoother=1, omega=0.8,
                           cheb_degree=2, nu_pre=1, nu_post=1, tol=1e-10, rhs="const",
                           precision="mixed", k="blocks16"),
}


# The paper's own elements on tetrahedra (P1 and P2 on the Kuhn tetrahedra of the cube
# grid), at about two million DOFs like the Q1 workload.
TET_CONFIGS = {
    "p1_3d_128_cheb": dict(dim=3, element=2, n_cells=128, n_levels=6, smoother=1, omega=0.8,
                           cheb_degree=2, nu_pre=1, nu_post=1, tol=1e-10, rhs="manufactured",
                           precision="fp64"),
    "p2_3d_64_cheb": dict(dim=3, element=3, n_cells=64, n_levels=5, smoother=1, omega=0.8,
                          cheb_degree=2, nu_pre=1, nu_post=1, tol=1e-10, rhs="manufactured",
                          precision="fp64"),
}


def serving_trace(n_requests=4096, rate=None, seed=4096, dims=(2, 3), levels2=(6, 11),
                  levels3=(4, 7), n_modes=4, kmax=8):
    """The seeded serving workload: a list of request dicts in arrival order.

    Each request: half 2D with 2^L x 2^L cells, L uniform in levels2, half 3D with
    2^L cubed cells, L uniform in levels3; right-hand side from n_modes sine modes with
    integer frequencies U{1..kmax} and N(0,1) amplitudes. Arrivals are a Poisson process
    of the given rate (requests per second); rate None gives all arrivals at t = 0.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    rng_t = np.random.Generator(np.random.PCG64(seed + 1))  # arrivals: a stream of their own
    out = []
    t = 0.0
    for r in range(n_requests):
        dim = int(dims[0] if rng.random() < 0.5 else dims[1])
        lo, hi = levels2 if dim == 2 else levels3
        L = int(rng.integers(lo, hi + 1))
        freq = rng.integers(1, kmax + 1, size=(n_modes, dim))
        amp = rng.standard_normal(n_modes)
        if rate:
            t += float(rng_t.exponential(1.0 / rate))
        modes = [(float(amp[m]), tuple(int(v) for v in freq[m])) for m in range(n_modes)]
        out.append(dict(id=r, dim=dim, n_cells=2 ** L, level_exp=L, modes=modes, arrival=t))
    return out
