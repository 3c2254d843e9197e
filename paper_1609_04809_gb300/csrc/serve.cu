// serve.cu -- continuous-batching multigrid server (mg_serve_* of include/mg.h).
//
// Requests are Q1 Poisson solves of different sizes and dimensions, run in mixed
// precision (FP32 V-cycle inside FP64 defect correction). The server keeps
//   * one operator set (level matrices, FP64 finest matrix, coarsest LU) per problem
//     shape (dim, cells, levels), shared by every request of that shape and cached
//     while memory allows;
//   * one workspace (level vectors, FP64 iterate and right-hand side) per admitted
//     request;
// all inside one device arena of the HBM budget, so the budget is the admission rule.
//
// Every defect-correction iteration of all admitted requests is one CUDA graph of
// phase launches: the FP64 outer residual of every request, then the V-cycle phases
// aligned by depth below each request's finest level (pre-smoothing steps, residual,
// restriction, coarsest solve, prolongation, post-smoothing steps), then x += c. Each
// phase is one persistent launch over a device tile list covering the same step of
// every request that has that depth. The tile lists are rewritten (one host-to-device
// copy) only when the set of admitted requests changes, so the graph for a given depth
// is captured once. The outer-residual phase also decides convergence on the device:
// later phases skip converged requests, so their iterate stays the one that met the
// tolerance. After each iteration the host reads the residual norms, retires finished
// requests (their slot and workspace are freed) and admits queued ones.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host_setup.h"
#include "kernels.cuh"
#include "mg.h"
#include "mg_internal.h"

using mgi::Error;
using namespace mgk;

#define SCK(call)                                                                                   \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) throw mgi::Error(MG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

namespace {

using Clock = std::chrono::steady_clock;

static inline int64_t rup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// ------------------------------------------------------------------------------------
// Device arena: first fit over 256-byte units, coalescing on free
// ------------------------------------------------------------------------------------
struct Arena {
    char *base = nullptr;
    size_t size = 0, in_use = 0, peak = 0;
    std::map<size_t, size_t> free_;  // offset -> size
    std::mutex mu;

    void init(char *b, size_t s)
    {
        base = b;
        size = s;
        free_.clear();
        free_[0] = s;
    }
    void *alloc(size_t bytes)
    {
        bytes = (size_t)rup((int64_t)std::max<size_t>(bytes, 1), 256);
        std::lock_guard<std::mutex> lk(mu);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            size_t off = it->first, sz = it->second;
            free_.erase(it);
            if (sz > bytes) free_[off + bytes] = sz - bytes;
            in_use += bytes;
            peak = std::max(peak, in_use);
            return base + off;
        }
        return nullptr;
    }
    void release(void *p, size_t bytes)
    {
        if (!p) return;
        bytes = (size_t)rup((int64_t)std::max<size_t>(bytes, 1), 256);
        std::lock_guard<std::mutex> lk(mu);
        size_t off = (size_t)((char *)p - base);
        in_use -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
};

void *arena_alloc_cb(size_t bytes, void *ctx) { return ((Arena *)ctx)->alloc(bytes); }
void arena_free_cb(void *p, size_t bytes, void *ctx) { ((Arena *)ctx)->release(p, bytes); }

// ------------------------------------------------------------------------------------
// Device descriptors
// ------------------------------------------------------------------------------------
constexpr int SV_MAXK = 21;   // DIA slots of the Q1 stiffness (9 in 2D, 21 in 3D)
constexpr int SV_MAXDEG = 4;  // Chebyshev degree supported by the server

struct SvLevel {  // one level of one request, FP32
    const float *val;  // DIA values (nullptr: a constant stencil, values in sv)
    int64_t ld;
    int K, n, N, dim;
    int slot;
    int32_t offs[SV_MAXK];
    int32_t pos[SV_MAXK];  // stencil: position (dx+1) + 3(dy+1) + 9(dz+1) of each slot
    float sv[SV_MAXK];     // stencil: the value of each slot
    float sdinv;           // stencil: 1 / a_ii
    float *x[2];
    float *b, *t, *d;
    float omega, c0;
    float c1[SV_MAXDEG], c2[SV_MAXDEG];
};

struct SvReq {  // one request's FP64 outer data and coarsest factors
    const double *A64;
    int64_t ld64;
    int K, n;
    int32_t offs[SV_MAXK];
    double *x64;
    const double *b64;
    const double *lu;
    const int *piv;
    int n0;
    int max_iters;
    double tol2;  // tol^2
};

struct SvState {  // mutable per slot, written only by the device after admission
    double norm2, nb2;
    unsigned ticket;
    int first;
    int converged;  // 0 running, 1 converged, 2 max_iters reached
    int iter;       // corrections applied so far
};

enum SvOp { OP_OUTER = 0, OP_SWEEP, OP_RESTRICT, OP_COARSE, OP_PROLONG, OP_UPDATE };

struct SvPhase {
    int op, mode, in, out, step;
    int item_off, nitems, ntiles;  // items carry their first tile index in .w
};

struct Plan {  // device-side layout of the per-composition plan buffer
    SvPhase *phases;
    int4 *items;
    SvLevel *levels;
    SvReq *reqs;
    SvState *state;
    double *partial;  // one slot per outer-residual tile
};

__device__ __forceinline__ bool slot_done(const Plan &P, int slot) { return P.state[slot].converged != 0; }

// item of phase tile t: the last item whose first tile (.w) is <= t
__device__ __forceinline__ int find_item(const int4 *items, int n, int t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (items[mid].w <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---- phase kernels (persistent: blocks stride over the phase's tiles) ----

template <int MODE, int RPT>
__device__ __forceinline__ void sv_sweep_tile(const SvLevel &L, int row0, int in, int out, int step)
{
    float c1 = MODE == SW_JACOBI || MODE == SW_JACOBI_Z ? L.omega : (MODE == SW_CHEB ? L.c1[step] : L.c0);
    float c2 = MODE == SW_CHEB ? L.c2[step] : 0.f;
    const float *x = L.x[in];
    float *o = MODE == SW_RESID ? L.t : L.x[out];
    for (int r = 0; r < RPT; r++) {
        int i = row0 + r * 256 + threadIdx.x;
        if (i >= L.n) return;
        if (!L.val) {  // constant stencil: the row's neighbours masked from its coordinates
            if (IsZero<MODE>::value) {
                sweep_out<float, MODE>(i, 0.f, L.sdinv, 0.f, L.b, o, L.d, c1, c2);
                continue;
            }
            const int n1 = L.N - 1;
            const int vx = i % n1, vy = (i / n1) % n1, vz = L.dim == 3 ? i / (n1 * n1) : 0;
            unsigned mx = 2u | (vx > 0 ? 1u : 0u) | (vx < n1 - 1 ? 4u : 0u);
            unsigned my = 2u | (vy > 0 ? 1u : 0u) | (vy < n1 - 1 ? 4u : 0u);
            unsigned m = ((my & 1u) ? mx : 0u) | ((my & 2u) ? mx << 3 : 0u) | ((my & 4u) ? mx << 6 : 0u);
            if (L.dim == 3) {
                unsigned mz = 2u | (vz > 0 ? 1u : 0u) | (vz < n1 - 1 ? 4u : 0u);
                m = ((mz & 1u) ? m : 0u) | ((mz & 2u) ? m << 9 : 0u) | ((mz & 4u) ? m << 18 : 0u);
            }
            const int cp = L.dim == 3 ? 13 : 4;  // the centre position
            float s = 0.f, xi = 0.f;
            if (L.K == 21) {
                float xv[21];
#pragma unroll
                for (int k = 0; k < 21; k++) xv[k] = __ldg(x + i + L.offs[k]);
#pragma unroll
                for (int k = 0; k < 21; k++)
                    if (L.pos[k] == cp || ((m >> L.pos[k]) & 1u)) s = fmaf(L.sv[k], xv[k], s);
                xi = xv[10];
            } else {
                float xv[9];
#pragma unroll
                for (int k = 0; k < 9; k++) xv[k] = __ldg(x + i + L.offs[k]);
#pragma unroll
                for (int k = 0; k < 9; k++)
                    if (L.pos[k] == cp || ((m >> L.pos[k]) & 1u)) s = fmaf(L.sv[k], xv[k], s);
                xi = xv[4];
            }
            sweep_out<float, MODE>(i, s, L.sdinv, xi, L.b, o, L.d, c1, c2);
            continue;
        }
        if (IsZero<MODE>::value) {
            float dg = __ldcs(L.val + (int64_t)(L.K / 2) * L.ld + i);
            sweep_out<float, MODE>(i, 0.f, Ar<float>::rcp(dg), 0.f, L.b, o, L.d, c1, c2);
            continue;
        }
        float s = 0.f, dg = 0.f, xi = 0.f;
        if (L.K == 21) {
            float a[21], xv[21];
#pragma unroll
            for (int k = 0; k < 21; k++) a[k] = __ldcs(L.val + (int64_t)k * L.ld + i);
#pragma unroll
            for (int k = 0; k < 21; k++) xv[k] = __ldg(x + i + L.offs[k]);
#pragma unroll
            for (int k = 0; k < 21; k++) s = fmaf(a[k], xv[k], s);
            dg = a[10];
            xi = xv[10];
        } else {
            float a[9], xv[9];
#pragma unroll
            for (int k = 0; k < 9; k++) a[k] = __ldcs(L.val + (int64_t)k * L.ld + i);
#pragma unroll
            for (int k = 0; k < 9; k++) xv[k] = __ldg(x + i + L.offs[k]);
#pragma unroll
            for (int k = 0; k < 9; k++) s = fmaf(a[k], xv[k], s);
            dg = a[4];
            xi = xv[4];
        }
        sweep_out<float, MODE>(i, s, Ar<float>::rcp(dg), xi, L.b, o, L.d, c1, c2);
    }
}

template <int MODE, int RPT>
__global__ void __launch_bounds__(256) k_sv_sweep(Plan P, int p)
{
    SvPhase ph = P.phases[p];
    const int4 *items = P.items + ph.item_off;
    for (int t = blockIdx.x; t < ph.ntiles; t += gridDim.x) {
        int4 it = items[find_item(items, ph.nitems, t)];
        const SvLevel &L = P.levels[it.x];
        if (slot_done(P, L.slot)) continue;
        sv_sweep_tile<MODE, RPT>(L, (t - it.w) * 256 * RPT, ph.in, ph.out, ph.step);
    }
}

template <int RPT>
__global__ void __launch_bounds__(256) k_sv_restrict(Plan P, int p)
{
    SvPhase ph = P.phases[p];
    const int4 *items = P.items + ph.item_off;
    for (int t = blockIdx.x; t < ph.ntiles; t += gridDim.x) {
        int4 it = items[find_item(items, ph.nitems, t)];
        const SvLevel &F = P.levels[it.x];
        const SvLevel &C = P.levels[it.y];
        if (slot_done(P, F.slot)) continue;
        const float *r = it.z ? F.b : F.t;  // no pre-smoothing: restrict b itself
        int nc1 = C.N - 1, nf1 = F.N - 1;
        int row0 = (t - it.w) * 256 * RPT;
        for (int q = 0; q < RPT; q++) {
            int I = row0 + q * 256 + threadIdx.x;
            if (I >= C.n) break;
            int X = I % nc1 + 1, Y = (I / nc1) % nc1 + 1;
            float s = 0.f;
            if (F.dim == 3) {
                int Z = I / (nc1 * nc1) + 1;
#pragma unroll
                for (int dz = -1; dz <= 1; dz++)
#pragma unroll
                    for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                        for (int dx = -1; dx <= 1; dx++) {
                            float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f) * (dz ? 0.5f : 1.f);
                            int64_t j = (2 * X + dx - 1) + (int64_t)nf1 * ((2 * Y + dy - 1) + (int64_t)nf1 * (2 * Z + dz - 1));
                            s = fmaf(w, __ldg(r + j), s);
                        }
            } else {
#pragma unroll
                for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                    for (int dx = -1; dx <= 1; dx++) {
                        float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f);
                        int64_t j = (2 * X + dx - 1) + (int64_t)nf1 * (2 * Y + dy - 1);
                        s = fmaf(w, __ldg(r + j), s);
                    }
            }
            C.b[I] = s;
        }
    }
}

template <int RPT>
__global__ void __launch_bounds__(256) k_sv_prolong(Plan P, int p)
{
    SvPhase ph = P.phases[p];
    const int4 *items = P.items + ph.item_off;
    for (int t = blockIdx.x; t < ph.ntiles; t += gridDim.x) {
        int4 it = items[find_item(items, ph.nitems, t)];
        const SvLevel &F = P.levels[it.x];
        const SvLevel &C = P.levels[it.y];
        if (slot_done(P, F.slot)) continue;
        const float *xc = C.x[it.z];
        float *xf = F.x[ph.out];
        int Nc = C.N, nf1 = F.N - 1, nc1 = Nc - 1;
        int row0 = (t - it.w) * 256 * RPT;
        for (int q = 0; q < RPT; q++) {
            int i = row0 + q * 256 + threadIdx.x;
            if (i >= F.n) break;
            int v0 = i % nf1 + 1, v1 = (i / nf1) % nf1 + 1, v2 = F.dim == 3 ? i / (nf1 * nf1) + 1 : 2;
            int odd = (v0 & 1) + (v1 & 1) + (F.dim == 3 ? (v2 & 1) : 0);
            float w = odd == 0 ? 1.f : (odd == 1 ? 0.5f : (odd == 2 ? 0.25f : 0.125f));
            int x0 = max(v0 >> 1, 1), x1 = min((v0 + 1) >> 1, Nc - 1);
            int y0 = max(v1 >> 1, 1), y1 = min((v1 + 1) >> 1, Nc - 1);
            int z0 = F.dim == 3 ? max(v2 >> 1, 1) : 1, z1 = F.dim == 3 ? min((v2 + 1) >> 1, Nc - 1) : 1;
            float acc = 0.f;
            for (int Z = z0; Z <= z1; Z++)
                for (int Y = y0; Y <= y1; Y++) {
                    int64_t row = (int64_t)nc1 * ((Y - 1) + (F.dim == 3 ? (int64_t)nc1 * (Z - 1) : 0)) - 1;
                    for (int X = x0; X <= x1; X++) acc = fmaf(w, __ldg(xc + row + X), acc);
                }
            xf[i] = xf[i] + acc;
        }
    }
}

// coarsest solve: one warp per request (n0 <= 64), the factors in shared memory
__global__ void __launch_bounds__(32) k_sv_coarse(Plan P, int p)
{
    SvPhase ph = P.phases[p];
    __shared__ double Ls[64 * 64];
    __shared__ double xs[64];
    __shared__ int ps[64];
    for (int it_i = blockIdx.x; it_i < ph.nitems; it_i += gridDim.x) {
        int4 it = P.items[ph.item_off + it_i];
        const SvReq &R = P.reqs[it.x];
        const SvLevel &C = P.levels[it.y];
        if (slot_done(P, it.x)) continue;
        int n = R.n0, l = threadIdx.x;
        __syncwarp();
        // stage the factors, pivots and right-hand side with independent loads in flight
        int pv0 = l < n ? R.piv[l] : 0, pv1 = l + 32 < n ? R.piv[l + 32] : 0;
#pragma unroll 8
        for (int k = l; k < n * n; k += 32) Ls[k] = R.lu[k];
        for (int k = l; k < n; k += 32) xs[k] = (double)C.b[k];
        if (l < n) ps[l] = pv0;
        if (l + 32 < n) ps[l + 32] = pv1;
        __syncwarp();
        if (l == 0)
            for (int k = 0; k < n; k++) {
                int q = ps[k];
                if (q != k) {
                    double tmp = xs[k];
                    xs[k] = xs[q];
                    xs[q] = tmp;
                }
            }
        __syncwarp();
        lu_substitute_warp(Ls, xs, n, l);
        for (int k = l; k < n; k += 32) C.x[0][k] = (float)xs[k];
    }
}

// FP64 outer residual r = b - A64 x64 per request, the norm of each request reduced in
// tile order by its last tile, and the convergence decision
template <int RPT>
__global__ void __launch_bounds__(256) k_sv_outer(Plan P, int p)
{
    SvPhase ph = P.phases[p];
    __shared__ double sh[32];
    __shared__ bool last;
    const int4 *items = P.items + ph.item_off;
    for (int t = blockIdx.x; t < ph.ntiles; t += gridDim.x) {
        int4 it = items[find_item(items, ph.nitems, t)];  // slot, finest level, tile count, first tile
        const SvReq &R = P.reqs[it.x];
        const SvLevel &F = P.levels[it.y];
        int row0 = (t - it.w) * 256 * RPT;
        double sq = 0.0;
        for (int q = 0; q < RPT; q++) {
            int i = row0 + q * 256 + threadIdx.x;
            if (i >= R.n) break;
            double s = 0.0;
            if (R.K == 21) {
#pragma unroll
                for (int k = 0; k < 21; k++)
                    s = __fma_rn(__ldcs(R.A64 + (int64_t)k * R.ld64 + i), __ldg(R.x64 + i + R.offs[k]), s);
            } else {
#pragma unroll
                for (int k = 0; k < 9; k++)
                    s = __fma_rn(__ldcs(R.A64 + (int64_t)k * R.ld64 + i), __ldg(R.x64 + i + R.offs[k]), s);
            }
            double ri = __dsub_rn(R.b64[i], s);
            F.b[i] = (float)ri;
            sq += ri * ri;
        }
        double bs = block_sum(sq, sh);
        if (threadIdx.x == 0) {
            P.partial[t] = bs;
            __threadfence();
            unsigned k = atomicAdd(&P.state[it.x].ticket, 1u);
            last = (k == (unsigned)it.z - 1);
        }
        __syncthreads();
        if (last) {
            __threadfence();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int k = 0; k < it.z; k++) tot += ((volatile double *)P.partial)[it.w + k];
                SvState &S = P.state[it.x];
                if (S.first) {
                    S.nb2 = tot;
                    S.first = 0;
                }
                S.norm2 = tot;
                if (tot <= R.tol2 * S.nb2) {
                    S.converged = 1;
                } else if (S.iter >= R.max_iters) {
                    S.converged = 2;
                } else {
                    S.converged = 0;
                    S.iter = S.iter + 1;  // this iteration's correction will be applied
                }
                S.ticket = 0u;
            }
        }
        __syncthreads();
    }
}

template <int RPT>
__global__ void __launch_bounds__(256) k_sv_update(Plan P, int p)
{
    SvPhase ph = P.phases[p];
    const int4 *items = P.items + ph.item_off;
    for (int t = blockIdx.x; t < ph.ntiles; t += gridDim.x) {
        int4 it = items[find_item(items, ph.nitems, t)];
        if (slot_done(P, it.x)) continue;
        const SvReq &R = P.reqs[it.x];
        const float *c = P.levels[it.y].x[ph.in];
        int row0 = (t - it.w) * 256 * RPT;
        for (int q = 0; q < RPT; q++) {
            int i = row0 + q * 256 + threadIdx.x;
            if (i >= R.n) break;
            R.x64[i] = __dadd_rn(R.x64[i], (double)c[i]);
        }
    }
}

// Right-hand side of a request given by sine modes (mg_serve_submit_rhs), formed on the
// device from its per-mode, per-axis factors: b_i = sum_m c[m] * ((v[m][0][ix] *
// v[m][1][iy]) [* v[m][2][iz]]), mode order, every product and sum rounded once (the
// evaluation of the host's mg_load_vector_separable, so both give the same bits).
// rv: nm x 3 x n1 factors then nm coefficients.
__global__ void __launch_bounds__(256) k_sv_rhs(double *__restrict__ b, const double *__restrict__ rv, int nm, int n1,
                                                int dim, int64_t n)
{
    const double *c = rv + (int64_t)nm * 3 * n1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t ix = i % n1, iy = (i / n1) % n1, iz = dim == 3 ? i / ((int64_t)n1 * n1) : 0;
        double s = 0.0;
        for (int m = 0; m < nm; m++) {
            const double *vm = rv + (int64_t)m * 3 * n1;
            double t = __dmul_rn(vm[ix], vm[n1 + iy]);
            if (dim == 3) t = __dmul_rn(t, vm[2 * n1 + iz]);
            s = __dadd_rn(s, __dmul_rn(c[m], t));
        }
        b[i] = s;
    }
}

// ------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------
struct OpSet {
    int dim = 0, N = 0, nlev = 0;
    mg_hierarchy *h = nullptr;
    int refs = 0;
    uint64_t last_use = 0;
    size_t bytes = 0;
};

struct Work {  // per-request device workspace (from the arena)
    std::vector<std::pair<void *, size_t>> blocks;
    std::vector<float *> x0, x1, b, t, d;  // per level
    double *x64 = nullptr, *b64 = nullptr;
    double *rv = nullptr;  // right-hand-side factors (requests given by sine modes)
};

struct Request {
    uint64_t ticket = 0;
    int dim = 0, N = 0, nlev = 0;
    double tol = 0;
    std::vector<double> b;
    std::vector<double> x;
    std::vector<double> hist;
    int iters = 0;
    mg_status status = MG_PENDING;
    std::string err;
    Clock::time_point t_submit, t_admit, t_done;
    OpSet *ops = nullptr;
    Work ws;
    int slot = -1;
    bool has_rhs = false;
    std::vector<double> amp;
    std::vector<int> freq;
    double f_const = 0.0;
    std::vector<double> rv;  // factors of the right-hand side (load_vector_factors), then c
    int nm = 0;
    int outcome = 0;  // after retirement: 1 converged, 2 max_iters reached
};

}  // namespace

struct mg_server {
    mg_device dev{};
    bool own_alloc = false;
    int device = 0;
    Arena arena;
    cudaStream_t s = nullptr;
    mg_options opt{};
    int max_active = 256;
    int rpt = 4;  // rows per thread (tile = 256 * rpt rows)
    int bps = 4;  // persistent blocks per SM
    int nsm = 0;
    std::mutex mu;
    std::condition_variable cv_sched, cv_setup, cv_done;
    std::deque<Request *> setup_q, ready_q;
    std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
    std::vector<Request *> active;       // admitted
    std::vector<int> free_slots;
    std::map<std::tuple<int, int, int>, std::unique_ptr<OpSet>> opsets;
    std::atomic<uint64_t> next_ticket{1};
    std::atomic<bool> stop{false};
    std::thread sched, setup;
    uint64_t clock = 0;
    // device plan buffers
    void *d_plan = nullptr;
    size_t plan_bytes = 0;
    char *h_plan = nullptr;  // pinned staging
    SvState *d_state = nullptr;
    SvState *h_state = nullptr;  // pinned
    double *d_partial = nullptr;
    int max_phases = 0, max_items = 0, max_tiles = 0;
    Plan plan{};
    bool plan_dirty = true;
    int cur_depth = -1;
    std::map<int, cudaGraphExec_t> graphs;  // by depth
    std::vector<SvPhase> phases;
    std::vector<int> phase_kernel;           // kernel id per phase (for capture)
    double *h_xstage = nullptr;              // pinned result staging
    size_t xstage_elems = 0;
    // ping-pong schedule (same for every request and level)
    int pre_cur = -1, post_cur = 0;
    std::vector<std::tuple<int, int, int, int>> pre_steps, post_steps;  // (mode, in, out, step)
    // statistics
    std::vector<double> latencies_ms;
    uint64_t completed = 0, cycles = 0, batch_sum = 0;
    double gpu_ms = 0.0, setup_ms = 0.0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // finished requests whose solutions are still on the device: copied back on the copy
    // stream while the next batched iteration runs
    cudaStream_t cs = nullptr;
    std::vector<Request *> draining;
    Clock::time_point t_first_submit, t_last_done;
    bool any_submit = false;
    std::string fatal;
};

static thread_local std::string g_setup_err;  // setup-thread failure detail

namespace {

int64_t level_pad(int dim, int N)
{
    int64_t n1 = N - 1;
    return rup(dim == 3 ? n1 * n1 + n1 + 1 : n1 + 1, 64);
}

// smoother step sequence: (mode, in, out, coefficient step) with buffer ping-pong
void make_schedule(mg_server *S)
{
    const mg_options &o = S->opt;
    auto apply = [&](int &c, std::vector<std::tuple<int, int, int, int>> &out) {
        if (o.smoother == MG_JACOBI) {
            if (c < 0) {
                out.emplace_back(SW_JACOBI_Z, 0, 0, 0);
                c = 0;
            } else {
                out.emplace_back(SW_JACOBI, c, 1 - c, 0);
                c = 1 - c;
            }
            return;
        }
        if (c < 0) {
            out.emplace_back(SW_CHEBF_Z, 0, 0, 0);
            c = 0;
        } else {
            out.emplace_back(SW_CHEBF, c, 1 - c, 0);
            c = 1 - c;
        }
        for (int j = 1; j < o.cheb_degree; j++) {
            out.emplace_back(SW_CHEB, c, 1 - c, j);
            c = 1 - c;
        }
    };
    int c = -1;
    S->pre_steps.clear();
    S->post_steps.clear();
    for (int a = 0; a < o.nu_pre; a++) apply(c, S->pre_steps);
    S->pre_cur = c;
    for (int a = 0; a < o.nu_post; a++) apply(c, S->post_steps);
    S->post_cur = c;
}

size_t workspace_bytes(const OpSet &ops)
{
    size_t tot = 0;
    for (int l = 0; l < ops.nlev; l++) {
        const mgi::LevelD &L = ops.h->lev[l];
        int64_t ld = L.A.ld, pad = level_pad(ops.dim, L.N);
        tot += 2 * rup((ld + 2 * pad) * 4, 256) + 3 * rup(ld * 4, 256);
    }
    const mgi::LevelD &F = ops.h->lev[ops.nlev - 1];
    tot += rup((F.A.ld + 2 * level_pad(ops.dim, F.N)) * 8, 256) + rup(F.A.ld * 8, 256);
    return tot;
}

bool alloc_workspace(mg_server *S, Request *r)
{
    OpSet &ops = *r->ops;
    Work &w = r->ws;
    auto take = [&](size_t bytes) -> void * {
        void *p = S->arena.alloc(bytes);
        if (p) w.blocks.emplace_back(p, bytes);
        return p;
    };
    bool ok = true;
    w.x0.assign(ops.nlev, nullptr);
    w.x1 = w.b = w.t = w.d = w.x0;
    for (int l = 0; l < ops.nlev && ok; l++) {
        const mgi::LevelD &L = ops.h->lev[l];
        int64_t ld = L.A.ld, pad = level_pad(ops.dim, L.N);
        char *a = (char *)take((ld + 2 * pad) * 4), *b = (char *)take((ld + 2 * pad) * 4);
        w.b[l] = (float *)take(ld * 4);
        w.t[l] = (float *)take(ld * 4);
        w.d[l] = (float *)take(ld * 4);
        ok = a && b && w.b[l] && w.t[l] && w.d[l];
        if (ok) {
            w.x0[l] = (float *)(a + pad * 4);
            w.x1[l] = (float *)(b + pad * 4);
        }
    }
    if (ok) {
        const mgi::LevelD &F = ops.h->lev[ops.nlev - 1];
        int64_t pad = level_pad(ops.dim, F.N);
        char *x = (char *)take((F.A.ld + 2 * pad) * 8);
        w.b64 = (double *)take(F.A.ld * 8);
        ok = x && w.b64;
        if (ok) w.x64 = (double *)(x + pad * 8);
        if (ok && r->has_rhs) {
            w.rv = (double *)take(r->rv.size() * 8);
            ok = w.rv != nullptr;
        }
    }
    if (!ok) {
        for (auto &bl : w.blocks) S->arena.release(bl.first, bl.second);
        w.blocks.clear();
    }
    return ok;
}

void free_workspace(mg_server *S, Request *r)
{
    for (auto &bl : r->ws.blocks) S->arena.release(bl.first, bl.second);
    r->ws.blocks.clear();
}

// evict cached operator sets nobody uses, least recently used first; true if any freed
bool evict_one(mg_server *S, const OpSet *keep)
{
    OpSet *victim = nullptr;
    std::tuple<int, int, int> vkey;
    for (auto &kv : S->opsets) {
        OpSet *o = kv.second.get();
        if (o->refs > 0 || o == keep) continue;
        if (!victim || o->last_use < victim->last_use) {
            victim = o;
            vkey = kv.first;
        }
    }
    if (!victim) return false;
    mg_hierarchy_free(victim->h);
    S->opsets.erase(vkey);
    return true;
}

// ---- plan: phases of one iteration for the admitted requests, aligned by depth ----
void build_plan(mg_server *S, std::vector<SvPhase> &phases, std::vector<int4> &items, std::vector<SvLevel> &levels,
                std::vector<SvReq> &reqs, int &depth)
{
    int tile_rows = 256 * S->rpt;
    phases.clear();
    items.clear();
    levels.clear();
    reqs.assign(S->max_active, SvReq{});
    depth = 0;
    // level table: per request, its levels (index base[r] + l)
    std::vector<int> base(S->active.size());
    for (size_t a = 0; a < S->active.size(); a++) {
        Request *r = S->active[a];
        OpSet &ops = *r->ops;
        mg_hierarchy *h = ops.h;
        depth = std::max(depth, ops.nlev - 1);
        base[a] = (int)levels.size();
        for (int l = 0; l < ops.nlev; l++) {
            const mgi::LevelD &L = h->lev[l];
            SvLevel v{};
            v.val = L.A.fmt == MG_STORAGE_STENCIL ? nullptr : (const float *)L.A.val;
            v.ld = L.A.ld;
            v.K = L.A.K;
            v.n = (int)L.n;
            v.N = L.N;
            v.dim = ops.dim;
            v.slot = r->slot;
            for (int k = 0; k < L.A.K && k < SV_MAXK; k++) {
                v.offs[k] = L.A.offs.o[k];
                v.pos[k] = L.A.full_of[k];
                v.sv[k] = (float)L.A.sval[k];
            }
            v.sdinv = (float)L.A.sdinv;
            v.x[0] = r->ws.x0[l];
            v.x[1] = r->ws.x1[l];
            v.b = r->ws.b[l];
            v.t = r->ws.t[l];
            v.d = r->ws.d[l];
            v.omega = (float)L.omega;
            v.c0 = (float)L.cheb_c0;
            for (int j = 0; j < SV_MAXDEG; j++) {
                v.c1[j] = j < (int)L.cheb_c1.size() ? (float)L.cheb_c1[j] : 0.f;
                v.c2[j] = j < (int)L.cheb_c2.size() ? (float)L.cheb_c2[j] : 0.f;
            }
            levels.push_back(v);
        }
        SvReq q{};
        q.A64 = (const double *)h->A64.val;
        q.ld64 = h->A64.ld;
        q.K = h->A64.K;
        q.n = (int)h->A64.n;
        for (int k = 0; k < h->A64.K && k < SV_MAXK; k++) q.offs[k] = h->A64.offs.o[k];
        q.x64 = r->ws.x64;
        q.b64 = r->ws.b64;
        q.lu = h->lu;
        q.piv = h->piv;
        q.n0 = h->n0;
        q.tol2 = r->tol * r->tol;
        q.max_iters = S->opt.max_iters;
        reqs[r->slot] = q;
    }
    auto add_phase = [&](int op, int mode, int in, int out, int step) -> SvPhase & {
        SvPhase ph{};
        ph.op = op;
        ph.mode = mode;
        ph.in = in;
        ph.out = out;
        ph.step = step;
        ph.item_off = (int)items.size();
        phases.push_back(ph);
        return phases.back();
    };
    auto add_item = [&](SvPhase &ph, int4 it, int rows) {
        it.w = ph.ntiles;  // first tile of this item within the phase
        items.push_back(it);
        ph.nitems++;
        ph.ntiles += (rows + tile_rows - 1) / tile_rows;
    };
    // outer residual
    {
        add_phase(OP_OUTER, 0, 0, 0, 0);
        for (size_t a = 0; a < S->active.size(); a++) {
            Request *r = S->active[a];
            int n = (int)r->ops->h->A64.n;
            int ntl = (n + tile_rows - 1) / tile_rows;
            add_item(phases.back(), make_int4(r->slot, base[a] + r->ops->nlev - 1, ntl, 0), n);
        }
    }
    // down: depth d acts on level L_r - d (>= 1) of every request deep enough
    for (int d = 0; d < depth; d++) {
        for (auto &st : S->pre_steps) {
            SvPhase &ph = add_phase(OP_SWEEP, std::get<0>(st), std::get<1>(st), std::get<2>(st), std::get<3>(st));
            for (size_t a = 0; a < S->active.size(); a++) {
                int l = S->active[a]->ops->nlev - 1 - d;
                if (l >= 1) add_item(phases.back(), make_int4(base[a] + l, 0, 0, 0), levels[base[a] + l].n);
            }
            (void)ph;
        }
        if (S->pre_cur >= 0) {
            add_phase(OP_SWEEP, SW_RESID, S->pre_cur, 0, 0);
            for (size_t a = 0; a < S->active.size(); a++) {
                int l = S->active[a]->ops->nlev - 1 - d;
                if (l >= 1) add_item(phases.back(), make_int4(base[a] + l, 0, 0, 0), levels[base[a] + l].n);
            }
        }
        add_phase(OP_RESTRICT, 0, 0, 0, 0);
        for (size_t a = 0; a < S->active.size(); a++) {
            int l = S->active[a]->ops->nlev - 1 - d;
            if (l >= 1)
                add_item(phases.back(), make_int4(base[a] + l, base[a] + l - 1, S->pre_cur < 0 ? 1 : 0, 0),
                         levels[base[a] + l - 1].n);
        }
        add_phase(OP_COARSE, 0, 0, 0, 0);
        for (size_t a = 0; a < S->active.size(); a++) {
            int l = S->active[a]->ops->nlev - 1 - d;
            if (l == 1) {
                SvPhase &ph = phases.back();
                items.push_back(make_int4(S->active[a]->slot, base[a], 0, 0));
                ph.nitems++;
            }
        }
    }
    // up
    for (int d = depth - 1; d >= 0; d--) {
        int pre_buf = S->pre_cur < 0 ? 0 : S->pre_cur;
        add_phase(OP_PROLONG, 0, 0, pre_buf, 0);
        for (size_t a = 0; a < S->active.size(); a++) {
            int l = S->active[a]->ops->nlev - 1 - d;
            if (l >= 1) {
                int cbuf = l - 1 == 0 ? 0 : S->post_cur;
                add_item(phases.back(), make_int4(base[a] + l, base[a] + l - 1, cbuf, 0), levels[base[a] + l].n);
            }
        }
        for (auto &st : S->post_steps) {
            add_phase(OP_SWEEP, std::get<0>(st), std::get<1>(st), std::get<2>(st), std::get<3>(st));
            for (size_t a = 0; a < S->active.size(); a++) {
                int l = S->active[a]->ops->nlev - 1 - d;
                if (l >= 1) add_item(phases.back(), make_int4(base[a] + l, 0, 0, 0), levels[base[a] + l].n);
            }
        }
    }
    // x += c (the finest correction is in buffer post_cur; a one-level request: buffer 0)
    add_phase(OP_UPDATE, 0, S->post_cur, 0, 0);
    for (size_t a = 0; a < S->active.size(); a++) {
        Request *r = S->active[a];
        add_item(phases.back(), make_int4(r->slot, base[a] + r->ops->nlev - 1, 0, 0), (int)r->ops->h->A64.n);
    }
}

template <int RPT>
void launch_phase(mg_server *S, const SvPhase &ph, int p, cudaStream_t s)
{
    int grid = S->nsm * S->bps;
    switch (ph.op) {
    case OP_OUTER: k_sv_outer<RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
    case OP_RESTRICT: k_sv_restrict<RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
    case OP_PROLONG: k_sv_prolong<RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
    case OP_COARSE: k_sv_coarse<<<std::min(S->max_active, 4 * S->nsm), 32, 0, s>>>(S->plan, p); break;
    case OP_UPDATE: k_sv_update<RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
    default:
        switch (ph.mode) {
        case SW_RESID: k_sv_sweep<SW_RESID, RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
        case SW_JACOBI: k_sv_sweep<SW_JACOBI, RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
        case SW_CHEBF: k_sv_sweep<SW_CHEBF, RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
        case SW_CHEB: k_sv_sweep<SW_CHEB, RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
        case SW_JACOBI_Z: k_sv_sweep<SW_JACOBI_Z, RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
        default: k_sv_sweep<SW_CHEBF_Z, RPT><<<grid, 256, 0, s>>>(S->plan, p); break;
        }
    }
}

void enqueue_cycle(mg_server *S, cudaStream_t s)
{
    for (size_t p = 0; p < S->phases.size(); p++) {
        switch (S->rpt) {
        case 1: launch_phase<1>(S, S->phases[p], (int)p, s); break;
        case 2: launch_phase<2>(S, S->phases[p], (int)p, s); break;
        case 8: launch_phase<8>(S, S->phases[p], (int)p, s); break;
        default: launch_phase<4>(S, S->phases[p], (int)p, s); break;
        }
        SCK(cudaGetLastError());
    }
}

// upload the plan for the admitted set; returns the depth
int upload_plan(mg_server *S)
{
    std::vector<SvPhase> phases;
    std::vector<int4> items;
    std::vector<SvLevel> levels;
    std::vector<SvReq> reqs;
    int depth = 0;
    build_plan(S, phases, items, levels, reqs, depth);
    if ((int)phases.size() > S->max_phases || (int)items.size() > S->max_items ||
        (int)levels.size() > S->max_active * MG_MAX_LEVELS || phases[0].ntiles > S->max_tiles)
        throw Error(MG_ENOMEM, "serving plan exceeds its capacity");
    // packed layout inside the plan buffer (fixed offsets)
    char *hp = S->h_plan;
    size_t off_ph = 0, off_it = rup((int64_t)S->max_phases * sizeof(SvPhase), 256);
    size_t off_lv = off_it + rup((int64_t)S->max_items * sizeof(int4), 256);
    size_t off_rq = off_lv + rup((int64_t)S->max_active * MG_MAX_LEVELS * sizeof(SvLevel), 256);
    std::memcpy(hp + off_ph, phases.data(), phases.size() * sizeof(SvPhase));
    std::memcpy(hp + off_it, items.data(), items.size() * sizeof(int4));
    std::memcpy(hp + off_lv, levels.data(), levels.size() * sizeof(SvLevel));
    std::memcpy(hp + off_rq, reqs.data(), reqs.size() * sizeof(SvReq));
    size_t bytes = off_rq + reqs.size() * sizeof(SvReq);
    SCK(cudaMemcpyAsync(S->d_plan, hp, bytes, cudaMemcpyHostToDevice, S->s));
    S->phases = phases;
    return depth;
}

cudaGraphExec_t graph_for(mg_server *S, int depth)
{
    auto it = S->graphs.find(depth);
    if (it != S->graphs.end()) return it->second;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    SCK(cudaStreamBeginCapture(S->s, cudaStreamCaptureModeThreadLocal));
    try {
        enqueue_cycle(S, S->s);
    } catch (...) {
        cudaStreamEndCapture(S->s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    SCK(cudaStreamEndCapture(S->s, &g));
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) throw Error(MG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    S->graphs[depth] = ge;
    return ge;
}

void finish_request(mg_server *S, Request *r, mg_status st, const std::string &err)
{
    r->status = st;
    r->err = err;
    r->t_done = Clock::now();
    if (st == MG_OK || st == MG_ENOCONV) {
        S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        S->completed++;
        S->t_last_done = r->t_done;
    }
    r->b.clear();
    r->b.shrink_to_fit();
    r->rv.clear();
    r->rv.shrink_to_fit();
}

// device bytes of a Q1 operator set (FP32 level matrices, FP64 finest matrix, LU and
// small buffers), from the level sizes: 21 stored diagonals in 3D, 9 in 2D
size_t opset_bytes_estimate(int dim, int N, int nlev)
{
    int K = dim == 3 ? 21 : 9;
    size_t tot = 4096;
    for (int l = 0; l < nlev; l++) {
        int64_t ld = rup(std::max<int64_t>(mgh::ndofs(dim, MG_Q1, N >> (nlev - 1 - l)), 1), 64);
        tot += (size_t)rup((int64_t)K * ld * 4, 256);
        if (l == nlev - 1) tot += (size_t)rup((int64_t)K * ld * 8, 256) + (size_t)rup((ld + 255) / 256 * 8, 256);
    }
    int64_t n0 = mgh::ndofs(dim, MG_Q1, N >> (nlev - 1));
    tot += (size_t)rup(n0 * n0 * 8, 256) + (size_t)rup(n0 * 4, 256);
    return tot;
}

// ---- setup thread: right-hand sides and operator sets ----
OpSet *get_opset(mg_server *S, int dim, int N, int nlev, std::unique_lock<std::mutex> &lk)
{
    auto key = std::make_tuple(dim, N, nlev);
    auto it = S->opsets.find(key);
    if (it != S->opsets.end()) return it->second.get();
    // an operator set larger than the whole budget can never be admitted
    if (opset_bytes_estimate(dim, N, nlev) > S->arena.size) {
        g_setup_err = "operator set larger than the budget";
        return nullptr;
    }
    // build outside the lock (host assembly and upload take time)
    lk.unlock();
    mg_problem p{dim, MG_Q1, N, nlev, nullptr};
    mg_options o = S->opt;
    o.precision = MG_MIXED;
    // FP32 levels of at least 32768 rows as the constant stencil (every request has k = 1),
    // the smaller ones in DIA: the same storage mg_setup gives MG_STORAGE_STENCIL
    o.storage = MG_STORAGE_STENCIL;
    o.use_graph = 0;
    mg_device dev{arena_alloc_cb, arena_free_cb, &S->arena, nullptr};
    std::unique_ptr<OpSet> ops(new OpSet());
    ops->dim = dim;
    ops->N = N;
    ops->nlev = nlev;
    mg_status st = MG_ENOMEM;
    std::string err;
    for (int attempt = 0; attempt < 64 && !S->stop; attempt++) {
        std::unique_ptr<mg_hierarchy> h(new mg_hierarchy());
        try {
            mgi::build_hierarchy(h.get(), &p, &o, &dev, false);
            ops->h = h.release();
            ops->bytes = ops->h->slab.size;
            st = MG_OK;
            break;
        } catch (const Error &e) {
            st = e.st;
            err = e.msg;
        }
        if (st != MG_ENOMEM) break;
        // out of budget: evict an unused operator set or wait for requests to finish
        lk.lock();
        bool freed = evict_one(S, nullptr);
        if (!freed) S->cv_setup.wait_for(lk, std::chrono::milliseconds(20));
        lk.unlock();
    }
    lk.lock();
    if (st != MG_OK) {
        g_setup_err = err;
        return nullptr;
    }
    OpSet *raw = ops.get();
    S->opsets[key] = std::move(ops);
    return raw;
}

void setup_loop(mg_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        if (S->setup_q.empty()) {
            S->cv_setup.wait(lk);
            continue;
        }
        Request *r = S->setup_q.front();
        S->setup_q.pop_front();
        auto t0 = Clock::now();
        if (r->has_rhs) {  // the per-mode, per-axis factors; the device forms b at admission
            lk.unlock();
            mg_rhs f{(int)r->amp.size(), r->amp.data(), r->freq.data(), r->f_const};
            std::vector<double> c;
            mgh::load_vector_factors(r->dim, r->N, &f, r->rv, c);
            r->nm = (int)c.size();
            r->rv.insert(r->rv.end(), c.begin(), c.end());
            lk.lock();
        }
        OpSet *ops = get_opset(S, r->dim, r->N, r->nlev, lk);
        S->setup_ms += std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
        if (!ops) {
            finish_request(S, r, MG_EBUDGET, "operators do not fit the device budget: " + g_setup_err);
            S->cv_done.notify_all();
            continue;
        }
        ops->refs++;
        r->ops = ops;
        S->ready_q.push_back(r);
        S->cv_sched.notify_all();
    }
}

// ---- scheduler thread ----
void admit(mg_server *S)
{
    bool changed = false;
    while (!S->ready_q.empty() && !S->free_slots.empty()) {
        Request *r = S->ready_q.front();
        if (!alloc_workspace(S, r)) {
            if (!S->active.empty()) break;  // wait for retirements
            if (evict_one(S, r->ops)) continue;
            S->ready_q.pop_front();
            r->ops->refs--;
            finish_request(S, r, MG_EBUDGET, "request does not fit the device budget");
            S->cv_done.notify_all();
            continue;
        }
        S->ready_q.pop_front();
        r->slot = S->free_slots.back();
        S->free_slots.pop_back();
        r->t_admit = Clock::now();
        const mgi::LevelD &F = r->ops->h->lev[r->ops->nlev - 1];
        int64_t n = F.n, pad = level_pad(r->dim, F.N);
        // zero the padded iterate (x0 = 0, zero halo) and the level vectors' halos
        SCK(cudaMemsetAsync((char *)r->ws.x64 - pad * 8, 0, (size_t)(F.A.ld + 2 * pad) * 8, S->s));
        for (int l = 0; l < r->ops->nlev; l++) {
            const mgi::LevelD &L = r->ops->h->lev[l];
            int64_t pl = level_pad(r->dim, L.N);
            SCK(cudaMemsetAsync((char *)r->ws.x0[l] - pl * 4, 0, (size_t)(L.A.ld + 2 * pl) * 4, S->s));
            SCK(cudaMemsetAsync((char *)r->ws.x1[l] - pl * 4, 0, (size_t)(L.A.ld + 2 * pl) * 4, S->s));
        }
        if (r->has_rhs) {
            SCK(cudaMemcpyAsync(r->ws.rv, r->rv.data(), r->rv.size() * 8, cudaMemcpyHostToDevice, S->s));
            int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)S->nsm * 8);
            k_sv_rhs<<<grid, 256, 0, S->s>>>(r->ws.b64, r->ws.rv, r->nm, F.N - 1, r->dim, n);
            SCK(cudaGetLastError());
        } else {
            SCK(cudaMemcpyAsync(r->ws.b64, r->b.data(), (size_t)n * 8, cudaMemcpyHostToDevice, S->s));
        }
        SvState init{};
        init.first = 1;
        SCK(cudaMemcpyAsync(&S->d_state[r->slot], &init, sizeof(SvState), cudaMemcpyHostToDevice, S->s));
        S->active.push_back(r);
        changed = true;
    }
    if (changed) S->plan_dirty = true;
}

// requests that met their tolerance (or max_iters) leave the batch: their slots are free
// at once, their workspaces once their solutions have been copied back (drain)
void retire(mg_server *S)
{
    std::vector<Request *> keep;
    bool changed = false;
    for (Request *r : S->active) {
        SvState &st = S->h_state[r->slot];
        double rel = st.nb2 > 0.0 ? std::sqrt(st.norm2 / st.nb2) : std::sqrt(st.norm2);
        r->hist.push_back(rel);
        r->iters = st.iter;
        if (st.converged == 0) {
            keep.push_back(r);
            continue;
        }
        S->free_slots.push_back(r->slot);
        r->slot = -1;
        r->outcome = st.converged;
        S->draining.push_back(r);
        changed = true;
    }
    S->active.swap(keep);
    if (changed) S->plan_dirty = true;
}

// copy the solutions of the retired requests to the host (copy stream, pinned staging),
// called without the lock while the next iteration runs on the compute stream; the
// requests' workspaces are not in that iteration's plan
void drain_copy(mg_server *S, const std::vector<Request *> &batch)
{
    for (Request *r : batch) {
        int64_t n = r->ops->h->A64.n;
        if ((size_t)n > S->xstage_elems) {
            if (S->h_xstage) cudaFreeHost(S->h_xstage);
            S->h_xstage = nullptr;
            SCK(cudaMallocHost(&S->h_xstage, (size_t)n * 8));
            S->xstage_elems = (size_t)n;
        }
        SCK(cudaMemcpyAsync(S->h_xstage, r->ws.x64, (size_t)n * 8, cudaMemcpyDeviceToHost, S->cs));
        SCK(cudaStreamSynchronize(S->cs));
        r->x.assign(S->h_xstage, S->h_xstage + n);
    }
}

// with the lock: release the drained requests' workspaces and finish them
void drain_finish(mg_server *S, const std::vector<Request *> &batch)
{
    for (Request *r : batch) {
        bool done = r->outcome == 1;
        free_workspace(S, r);
        r->ops->refs--;
        r->ops->last_use = ++S->clock;
        finish_request(S, r, done ? MG_OK : MG_ENOCONV, done ? "" : "max_iters reached");
    }
    if (!batch.empty()) {
        S->cv_done.notify_all();
        S->cv_setup.notify_all();
    }
}

void sched_loop(mg_server *S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    try {
        while (!S->stop) {
            admit(S);
            std::vector<Request *> batch;
            batch.swap(S->draining);
            if (S->active.empty()) {
                if (!batch.empty()) {  // nothing to overlap with: copy back now
                    lk.unlock();
                    drain_copy(S, batch);
                    lk.lock();
                    drain_finish(S, batch);
                    continue;
                }
                S->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
            if (S->plan_dirty) {
                S->cur_depth = upload_plan(S);
                S->plan_dirty = false;
            }
            cudaGraphExec_t g = graph_for(S, S->cur_depth);
            // the graph's phase count depends only on the depth; contents come from the plan
            lk.unlock();
            SCK(cudaEventRecord(S->ev0, S->s));
            SCK(cudaGraphLaunch(g, S->s));
            SCK(cudaEventRecord(S->ev1, S->s));
            SCK(cudaMemcpyAsync(S->h_state, S->d_state, sizeof(SvState) * S->max_active, cudaMemcpyDeviceToHost, S->s));
            drain_copy(S, batch);  // overlaps the iteration just launched
            SCK(cudaStreamSynchronize(S->s));
            float gms = 0.f;
            SCK(cudaEventElapsedTime(&gms, S->ev0, S->ev1));
            lk.lock();
            drain_finish(S, batch);
            S->gpu_ms += gms;
            S->cycles++;
            S->batch_sum += S->active.size();
            retire(S);
        }
    } catch (const Error &e) {
        S->fatal = e.msg;
        for (Request *r : S->active) finish_request(S, r, e.st, e.msg);
        for (Request *r : S->draining) finish_request(S, r, e.st, e.msg);
        S->active.clear();
        S->draining.clear();
        S->cv_done.notify_all();
    }
}

}  // namespace

// ------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------
extern "C" void mg_serve_config_default(mg_serve_config *c)
{
    std::memset(c, 0, sizeof(*c));
    c->hbm_budget_bytes = (size_t)4 << 30;
    c->max_active = 256;
    c->rows_per_thread = 4;
    c->blocks_per_sm = 4;
    mg_options_default(&c->options);
    c->options.smoother = MG_CHEBYSHEV;
    c->options.nu_pre = 1;
    c->options.nu_post = 1;
    c->options.precision = MG_MIXED;
}

extern "C" mg_status mg_serve_create(const mg_serve_config *cfg, const mg_device *dev, mg_server **out)
{
    if (!cfg || !out) {
        mgi::set_error("NULL argument");
        return MG_EINVAL;
    }
    *out = nullptr;
    std::unique_ptr<mg_server> S(new mg_server());
    try {
        const mg_options &o = cfg->options;
        if (o.smoother == MG_GAUSS_SEIDEL)
            throw Error(MG_EINVAL, "the Gauss-Seidel smoother is not available to the serving API");
        if (o.smoother != MG_JACOBI && o.smoother != MG_CHEBYSHEV) throw Error(MG_EINVAL, "bad smoother");
        if (o.smoother == MG_CHEBYSHEV && (o.cheb_degree < 1 || o.cheb_degree > SV_MAXDEG))
            throw Error(MG_EINVAL, "serving supports Chebyshev degree 1..4");
        if (o.nu_pre < 1 || o.nu_post < 0) throw Error(MG_EINVAL, "serving needs nu_pre >= 1");
        if (cfg->max_active < 1 || cfg->max_active > 4096) throw Error(MG_EINVAL, "max_active out of range");
        if (cfg->rows_per_thread != 1 && cfg->rows_per_thread != 2 && cfg->rows_per_thread != 4 &&
            cfg->rows_per_thread != 8)
            throw Error(MG_EINVAL, "rows_per_thread must be 1, 2, 4 or 8");
        if (cfg->blocks_per_sm < 1 || cfg->blocks_per_sm > 8) throw Error(MG_EINVAL, "blocks_per_sm out of range");
        S->opt = o;
        S->opt.precision = MG_MIXED;
        S->max_active = cfg->max_active;
        S->rpt = cfg->rows_per_thread;
        S->bps = cfg->blocks_per_sm;
        if (dev) S->dev = *dev;
        S->own_alloc = !S->dev.alloc;
        SCK(cudaGetDevice(&S->device));
        SCK(cudaDeviceGetAttribute(&S->nsm, cudaDevAttrMultiProcessorCount, S->device));
        SCK(cudaStreamCreateWithFlags(&S->s, cudaStreamNonBlocking));
        SCK(cudaStreamCreateWithFlags(&S->cs, cudaStreamNonBlocking));
        SCK(cudaEventCreate(&S->ev0));
        SCK(cudaEventCreate(&S->ev1));
        size_t budget = (size_t)rup((int64_t)cfg->hbm_budget_bytes, 256);
        void *base = nullptr;
        if (S->own_alloc) {
            if (cudaMalloc(&base, budget) != cudaSuccess) {
                cudaGetLastError();
                throw Error(MG_ENOMEM, "cannot reserve the serving budget");
            }
        } else {
            base = S->dev.alloc(budget, S->dev.ctx);
            if (!base) throw Error(MG_ENOMEM, "cannot reserve the serving budget");
        }
        S->arena.init((char *)base, budget);
        make_schedule(S.get());
        // plan capacity
        int steps = (int)(S->pre_steps.size() + S->post_steps.size());
        S->max_phases = 2 + MG_MAX_LEVELS * (steps + 4);
        S->max_items = S->max_phases * S->max_active;
        S->max_tiles = 1 << 20;  // outer-residual tiles per iteration (partial sums)
        size_t off = 0;
        off += rup((int64_t)S->max_phases * sizeof(SvPhase), 256);
        size_t off_it = off;
        off += rup((int64_t)S->max_items * sizeof(int4), 256);
        size_t off_lv = off;
        off += rup((int64_t)S->max_active * MG_MAX_LEVELS * sizeof(SvLevel), 256);
        size_t off_rq = off;
        off += rup((int64_t)S->max_active * sizeof(SvReq), 256);
        S->plan_bytes = off;
        S->d_plan = S->arena.alloc(off);
        S->d_state = (SvState *)S->arena.alloc(sizeof(SvState) * S->max_active);
        S->d_partial = (double *)S->arena.alloc(sizeof(double) * S->max_tiles);
        if (!S->d_plan || !S->d_state || !S->d_partial) throw Error(MG_ENOMEM, "budget too small for the plan buffers");
        SCK(cudaMallocHost(&S->h_plan, off));
        SCK(cudaMallocHost(&S->h_state, sizeof(SvState) * S->max_active));
        SCK(cudaMemset(S->d_state, 0, sizeof(SvState) * S->max_active));
        char *dp = (char *)S->d_plan;
        S->plan.phases = (SvPhase *)dp;
        S->plan.items = (int4 *)(dp + off_it);
        S->plan.levels = (SvLevel *)(dp + off_lv);
        S->plan.reqs = (SvReq *)(dp + off_rq);
        S->plan.state = S->d_state;
        S->plan.partial = S->d_partial;
        for (int k = S->max_active - 1; k >= 0; k--) S->free_slots.push_back(k);
        mg_server *raw = S.get();
        S->sched = std::thread(sched_loop, raw);
        S->setup = std::thread(setup_loop, raw);
    } catch (const Error &e) {
        mgi::set_error(e.msg);
        return e.st;
    }
    *out = S.release();
    return MG_OK;
}

static mg_status submit_common(mg_server *S, const mg_problem *p, const double *b_host, const mg_rhs *f, double tol,
                               uint64_t *ticket)
{
    if (!S || !p || !ticket) {
        mgi::set_error("NULL argument");
        return MG_EINVAL;
    }
    if (p->element != MG_Q1 || p->k_cell || mg_ndofs(p->dim, p->element, p->n_cells) < 0 || p->n_levels < 2 ||
        p->n_levels > MG_MAX_LEVELS) {
        mgi::set_error("serving takes Q1 Poisson problems (k = 1) with at least two levels");
        return MG_EINVAL;
    }
    int Nc = p->n_cells >> (p->n_levels - 1);
    if (Nc < 2 || (Nc << (p->n_levels - 1)) != p->n_cells) {
        mgi::set_error("n_cells must be the coarsest size (>= 2) times 2^(n_levels-1)");
        return MG_EINVAL;
    }
    int64_t n0 = mgh::ndofs(p->dim, MG_Q1, Nc);
    if (n0 > 64) {
        mgi::set_error("serving needs a coarsest level of at most 64 DOFs");
        return MG_EINVAL;
    }
    if (!(tol > 0.0)) {
        mgi::set_error("tolerance must be positive");
        return MG_EINVAL;
    }
    std::unique_ptr<Request> r(new Request());
    r->dim = p->dim;
    r->N = p->n_cells;
    r->nlev = p->n_levels;
    r->tol = tol;
    int64_t n = mgh::ndofs(p->dim, MG_Q1, p->n_cells);
    if (b_host) {
        for (int64_t i = 0; i < n; i++)
            if (!std::isfinite(b_host[i])) {
                mgi::set_error("the right-hand side holds a NaN or an infinity");
                return MG_EINVAL;
            }
        r->b.assign(b_host, b_host + n);
    } else {
        if (!f || f->n_modes < 0 || (f->n_modes > 0 && (!f->amp || !f->freq))) {
            mgi::set_error("bad right-hand side");
            return MG_EINVAL;
        }
        bool finite = std::isfinite(f->f_const);
        for (int m = 0; m < f->n_modes; m++) finite = finite && std::isfinite(f->amp[m]);
        if (!finite) {
            mgi::set_error("the right-hand side holds a NaN or an infinity");
            return MG_EINVAL;
        }
        r->has_rhs = true;
        r->amp.assign(f->amp, f->amp + f->n_modes);
        r->freq.assign(f->freq, f->freq + 3 * f->n_modes);
        r->f_const = f->f_const;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->fatal.empty()) {
        mgi::set_error("server stopped: " + S->fatal);
        return MG_ECUDA;
    }
    r->ticket = S->next_ticket++;
    r->t_submit = Clock::now();
    if (!S->any_submit) {
        S->any_submit = true;
        S->t_first_submit = r->t_submit;
    }
    *ticket = r->ticket;
    Request *raw = r.get();
    S->reqs[r->ticket] = std::move(r);
    S->setup_q.push_back(raw);
    S->cv_setup.notify_all();
    return MG_OK;
}

extern "C" mg_status mg_serve_submit(mg_server *S, const mg_problem *p, const double *b_host, double rel_tol,
                                     uint64_t *ticket)
{
    if (!b_host) {
        mgi::set_error("b_host is NULL");
        return MG_EINVAL;
    }
    return submit_common(S, p, b_host, nullptr, rel_tol, ticket);
}

extern "C" mg_status mg_serve_submit_rhs(mg_server *S, const mg_problem *p, const mg_rhs *f, double rel_tol,
                                         uint64_t *ticket)
{
    return submit_common(S, p, nullptr, f, rel_tol, ticket);
}

static mg_status take_result(mg_server *S, uint64_t ticket, double *x_host, int *iters, double *res_hist,
                             int hist_len)
{
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
        mgi::set_error("unknown ticket");
        return MG_ENOTFOUND;
    }
    Request *r = it->second.get();
    if (r->status == MG_PENDING) return MG_PENDING;
    mg_status st = r->status;
    if (x_host && !r->x.empty()) std::memcpy(x_host, r->x.data(), r->x.size() * 8);
    if (iters) *iters = r->iters;
    if (res_hist)
        for (int k = 0; k < hist_len && k < (int)r->hist.size(); k++) res_hist[k] = r->hist[k];
    if (st != MG_OK) mgi::set_error(r->err);
    S->reqs.erase(it);
    return st;
}

extern "C" mg_status mg_serve_poll(mg_server *S, uint64_t ticket, double *x_host, int *iters)
{
    if (!S) {
        mgi::set_error("NULL server");
        return MG_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    return take_result(S, ticket, x_host, iters, nullptr, 0);
}

extern "C" mg_status mg_serve_wait(mg_server *S, uint64_t ticket, double timeout_s, double *x_host, int *iters,
                                   double *res_hist, int hist_len)
{
    if (!S) {
        mgi::set_error("NULL server");
        return MG_EINVAL;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    for (;;) {
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) {
            mgi::set_error("unknown ticket");
            return MG_ENOTFOUND;
        }
        if (it->second->status != MG_PENDING) return take_result(S, ticket, x_host, iters, res_hist, hist_len);
        if (!S->fatal.empty()) {
            mgi::set_error("server stopped: " + S->fatal);
            return MG_ECUDA;
        }
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            mgi::set_error("wait timed out");
            return MG_ETIMEOUT;
        }
    }
}

extern "C" mg_status mg_serve_get_stats(mg_server *S, mg_serve_stats *out)
{
    if (!S || !out) {
        mgi::set_error("NULL argument");
        return MG_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = S->completed;
    out->cycles = S->cycles;
    out->active = (int)S->active.size();
    out->queued = (int)(S->setup_q.size() + S->ready_q.size());
    out->mean_batch = S->cycles ? (double)S->batch_sum / (double)S->cycles : 0.0;
    out->device_bytes_in_use = S->arena.in_use;
    out->device_bytes_peak = S->arena.peak;
    out->operator_sets = (int)S->opsets.size();
    out->gpu_ms = S->gpu_ms;
    out->setup_ms = S->setup_ms;
    if (!S->latencies_ms.empty()) {
        std::vector<double> v = S->latencies_ms;
        std::sort(v.begin(), v.end());
        auto q = [&](double f) { return v[std::min(v.size() - 1, (size_t)std::floor(f * (double)(v.size() - 1) + 0.5))]; };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = v.back();
        double span = std::chrono::duration<double>(S->t_last_done - S->t_first_submit).count();
        out->solves_per_s = span > 0 ? (double)S->completed / span : 0.0;
        out->span_ms = 1e3 * span;
    }
    return MG_OK;
}

extern "C" mg_status mg_serve_reset_stats(mg_server *S)
{
    if (!S) {
        mgi::set_error("NULL server");
        return MG_EINVAL;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    S->latencies_ms.clear();
    S->completed = S->cycles = S->batch_sum = 0;
    S->gpu_ms = S->setup_ms = 0.0;
    S->any_submit = false;
    S->arena.peak = S->arena.in_use;
    return MG_OK;
}

// Autotuner: time every candidate tile shape on `repeats` copies of each given shape,
// solved together as one batch (right-hand side f = 1), and keep the fastest.
extern "C" mg_status mg_serve_tune(mg_server *S, const mg_problem *shapes, int nshapes, int repeats, double rel_tol,
                                   int *rows_per_thread, int *blocks_per_sm)
{
    if (!S || !shapes || nshapes < 1 || repeats < 1) {
        mgi::set_error("bad arguments");
        return MG_EINVAL;
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (!S->active.empty() || !S->ready_q.empty() || !S->setup_q.empty()) {
            mgi::set_error("mg_serve_tune needs an idle server");
            return MG_EINVAL;
        }
    }
    static const int rpts[] = {1, 2, 4, 8};
    static const int bpss[] = {2, 4, 8};
    double best = 1e300;
    int best_r = S->rpt, best_b = S->bps;
    mg_rhs f{0, nullptr, nullptr, 1.0};
    for (int r : rpts)
        for (int b : bpss) {
            {
                std::lock_guard<std::mutex> lk(S->mu);
                S->rpt = r;
                S->bps = b;
                for (auto &kv : S->graphs) cudaGraphExecDestroy(kv.second);
                S->graphs.clear();
                S->plan_dirty = true;
            }
            for (int pass = 0; pass < 2; pass++) {  // the first pass builds graphs and caches
                std::vector<uint64_t> tickets;
                auto t0 = Clock::now();
                for (int k = 0; k < repeats; k++)
                    for (int s = 0; s < nshapes; s++) {
                        uint64_t t = 0;
                        mg_status st = mg_serve_submit_rhs(S, &shapes[s], &f, rel_tol, &t);
                        if (st != MG_OK) return st;
                        tickets.push_back(t);
                    }
                for (uint64_t t : tickets) {
                    mg_status st = mg_serve_wait(S, t, 600.0, nullptr, nullptr, nullptr, 0);
                    if (st != MG_OK && st != MG_ENOCONV) return st;
                }
                double dt = std::chrono::duration<double>(Clock::now() - t0).count();
                if (pass == 1 && dt < best) {
                    best = dt;
                    best_r = r;
                    best_b = b;
                }
            }
        }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->rpt = best_r;
        S->bps = best_b;
        for (auto &kv : S->graphs) cudaGraphExecDestroy(kv.second);
        S->graphs.clear();
        S->plan_dirty = true;
    }
    mg_serve_reset_stats(S);
    if (rows_per_thread) *rows_per_thread = best_r;
    if (blocks_per_sm) *blocks_per_sm = best_b;
    return MG_OK;
}

extern "C" mg_status mg_serve_destroy(mg_server *S)
{
    if (!S) return MG_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_sched.notify_all();
    S->cv_setup.notify_all();
    if (S->sched.joinable()) S->sched.join();
    if (S->setup.joinable()) S->setup.join();
    cudaStreamSynchronize(S->s);
    for (auto &kv : S->graphs) cudaGraphExecDestroy(kv.second);
    for (auto &kv : S->opsets) mg_hierarchy_free(kv.second->h);
    S->opsets.clear();
    if (S->h_plan) cudaFreeHost(S->h_plan);
    if (S->h_state) cudaFreeHost(S->h_state);
    if (S->h_xstage) cudaFreeHost(S->h_xstage);
    if (S->arena.base) {
        if (S->own_alloc)
            cudaFree(S->arena.base);
        else if (S->dev.free)
            S->dev.free(S->arena.base, S->arena.size, S->dev.ctx);
    }
    if (S->cs) {
        cudaStreamSynchronize(S->cs);
        cudaStreamDestroy(S->cs);
    }
    if (S->ev0) cudaEventDestroy(S->ev0);
    if (S->ev1) cudaEventDestroy(S->ev1);
    if (S->s) cudaStreamDestroy(S->s);
    delete S;
    return MG_OK;
}

