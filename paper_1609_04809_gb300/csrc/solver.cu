// solver.cu -- device hierarchy, V-cycle schedule, CUDA graphs and the C ABI of libmg.so.
//
// One defect-correction iteration is two CUDA graphs replayed on a private stream:
//   G_r: FP64 outer residual r = b - A64 x64 (written in the inner precision into the
//        finest level's right-hand side) and ||r||^2;
//   G_v: one V-cycle on that right-hand side (Sec. 5.3: pre-smoothing, restriction of
//        the residual level by level, exact coarsest solve, prolongation with
//        correction and post-smoothing on the way up), then x64 += c.
// The host reads ||r||^2 after G_r (one 8-byte copy) for the stopping test.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <string>
#include <vector>

#include "host_setup.h"
#include "kernels.cuh"
#include "gs.cuh"
#include "krylov.cuh"
#include "heat.cuh"
#include "mg.h"
#include "mg_internal.h"

using namespace mgk;

// ------------------------------------------------------------------------------------
// Errors
// ------------------------------------------------------------------------------------
static thread_local std::string g_err;

namespace mgi {
void set_error(const std::string &m) { g_err = m; }
}  // namespace mgi

extern "C" const char *mg_last_error(void) { return g_err.c_str(); }

#define CK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) throw mgi::Error(MG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CKL()                                                                                       \
    do {                                                                                            \
        cudaError_t e_ = cudaGetLastError();                                                        \
        if (e_ != cudaSuccess) throw mgi::Error(MG_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

// ------------------------------------------------------------------------------------
// Non-template kernels
// ------------------------------------------------------------------------------------
namespace mgk {
__global__ void k_lu_factor(double *a, int n, int *piv, int *info)
{
    __shared__ int p_sh;
    int t = threadIdx.x;
    for (int k = 0; k < n; k++) {
        if (t == 0) {
            int p = k;
            double best = fabs(a[(int64_t)k * n + k]);
            for (int i = k + 1; i < n; i++) {
                double v = fabs(a[(int64_t)i * n + k]);
                if (v > best) {
                    best = v;
                    p = i;
                }
            }
            piv[k] = p;
            p_sh = p;
            if (best == 0.0) *info = 1;
        }
        __syncthreads();
        int p = p_sh;
        if (p != k)
            for (int j = t; j < n; j += blockDim.x) {
                double tmp = a[(int64_t)k * n + j];
                a[(int64_t)k * n + j] = a[(int64_t)p * n + j];
                a[(int64_t)p * n + j] = tmp;
            }
        __syncthreads();
        for (int i = k + 1 + t; i < n; i += blockDim.x) {
            double l = __ddiv_rn(a[(int64_t)i * n + k], a[(int64_t)k * n + k]);
            a[(int64_t)i * n + k] = l;
            for (int j = k + 1; j < n; j++)
                a[(int64_t)i * n + j] = __dsub_rn(a[(int64_t)i * n + j], __dmul_rn(l, a[(int64_t)k * n + j]));
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256, 6) k_norm2(const double *__restrict__ v, int n, double *partial, unsigned *ticket,
                                               double *norm2)
{
    double sq = 0.0;
    const int st = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * st < n; i += 4 * st) {  // four loads in flight, rows in order
        double v0 = v[i], v1 = v[i + st], v2 = v[i + 2 * st], v3 = v[i + 3 * st];
        sq = __fma_rn(v0, v0, sq);
        sq = __fma_rn(v1, v1, sq);
        sq = __fma_rn(v2, v2, sq);
        sq = __fma_rn(v3, v3, sq);
    }
    for (; i < n; i += st) sq = __fma_rn(v[i], v[i], sq);
    finish_norm(sq, partial, ticket, norm2);
}

__global__ void k_coef_dinv(const float *__restrict__ kap, int n1, float *__restrict__ dinv)
{
    const int vx = blockIdx.x * blockDim.x + threadIdx.x, vy = blockIdx.y, vz = blockIdx.z;
    if (vx >= n1) return;
    const int64_t nc = n1 + 1;
    const float *k0 = kap + vx + nc * (vy + nc * (int64_t)vz), *k1 = k0 + nc * nc;
    const float kc = (k0[0] + k0[1]) + (k0[nc] + k0[nc + 1]), kn = (k1[0] + k1[1]) + (k1[nc] + k1[nc + 1]);
    dinv[vx + (int64_t)n1 * (vy + (int64_t)n1 * vz)] = Ar<float>::rcp(4.0f * (kc + kn));
}
}  // namespace mgk

// ------------------------------------------------------------------------------------
// Helpers
// ------------------------------------------------------------------------------------
using mgi::DevMat;
using mgi::Error;
using mgi::LevelD;

static inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }
static inline unsigned grid_for(int64_t n) { return (unsigned)((n + 255) / 256); }
// grid of a kernel that ends in a block-partial reduction (finish_norm)
static inline unsigned reduce_grid(int64_t n) { return std::min<unsigned>(std::max<unsigned>(grid_for(n), 1u), kReduceBlocks); }
// grid of a kernel that applies an FP64 operator row by row: one wave at the residency it
// is compiled for (mgk::fp64_rows_blocks_per_sm; the storage codes equal its FMT codes)
static inline unsigned fp64_rows_grid(const DevMat &A, int64_t n)
{
    return std::min<unsigned>(reduce_grid(n), 152u * (unsigned)mgk::fp64_rows_blocks_per_sm(A.fmt));
}

// threads per block of a row sweep: 256, or 64 below two blocks of 256 per SM of the 152,
// so that the few rows of a small level spread over every SM (rows are independent)
static inline unsigned sweep_block(int64_t n) { return n < 152 * 256 * 2 ? 64u : 256u; }

// threads per block of a transfer over grid lines of l1 points: the line rounded up to
// whole warps, at most 128 (a 128-thread block over a 63-point line idles half its threads)
static inline unsigned line_block(unsigned l1) { return std::min(128u, std::max(32u, (l1 + 31) / 32 * 32)); }

// f(std::integral_constant<int, K>()) for the stored slot count K of a DIA matrix: the
// instantiated counts are 7 and 15 (P1, P1 + mass), 9 (2D Q1), 21 and 27 (3D Q1).
template <typename F>
static void with_dia_k(int K, F &&f)
{
    switch (K) {
    case 7: f(std::integral_constant<int, 7>()); break;
    case 9: f(std::integral_constant<int, 9>()); break;
    case 15: f(std::integral_constant<int, 15>()); break;
    case 21: f(std::integral_constant<int, 21>()); break;
    case 27: f(std::integral_constant<int, 27>()); break;
    default: throw mgi::Error(MG_EINVAL, "no DIA kernel for " + std::to_string(K) + " stored diagonals");
    }
}

void mgi::Slab::reserve(size_t bytes)
{
    used = round_up((int64_t)used, 256) + bytes;
}

void *mgi::Slab::take(size_t bytes)
{
    size_t off = (size_t)round_up((int64_t)used, 256);
    if (off + bytes > size) throw Error(MG_ENOMEM, "device slab overflow");
    used = off + bytes;
    return base + off;
}

template <typename T>
static MatView<T> view(const DevMat &m)
{
    MatView<T> v;
    v.val = (const T *)m.val;
    v.col = m.col;
    v.rowptr = m.rowptr;
    v.perm = m.perm;
    v.dinv = (const T *)m.dinv;
    v.ld = m.ld;
    v.K = m.K;
    v.center = m.center;
    v.offs = m.offs;
    return v;
}

// ------------------------------------------------------------------------------------
// Profiling: CUDA events around launches
// ------------------------------------------------------------------------------------
void mgi::Prof::begin(cudaStream_t s, int kclass, int level, double bytes, double flops, std::vector<Rec> *sink,
                      bool capturing)
{
    Rec r;
    r.kclass = kclass;
    r.level = level;
    r.bytes = bytes;
    r.flops = flops;
    CK(cudaEventCreate(&r.e0));
    CK(cudaEventCreate(&r.e1));
    if (capturing)
        CK(cudaEventRecordWithFlags(r.e0, s, cudaEventRecordExternal));
    else
        CK(cudaEventRecord(r.e0, s));
    sink->push_back(r);
}

void mgi::Prof::end(cudaStream_t s, std::vector<Rec> *sink, bool capturing)
{
    Rec &r = sink->back();
    if (capturing)
        CK(cudaEventRecordWithFlags(r.e1, s, cudaEventRecordExternal));
    else
        CK(cudaEventRecord(r.e1, s));
}

void mgi::Prof::collect(std::vector<Rec> &recs)
{
    for (auto &r : recs) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.e0, r.e1));
        int k = r.kclass * MG_MAX_LEVELS + r.level;
        ms_total[k] += ms;
        launches[k] += 1;
        bytes_total[k] += r.bytes;
        flops_total[k] += r.flops;
    }
}

void mgi::Prof::release(std::vector<Rec> &recs)
{
    for (auto &r : recs) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    recs.clear();
}

// ------------------------------------------------------------------------------------
// The hierarchy
// ------------------------------------------------------------------------------------
static void destroy_graphs(mg_hierarchy *h)
{
    if (h->g_r) cudaGraphExecDestroy(h->g_r);
    if (h->g_v) cudaGraphExecDestroy(h->g_v);
    if (h->g_pi) cudaGraphExecDestroy(h->g_pi);
    if (h->g_pc) cudaGraphExecDestroy(h->g_pc);
    h->g_r = h->g_v = h->g_pi = h->g_pc = nullptr;
    h->prof.release(h->rec_r);
    h->prof.release(h->rec_v);
    h->prof.release(h->rec_pi);
    h->prof.release(h->rec_pc);
}

mg_hierarchy::~mg_hierarchy()
{
    destroy_graphs(this);
    prof.release(rec_eager);
    if (s) cudaStreamSynchronize(s);
    if (slab.base) {
        if (own_alloc)
            cudaFree(slab.base);
        else if (dev.free)
            dev.free(slab.base, slab.size, dev.ctx);
    }
    if (h_norm2) cudaFreeHost(h_norm2);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (s) cudaStreamDestroy(s);
}

// launch bookkeeping: profiling events and launch counting
struct LaunchScope {
    mg_hierarchy *h;
    cudaStream_t s;
    bool on;
    LaunchScope(mg_hierarchy *h_, cudaStream_t s_, int kclass, int level, double bytes, double flops = 0.0)
        : h(h_), s(s_)
    {
        if (h->counting) h->kernels_per_cycle++;
        on = h->profiling && ((h->prof_class_mask >> kclass) & 1) && ((h->prof_level_mask >> level) & 1);
        if (on) h->prof.begin(s, kclass, level, bytes, flops, h->sink, h->capturing);
    }
    ~LaunchScope() noexcept(false)
    {
        if (on) h->prof.end(s, h->sink, h->capturing);
    }
};

static double mat_bytes(const DevMat &m, int sv)
{
    switch (m.fmt) {
    case MG_STORAGE_DIA: return (double)m.K * (double)m.n * sv;
    case MG_STORAGE_STENCIL: return 0.0;  // the values are launch parameters
    case MG_STORAGE_COEF: return 4.0 * (double)(m.n1 + 1) * (m.n1 + 1) * (m.n1 + 1);  // one FP32 value per cell
    case MG_STORAGE_ELL: return (double)m.K * (double)m.n * (sv + 4);
    case MG_STORAGE_SELL: return (double)m.padded * (sv + 4) + 8.0 * (double)(m.nslices + 1) + 4.0 * (double)m.n;
    default: return (double)m.nnz * (sv + 4) + 8.0 * (double)(m.n + 1);
    }
}

// stored entries one pass over the matrix multiplies (padding included)
static double mat_entries(const DevMat &m)
{
    switch (m.fmt) {
    case MG_STORAGE_CSR: return (double)m.nnz;
    case MG_STORAGE_SELL: return (double)m.padded;
    default: return (double)m.K * (double)m.n;
    }
}

// ------------------------------------------------------------------------------------
// Kernel dispatch
// ------------------------------------------------------------------------------------
// Launch with programmatic dependent launch when pdl is set: the kernel may be scheduled
// while the previous one in the stream finishes; it waits for it in pdl_enter().
template <typename... KArgs, typename... Args>
static void klaunch(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                    Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    if (e != cudaSuccess) throw Error(MG_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

// stencil position sets with fixed-position kernels: bit (dx+1) + 3(dy+1) + 9(dz+1)
constexpr unsigned kStencil27 = 0x7FFFFFFu;  // every position (Q1 + mass shift)
constexpr unsigned kFaces = (1u << 4) | (1u << 10) | (1u << 12) | (1u << 14) | (1u << 16) | (1u << 22);
constexpr unsigned kStencilQ1 = kStencil27 & ~kFaces;   // 3D Q1: face couplings are zero
constexpr unsigned kStencilP1 = kFaces | (1u << 13);    // P1 on the Kuhn mesh: seven points
constexpr unsigned kStencil9 = 0x1FFu;                  // 2D Q1

// whether a sweep of this level can also apply the finest correction to x64 (fused_update)
template <typename T>
static bool can_fuse_update(const DevMat &A)
{
    if (!std::is_same<T, float>::value) return false;
    if (A.fmt == MG_STORAGE_COEF) return true;
    if (A.fmt != MG_STORAGE_STENCIL) return false;
    if (A.elem == MG_RQ1) return true;
    unsigned pm = 0;
    for (int k = 0; k < A.K; k++) pm |= 1u << A.full_of[k];
    return A.dim == 3 && (pm == kStencilQ1 || pm == kStencil27 || pm == kStencilP1);
}

// upd: x64 for the sweep that also applies the correction (only where can_fuse_update)
template <typename T, int MODE>
static void sweep_fmt(const DevMat &A, int n, const T *x, const T *b, T *out, T *d, T c1, T c2, cudaStream_t s,
                      bool pdl = false, double *upd = nullptr)
{
    if (upd && !can_fuse_update<T>(A)) throw Error(MG_EINVAL, "this storage does not apply the update");
    if (A.fmt == MG_STORAGE_COEF) {
        if constexpr (std::is_same<T, float>::value) {
            // planes per thread: up to 16, fewer where the columns alone would not give about
            // MG_COEF_THREADS threads on each of the 152 SMs (two waves of 2048)
            int n1 = A.n1;
            int zc = (int)std::max<int64_t>(1, std::min<int64_t>(16, (int64_t)n1 * n1 * n1 / ((int64_t)MG_COEF_THREADS * 152)));
            CoefView S{(const float *)A.val, n1, zc};
            unsigned bx = line_block((unsigned)n1), by = std::min(256u / bx, (unsigned)n1);
            dim3 g((unsigned)((n1 + bx - 1) / bx), (unsigned)((n1 + by - 1) / by), (unsigned)((n1 + zc - 1) / zc)),
                blk(bx, by);
            if constexpr (MODE == SW_RESID) {  // the pair-carrying march: faster for the residual
                klaunch(pdl, k_coef_resid<SW_RESID>, g, blk, 0, s, S, x, b, out, d, c1, c2, upd);
                return;
            }
            klaunch(pdl, k_coef_sweep<MODE>, g, blk, 0, s, S, x, b, out, d, c1, c2, upd);
            return;
        } else {
            throw Error(MG_EINVAL, "coefficient storage holds FP32 levels only");
        }
    }
    if (A.fmt == MG_STORAGE_STENCIL && A.elem == MG_RQ1) {
        if constexpr (std::is_same<T, float>::value) {
            // slabs per thread: up to 8, fewer where the blocks would not give about two
            // waves of 2048 threads on each of the 152 SMs
            unsigned N = (unsigned)(A.n1 + 1), bx = line_block(N), by = std::min(256u / bx, N);
            int cz = (int)std::max<int64_t>(1, std::min<int64_t>(8, 3 * (int64_t)N * N * N / (2 * 2048 * 152)));
            Rq1View S{A.n1 + 1, (float)A.sval[1], (float)A.sdinv, cz};
            dim3 g((N + bx - 1) / bx, (N + by - 1) / by, 3 * ((N + cz - 1) / cz)), blk(bx, by);
            klaunch(pdl, k_stencil_rq1<MODE>, g, blk, 0, s, S, x, b, out, d, c1, c2, upd);
            return;
        } else {
            throw Error(MG_EINVAL, "the face stencil holds FP32 levels only");
        }
    }
    if (A.fmt == MG_STORAGE_STENCIL) {
        StencilView<T> S{};
        for (int k = 0; k < A.K; k++) {
            S.a[k] = (T)A.sval[k];
            S.off[k] = A.offs.o[k];
            S.pos[k] = A.full_of[k];
        }
        S.dinv = (T)A.sdinv;
        S.n1 = A.n1;
        unsigned n1 = (unsigned)A.n1, bx = line_block(n1), by = std::min(256u / bx, n1);
        dim3 g((n1 + bx - 1) / bx, (n1 + by - 1) / by, A.dim == 3 ? n1 : 1u), blk(bx, by);
        unsigned pm = 0;  // the stored positions; the common sets have fixed-position kernels
        for (int k = 0; k < A.K; k++) pm |= 1u << A.full_of[k];
        if (A.dim == 3 && (pm == kStencilQ1 || pm == kStencil27 || pm == kStencilP1)) {
            // 3D: each thread marches along z through up to 16 planes of its column (fewer where
            // the columns alone would not give about two waves of 2048 threads per SM)
            int zc = (int)std::max<int64_t>(1, std::min<int64_t>(16, (int64_t)n1 * n1 * n1 / (2 * 2048 * 152)));
            dim3 gz(g.x, g.y, (n1 + zc - 1) / zc);
            if (pm == kStencilQ1)
                klaunch(pdl, k_stencil_march<T, kStencilQ1, MODE>, gz, blk, 0, s, S, zc, x, b, out, d, c1, c2, upd);
            else if (pm == kStencil27)
                klaunch(pdl, k_stencil_march<T, kStencil27, MODE>, gz, blk, 0, s, S, zc, x, b, out, d, c1, c2, upd);
            else
                klaunch(pdl, k_stencil_march<T, kStencilP1, MODE>, gz, blk, 0, s, S, zc, x, b, out, d, c1, c2, upd);
            return;
        }
        if (A.dim == 2 && pm == kStencil9) {
            klaunch(pdl, k_stencil_fixed<T, kStencil9, MODE, 2>, g, blk, 0, s, S, x, b, out, d, c1, c2);
            return;
        }
        with_dia_k(A.K, [&](auto k) {
            if (A.dim == 3)
                klaunch(pdl, k_stencil_sweep<T, decltype(k)::value, MODE, 3>, g, blk, 0, s, S, x, b, out, d, c1, c2);
            else
                klaunch(pdl, k_stencil_sweep<T, decltype(k)::value, MODE, 2>, g, blk, 0, s, S, x, b, out, d, c1, c2);
        });
        return;
    }
    MatView<T> v = view<T>(A);
    unsigned bs = sweep_block(n);
    dim3 g((unsigned)((n + bs - 1) / bs)), blk(bs);
    if (A.fmt == MG_STORAGE_DIA) {
        with_dia_k(A.K, [&](auto k) {
            klaunch(pdl, k_dia_sweep<T, decltype(k)::value, MODE>, g, blk, 0, s, v, n, x, b, out, d, c1, c2);
        });
    } else if (A.fmt == MG_STORAGE_ELL) {
        klaunch(pdl, k_ell_sweep<T, MODE>, g, blk, 0, s, v, n, x, b, out, d, c1, c2);
    } else if (A.fmt == MG_STORAGE_SELL) {
        klaunch(pdl, k_sell_sweep<T, MODE>, g, blk, 0, s, v, n, x, b, out, d, c1, c2);
    } else {
        klaunch(pdl, k_csr_sweep<T, MODE>, g, blk, 0, s, v, n, x, b, out, d, c1, c2);
    }
}

template <typename T>
static void sweep(mg_hierarchy *h, int l, int mode, const T *x, const T *b, T *out, T *d, double c1, double c2,
                  cudaStream_t s, bool fuse = false)
{
    LevelD &L = h->lev[l];
    // the iteration's update x64 += c in this sweep (the finest level's last one), where the
    // level's storage has a kernel that applies it
    double *upd = fuse && l == h->Lf && !(h->tail_rec && l <= h->tail_level) && can_fuse_update<T>(L.A) ? h->x64
                                                                                                       : nullptr;
    if (upd) h->update_fused = true;
    if (h->tail_rec && l <= h->tail_level) {  // part of the coarse-level tail launch
        TailOp op{};
        op.kind = TAIL_SWEEP;
        op.level = l;
        op.mode = mode;
        op.in = x == (const T *)L.x[1] ? 1 : 0;
        op.out = out == (T *)L.t ? 2 : (out == (T *)L.x[1] ? 1 : 0);
        op.c1 = c1;
        op.c2 = c2;
        h->tail_ops.push_back(op);
        return;
    }
    int sv = sizeof(T);
    double n = (double)L.n;
    double bytes;
    int kclass;
    bool zero = mode == SW_JACOBI_Z || mode == SW_CHEBF_Z;
    if (zero) {  // the diagonal (stored D^-1, the DIA diagonal slot, or a row scan), b, out [, d]
        kclass = MG_K_SMOOTH0;
        double diag = L.A.fmt == MG_STORAGE_STENCIL
                          ? 0.0
                          : (L.A.dinv ? n * sv : (L.A.fmt == MG_STORAGE_DIA ? n * sv : mat_bytes(L.A, sv)));
        bytes = diag + 2 * n * sv + (mode == SW_CHEBF_Z ? n * sv : 0);
    } else {  // the matrix, x, b, out [, D^-1] [, d read and/or write]
        kclass = mode == SW_RESID ? MG_K_RESID : MG_K_SMOOTH;
        bytes = mat_bytes(L.A, sv) + 3 * n * sv;
        if (mode != SW_RESID && L.A.dinv && sv == 8) bytes += n * sv;  // FP32 sweeps use rcp(a_ii)
        if (mode == SW_CHEBF) bytes += n * sv;
        if (mode == SW_CHEB) bytes += 2 * n * sv;
    }
    if (upd) bytes += 16 * n;  // x64 read and written
    // algorithmic flops: two per stored entry (a multiply-add) plus the update's operations
    static const int kUpdateOps[6] = {1, 4, 4, 6, 2, 2};
    double entries = mat_entries(L.A);
    double flops = (zero ? 0.0 : 2.0 * entries) + kUpdateOps[mode] * n;
    LaunchScope ls(h, s, kclass, l, bytes, flops);
    int nn = (int)L.n;
    T a = (T)c1, bb = (T)c2;
    bool pdl = h->opt.use_pdl != 0;
    switch (mode) {
    case SW_RESID: sweep_fmt<T, SW_RESID>(L.A, nn, x, b, out, d, a, bb, s, pdl, upd); break;
    case SW_JACOBI: sweep_fmt<T, SW_JACOBI>(L.A, nn, x, b, out, d, a, bb, s, pdl, upd); break;
    case SW_CHEBF: sweep_fmt<T, SW_CHEBF>(L.A, nn, x, b, out, d, a, bb, s, pdl, upd); break;
    case SW_CHEB: sweep_fmt<T, SW_CHEB>(L.A, nn, x, b, out, d, a, bb, s, pdl, upd); break;
    case SW_JACOBI_Z: sweep_fmt<T, SW_JACOBI_Z>(L.A, nn, x, b, out, d, a, bb, s, pdl, upd); break;
    default: sweep_fmt<T, SW_CHEBF_Z>(L.A, nn, x, b, out, d, a, bb, s, pdl, upd); break;
    }
}

// one smoother application on level l; c: buffer holding x (-1: x = 0); returns new buffer
// one multicolour Gauss-Seidel sweep of level l on x in place: one launch per colour
// (or per pair of mutually uncoupled colours), colours ascending (descending in
// post-smoothing)
template <typename T>
static void gs_sweep(mg_hierarchy *h, int l, T *x, bool post, cudaStream_t s)
{
    LevelD &L = h->lev[l];
    const DevMat &G = L.G;
    MatView<T> v = view<T>(G);
    int ng = (int)L.gs_groups.size(), sv = sizeof(T);
    bool pdl = h->opt.use_pdl != 0;
    const T *b = (const T *)L.b;
    for (int gg = 0; gg < ng; gg++) {
        const auto &grp = L.gs_groups[post ? ng - 1 - gg : gg];
        int64_t r0 = grp.first;
        int nr = (int)(grp.second - r0);
        if (nr == 0) continue;
        // the colour's slice of the matrix (values, columns), perm, D^-1, b, and x read
        // and written at its rows; gathers of x at other rows count as cache hits
        double per_row = G.fmt == MG_STORAGE_CSR ? 0.0 : (double)G.K * (sv + (G.fmt == MG_STORAGE_ELL ? 4 : 0));
        double slice = G.fmt == MG_STORAGE_CSR
                           ? (double)(L.nnz) * (sv + 4) * nr / std::max<int64_t>(L.n, 1) + 8.0 * nr
                           : per_row * nr;
        double bytes = slice + nr * (4.0 + 3.0 * sv + (G.dinv ? sv : 0));
        double entries = G.fmt == MG_STORAGE_CSR ? (double)L.nnz * nr / std::max<int64_t>(L.n, 1) : (double)G.K * nr;
        LaunchScope ls(h, s, MG_K_SMOOTH, l, bytes, 2.0 * entries + 4.0 * nr);
        unsigned bs = sweep_block(nr);
        dim3 g((unsigned)((nr + bs - 1) / bs)), blk(bs);
        if (G.fmt == MG_STORAGE_DIA) {
            with_dia_k(G.K, [&](auto k) {
                klaunch(pdl, k_gs_dia<T, decltype(k)::value>, g, blk, 0, s, v, (const int32_t *)L.perm, r0, nr, x, b);
            });
        } else if (G.fmt == MG_STORAGE_ELL) {
            klaunch(pdl, k_gs_ell<T>, g, blk, 0, s, v, (const int32_t *)L.perm, r0, nr, x, b);
        } else {
            klaunch(pdl, k_gs_csr<T>, g, blk, 0, s, v, (const int32_t *)L.perm, r0, nr, x, b);
        }
    }
}

template <typename T>
static int smooth(mg_hierarchy *h, int l, int c, bool post, cudaStream_t s, bool fuse_last = false,
                  bool first_done = false)
{
    // first_done: the step from x = 0 was taken by the kernel that made the level's
    // right-hand side (zfuse, outer_z)
    LevelD &L = h->lev[l];
    T *b = (T *)L.b, *d = (T *)L.d;
    const int last = h->opt.smoother == MG_JACOBI ? 0 : h->opt.cheb_degree - 1;  // the last step of this application
    if (h->opt.smoother == MG_GAUSS_SEIDEL) {  // in place: the buffer does not change
        if (c < 0) {
            CK(cudaMemsetAsync(L.x[0], 0, (size_t)L.n * sizeof(T), s));
            c = 0;
        }
        gs_sweep<T>(h, l, (T *)L.x[c], post, s);
        return c;
    }
    if (h->opt.smoother == MG_JACOBI) {
        if (c < 0) {
            if (!first_done) sweep<T>(h, l, SW_JACOBI_Z, nullptr, b, (T *)L.x[0], d, L.omega, 0.0, s, fuse_last);
            return 0;
        }
        sweep<T>(h, l, SW_JACOBI, (T *)L.x[c], b, (T *)L.x[1 - c], d, L.omega, 0.0, s, fuse_last);
        return 1 - c;
    }
    if (c < 0) {
        if (!first_done)
            sweep<T>(h, l, SW_CHEBF_Z, nullptr, b, (T *)L.x[0], d, L.cheb_c0, 0.0, s, fuse_last && last == 0);
        c = 0;
    } else {
        sweep<T>(h, l, SW_CHEBF, (T *)L.x[c], b, (T *)L.x[1 - c], d, L.cheb_c0, 0.0, s, fuse_last && last == 0);
        c = 1 - c;
    }
    for (int j = 1; j < h->opt.cheb_degree; j++) {
        sweep<T>(h, l, SW_CHEB, (T *)L.x[c], b, (T *)L.x[1 - c], d, L.cheb_c1[j], L.cheb_c2[j], s,
                 fuse_last && j == last);
        c = 1 - c;
    }
    return c;
}

// The first pre-smoothing step of level l (from x = 0) as a ZStep for the kernel that
// produces the level's right-hand side; bytes: what that step adds to the kernel's traffic
template <typename T>
static mgk::ZStep<T> zstep_of(mg_hierarchy *h, int l, double *bytes)
{
    LevelD &L = h->lev[l];
    const DevMat &M = L.A;
    const int sv = sizeof(T);
    mgk::ZStep<T> Z{};
    if (M.fmt == MG_STORAGE_COEF)
        Z.dinv = (const T *)L.zdinv;
    else if (M.fmt == MG_STORAGE_STENCIL)
        Z.cdinv = (T)M.sdinv;
    else if (M.dinv)  // FP64 levels; FP32 ELL, CSR and SELL levels
        Z.dinv = (const T *)M.dinv;
    else if (M.fmt == MG_STORAGE_DIA)
        Z.diag = (const T *)M.val + (int64_t)M.center * M.ld;
    else
        throw Error(MG_EINVAL, "level has no diagonal for the fused first smoothing step");
    if (M.fmt == MG_STORAGE_COEF && !L.zdinv) throw Error(MG_EINVAL, "coefficient level without D^-1");
    const bool cheb = h->opt.smoother == MG_CHEBYSHEV;
    Z.out = (T *)L.x[0];
    Z.d = (T *)L.d;
    Z.c1 = (T)(cheb ? L.cheb_c0 : L.omega);
    *bytes += (M.fmt == MG_STORAGE_STENCIL ? 0.0 : (double)L.n * sv) + (cheb ? 2.0 : 1.0) * L.n * sv;
    return Z;
}

// zf: level l - 1's first smoothing step rides on the restriction (zfuse)
template <typename T>
static void restrict_to(mg_hierarchy *h, int l, const T *r, cudaStream_t s, bool zf = false)
{
    LevelD &F = h->lev[l], &C = h->lev[l - 1];
    if (h->tail_rec && l <= h->tail_level) {
        TailOp op{};
        op.kind = TAIL_RESTRICT;
        op.level = l;
        op.aux = r == (const T *)F.b ? 1 : 0;
        h->tail_ops.push_back(op);
        return;
    }
    int sv = sizeof(T);
    double bytes = (double)F.n * sv + (double)C.n * sv;
    if (!F.structured) bytes += mat_bytes(F.R, sv);
    mgk::ZStep<T> Z{};
    if (zf) Z = zstep_of<T>(h, l - 1, &bytes);
    LaunchScope ls(h, s, MG_K_RESTRICT, l, bytes);
    const bool pdl = h->opt.use_pdl != 0;
    auto go = [&](auto zm) {
        constexpr int ZM = decltype(zm)::value;
        if (F.structured) {
            unsigned l1 = (unsigned)(C.N - 1), bx = line_block(l1);
            dim3 g((l1 + bx - 1) / bx, l1, h->dim == 3 ? l1 : 1);
            if (h->dim == 3)
                klaunch(pdl, k_restrict_q1<T, 3, ZM>, g, dim3(bx), 0, s, r, (T *)C.b, C.N, Z);
            else
                klaunch(pdl, k_restrict_q1<T, 2, ZM>, g, dim3(bx), 0, s, r, (T *)C.b, C.N, Z);
        } else {  // explicit R in SELL-32
            klaunch(pdl, k_sell_apply<T, false, ZM>, dim3(grid_for(C.n)), dim3(256), 0, s,
                    (const int64_t *)F.R.rowptr, (const int32_t *)F.R.col, (const T *)F.R.val,
                    (const int32_t *)F.R.perm, (int)C.n, r, (T *)C.b, Z);
        }
    };
    if (!zf)
        go(std::integral_constant<int, 0>());
    else if (h->opt.smoother == MG_CHEBYSHEV)
        go(std::integral_constant<int, SW_CHEBF_Z>());
    else
        go(std::integral_constant<int, SW_JACOBI_Z>());
}

template <typename T>
static void prolong_add(mg_hierarchy *h, int l, const T *xc, T *xf, cudaStream_t s)
{
    LevelD &F = h->lev[l], &C = h->lev[l - 1];
    if (h->tail_rec && l <= h->tail_level) {
        TailOp op{};
        op.kind = TAIL_PROLONG;
        op.level = l;
        op.out = xf == (T *)F.x[1] ? 1 : 0;
        op.aux = xc == (const T *)C.x[1] ? 1 : 0;
        h->tail_ops.push_back(op);
        return;
    }
    int sv = sizeof(T);
    double bytes = 2.0 * F.n * sv + (double)C.n * sv;
    if (!F.structured) bytes += mat_bytes(F.P, sv);
    LaunchScope ls(h, s, MG_K_PROLONG, l, bytes);
    if (F.structured) {
        unsigned nx = (unsigned)C.N, bx = line_block(nx);  // one thread per coarse cell corner (X, Y[, Z])
        dim3 g((nx + bx - 1) / bx, nx, h->dim == 3 ? nx : 1);
        bool pdl = h->opt.use_pdl != 0;
        if (h->dim == 3)
            klaunch(pdl, k_prolong_q1<T, 3>, g, dim3(bx), 0, s, xc, xf, C.N);
        else
            klaunch(pdl, k_prolong_q1<T, 2>, g, dim3(bx), 0, s, xc, xf, C.N);
    } else {  // explicit P in SELL-32
        klaunch(h->opt.use_pdl != 0, k_sell_apply<T, true>, dim3(grid_for(F.n)), dim3(256), 0, s,
                (const int64_t *)F.P.rowptr, (const int32_t *)F.P.col, (const T *)F.P.val, (const int32_t *)F.P.perm,
                (int)F.n, xc, xf, mgk::ZStep<T>{});
    }
}

// V-cycle on the finest level's right-hand side (the defect); returns the buffer of the
// finest level holding the correction
template <typename T>
static void launch_tail(mg_hierarchy *h, cudaStream_t s)
{
    TailProg<T> P{};
    if ((int)h->tail_ops.size() > TAIL_MAX_OPS) throw Error(MG_EINVAL, "coarse-level tail has too many operations");
    for (int l = 0; l <= h->tail_level; l++) {
        LevelD &L = h->lev[l];
        P.lev[l].A = view<T>(L.A);
        P.lev[l].n = (int)L.n;
        P.lev[l].N = L.N;
        P.lev[l].x[0] = (T *)L.x[0];
        P.lev[l].x[1] = (T *)L.x[1];
        P.lev[l].b = (T *)L.b;
        P.lev[l].t = (T *)L.t;
        P.lev[l].d = (T *)L.d;
    }
    for (size_t k = 0; k < h->tail_ops.size(); k++) P.ops[k] = h->tail_ops[k];
    P.nops = (int)h->tail_ops.size();
    P.dim = h->dim;
    P.K = h->lev[h->tail_level].A.K;
    P.lu = h->lu;
    P.piv = h->piv;
    P.n0 = h->n0;
    LaunchScope ls(h, s, MG_K_COARSE, 0, 0.0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(h->tail_cluster);
    cfg.blockDim = dim3(512);
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = h->tail_cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = h->opt.use_pdl ? 2 : 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_tail<T>, P);
    if (e != cudaSuccess) throw Error(MG_ECUDA, std::string("coarse-level tail launch: ") + cudaGetErrorString(e));
    h->tail_ops.clear();
}

// first_done: the finest level's first smoothing step was taken by the outer residual
template <typename T>
static int enqueue_vcycle(mg_hierarchy *h, cudaStream_t s, bool first_done = false)
{
    int Lf = h->Lf;
    std::vector<int> cur((size_t)h->nlev, -1);
    h->tail_ops.clear();
    h->tail_rec = h->tail_level >= 1;
    // fz[l]: level l's first smoothing step was taken by the kernel that produced its
    // right-hand side (the outer residual on the finest level, the restriction below it)
    std::vector<char> fz((size_t)h->nlev, 0);
    fz[Lf] = first_done;
    for (int l = 1; l < Lf; l++) fz[l] = h->zfuse && !(h->tail_rec && l <= h->tail_level);
    for (int l = Lf; l >= 1; l--) {  // pre-smoothing and restriction of the residual
        LevelD &L = h->lev[l];
        int c = -1;
        for (int a = 0; a < h->opt.nu_pre; a++) c = smooth<T>(h, l, c, false, s, false, fz[l] && a == 0);
        const T *r;
        if (c < 0) {
            r = (const T *)L.b;  // b - A 0 = b
        } else {
            sweep<T>(h, l, SW_RESID, (T *)L.x[c], (T *)L.b, (T *)L.t, nullptr, 0.0, 0.0, s);
            r = (const T *)L.t;
        }
        restrict_to<T>(h, l, r, s, l - 1 >= 1 && fz[l - 1]);
        cur[l] = c;
    }
    if (h->tail_rec) {  // the coarsest solve belongs to the tail launch
        TailOp op{};
        op.kind = TAIL_COARSE;
        op.level = 0;
        h->tail_ops.push_back(op);
        cur[0] = 0;
    } else {  // exact solve on the coarsest level
        LevelD &C = h->lev[0];
        LaunchScope ls(h, s, MG_K_COARSE, 0, (double)h->n0 * h->n0 * 8 + 2.0 * h->n0 * sizeof(T));
        bool pdl = h->opt.use_pdl != 0;
        const double *lu = h->lu;
        const int *piv = h->piv;
        if (h->n0 <= 64) {
            klaunch(pdl, k_coarse_solve_warp<T>, dim3(1), dim3(256), 0, s, lu, piv, h->n0, (const T *)C.b,
                    (T *)C.x[0]);
        } else {
            int thr = (int)round_up(h->n0, 32);
            klaunch(pdl, k_coarse_solve<T>, dim3(1), dim3(thr), (size_t)h->n0 * sizeof(double), s, lu, piv, h->n0,
                    (const T *)C.b, (T *)C.x[0]);
        }
        cur[0] = 0;
    }
    for (int l = 1; l <= Lf; l++) {  // prolongation, correction and post-smoothing
        LevelD &L = h->lev[l];
        if (h->tail_rec && l == h->tail_level + 1) {  // leaving the tail: replay it in one launch
            launch_tail<T>(h, s);
            h->tail_rec = false;
        }
        if (cur[l] < 0) {
            if (h->tail_rec && l <= h->tail_level) {
                TailOp op{};
                op.kind = TAIL_ZERO;
                op.level = l;
                op.out = 0;
                h->tail_ops.push_back(op);
            } else {
                CK(cudaMemsetAsync(L.x[0], 0, (size_t)L.n * sizeof(T), s));
            }
            cur[l] = 0;
        }
        prolong_add<T>(h, l, (const T *)h->lev[l - 1].x[cur[l - 1]], (T *)L.x[cur[l]], s);
        for (int a = 0; a < h->opt.nu_post; a++)
            cur[l] = smooth<T>(h, l, cur[l], true, s, h->fuse_update && l == Lf && a == h->opt.nu_post - 1);
    }
    if (h->tail_rec) {  // the whole hierarchy was the tail
        launch_tail<T>(h, s);
        h->tail_rec = false;
    }
    return cur[Lf];
}

template <typename MK>
static void launch_fp64_rows(mg_hierarchy *h, const DevMat &A, MK &&mk)
{
    if (A.fmt == MG_STORAGE_DIA) {
        with_dia_k(A.K, [&](auto k) { mk(std::integral_constant<int, 3>(), k); });
    } else if (A.fmt == MG_STORAGE_ELL) {
        mk(std::integral_constant<int, 2>(), std::integral_constant<int, 1>());
    } else if (A.fmt == MG_STORAGE_SELL) {
        mk(std::integral_constant<int, 4>(), std::integral_constant<int, 1>());
    } else {
        mk(std::integral_constant<int, 1>(), std::integral_constant<int, 1>());
    }
}

template <typename T>
static void enqueue_outer(mg_hierarchy *h, cudaStream_t s)
{
    LevelD &F = h->lev[h->Lf];
    const DevMat &A = h->A64;
    int n = (int)F.n;
    double bytes = mat_bytes(A, 8) + 16.0 * n + (double)n * sizeof(T);
    double entries = mat_entries(A);
    MatView<double> v = view<double>(A);
    dim3 g(fp64_rows_grid(A, n)), blk(256);
    T *r = (T *)F.b;
    bool pdl = h->opt.use_pdl != 0;
    const double *x = h->x64, *b = h->b64;
    if constexpr (std::is_same<T, float>::value) {
        if (h->outer_z) {  // and the finest level's first smoothing step (from x = 0)
            const bool cheb = h->opt.smoother == MG_CHEBYSHEV;
            mgk::ZStep<float> Z = zstep_of<float>(h, h->Lf, &bytes);
            LaunchScope ls(h, s, MG_K_OUTER, h->Lf, bytes, 2.0 * entries + 5.0 * n);
            launch_fp64_rows(h, A, [&](auto fmt, auto k) {
                constexpr int FMT = decltype(fmt)::value, K = decltype(k)::value;
                if (cheb)
                    klaunch(pdl, k_outer_resid<float, FMT, K, SW_CHEBF_Z>, g, blk, 0, s, v, n, x, b, r, h->partial,
                            h->ticket, h->norm2, Z);
                else
                    klaunch(pdl, k_outer_resid<float, FMT, K, SW_JACOBI_Z>, g, blk, 0, s, v, n, x, b, r, h->partial,
                            h->ticket, h->norm2, Z);
            });
            return;
        }
    }
    LaunchScope ls(h, s, MG_K_OUTER, h->Lf, bytes, 2.0 * entries + 3.0 * n);
    if (A.fmt == MG_STORAGE_DIA) {
        with_dia_k(A.K, [&](auto k) {
            klaunch(pdl, k_outer_resid<T, 3, decltype(k)::value>, g, blk, 0, s, v, n, x, b, r, h->partial, h->ticket,
                    h->norm2, mgk::ZStep<float>{});
        });
    } else if (A.fmt == MG_STORAGE_ELL) {
        klaunch(pdl, k_outer_resid<T, 2, 1>, g, blk, 0, s, v, n, x, b, r, h->partial, h->ticket, h->norm2,
                mgk::ZStep<float>{});
    } else if (A.fmt == MG_STORAGE_SELL) {
        klaunch(pdl, k_outer_resid<T, 4, 1>, g, blk, 0, s, v, n, x, b, r, h->partial, h->ticket, h->norm2,
                mgk::ZStep<float>{});
    } else {
        klaunch(pdl, k_outer_resid<T, 1, 1>, g, blk, 0, s, v, n, x, b, r, h->partial, h->ticket, h->norm2,
                mgk::ZStep<float>{});
    }
}

template <typename T>
static void enqueue_update(mg_hierarchy *h, int cur, cudaStream_t s)
{
    LevelD &F = h->lev[h->Lf];
    int n = (int)F.n;
    LaunchScope ls(h, s, MG_K_UPDATE, h->Lf, 16.0 * n + (double)n * sizeof(T));
    klaunch(h->opt.use_pdl != 0, k_update<T>, dim3(grid_for(n)), dim3(256), 0, s, h->x64, (const T *)F.x[cur], n);
}

static void enqueue_r(mg_hierarchy *h, cudaStream_t s)
{
    if (h->mixed)
        enqueue_outer<float>(h, s);
    else
        enqueue_outer<double>(h, s);
}

// one V-cycle and x64 += c; the update rides on the finest level's last post-smoothing
// sweep where its storage has a kernel for that, else it is a launch of its own
static void enqueue_v(mg_hierarchy *h, cudaStream_t s)
{
    h->update_fused = false;
    h->fuse_update = true;
    if (h->mixed) {
        int c = enqueue_vcycle<float>(h, s, h->outer_z);
        h->fuse_update = false;
        if (!h->update_fused) enqueue_update<float>(h, c, s);
    } else {
        int c = enqueue_vcycle<double>(h, s);
        h->fuse_update = false;
        if (!h->update_fused) enqueue_update<double>(h, c, s);
    }
}

// ---- preconditioned CG ----

// r_0 = b - A x_0 (FP64, and in the inner precision as the V-cycle's right-hand side)
template <typename T>
static void enqueue_pcg_init(mg_hierarchy *h, cudaStream_t s)
{
    LevelD &F = h->lev[h->Lf];
    const DevMat &A = h->A64;
    int n = (int)F.n;
    double entries = mat_entries(A);
    double bytes = mat_bytes(A, 8) + 32.0 * n + (double)n * sizeof(T);
    mgk::ZStep<float> Z{};
    const bool zf = std::is_same<T, float>::value && h->outer_z;  // and the finest level's first step
    if (zf) Z = zstep_of<float>(h, h->Lf, &bytes);
    LaunchScope ls(h, s, MG_K_OUTER, h->Lf, bytes, 2.0 * entries + (zf ? 5.0 : 3.0) * n);
    MatView<double> v = view<double>(A);
    bool pdl = h->opt.use_pdl != 0;
    dim3 g(fp64_rows_grid(A, n)), blk(256);
    const int zm = !zf ? 0 : (h->opt.smoother == MG_CHEBYSHEV ? (int)SW_CHEBF_Z : (int)SW_JACOBI_Z);
    launch_fp64_rows(h, A, [&](auto fmt, auto k) {
        constexpr int FMT = decltype(fmt)::value, K = decltype(k)::value;
        auto go = [&](auto kern) {
            klaunch(pdl, kern, g, blk, 0, s, v, n, (const double *)h->x64, (const double *)h->b64, h->pcg_r,
                    (T *)F.b, h->pcg_p, h->pcg_scal, h->partial, h->ticket, h->norm2, Z);
        };
        if constexpr (std::is_same<T, float>::value) {
            if (zm == SW_CHEBF_Z) return go(k_pcg_init<T, FMT, K, SW_CHEBF_Z>);
            if (zm == SW_JACOBI_Z) return go(k_pcg_init<T, FMT, K, SW_JACOBI_Z>);
        }
        go(k_pcg_init<T, FMT, K, 0>);
    });
}

// one CG iteration: z = V(r), rz, p, q = A p, x and r
template <typename T>
static void enqueue_pcg_iter(mg_hierarchy *h, cudaStream_t s)
{
    LevelD &F = h->lev[h->Lf];
    const DevMat &A = h->A64;
    int n = (int)F.n, sv = sizeof(T);
    bool pdl = h->opt.use_pdl != 0;
    dim3 g(grid_for(n)), blk(256);
    // the V-cycle's finest first step was taken by the kernel that wrote r (init or update)
    int c = enqueue_vcycle<T>(h, s, std::is_same<T, float>::value && h->outer_z);
    const T *z = (const T *)F.x[c];
    dim3 gr(reduce_grid(n));  // the kernels that end in an inner product
    {
        LaunchScope ls(h, s, MG_K_KRYLOV, h->Lf, 8.0 * n + (double)n * sv, 2.0 * n);
        klaunch(pdl, k_pcg_rz<T>, gr, blk, 0, s, (const double *)h->pcg_r, z, n, h->partial, h->ticket,
                h->pcg_scal);
    }
    {
        LaunchScope ls(h, s, MG_K_KRYLOV, h->Lf, 16.0 * n + (double)n * sv, 2.0 * n);
        klaunch(pdl, k_pcg_dir<T>, g, blk, 0, s, z, h->pcg_p, n, (const double *)h->pcg_scal);
    }
    {
        double entries = mat_entries(A);
        LaunchScope ls(h, s, MG_K_KRYLOV, h->Lf, mat_bytes(A, 8) + 16.0 * n, 2.0 * entries + 2.0 * n);
        MatView<double> v = view<double>(A);
        dim3 ga(fp64_rows_grid(A, n));
        launch_fp64_rows(h, A, [&](auto fmt, auto k) {
            klaunch(pdl, k_pcg_apply<decltype(fmt)::value, decltype(k)::value>, ga, blk, 0, s, v, n,
                    (const double *)h->pcg_p, h->pcg_q, h->partial, h->ticket, h->pcg_scal);
        });
    }
    {
        double bytes = 48.0 * n + (double)n * sv;
        mgk::ZStep<float> Z{};
        const bool zf = std::is_same<T, float>::value && h->outer_z;  // and the next V-cycle's first step
        if (zf) Z = zstep_of<float>(h, h->Lf, &bytes);
        LaunchScope ls(h, s, MG_K_KRYLOV, h->Lf, bytes, (zf ? 8.0 : 6.0) * n);
        auto go = [&](auto kern) {
            klaunch(pdl, kern, gr, blk, 0, s, h->x64, h->pcg_r, (T *)F.b, (const double *)h->pcg_p,
                    (const double *)h->pcg_q, n, h->pcg_scal, h->partial, h->ticket, h->norm2, Z);
        };
        if constexpr (std::is_same<T, float>::value) {
            if (zf && h->opt.smoother == MG_CHEBYSHEV)
                go(k_pcg_update<T, SW_CHEBF_Z>);
            else if (zf)
                go(k_pcg_update<T, SW_JACOBI_Z>);
            else
                go(k_pcg_update<T, 0>);
        } else {
            go(k_pcg_update<T, 0>);
        }
    }
}

static void enqueue_pi(mg_hierarchy *h, cudaStream_t s)
{
    if (h->mixed)
        enqueue_pcg_init<float>(h, s);
    else
        enqueue_pcg_init<double>(h, s);
}

static void enqueue_pc(mg_hierarchy *h, cudaStream_t s)
{
    if (h->mixed)
        enqueue_pcg_iter<float>(h, s);
    else
        enqueue_pcg_iter<double>(h, s);
}

static cudaGraphExec_t capture(mg_hierarchy *h, void (*fn)(mg_hierarchy *, cudaStream_t), std::vector<mgi::Prof::Rec> *sink)
{
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    h->sink = sink;
    h->capturing = true;
    CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
    try {
        fn(h, h->s);
    } catch (...) {
        cudaStreamEndCapture(h->s, &g);
        if (g) cudaGraphDestroy(g);
        h->capturing = false;
        throw;
    }
    CK(cudaStreamEndCapture(h->s, &g));
    h->capturing = false;
    cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) throw Error(MG_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    return ge;
}

static void ensure_graphs(mg_hierarchy *h)
{
    if (!h->opt.use_graph || (h->g_r && h->g_v)) return;
    destroy_graphs(h);
    h->g_r = capture(h, enqueue_r, &h->rec_r);
    h->g_v = capture(h, enqueue_v, &h->rec_v);
}

// median device time of the captured V-cycle (with the update), from the hierarchy's own
// vectors; used at setup to choose between launch plans that compute the same bits
static double time_vcycle_graph(mg_hierarchy *h)
{
    cudaGraphExec_t ge = capture(h, enqueue_v, nullptr);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<float> ms;
    for (int r = 0; r < 25; r++) {
        CK(cudaEventRecord(e0, h->s));
        CK(cudaGraphLaunch(ge, h->s));
        CK(cudaEventRecord(e1, h->s));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        if (r >= 5) ms.push_back(t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGraphExecDestroy(ge);
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
}

static void ensure_pcg_graphs(mg_hierarchy *h)
{
    if (!h->opt.use_graph || (h->g_pi && h->g_pc)) return;
    h->g_pi = capture(h, enqueue_pi, &h->rec_pi);
    h->g_pc = capture(h, enqueue_pc, &h->rec_pc);
}

static void run_graph_or_eager(mg_hierarchy *h, cudaGraphExec_t g, void (*fn)(mg_hierarchy *, cudaStream_t))
{
    if (h->opt.use_graph) {
        CK(cudaGraphLaunch(g, h->s));
    } else {
        h->sink = &h->rec_eager;
        fn(h, h->s);
    }
}

static void run_r(mg_hierarchy *h)
{
    if (h->opt.use_graph) {
        CK(cudaGraphLaunch(h->g_r, h->s));
    } else {
        h->sink = &h->rec_eager;
        enqueue_r(h, h->s);
    }
}

static void run_v(mg_hierarchy *h)
{
    if (h->opt.use_graph) {
        CK(cudaGraphLaunch(h->g_v, h->s));
    } else {
        h->sink = &h->rec_eager;
        enqueue_v(h, h->s);
    }
}

// after a synchronisation of h->s: fold the finished launches into the profile
static void prof_collect(mg_hierarchy *h, bool r_ran, bool v_ran)
{
    if (!h->profiling) return;
    if (h->opt.use_graph) {
        if (r_ran) h->prof.collect(h->rec_r);
        if (v_ran) h->prof.collect(h->rec_v);
    } else {
        h->prof.collect(h->rec_eager);
        h->prof.release(h->rec_eager);
    }
}

static void prof_collect_pcg(mg_hierarchy *h, bool init_ran, bool iter_ran)
{
    if (!h->profiling) return;
    if (h->opt.use_graph) {
        if (init_ran) h->prof.collect(h->rec_pi);
        if (iter_ran) h->prof.collect(h->rec_pc);
    } else {
        h->prof.collect(h->rec_eager);
        h->prof.release(h->rec_eager);
    }
}

static double read_norm2(mg_hierarchy *h)
{
    CK(cudaMemcpyAsync(h->h_norm2, h->norm2, sizeof(double), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    return *h->h_norm2;
}

static double norm_b(mg_hierarchy *h)
{
    int n = (int)h->lev[h->Lf].n;
    k_norm2<<<reduce_grid(n), 256, 0, h->s>>>(h->b64, n, h->partial, h->ticket, h->norm2);
    CKL();
    return std::sqrt(read_norm2(h));
}

// ------------------------------------------------------------------------------------
// Setup
// ------------------------------------------------------------------------------------
extern "C" void mg_options_default(mg_options *o)
{
    std::memset(o, 0, sizeof(*o));
    o->smoother = MG_JACOBI;
    o->omega = 0.8;
    o->cheb_degree = 2;
    o->nu_pre = 2;
    o->nu_post = 2;
    o->cheb_hi = 1.1;
    o->cheb_ratio = 4.0;
    o->power_iters = 20;
    o->power_seed = 1609;
    o->precision = MG_FP64;
    o->storage = MG_STORAGE_AUTO;
    o->max_iters = 100;
    o->use_graph = 1;
    o->use_pdl = 1;
    o->coarse_tail = 2;
    o->fuse_first = 1;
}

extern "C" int64_t mg_ndofs(int dim, int element, int n_cells)
{
    if (n_cells < 1 || !((element == MG_Q1 && (dim == 2 || dim == 3)) ||
                         ((element == MG_RQ1 || element == MG_P1 || element == MG_P2) && dim == 3)))
        return -1;
    return mgh::ndofs(dim, element, n_cells);
}

static void validate_problem(const mg_problem *p)
{
    if (!p) throw Error(MG_EINVAL, "problem is NULL");
    if (mg_ndofs(p->dim, p->element, p->n_cells) < 0) throw Error(MG_EINVAL, "invalid dim/element/n_cells");
    if (p->n_levels < 1 || p->n_levels > MG_MAX_LEVELS) throw Error(MG_EINVAL, "n_levels out of range");
    int Nc = p->n_cells >> (p->n_levels - 1);
    if (Nc < 2 || (Nc << (p->n_levels - 1)) != p->n_cells)
        throw Error(MG_EINVAL, "n_cells must be the coarsest size (>= 2) times 2^(n_levels-1)");
    int64_t n = mgh::ndofs(p->dim, p->element, p->n_cells);
    if (n > (int64_t)INT32_MAX / 32) throw Error(MG_EINVAL, "problem too large for 32-bit row indices");
    if (!(p->mass >= 0.0) || !std::isfinite(p->mass)) throw Error(MG_EINVAL, "mass must be finite and >= 0");
    if (p->mass != 0.0 && p->element == MG_RQ1) throw Error(MG_EINVAL, "the mass shift is built for Q1, P1 and P2");
}

extern "C" mg_status mg_load_vector(const mg_problem *p, const mg_rhs *f, double *b_host)
{
    try {
        validate_problem(p);
        if (!f || !b_host) throw Error(MG_EINVAL, "rhs or output is NULL");
        if (f->n_modes < 0 || (f->n_modes > 0 && (!f->amp || !f->freq))) throw Error(MG_EINVAL, "bad rhs modes");
        mgh::load_vector(p->dim, p->element, p->n_cells, f, b_host);
        return MG_OK;
    } catch (const Error &e) {
        g_err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        return MG_ENOMEM;
    }
}

extern "C" mg_status mg_load_vector_separable(const mg_problem *p, const mg_rhs *f, double *b_host)
{
    try {
        validate_problem(p);
        if (p->element != MG_Q1) throw Error(MG_EINVAL, "the factorised load vector is for Q1");
        if (!f || !b_host) throw Error(MG_EINVAL, "rhs or output is NULL");
        if (f->n_modes < 0 || (f->n_modes > 0 && (!f->amp || !f->freq))) throw Error(MG_EINVAL, "bad rhs modes");
        mgh::load_vector_separable(p->dim, p->n_cells, f, b_host);
        return MG_OK;
    } catch (const Error &e) {
        g_err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        return MG_ENOMEM;
    }
}

// device format of a level operator
// SELL-32 layout: rows sorted by length, longest first (ties by row index), slices of 32
// positions; slice s holds 32 * K_s slots from sptr[s] (K_s = its longest row).
static void sell_layout(const mgh::Csr &A, std::vector<int32_t> &perm, std::vector<int64_t> &sptr)
{
    int64_t n = A.nrows;
    perm.resize((size_t)n);
    for (int64_t i = 0; i < n; i++) perm[i] = (int32_t)i;
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) {
        return A.rowptr[a + 1] - A.rowptr[a] > A.rowptr[b + 1] - A.rowptr[b];
    });
    int64_t ns = (n + 31) / 32;
    sptr.assign((size_t)ns + 1, 0);
    for (int64_t s = 0; s < ns; s++) {
        int32_t first = perm[(size_t)s * 32];
        int64_t Ks = std::max<int64_t>(A.rowptr[first + 1] - A.rowptr[first], 1);
        sptr[s + 1] = sptr[s] + 32 * Ks;
    }
}

// Constant stencil (Q1, P1 on the grid vertices): by_pos[p] receives the values of the
// row of grid point (2, 2[, 2]) by stencil position p = (dx+1) + 3(dy+1) [+ 9(dz+1)], in the
// inner precision (FP32: that row's row-sum-preserving rounding, as round_fp32 forms it).
// True only if every row of A holds exactly these FP64 values at its in-grid neighbours:
// no entry outside the 3^d box, the stencil's nonzero positions all present where the
// neighbour is in the grid, any other entry zero.
static bool constant_stencil(const mgh::Csr &A, int dim, int N, int sv, double by_pos[27])
{
    if (N < 4) return false;
    const int npos = dim == 3 ? 27 : 9;
    const int64_t n1 = N - 1;
    const int64_t i0 = 1 + n1 * (1 + (dim == 3 ? n1 : 0));
    double st[27] = {};
    bool has[27] = {};
    auto pos_of = [&](const int *ci, const int *cj, int &p) {
        int q[3] = {0, 0, 0};
        for (int a = 0; a < dim; a++) {
            q[a] = cj[a] - ci[a];
            if (q[a] < -1 || q[a] > 1) return false;
        }
        p = (q[0] + 1) + 3 * (q[1] + 1) + (dim == 3 ? 9 * (q[2] + 1) : 0);
        return true;
    };
    int ci[3], cj[3], p;
    mgh::q1_coords(dim, N, i0, ci);
    for (int64_t k = A.rowptr[i0]; k < A.rowptr[i0 + 1]; k++) {
        mgh::q1_coords(dim, N, A.col[k], cj);
        if (!pos_of(ci, cj, p)) return false;
        st[p] = A.val[k];
        has[p] = true;
    }
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < A.nrows; i++) {
        int vi[3], vj[3], q;
        mgh::q1_coords(dim, N, i, vi);
        unsigned seen = 0;
        bool ok = true;
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1] && ok; k++) {
            mgh::q1_coords(dim, N, A.col[k], vj);
            ok = pos_of(vi, vj, q) && A.val[k] == (has[q] ? st[q] : 0.0);
            if (ok) seen |= 1u << q;
        }
        for (int pp = 0; pp < npos && ok; pp++) {
            if (!has[pp] || st[pp] == 0.0 || ((seen >> pp) & 1u)) continue;
            int dd[3] = {pp % 3 - 1, (pp / 3) % 3 - 1, pp / 9 - 1};
            bool in = true;
            for (int a = 0; a < dim; a++) in = in && vi[a] + dd[a] >= 1 && vi[a] + dd[a] <= N - 1;
            ok = !in;  // a stencil neighbour inside the grid is missing from the row
        }
        if (!ok) bad++;
    }
    if (bad) return false;
    for (int pp = 0; pp < 27; pp++) by_pos[pp] = st[pp];
    if (sv == 4) {  // the row-sum-preserving FP32 rounding of row i0
        double rowsum = 0.0, off32 = 0.0;
        int pc = -1;
        for (int64_t k = A.rowptr[i0]; k < A.rowptr[i0 + 1]; k++) {
            mgh::q1_coords(dim, N, A.col[k], cj);
            pos_of(ci, cj, p);
            rowsum = rowsum + A.val[k];
            if (A.col[k] == i0) {
                pc = p;
            } else {
                by_pos[p] = (double)(float)A.val[k];
                off32 = off32 + by_pos[p];
            }
        }
        if (pc >= 0) by_pos[pc] = (double)(float)(rowsum - off32);
    }
    return true;
}

// The in-grid neighbours of rotated-Q1 face r on N cells per axis (the same enumeration
// as k_stencil_rq1): col[], role[] (0 the face itself, 1 a face opposite it in one of its
// two cells, 2 one of the other faces of those cells). Returns the count.
static int rq1_neighbours(int N, int64_t r, int64_t *col, int *role)
{
    const int64_t M = N - 1, ny0 = M * N * N, nz0 = 2 * M * N * N;
    int f = r < ny0 ? 0 : (r < nz0 ? 1 : 2);
    int64_t loc = r - (f == 0 ? 0 : (f == 1 ? ny0 : nz0));
    int p, q, c;  // the kernel's thread coordinates (fast, line, slab) of the face
    if (f == 0) {
        p = (int)(loc % M);
        q = (int)((loc / M) % N);
        c = (int)(loc / (M * N));
    } else if (f == 1) {
        p = (int)(loc % N);
        q = (int)((loc / N) % M);
        c = (int)(loc / (N * M));
    } else {
        p = (int)(loc % N);
        q = (int)((loc / N) % N);
        c = (int)(loc / ((int64_t)N * N));
    }
    int cnt = 0;
    auto add = [&](bool in, int64_t j, int ro) {
        if (!in) return;
        col[cnt] = j;
        role[cnt] = ro;
        cnt++;
    };
    add(true, r, 0);
    int t0 = f == 0 ? p : (f == 1 ? q : c);  // position along the normal minus 1
    int64_t step = f == 0 ? 1 : (f == 1 ? N : (int64_t)N * N);
    add(t0 >= 1, r - step, 1);
    add(t0 + 1 <= M - 1, r + step, 1);
    for (int s2 = 0; s2 < 2; s2++)
        for (int t = 0; t < 2; t++) {
            if (f == 0) {
                int cx = p + s2, jy = q + t, kz = c + t;
                add(jy >= 1 && jy <= M, ny0 + cx + N * ((jy - 1) + M * c), 2);
                add(kz >= 1 && kz <= M, nz0 + cx + N * (q + (int64_t)N * (kz - 1)), 2);
            } else if (f == 1) {
                int cy = q + s2, ix = p + t, kz = c + t;
                add(ix >= 1 && ix <= M, (ix - 1) + M * (cy + (int64_t)N * c), 2);
                add(kz >= 1 && kz <= M, nz0 + p + N * (cy + (int64_t)N * (kz - 1)), 2);
            } else {
                int cz = c + s2, ix = p + t, jy = q + t;
                add(ix >= 1 && ix <= M, (ix - 1) + M * (q + (int64_t)N * cz), 2);
                add(jy >= 1 && jy <= M, ny0 + p + N * ((jy - 1) + M * cz), 2);
            }
        }
    return cnt;
}

// Constant face stencil of a rotated-Q1 level (MG_STORAGE_STENCIL): true if every row of
// A holds exactly its in-grid neighbours of rq1_neighbours, with one FP64 value per role
// taken from an interior row: the diagonal 6 v, the opposite faces v, the other faces -v
// (each within 1e-13 of the diagonal, the values of a constant coefficient). vals
// receives (diagonal, opposite, other).
static bool rq1_constant_stencil(const mgh::Csr &A, int N, double vals[3])
{
    // the face-stencil kernel indexes faces in 32 bits
    if (N < 4 || A.nrows != mgh::ndofs(3, MG_RQ1, N) || A.nrows >= ((int64_t)1 << 31)) return false;
    const int64_t M = N - 1;
    const int64_t r0 = 1 + M * (1 + (int64_t)N * 1);  // x-face at position 2 over cell (1, 1)
    double ref[3] = {0.0, 0.0, 0.0};
    {
        int64_t col[11];
        int role[11];
        int cnt = rq1_neighbours(N, r0, col, role);
        if (cnt != 11 || A.rowptr[r0 + 1] - A.rowptr[r0] != 11) return false;
        for (int64_t q = A.rowptr[r0]; q < A.rowptr[r0 + 1]; q++)
            for (int k = 0; k < cnt; k++)
                if (col[k] == A.col[q]) ref[role[k]] = A.val[q];
    }
    const double tol = 1e-13 * std::fabs(ref[0]);
    if (!(ref[0] > 0.0) || std::fabs(ref[0] - 6.0 * ref[1]) > tol || std::fabs(ref[2] + ref[1]) > tol) return false;
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t r = 0; r < A.nrows; r++) {
        int64_t col[11];
        int role[11];
        int cnt = rq1_neighbours(N, r, col, role);
        bool ok = A.rowptr[r + 1] - A.rowptr[r] == cnt;
        for (int64_t q = A.rowptr[r]; q < A.rowptr[r + 1] && ok; q++) {
            bool hit = false;
            for (int k = 0; k < cnt && !hit; k++)
                if (col[k] == A.col[q]) hit = A.val[q] == ref[role[k]];
            ok = hit;
        }
        if (!ok) bad++;
    }
    if (bad) return false;
    for (int k = 0; k < 3; k++) vals[k] = ref[k];
    return true;
}

// Per-cell coefficient form of a 3D Q1 level (MG_STORAGE_COEF): true if every row of A is
// the rediscretisation of the per-cell coefficient k of this level's N^3 cells (x fastest)
// with the unit-cube Q1 stiffness: a_ii = (h/3) sum of the 8 k_e around vertex i, a_ij =
// -(h/12) sum of k_e over the cells holding both corners for a corner across a face (2
// cells) or the body (1 cell), 0 across an edge; every entry within 1e-12 of the row's
// diagonal, every in-grid corner across a face or the body present. kap receives the
// stored values k_e h / 12 in FP32.
static bool coef_form(const mgh::Csr &A, int N, const std::vector<double> &k, std::vector<float> &kap)
{
    if (N < 4 || (int64_t)k.size() != (int64_t)N * N * N) return false;
    const double h = 1.0 / N;
    const int64_t nc = N;
    int64_t bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < A.nrows; i++) {
        int vi[3], vj[3];
        mgh::q1_coords(3, N, i, vi);
        // k of the cell on side (a, b, c) of the vertex: cell (X - 1 + a, Y - 1 + b, Z - 1 + c)
        auto kc = [&](int a, int b, int c) { return k[(size_t)((vi[0] - 1 + a) + nc * ((vi[1] - 1 + b) + nc * (vi[2] - 1 + c)))]; };
        double ks = 0.0;
        for (int e = 0; e < 8; e++) ks += kc(e & 1, (e >> 1) & 1, e >> 2);
        const double diag = ks * h / 3.0, tol = 1e-12 * std::fabs(diag);
        int found = 0, want = 1;
        for (int p = 0; p < 27; p++) {  // the in-grid corners across a face or the body
            int d[3] = {p % 3 - 1, (p / 3) % 3 - 1, p / 9 - 1};
            int nz = (d[0] != 0) + (d[1] != 0) + (d[2] != 0);
            bool in = true;
            for (int a = 0; a < 3; a++) in = in && vi[a] + d[a] >= 1 && vi[a] + d[a] <= N - 1;
            if (in && nz >= 2) want++;
        }
        bool ok = true;
        for (int64_t q = A.rowptr[i]; q < A.rowptr[i + 1] && ok; q++) {
            mgh::q1_coords(3, N, A.col[q], vj);
            int d[3] = {vj[0] - vi[0], vj[1] - vi[1], vj[2] - vi[2]};
            for (int a = 0; a < 3; a++) ok = ok && d[a] >= -1 && d[a] <= 1;
            if (!ok) break;
            int nz = (d[0] != 0) + (d[1] != 0) + (d[2] != 0);
            double expect = 0.0;
            if (nz == 0) {
                expect = diag;
            } else if (nz >= 2) {
                double sk = 0.0;
                for (int e = 0; e < 8; e++) {
                    int side[3] = {e & 1, (e >> 1) & 1, e >> 2};
                    bool both = true;
                    for (int a = 0; a < 3; a++)
                        if (d[a] != 0 && side[a] != (d[a] > 0 ? 1 : 0)) both = false;
                    if (both) sk += kc(side[0], side[1], side[2]);
                }
                expect = -sk * h / 12.0;
            }
            ok = std::fabs(A.val[q] - expect) <= tol;
            if (ok && nz != 1) found++;
        }
        if (!ok || found != want) bad++;
    }
    if (bad) return false;
    kap.resize(k.size());
    for (size_t e = 0; e < k.size(); e++) kap[e] = (float)(k[e] * h / 12.0);
    return true;
}

// stencil_vals: STENCIL only, the values by stencil position (constant_stencil)
static void plan_matrix(DevMat &m, const mgh::Csr &A, int fmt, int dim, int N, int sv, mgi::Slab &slab, bool take,
                        const double *stencil_vals = nullptr, int elem = MG_Q1)
{
    m.fmt = fmt;
    m.n = A.nrows;
    m.nnz = A.nnz();
    m.ld = round_up(std::max<int64_t>(m.n, 1), 64);
    m.elem_size = sv;
    m.n1 = N - 1;
    m.dim = dim;
    m.elem = elem;
    if (fmt == MG_STORAGE_STENCIL && elem == MG_RQ1) {  // face stencil: three values, nothing stored
        if (!stencil_vals) throw Error(MG_EINVAL, "stencil storage without stencil values");
        m.K = 11;
        for (int q = 0; q < 3; q++) m.sval[q] = stencil_vals[q];
        // the FP32 sweep forms hv * (6 x_i - ...): a_ii = 6 hv in FP32
        float hv = (float)m.sval[1];
        m.sdinv = sv == 8 ? 1.0 / m.sval[0] : (double)(1.0f / (6.0f * hv));
        return;
    }
    if (fmt == MG_STORAGE_COEF) {  // 3D Q1: the 21 positions of the stencil, one value per cell
        if (dim != 3) throw Error(MG_EINVAL, "coefficient storage is 3D Q1 only");
        int64_t n1 = N - 1;
        int k = 0;
        for (int p = 0; p < 27; p++) {
            int dx = p % 3 - 1, dy = (p / 3) % 3 - 1, dz = p / 9 - 1;
            if ((dx != 0) + (dy != 0) + (dz != 0) == 1) continue;  // edge-adjacent: coupling 0
            m.offs.o[k] = (int32_t)(dx + n1 * dy + n1 * n1 * dz);
            m.full_of[k] = p;
            if (p == 13) m.center = k;
            k++;
        }
        m.K = k;
        size_t bytes = (size_t)N * N * N * 4;
        if (take)
            m.val = slab.take(bytes);
        else
            slab.reserve(bytes);
        return;
    }
    if (fmt == MG_STORAGE_DIA || fmt == MG_STORAGE_STENCIL) {
        // keep the stencil positions that hold a nonzero anywhere (ascending offset),
        // padded with unused positions up to an instantiated slot count (9, 21 or 27).
        // A symmetric matrix uses position p iff it uses npos-1-p, and padding adds such
        // pairs, so the diagonal is always the middle slot K/2.
        int npos = dim == 3 ? 27 : 9, cpos = npos / 2;
        bool used[27] = {};
        used[cpos] = true;
        for (int64_t i = 0; i < A.nrows; i++) {
            int ci[3], cj[3];
            mgh::q1_coords(dim, N, i, ci);
            for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) {
                if (A.val[k] == 0.0) continue;
                mgh::q1_coords(dim, N, A.col[k], cj);
                used[(cj[0] - ci[0] + 1) + 3 * (cj[1] - ci[1] + 1) + (dim == 3 ? 9 * (cj[2] - ci[2] + 1) : 0)] = true;
            }
        }
        for (int p = 0; p < npos; p++)  // symmetrise (a Galerkin product may round asymmetrically)
            if (used[p]) used[npos - 1 - p] = true;
        int cnt = 0;
        for (int p = 0; p < npos; p++) cnt += used[p];
        // the smallest instantiated slot count that holds them: 9 in 2D; 7, 15, 21, 27 in 3D
        int K = 9;
        if (dim == 3) K = cnt <= 7 ? 7 : (cnt <= 15 ? 15 : (cnt <= 21 ? 21 : 27));
        for (int p = 0; p < cpos && cnt < K; p++)
            if (!used[p]) {
                used[p] = used[npos - 1 - p] = true;
                cnt += 2;
            }
        m.K = K;
        int64_t n1 = N - 1;
        int k = 0;
        for (int p = 0; p < npos; p++) {
            if (!used[p]) continue;
            int dx = p % 3 - 1, dy = (p / 3) % 3 - 1, dz = dim == 3 ? p / 9 - 1 : 0;
            m.offs.o[k] = (int32_t)(dx + n1 * dy + n1 * n1 * dz);
            m.full_of[k] = p;
            if (p == cpos) m.center = k;
            k++;
        }
        if (k != K || m.center != K / 2) throw Error(MG_EINVAL, "DIA slot selection is not symmetric");
        if (fmt == MG_STORAGE_STENCIL) {  // values as launch parameters; nothing stored
            if (!stencil_vals) throw Error(MG_EINVAL, "stencil storage without stencil values");
            for (int q = 0; q < K; q++) m.sval[q] = stencil_vals[m.full_of[q]];
            double ac = m.sval[m.center];
            m.sdinv = sv == 8 ? 1.0 / ac : (double)(1.0f / (float)ac);
            return;
        }
        size_t bytes = (size_t)m.K * m.ld * sv;
        if (take)
            m.val = slab.take(bytes);
        else
            slab.reserve(bytes);
    } else if (fmt == MG_STORAGE_SELL) {
        std::vector<int32_t> perm;
        std::vector<int64_t> sptr;
        sell_layout(A, perm, sptr);
        m.nslices = (int64_t)sptr.size() - 1;
        m.padded = sptr.back();
        m.K = (int)(m.nslices ? (sptr[1] - sptr[0]) / 32 : 1);  // the widest slice
        size_t vb = (size_t)std::max<int64_t>(m.padded, 1) * sv, cb = (size_t)std::max<int64_t>(m.padded, 1) * 4,
               sb = (size_t)(m.nslices + 1) * 8, pb = (size_t)std::max<int64_t>(m.n, 1) * 4;
        if (take) {
            m.val = slab.take(vb);
            m.col = (int32_t *)slab.take(cb);
            m.rowptr = (int64_t *)slab.take(sb);
            m.perm = (int32_t *)slab.take(pb);
        } else {
            slab.reserve(vb);
            slab.reserve(cb);
            slab.reserve(sb);
            slab.reserve(pb);
        }
    } else if (fmt == MG_STORAGE_ELL) {
        int K = 0;
        for (int64_t i = 0; i < A.nrows; i++) K = std::max<int>(K, (int)(A.rowptr[i + 1] - A.rowptr[i]));
        m.K = std::max(K, 1);
        size_t vb = (size_t)m.K * m.ld * sv, cb = (size_t)m.K * m.ld * 4;
        if (take) {
            m.val = slab.take(vb);
            m.col = (int32_t *)slab.take(cb);
        } else {
            slab.reserve(vb);
            slab.reserve(cb);
        }
    } else {
        m.K = 0;
        size_t vb = (size_t)std::max<int64_t>(m.nnz, 1) * sv, cb = (size_t)std::max<int64_t>(m.nnz, 1) * 4,
               rb = (size_t)(m.n + 1) * 8;
        if (take) {
            m.val = slab.take(vb);
            m.col = (int32_t *)slab.take(cb);
            m.rowptr = (int64_t *)slab.take(rb);
        } else {
            slab.reserve(vb);
            slab.reserve(cb);
            slab.reserve(rb);
        }
    }
}

template <typename T>
static void upload_matrix(const DevMat &m, const mgh::Csr &A, const std::vector<T> &vals, int dim, int N,
                          cudaStream_t s)
{
    if (m.fmt == MG_STORAGE_STENCIL || m.fmt == MG_STORAGE_COEF) return;  // no matrix values stored
    if (m.fmt == MG_STORAGE_DIA) {
        std::vector<T> v((size_t)m.K * m.ld, T(0));
        int k3 = dim == 3 ? 9 : 0;
        int slot_of[27];
        for (int p = 0; p < 27; p++) slot_of[p] = -1;
        for (int k = 0; k < m.K; k++) slot_of[m.full_of[k]] = k;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < A.nrows; i++) {
            int ci[3], cj[3];
            mgh::q1_coords(dim, N, i, ci);
            for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) {
                mgh::q1_coords(dim, N, A.col[k], cj);
                int slot = slot_of[(cj[0] - ci[0] + 1) + 3 * (cj[1] - ci[1] + 1) + k3 * (cj[2] - ci[2] + 1)];
                if (slot >= 0) v[(size_t)slot * m.ld + i] = vals[k];  // dropped positions hold only zeros
            }
        }
        CK(cudaMemcpyAsync(m.val, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    } else if (m.fmt == MG_STORAGE_SELL) {
        std::vector<int32_t> perm;
        std::vector<int64_t> sptr;
        sell_layout(A, perm, sptr);
        std::vector<T> v((size_t)std::max<int64_t>(m.padded, 1), T(0));
        std::vector<int32_t> c((size_t)std::max<int64_t>(m.padded, 1), 0);
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < m.nslices * 32; r++) {
            int64_t sl = r / 32, lane = r % 32, Ks = (sptr[sl + 1] - sptr[sl]) / 32;
            int64_t i = r < A.nrows ? perm[r] : -1;
            int64_t len = i >= 0 ? A.rowptr[i + 1] - A.rowptr[i] : 0;
            // padding: column i (square operators), else the row's first column, so that a
            // padded slot repeats a column of the row (lanes past n: any valid column)
            int64_t ir = i >= 0 ? i : perm[(size_t)sl * 32];
            int64_t lr = A.rowptr[ir + 1] - A.rowptr[ir];
            int32_t pad = (int32_t)(A.ncols == A.nrows ? ir : (lr > 0 ? A.col[A.rowptr[ir]] : 0));
            for (int64_t k = 0; k < Ks; k++) {
                size_t e = (size_t)(sptr[sl] + 32 * k + lane);
                if (k < len) {
                    c[e] = A.col[A.rowptr[i] + k];
                    v[e] = vals[A.rowptr[i] + k];
                } else {
                    c[e] = pad;
                }
            }
        }
        CK(cudaMemcpyAsync(m.val, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(m.col, c.data(), c.size() * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(m.rowptr, sptr.data(), sptr.size() * 8, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(m.perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    } else if (m.fmt == MG_STORAGE_ELL) {
        std::vector<T> v((size_t)m.K * m.ld, T(0));
        std::vector<int32_t> c((size_t)m.K * m.ld, 0);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < m.ld; i++) {
            int64_t len = i < A.nrows ? A.rowptr[i + 1] - A.rowptr[i] : 0;
            for (int k = 0; k < m.K; k++) {
                if (k < len) {
                    c[(size_t)k * m.ld + i] = A.col[A.rowptr[i] + k];
                    v[(size_t)k * m.ld + i] = vals[A.rowptr[i] + k];
                } else {
                    c[(size_t)k * m.ld + i] = (int32_t)std::min<int64_t>(i, std::max<int64_t>(A.nrows - 1, 0));
                }
            }
        }
        CK(cudaMemcpyAsync(m.val, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(m.col, c.data(), c.size() * 4, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    } else {
        CK(cudaMemcpyAsync(m.val, vals.data(), vals.size() * sizeof(T), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(m.col, A.col.data(), A.col.size() * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(m.rowptr, A.rowptr.data(), A.rowptr.size() * 8, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
}

// The colour-major copy G of level l's matrix: DIA / ELL slots and D^-1 gathered on the
// device from the level's own arrays (so both hold the same values in either precision),
// CSR rows reordered on the host.
static void upload_gs_copy(mg_hierarchy *h, int l, const mgh::Csr &A, const std::vector<int32_t> &perm)
{
    LevelD &L = h->lev[l];
    DevMat &G = L.G;
    int64_t n = L.n;
    if (n == 0) return;
    CK(cudaMemcpyAsync(L.perm, perm.data(), perm.size() * 4, cudaMemcpyHostToDevice, h->s));
    auto gather = [&](void *dst, const void *src, int K, int esz) {
        int64_t tot = n * K;
        unsigned grid = (unsigned)((tot + 255) / 256);
        if (esz == 8)
            k_gather_rows<double><<<grid, 256, 0, h->s>>>((double *)dst, (const double *)src, L.perm, n, G.ld, K);
        else if (esz == 4)
            k_gather_rows<float><<<grid, 256, 0, h->s>>>((float *)dst, (const float *)src, L.perm, n, G.ld, K);
        else
            k_gather_rows<int32_t><<<grid, 256, 0, h->s>>>((int32_t *)dst, (const int32_t *)src, L.perm, n, G.ld, K);
        CKL();
    };
    if (G.fmt == MG_STORAGE_DIA || G.fmt == MG_STORAGE_ELL) {
        gather(G.val, L.A.val, G.K, h->inner_size);
        if (G.fmt == MG_STORAGE_ELL) gather(G.col, L.A.col, G.K, -4);  // column indices
    } else {
        std::vector<int64_t> rp((size_t)n + 1, 0);
        for (int64_t r = 0; r < n; r++) rp[r + 1] = rp[r] + (A.rowptr[perm[r] + 1] - A.rowptr[perm[r]]);
        std::vector<int32_t> cols((size_t)A.nnz());
        std::vector<float> v32;
        if (h->mixed) mgh::round_fp32(A, v32);
        std::vector<double> vd(h->mixed ? 0 : (size_t)A.nnz());
        std::vector<float> vf(h->mixed ? (size_t)A.nnz() : 0);
        for (int64_t r = 0; r < n; r++) {
            int64_t src = A.rowptr[perm[r]], len = rp[r + 1] - rp[r];
            for (int64_t k = 0; k < len; k++) {
                cols[rp[r] + k] = A.col[src + k];
                if (h->mixed)
                    vf[rp[r] + k] = v32[src + k];
                else
                    vd[rp[r] + k] = A.val[src + k];
            }
        }
        if (h->mixed)
            CK(cudaMemcpyAsync(G.val, vf.data(), vf.size() * 4, cudaMemcpyHostToDevice, h->s));
        else
            CK(cudaMemcpyAsync(G.val, vd.data(), vd.size() * 8, cudaMemcpyHostToDevice, h->s));
        CK(cudaMemcpyAsync(G.col, cols.data(), cols.size() * 4, cudaMemcpyHostToDevice, h->s));
        CK(cudaMemcpyAsync(G.rowptr, rp.data(), rp.size() * 8, cudaMemcpyHostToDevice, h->s));
    }
    if (G.dinv) gather(G.dinv, L.A.dinv, 1, 8);
    CK(cudaStreamSynchronize(h->s));
}

static std::vector<float> to_f32(const std::vector<double> &v)
{
    std::vector<float> o(v.size());
    for (size_t i = 0; i < v.size(); i++) o[i] = (float)v[i];
    return o;
}

// Chebyshev coefficients of level l (the same recurrence as the smoother's definition)
static void cheb_coeffs(LevelD &L, const mg_options &o)
{
    double hi = o.cheb_hi * L.lambda;
    double lo = hi / o.cheb_ratio;
    double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
    double sigma = theta / delta;
    double rho0 = 1.0 / sigma;
    L.cheb_c0 = 1.0 / theta;
    L.cheb_c1.assign((size_t)std::max(o.cheb_degree, 1), 0.0);
    L.cheb_c2.assign((size_t)std::max(o.cheb_degree, 1), 0.0);
    for (int j = 1; j < o.cheb_degree; j++) {
        double rho1 = 1.0 / (2.0 * sigma - rho0);
        L.cheb_c1[j] = rho1 * rho0;
        L.cheb_c2[j] = (2.0 * rho1) / delta;
        rho0 = rho1;
    }
}

static int pick_storage(const mg_options &o, int elem)
{
    bool vertex_grid = elem == MG_Q1 || elem == MG_P1;  // DOFs on the grid vertices, stencil in the 27-point box
    if (o.storage == MG_STORAGE_DIA && !vertex_grid)
        throw Error(MG_EINVAL, "DIA storage needs Q1 or P1 (fixed stencil offsets)");
    if (o.storage == MG_STORAGE_STENCIL &&
        ((!vertex_grid && elem != MG_RQ1) || o.precision != MG_MIXED || o.smoother == MG_GAUSS_SEIDEL))
        throw Error(MG_EINVAL, "stencil storage needs Q1, P1 or rotated Q1, mixed precision and no Gauss-Seidel");
    if (o.storage == MG_STORAGE_COEF && (elem != MG_Q1 || o.precision != MG_MIXED || o.smoother == MG_GAUSS_SEIDEL))
        throw Error(MG_EINVAL, "coefficient storage needs 3D Q1, mixed precision and no Gauss-Seidel");
    if (o.storage != MG_STORAGE_AUTO) return o.storage == MG_STORAGE_STENCIL && elem == MG_RQ1 ? MG_STORAGE_STENCIL
                                                                                             : o.storage;
    return vertex_grid ? MG_STORAGE_DIA : MG_STORAGE_ELL;
}

// Storage chosen by measurement: every candidate format of this level's matrix is built
// in temporary device memory and timed on residual sweeps; the fastest wins. Choices are
// cached per (dim, element, cells, value size) for the life of the process.
template <typename T>
static double time_format(mg_hierarchy *h, const mgh::Csr &A, int fmt, int dim, int N, const double *svals,
                          const std::vector<float> *kap)
{
    mgi::Slab S;
    DevMat m;
    plan_matrix(m, A, fmt, dim, N, sizeof(T), S, false, svals, h->elem);
    int64_t n1 = N - 1;
    int64_t pad = (fmt == MG_STORAGE_DIA || fmt == MG_STORAGE_STENCIL || fmt == MG_STORAGE_COEF) && h->elem != MG_RQ1
                      ? round_up(dim == 3 ? n1 * n1 + n1 + 1 : n1 + 1, 64)
                      : 0;
    int64_t ld = round_up(std::max<int64_t>(A.nrows, 1), 64);
    S.reserve((size_t)(ld + 2 * pad) * sizeof(T));
    S.reserve((size_t)ld * sizeof(T) * 2);
    size_t bytes = S.used + 256;
    S.used = 0;
    S.size = bytes;
    S.base = h->own_alloc ? nullptr : (char *)h->dev.alloc(bytes, h->dev.ctx);
    if (h->own_alloc && cudaMalloc(&S.base, bytes) != cudaSuccess) {
        cudaGetLastError();
        S.base = nullptr;
    }
    if (!S.base) return 1e300;  // no room to try it: never chosen
    double ms_best = 1e300;
    try {
        plan_matrix(m, A, fmt, dim, N, sizeof(T), S, true, svals, h->elem);
        char *xb = (char *)S.take((size_t)(ld + 2 * pad) * sizeof(T));
        T *x = (T *)(xb + pad * sizeof(T));
        T *b = (T *)S.take((size_t)ld * sizeof(T)), *r = (T *)S.take((size_t)ld * sizeof(T));
        CK(cudaMemsetAsync(S.base, 0, S.size, h->s));
        std::vector<T> vals(A.val.begin(), A.val.end());
        upload_matrix<T>(m, A, vals, dim, N, h->s);
        if (fmt == MG_STORAGE_COEF) {
            if (!kap) throw Error(MG_EINVAL, "coefficient storage without coefficients");
            CK(cudaMemcpyAsync(m.val, kap->data(), kap->size() * 4, cudaMemcpyHostToDevice, h->s));
        }
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        // a busy GPU first (clocks leave their idle state), then the best of several runs.
        // An FP32 level is timed on what a V-cycle runs on it, three smoothing steps per
        // residual (the per-cell form has a separate residual kernel); an FP64 level on
        // residuals (its smoothing steps would read a D^-1 this trial does not build).
        auto four = [&]() {
            if constexpr (std::is_same<T, float>::value) {
                for (int k = 0; k < 3; k++)
                    sweep_fmt<T, SW_JACOBI>(m, (int)A.nrows, x, b, r, (T *)nullptr, T(0.8), T(0), h->s);
                sweep_fmt<T, SW_RESID>(m, (int)A.nrows, x, b, r, (T *)nullptr, T(0), T(0), h->s);
            } else {
                for (int k = 0; k < 4; k++)
                    sweep_fmt<T, SW_RESID>(m, (int)A.nrows, x, b, r, (T *)nullptr, T(0), T(0), h->s);
            }
        };
        for (int rep = 0; rep < 50; rep++) four();
        for (int rep = 0; rep < 10; rep++) {
            CK(cudaEventRecord(e0, h->s));
            four();
            CK(cudaEventRecord(e1, h->s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            ms_best = std::min(ms_best, (double)ms / 4.0);
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    } catch (...) {
        ms_best = 1e300;
    }
    CK(cudaStreamSynchronize(h->s));
    if (h->own_alloc)
        cudaFree(S.base);
    else
        h->dev.free(S.base, S.size, h->dev.ctx);
    return ms_best;
}

// svals: the level's constant stencil (constant_stencil) when it may be stored as one
// kap: the level's per-cell coefficients (coef_form) when it may be stored in that form
static int tune_storage(mg_hierarchy *h, const mgh::Csr &A, int dim, int elem, int N, const double *svals,
                        const std::vector<float> *kap)
{
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, bool, bool, bool>, int> cache;
    auto key = std::make_tuple(dim, elem, N, h->inner_size, h->mass != 0.0, svals != nullptr, kap != nullptr);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    std::vector<int> cands;
    if (elem == MG_Q1 || elem == MG_P1) cands.push_back(MG_STORAGE_DIA);
    cands.push_back(MG_STORAGE_ELL);
    cands.push_back(MG_STORAGE_CSR);
    if (elem == MG_RQ1 || elem == MG_P2) cands.push_back(MG_STORAGE_SELL);  // uneven rows (P2) or no DIA
    if (svals) cands.push_back(MG_STORAGE_STENCIL);
    if (kap && h->mixed) cands.push_back(MG_STORAGE_COEF);
    int best = cands[0];
    double best_ms = 1e300;
    for (int f : cands) {
        double ms = h->mixed ? time_format<float>(h, A, f, dim, N, svals, kap)
                             : time_format<double>(h, A, f, dim, N, svals, kap);
        if (ms < best_ms) {
            best_ms = ms;
            best = f;
        }
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = best;
    return best;
}

void mgi::build_hierarchy(mg_hierarchy *h, const mg_problem *p, const mg_options *o, const mg_device *dev,
                          bool with_vectors)
{
    validate_problem(p);
    h->with_vectors = with_vectors;
    if (o->smoother != MG_JACOBI && o->smoother != MG_CHEBYSHEV && o->smoother != MG_GAUSS_SEIDEL)
        throw Error(MG_EINVAL, "bad smoother");
    if (o->smoother == MG_CHEBYSHEV && (o->cheb_degree < 1 || !(o->cheb_ratio > 1.0) || !(o->cheb_hi > 0.0) || o->power_iters < 1))
        throw Error(MG_EINVAL, "bad Chebyshev parameters");
    if (o->nu_pre < 0 || o->nu_post < 0 || o->max_iters < 0) throw Error(MG_EINVAL, "negative counts");
    if (o->precision != MG_FP64 && o->precision != MG_MIXED) throw Error(MG_EINVAL, "bad precision");
    if (o->storage < MG_STORAGE_AUTO || o->storage > MG_STORAGE_COEF) throw Error(MG_EINVAL, "bad storage");
    if (o->storage == MG_STORAGE_COEF && (p->dim != 3 || p->mass != 0.0))
        throw Error(MG_EINVAL, "coefficient storage needs 3D Q1 without a mass shift");
    h->prob = *p;
    h->prob.k_cell = nullptr;
    h->opt = *o;
    h->dim = p->dim;
    h->elem = p->element;
    h->nlev = p->n_levels;
    h->Lf = p->n_levels - 1;
    h->mixed = o->precision == MG_MIXED;
    // the first pre-smoothing step of a level (from x = 0) rides on the kernel that makes
    // the level's right-hand side: the restriction on the levels below the finest, the
    // outer residual on the finest level of a mixed hierarchy
    h->zfuse = o->fuse_first != 0 && h->Lf >= 1 && o->nu_pre >= 1 &&
               (o->smoother == MG_JACOBI || o->smoother == MG_CHEBYSHEV);
    h->outer_z = h->zfuse && h->mixed;
    h->inner_size = h->mixed ? 4 : 8;
    if (dev) h->dev = *dev;
    h->own_alloc = !h->dev.alloc;
    CK(cudaGetDevice(&h->device));
    h->caller = (cudaStream_t)h->dev.stream;
    CK(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    CK(cudaMallocHost(&h->h_norm2, sizeof(double)));

    int dim = h->dim, elem = h->elem, nlev = h->nlev, Lf = h->Lf;
    h->lev.resize((size_t)nlev);
    // ---- host hierarchy, finest to coarsest ----
    mgh::HostHierarchy HH;
    mgh::build_hierarchy(dim, elem, p->n_cells, nlev, p->k_cell, 0, HH, p->mass);
    h->mass = p->mass;
    // Crank-Nicolson: B = sigma M - A of the finest level, entrywise on the common pattern
    mgh::Csr Bh;
    if (p->mass != 0.0 && with_vectors) {
        mgh::Csr Mf;
        mgh::assemble(dim, elem, p->n_cells, p->k_cell, Bh);
        mgh::assemble_mass(dim, elem, p->n_cells, Mf);
        for (size_t q = 0; q < Bh.val.size(); q++) Bh.val[q] = p->mass * Mf.val[q] - Bh.val[q];
    }
    std::vector<mgh::Csr> &A = HH.A, &P = HH.P, &R = HH.R;
    for (int l = Lf; l >= 0; l--) {
        LevelD &L = h->lev[l];
        L.N = HH.N[l];
        L.n = A[l].nrows;
        L.galerkin = HH.galerkin[l];
        L.nnz = A[l].nnz();
    }
    // ---- smoother parameters ----
    for (int l = 0; l <= Lf; l++) {
        LevelD &L = h->lev[l];
        L.omega = o->omega;
        if (l >= 1 && o->smoother == MG_CHEBYSHEV) {
            L.lambda = mgh::level_lambda(A[l], o->power_iters, o->power_seed);
            cheb_coeffs(L, *o);
        }
    }
    h->n0 = (int)h->lev[0].n;
    if (h->n0 > 1024) throw Error(MG_EINVAL, "coarsest level has more than 1024 DOFs; add levels");

    // ---- device memory plan (pass 0: count, pass 1: assign) ----
    int fmt = pick_storage(*o, elem);
    std::vector<int> lfmt((size_t)nlev, fmt);
    // constant-stencil storage: FP32 levels above the coarse-level tail whose every row is
    // the same stencil (checked exactly)
    std::vector<std::array<double, 27>> svals((size_t)nlev);
    std::vector<char> scan((size_t)nlev, 0);
    if (h->mixed && (elem == MG_Q1 || elem == MG_P1) && o->smoother != MG_GAUSS_SEIDEL)
        for (int l = 1; l <= Lf; l++)
            if (h->lev[l].n >= 32768) scan[l] = constant_stencil(A[l], dim, h->lev[l].N, 4, svals[l].data());
    if (h->mixed && elem == MG_RQ1 && o->smoother != MG_GAUSS_SEIDEL)
        for (int l = 1; l <= Lf; l++)
            if (h->lev[l].n >= 32768 && !h->lev[l].galerkin)
                scan[l] = rq1_constant_stencil(A[l], h->lev[l].N, svals[l].data());
    // per-cell coefficient storage: FP32 levels of 3D Q1 rediscretised with a per-cell
    // coefficient (checked against the assembled matrix)
    std::vector<std::vector<float>> kap((size_t)nlev);
    std::vector<char> coef((size_t)nlev, 0);
    if (h->mixed && elem == MG_Q1 && dim == 3 && p->mass == 0.0 && o->smoother != MG_GAUSS_SEIDEL &&
        (o->storage == MG_STORAGE_AUTO || o->storage == MG_STORAGE_COEF))
        for (int l = 1; l <= Lf; l++) {
            const LevelD &L = h->lev[l];
            if (L.n < 32768 || L.galerkin) continue;
            std::vector<double> kl;
            bool have = true;
            if (p->k_cell)
                have = mgh::coarse_coefficient(dim, p->n_cells, p->k_cell, L.N, kl);
            else
                kl.assign((size_t)L.N * L.N * L.N, 1.0);
            coef[l] = have && coef_form(A[l], L.N, kl, kap[l]);
        }
    if (o->storage == MG_STORAGE_AUTO) {  // measured on the levels large enough to be bandwidth-bound
        for (int l = 1; l <= Lf; l++)
            if (h->lev[l].n >= 32768)
                lfmt[l] = tune_storage(h, A[l], dim, elem, h->lev[l].N, scan[l] ? svals[l].data() : nullptr,
                                       coef[l] ? &kap[l] : nullptr);
    } else if (fmt == MG_STORAGE_STENCIL) {
        for (int l = 0; l <= Lf; l++)
            if (!scan[l]) lfmt[l] = elem == MG_RQ1 ? MG_STORAGE_ELL : MG_STORAGE_DIA;
    } else if (fmt == MG_STORAGE_COEF) {
        for (int l = 0; l <= Lf; l++)
            if (!coef[l]) lfmt[l] = MG_STORAGE_DIA;
    }
    int sv = h->inner_size;
    // ---- multicolour Gauss-Seidel: colour order of every smoothed level ----
    const bool gs = o->smoother == MG_GAUSS_SEIDEL;
    std::vector<std::vector<int32_t>> gs_perm((size_t)nlev);
    if (gs)
        for (int l = 1; l <= Lf; l++) {
            if (!mgh::colouring_valid(A[l], dim, elem, h->lev[l].N))
                throw Error(MG_EINVAL, "level " + std::to_string(l) + " couples two DOFs of one colour");
            mgh::colour_order(dim, elem, h->lev[l].N, gs_perm[l], h->lev[l].coff);
            h->lev[l].gs_groups = mgh::colour_launch_groups(A[l], dim, elem, h->lev[l].N, h->lev[l].coff);
        }
    for (int pass = 0; pass < 2; pass++) {
        bool take = pass == 1;
        mgi::Slab &S = h->slab;
        if (take) {
            size_t bytes = S.used + 256;
            S.used = 0;
            S.size = bytes;
            if (h->own_alloc) {
                cudaError_t e = cudaMalloc(&S.base, bytes);
                if (e != cudaSuccess) {
                    S.base = nullptr;
                    cudaGetLastError();
                    throw Error(MG_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
                }
            } else {
                S.base = (char *)h->dev.alloc(bytes, h->dev.ctx);
                if (!S.base) throw Error(MG_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
            }
        }
        auto vec = [&](size_t bytes) -> void * {
            if (take) return S.take(bytes);
            S.reserve(bytes);
            return nullptr;
        };
        for (int l = 0; l <= Lf; l++) {
            LevelD &L = h->lev[l];
            int lf = lfmt[l];
            L.fmt = lf;
            plan_matrix(L.A, A[l], lf, dim, L.N, sv, S, take, lf == MG_STORAGE_STENCIL ? svals[l].data() : nullptr, elem);
            if (!h->mixed && l >= 1) L.A.dinv = vec((size_t)L.A.ld * 8);  // FP64 smoothers read D^-1
            // FP32 sweeps from x = 0 on formats whose diagonal has no fixed slot read D^-1
            // instead of scanning the row (the same value: 1/a_ii rounded once)
            if (h->mixed && l >= 1 && lf != MG_STORAGE_DIA && lf != MG_STORAGE_STENCIL && lf != MG_STORAGE_COEF)
                L.A.dinv = vec((size_t)L.A.ld * 4);
            if (h->zfuse && l >= 1 && lf == MG_STORAGE_COEF) L.zdinv = vec((size_t)L.A.ld * 4);
            if (gs && l >= 1) {  // the colour-major copy of A for the Gauss-Seidel sweeps (CSR for SELL levels)
                plan_matrix(L.G, A[l], lf == MG_STORAGE_SELL ? MG_STORAGE_CSR : lf, dim, L.N, sv, S, take);
                if (!h->mixed) L.G.dinv = vec((size_t)L.G.ld * 8);
                L.perm = (int32_t *)vec((size_t)std::max<int64_t>(L.G.n, 1) * 4);
            }
            int64_t n1 = L.N - 1;
            L.pad = (lf == MG_STORAGE_DIA || lf == MG_STORAGE_STENCIL || lf == MG_STORAGE_COEF) && elem != MG_RQ1
                        ? round_up(dim == 3 ? n1 * n1 + n1 + 1 : n1 + 1, 64)
                        : 0;
            int64_t ld = L.A.ld;
            if (with_vectors) {
                for (int c = 0; c < 2; c++) {
                    char *base = (char *)vec((size_t)(ld + 2 * L.pad) * sv);
                    L.x[c] = take ? base + (size_t)L.pad * sv : nullptr;
                }
                L.b = vec((size_t)ld * sv);
                L.t = vec((size_t)ld * sv);
                L.d = vec((size_t)ld * sv);
            }
            if (l >= 1) {
                L.structured = elem == MG_Q1;
                if (!L.structured) {
                    plan_matrix(L.P, P[l], MG_STORAGE_SELL, dim, L.N, sv, S, take);
                    plan_matrix(L.R, R[l], MG_STORAGE_SELL, dim, L.N, sv, S, take);
                }
            }
        }
        LevelD &F = h->lev[Lf];
        if (h->mixed) {
            // the FP64 operator of the outer residual is stored (a stencil or coefficient level stores DIA)
            bool formed = F.fmt == MG_STORAGE_STENCIL || F.fmt == MG_STORAGE_COEF;
            int f64 = formed ? (elem == MG_RQ1 ? MG_STORAGE_SELL : MG_STORAGE_DIA) : F.fmt;
            plan_matrix(h->A64, A[Lf], f64, dim, F.N, 8, S, take);
        } else if (take) {
            h->A64 = F.A;
        }
        h->pad64 = F.pad;
        if (with_vectors) {
            char *base = (char *)vec((size_t)(F.A.ld + 2 * h->pad64) * 8);
            h->x64 = take ? (double *)(base + (size_t)h->pad64 * 8) : nullptr;
            h->b64 = (double *)vec((size_t)F.A.ld * 8);
            char *pb = (char *)vec((size_t)(F.A.ld + 2 * h->pad64) * 8);  // CG search direction
            h->pcg_p = take ? (double *)(pb + (size_t)h->pad64 * 8) : nullptr;
            h->pcg_r = (double *)vec((size_t)F.A.ld * 8);
            h->pcg_q = (double *)vec((size_t)F.A.ld * 8);
            h->pcg_scal = (double *)vec(PCG_NSCAL * 8);
            if (h->mass != 0.0) {
                bool formed = F.fmt == MG_STORAGE_STENCIL || F.fmt == MG_STORAGE_COEF;
                int f64 = formed ? (elem == MG_RQ1 ? MG_STORAGE_SELL : MG_STORAGE_DIA) : F.fmt;
                plan_matrix(h->B64, Bh, f64, dim, F.N, 8, S, take);
                h->bF64 = (double *)vec((size_t)F.A.ld * 8);
            }
        }
        h->lu = (double *)vec((size_t)h->n0 * h->n0 * 8);
        h->piv = (int *)vec((size_t)h->n0 * 4);
        h->d_info = (int *)vec(64);
        h->partial = (double *)vec((size_t)grid_for(F.A.ld) * 8);
        h->ticket = (unsigned *)vec(64);
        h->norm2 = (double *)vec(64);
    }
    // ---- upload ----
    CK(cudaMemsetAsync(h->slab.base, 0, h->slab.size, h->s));
    for (int l = 0; l <= Lf; l++) {
        LevelD &L = h->lev[l];
        if (h->mixed) {
            std::vector<float> v32;
            if (L.A.fmt == MG_STORAGE_COEF) {
                CK(cudaMemcpyAsync(L.A.val, kap[l].data(), kap[l].size() * 4, cudaMemcpyHostToDevice, h->s));
                if (L.zdinv) {
                    const int n1 = L.A.n1;
                    mgk::k_coef_dinv<<<dim3((unsigned)((n1 + 127) / 128), (unsigned)n1, (unsigned)n1), 128, 0, h->s>>>(
                        (const float *)L.A.val, n1, (float *)L.zdinv);
                    CK(cudaGetLastError());
                }
                CK(cudaStreamSynchronize(h->s));
            } else {
                mgh::round_fp32(A[l], v32);
                upload_matrix<float>(L.A, A[l], v32, dim, L.N, h->s);
            }
            if (L.A.dinv) {
                std::vector<float> dv((size_t)L.A.ld, 0.0f);
                for (int64_t i = 0; i < A[l].nrows; i++)
                    for (int64_t k = A[l].rowptr[i]; k < A[l].rowptr[i + 1]; k++)
                        if (A[l].col[k] == i) {
                            dv[i] = 1.0f / v32[k];
                            break;
                        }
                CK(cudaMemcpyAsync(L.A.dinv, dv.data(), dv.size() * 4, cudaMemcpyHostToDevice, h->s));
                CK(cudaStreamSynchronize(h->s));
            }
            if (l >= 1 && !L.structured) {
                upload_matrix<float>(L.P, P[l], to_f32(P[l].val), dim, L.N, h->s);
                upload_matrix<float>(L.R, R[l], to_f32(R[l].val), dim, L.N, h->s);
            }
        } else {
            upload_matrix<double>(L.A, A[l], A[l].val, dim, L.N, h->s);
            if (L.A.dinv) {
                std::vector<double> dv((size_t)L.A.ld, 0.0);
                for (int64_t i = 0; i < A[l].nrows; i++)
                    for (int64_t k = A[l].rowptr[i]; k < A[l].rowptr[i + 1]; k++)
                        if (A[l].col[k] == i) dv[i] = 1.0 / A[l].val[k];
                CK(cudaMemcpyAsync(L.A.dinv, dv.data(), dv.size() * 8, cudaMemcpyHostToDevice, h->s));
                CK(cudaStreamSynchronize(h->s));
            }
            if (l >= 1 && !L.structured) {
                upload_matrix<double>(L.P, P[l], P[l].val, dim, L.N, h->s);
                upload_matrix<double>(L.R, R[l], R[l].val, dim, L.N, h->s);
            }
        }
    }
    if (h->mixed) upload_matrix<double>(h->A64, A[Lf], A[Lf].val, dim, h->lev[Lf].N, h->s);
    if (gs)
        for (int l = 1; l <= Lf; l++) upload_gs_copy(h, l, A[l], gs_perm[l]);
    if (h->B64.val) upload_matrix<double>(h->B64, Bh, Bh.val, dim, h->lev[Lf].N, h->s);
    // ---- coarsest LU on the device ----
    {
        std::vector<double> dense((size_t)h->n0 * h->n0, 0.0);
        for (int i = 0; i < h->n0; i++)
            for (int64_t k = A[0].rowptr[i]; k < A[0].rowptr[i + 1]; k++) dense[(size_t)i * h->n0 + A[0].col[k]] = A[0].val[k];
        CK(cudaMemcpyAsync(h->lu, dense.data(), dense.size() * 8, cudaMemcpyHostToDevice, h->s));
        k_lu_factor<<<1, 256, 0, h->s>>>(h->lu, h->n0, h->piv, h->d_info);
        CKL();
        int info = 0;
        CK(cudaMemcpyAsync(&info, h->d_info, 4, cudaMemcpyDeviceToHost, h->s));
        CK(cudaStreamSynchronize(h->s));
        if (info) throw Error(MG_EINVAL, "coarsest matrix is singular");
    }
    // ---- coarse-level tail: the levels of at most 4096 rows in one cluster launch ----
    h->tail_level = -1;
    if (o->coarse_tail && h->n0 <= 64 && o->smoother != MG_GAUSS_SEIDEL) {
        int t = -1;
        for (int l = 0; l <= Lf; l++) {
            const LevelD &L = h->lev[l];
            bool ok = L.n <= 4096 && L.fmt == MG_STORAGE_DIA && (l == 0 || L.structured);
            if (!ok) break;
            t = l;
        }
        // operations one V-cycle records per tail level: the sweeps of pre- and post-smoothing,
        // the residual, the restriction, the zeroing of the correction and the prolongation
        int64_t spc = o->smoother == MG_JACOBI ? 1 : o->cheb_degree;
        int64_t per_level = ((int64_t)o->nu_pre + o->nu_post) * spc + 4;
        while (t >= 1 && 1 + t * per_level > TAIL_MAX_OPS) t--;
        if (t >= 1 && t < TAIL_MAX_LEVELS) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(h->tail_cluster);
            cfg.blockDim = dim3(512);
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = h->tail_cluster;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nclusters = 0;
            cudaError_t e = h->mixed ? cudaOccupancyMaxActiveClusters(&nclusters, k_tail<float>, &cfg)
                                     : cudaOccupancyMaxActiveClusters(&nclusters, k_tail<double>, &cfg);
            if (e == cudaSuccess && nclusters > 0)
                h->tail_level = t;
            else
                cudaGetLastError();
        }
    }
    // ---- launch count of one iteration, graphs ----
    if (!with_vectors) {
        CK(cudaStreamSynchronize(h->s));
        return;
    }
    if (o->coarse_tail == 2 && h->tail_level >= 1 && h->opt.use_graph) {
        // keep the tail only where the captured V-cycle is measurably faster with it
        double with_tail = time_vcycle_graph(h);
        int t = h->tail_level;
        h->tail_level = -1;
        destroy_graphs(h);
        double without = time_vcycle_graph(h);
        destroy_graphs(h);
        if (with_tail < 0.98 * without) h->tail_level = t;
    }
    h->counting = 1;
    h->kernels_per_cycle = 0;
    {
        // count by a dry enqueue on a capture that is discarded
        cudaGraph_t g = nullptr;
        h->capturing = true;
        CK(cudaStreamBeginCapture(h->s, cudaStreamCaptureModeThreadLocal));
        enqueue_r(h, h->s);
        enqueue_v(h, h->s);
        CK(cudaStreamEndCapture(h->s, &g));
        h->capturing = false;
        if (g) cudaGraphDestroy(g);
    }
    h->counting = 0;
    ensure_graphs(h);
    CK(cudaStreamSynchronize(h->s));
}

extern "C" mg_status mg_setup(const mg_problem *p, const mg_options *o, const mg_device *dev, mg_hierarchy **out)
{
    if (!out) {
        g_err = "out is NULL";
        return MG_EINVAL;
    }
    *out = nullptr;
    mg_options def;
    if (!o) {
        mg_options_default(&def);
        o = &def;
    }
    std::unique_ptr<mg_hierarchy> h(new (std::nothrow) mg_hierarchy());
    if (!h) {
        g_err = "host allocation failed";
        return MG_ENOMEM;
    }
    try {
        mgi::build_hierarchy(h.get(), p, o, dev, true);
    } catch (const Error &e) {
        g_err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        return MG_ENOMEM;
    }
    *out = h.release();
    return MG_OK;
}

extern "C" mg_status mg_hierarchy_free(mg_hierarchy *h)
{
    delete h;
    return MG_OK;
}

extern "C" mg_status mg_get_info(const mg_hierarchy *h, mg_info *info)
{
    if (!h || !info) {
        g_err = "NULL argument";
        return MG_EINVAL;
    }
    std::memset(info, 0, sizeof(*info));
    info->n_levels = h->nlev;
    info->precision = h->opt.precision;
    for (int l = 0; l < h->nlev; l++) {
        info->n[l] = h->lev[l].n;
        info->nnz[l] = h->lev[l].nnz;
        info->storage[l] = h->lev[l].fmt;
        info->galerkin[l] = h->lev[l].galerkin;
        info->lambda[l] = h->lev[l].lambda;
        info->transfer[l] = l == 0 ? MG_TRANSFER_NONE : (h->lev[l].structured ? MG_TRANSFER_GRID : MG_TRANSFER_SELL);
    }
    info->device_bytes = h->slab.size;
    info->kernels_per_cycle = h->kernels_per_cycle;
    info->tail_levels = h->tail_level + 1;
    return MG_OK;
}

// ------------------------------------------------------------------------------------
// Solve
// ------------------------------------------------------------------------------------
static void join_in(mg_hierarchy *h)
{
    CK(cudaEventRecord(h->ev_in, h->caller));
    CK(cudaStreamWaitEvent(h->s, h->ev_in, 0));
}

static void join_out(mg_hierarchy *h)
{
    CK(cudaEventRecord(h->ev_out, h->s));
    CK(cudaStreamWaitEvent(h->caller, h->ev_out, 0));
    CK(cudaStreamSynchronize(h->s));
}

// A right-hand side or initial guess holding a NaN or an infinity is rejected before the
// first cycle; a residual that stops being finite ends the iteration at once.
static void check_finite_start(double nb, double nr)
{
    if (!std::isfinite(nb)) throw Error(MG_EINVAL, "the right-hand side holds a NaN or an infinity");
    if (!std::isfinite(nr)) throw Error(MG_EINVAL, "the initial guess holds a NaN or an infinity");
}

static mg_status solve_internal(mg_hierarchy *h, double tol, int *iters, double *hist)
{
    ensure_graphs(h);
    double nb = norm_b(h);
    if (!std::isfinite(nb)) check_finite_start(nb, 0.0);
    int k = 0;
    mg_status st = MG_ENOCONV;
    run_r(h);
    double nr = std::sqrt(read_norm2(h));
    prof_collect(h, true, false);
    check_finite_start(nb, nr);
    bool diverged = false;
    for (;;) {
        double rel = nb > 0.0 ? nr / nb : nr;
        if (hist) hist[k] = rel;
        if (rel <= tol) {
            st = MG_OK;
            break;
        }
        if (!std::isfinite(rel)) {
            diverged = true;
            break;
        }
        if (k == h->opt.max_iters) break;
        run_v(h);
        run_r(h);
        nr = std::sqrt(read_norm2(h));
        prof_collect(h, true, true);
        k++;
    }
    if (iters) *iters = k;
    if (st == MG_ENOCONV) g_err = diverged ? "the residual is no longer finite" : "max_iters reached before the tolerance";
    return st;
}

// CG preconditioned by one V-cycle; hist[k] = ||r_k|| / ||b|| of the recursively updated
// residual, the same stopping rule as the defect correction
static mg_status pcg_internal(mg_hierarchy *h, double tol, int *iters, double *hist)
{
    if (h->opt.nu_pre != h->opt.nu_post)
        throw Error(MG_EINVAL, "conjugate gradients need a symmetric V-cycle (nu_pre == nu_post)");
    ensure_pcg_graphs(h);
    double nb = norm_b(h);
    if (!std::isfinite(nb)) check_finite_start(nb, 0.0);
    int k = 0;
    mg_status st = MG_ENOCONV;
    run_graph_or_eager(h, h->g_pi, enqueue_pi);
    double nr = std::sqrt(read_norm2(h));
    prof_collect_pcg(h, true, false);
    check_finite_start(nb, nr);
    bool diverged = false;
    for (;;) {
        double rel = nb > 0.0 ? nr / nb : nr;
        if (hist) hist[k] = rel;
        if (rel <= tol) {
            st = MG_OK;
            break;
        }
        if (!std::isfinite(rel)) {
            diverged = true;
            break;
        }
        if (k == h->opt.max_iters) break;
        run_graph_or_eager(h, h->g_pc, enqueue_pc);
        nr = std::sqrt(read_norm2(h));
        prof_collect_pcg(h, false, true);
        k++;
    }
    if (iters) *iters = k;
    if (st == MG_ENOCONV) g_err = diverged ? "the residual is no longer finite" : "max_iters reached before the tolerance";
    return st;
}

template <typename F>
static mg_status guarded(mg_hierarchy *h, F &&fn)
{
    if (!h) {
        g_err = "hierarchy is NULL";
        return MG_EINVAL;
    }
    std::lock_guard<std::mutex> lk(h->mu);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    mg_status st;
    try {
        st = fn();
    } catch (const Error &e) {
        g_err = e.msg;
        st = e.st;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        st = MG_ENOMEM;
    }
    if (prev != h->device) cudaSetDevice(prev);
    return st;
}

extern "C" mg_status mg_solve(mg_hierarchy *h, const double *b_dev, double *x_dev, double rel_tol, int *iters,
                              double *res_hist)
{
    return guarded(h, [&]() -> mg_status {
        if (!b_dev || !x_dev) throw Error(MG_EINVAL, "b or x is NULL");
        size_t bytes = (size_t)h->lev[h->Lf].n * 8;
        join_in(h);
        CK(cudaMemcpyAsync(h->b64, b_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
        CK(cudaMemcpyAsync(h->x64, x_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
        mg_status st = solve_internal(h, rel_tol, iters, res_hist);
        CK(cudaMemcpyAsync(x_dev, h->x64, bytes, cudaMemcpyDeviceToDevice, h->s));
        join_out(h);
        return st;
    });
}

extern "C" mg_status mg_solve_host(mg_hierarchy *h, const double *b_host, double *x_host, double rel_tol, int *iters,
                                   double *res_hist)
{
    return guarded(h, [&]() -> mg_status {
        if (!b_host || !x_host) throw Error(MG_EINVAL, "b or x is NULL");
        size_t bytes = (size_t)h->lev[h->Lf].n * 8;
        join_in(h);
        CK(cudaMemcpyAsync(h->b64, b_host, bytes, cudaMemcpyHostToDevice, h->s));
        CK(cudaMemcpyAsync(h->x64, x_host, bytes, cudaMemcpyHostToDevice, h->s));
        mg_status st = solve_internal(h, rel_tol, iters, res_hist);
        CK(cudaMemcpyAsync(x_host, h->x64, bytes, cudaMemcpyDeviceToHost, h->s));
        join_out(h);
        return st;
    });
}

extern "C" mg_status mg_pcg(mg_hierarchy *h, const double *b_dev, double *x_dev, double rel_tol, int *iters,
                            double *res_hist)
{
    return guarded(h, [&]() -> mg_status {
        if (!b_dev || !x_dev) throw Error(MG_EINVAL, "b or x is NULL");
        if (!h->with_vectors) throw Error(MG_EINVAL, "hierarchy has no vectors");
        size_t bytes = (size_t)h->lev[h->Lf].n * 8;
        join_in(h);
        CK(cudaMemcpyAsync(h->b64, b_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
        CK(cudaMemcpyAsync(h->x64, x_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
        mg_status st = pcg_internal(h, rel_tol, iters, res_hist);
        CK(cudaMemcpyAsync(x_dev, h->x64, bytes, cudaMemcpyDeviceToDevice, h->s));
        join_out(h);
        return st;
    });
}

extern "C" mg_status mg_pcg_host(mg_hierarchy *h, const double *b_host, double *x_host, double rel_tol, int *iters,
                                 double *res_hist)
{
    return guarded(h, [&]() -> mg_status {
        if (!b_host || !x_host) throw Error(MG_EINVAL, "b or x is NULL");
        if (!h->with_vectors) throw Error(MG_EINVAL, "hierarchy has no vectors");
        size_t bytes = (size_t)h->lev[h->Lf].n * 8;
        join_in(h);
        CK(cudaMemcpyAsync(h->b64, b_host, bytes, cudaMemcpyHostToDevice, h->s));
        CK(cudaMemcpyAsync(h->x64, x_host, bytes, cudaMemcpyHostToDevice, h->s));
        mg_status st = pcg_internal(h, rel_tol, iters, res_hist);
        CK(cudaMemcpyAsync(x_host, h->x64, bytes, cudaMemcpyDeviceToHost, h->s));
        join_out(h);
        return st;
    });
}

// Crank-Nicolson steps on the hierarchy's iterate x64 (u_k in, u_n out) with bF in bF64
static mg_status heat_internal(mg_hierarchy *h, const double *g, int n_steps, double tol, int method, int *iters)
{
    int n = (int)h->lev[h->Lf].n;
    MatView<double> v = view<double>(h->B64);
    bool pdl = h->opt.use_pdl != 0;
    for (int k = 0; k < n_steps; k++) {
        double t = g[k] + g[k + 1];
        {
            const DevMat &B = h->B64;
            double entries = mat_entries(B);
            LaunchScope ls(h, h->s, MG_K_OUTER, h->Lf, mat_bytes(B, 8) + 24.0 * n, 2.0 * entries + 2.0 * n);
            launch_fp64_rows(h, B, [&](auto fmt, auto kk) {
                klaunch(pdl, k_heat_rhs<decltype(fmt)::value, decltype(kk)::value>, dim3(grid_for(n)), dim3(256), 0,
                        h->s, v, n, (const double *)h->x64, (const double *)h->bF64, t, h->b64);
            });
        }
        int it = 0;
        mg_status st = method == MG_METHOD_PCG ? pcg_internal(h, tol, &it, nullptr) : solve_internal(h, tol, &it, nullptr);
        if (iters) iters[k] = it;
        if (st != MG_OK) return st;
    }
    return MG_OK;
}

static void heat_check(mg_hierarchy *h, const double *g, int n_steps, int method)
{
    if (h->mass == 0.0 || !h->B64.val) throw Error(MG_EINVAL, "the hierarchy has no mass shift (problem.mass)");
    if (!g || n_steps < 0) throw Error(MG_EINVAL, "bad g or n_steps");
    if (method != MG_METHOD_DC && method != MG_METHOD_PCG) throw Error(MG_EINVAL, "bad method");
}

extern "C" mg_status mg_heat(mg_hierarchy *h, const double *bF_dev, const double *g_host, int n_steps, double *u_dev,
                             double rel_tol, int method, int *iters)
{
    return guarded(h, [&]() -> mg_status {
        heat_check(h, g_host, n_steps, method);
        if (!bF_dev || !u_dev) throw Error(MG_EINVAL, "bF or u is NULL");
        size_t bytes = (size_t)h->lev[h->Lf].n * 8;
        ensure_graphs(h);
        join_in(h);
        CK(cudaMemcpyAsync(h->bF64, bF_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
        CK(cudaMemcpyAsync(h->x64, u_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
        mg_status st = heat_internal(h, g_host, n_steps, rel_tol, method, iters);
        CK(cudaMemcpyAsync(u_dev, h->x64, bytes, cudaMemcpyDeviceToDevice, h->s));
        join_out(h);
        return st;
    });
}

extern "C" mg_status mg_heat_host(mg_hierarchy *h, const double *bF_host, const double *g_host, int n_steps,
                                  double *u_host, double rel_tol, int method, int *iters)
{
    return guarded(h, [&]() -> mg_status {
        heat_check(h, g_host, n_steps, method);
        if (!bF_host || !u_host) throw Error(MG_EINVAL, "bF or u is NULL");
        size_t bytes = (size_t)h->lev[h->Lf].n * 8;
        ensure_graphs(h);
        join_in(h);
        CK(cudaMemcpyAsync(h->bF64, bF_host, bytes, cudaMemcpyHostToDevice, h->s));
        CK(cudaMemcpyAsync(h->x64, u_host, bytes, cudaMemcpyHostToDevice, h->s));
        mg_status st = heat_internal(h, g_host, n_steps, rel_tol, method, iters);
        CK(cudaMemcpyAsync(u_host, h->x64, bytes, cudaMemcpyDeviceToHost, h->s));
        join_out(h);
        return st;
    });
}

extern "C" mg_status mg_cycle(mg_hierarchy *h, const double *b_dev, double *x_dev, int n_cycles, double *rel_res)
{
    return guarded(h, [&]() -> mg_status {
        if (!b_dev || !x_dev || n_cycles < 0) throw Error(MG_EINVAL, "bad arguments");
        size_t bytes = (size_t)h->lev[h->Lf].n * 8;
        ensure_graphs(h);
        join_in(h);
        CK(cudaMemcpyAsync(h->b64, b_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
        CK(cudaMemcpyAsync(h->x64, x_dev, bytes, cudaMemcpyDeviceToDevice, h->s));
        double nb = norm_b(h);
        for (int c = 0; c < n_cycles; c++) {
            run_r(h);
            run_v(h);
            if (h->profiling) {
                CK(cudaStreamSynchronize(h->s));
                prof_collect(h, true, true);
            }
        }
        double nr = 0.0;
        if (n_cycles > 0) nr = std::sqrt(read_norm2(h));
        if (rel_res) *rel_res = nb > 0.0 ? nr / nb : nr;
        CK(cudaMemcpyAsync(x_dev, h->x64, bytes, cudaMemcpyDeviceToDevice, h->s));
        join_out(h);
        return MG_OK;
    });
}

// ------------------------------------------------------------------------------------
// Host-only assembly export
// ------------------------------------------------------------------------------------
extern "C" mg_status mg_assemble_operator(const mg_problem *p, int level, int which, int64_t *nrows, int64_t *nnz,
                                          int64_t *rowptr, int32_t *col, double *val)
{
    try {
        validate_problem(p);
        int Lf = p->n_levels - 1;
        if (level < 0 || level > Lf || which < 0 || which > 2 || (which > 0 && level < 1))
            throw Error(MG_EINVAL, "bad level/which");
        mgh::HostHierarchy HH;
        mgh::build_hierarchy(p->dim, p->element, p->n_cells, p->n_levels, p->k_cell, which == 0 ? level : level - 1, HH,
                             p->mass);
        const mgh::Csr &m = which == 0 ? HH.A[level] : (which == 1 ? HH.P[level] : HH.R[level]);
        if (nrows) *nrows = m.nrows;
        if (nnz) *nnz = m.nnz();
        if (rowptr) {
            std::memcpy(rowptr, m.rowptr.data(), m.rowptr.size() * 8);
            if (col) std::memcpy(col, m.col.data(), m.col.size() * 4);
            if (val) std::memcpy(val, m.val.data(), m.val.size() * 8);
        }
        return MG_OK;
    } catch (const Error &e) {
        g_err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        return MG_ENOMEM;
    }
}

extern "C" mg_status mg_constant_stencil(const mg_problem *p, int level, int *is_stencil)
{
    try {
        validate_problem(p);
        if (!is_stencil) throw Error(MG_EINVAL, "NULL argument");
        if (level < 0 || level > p->n_levels - 1) throw Error(MG_EINVAL, "bad level");
        *is_stencil = 0;
        if (p->element != MG_Q1 && p->element != MG_P1) return MG_OK;
        mgh::HostHierarchy HH;
        mgh::build_hierarchy(p->dim, p->element, p->n_cells, p->n_levels, p->k_cell, level, HH, p->mass);
        double vals[27];
        *is_stencil = constant_stencil(HH.A[level], p->dim, HH.N[level], 8, vals) ? 1 : 0;
        return MG_OK;
    } catch (const Error &e) {
        g_err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        g_err = "host allocation failed";
        return MG_ENOMEM;
    }
}

// ------------------------------------------------------------------------------------
// Export and profiling
// ------------------------------------------------------------------------------------
template <typename T>
static std::vector<double> download_vals(const DevMat &m, size_t count)
{
    std::vector<T> v(count);
    CK(cudaMemcpy(v.data(), m.val, count * sizeof(T), cudaMemcpyDeviceToHost));
    return std::vector<double>(v.begin(), v.end());
}

// transfers: the padding of a row without entries is a zero in column 0; transfer
// operators hold no stored zeros, so drop_zero removes exactly the padding
static void export_dev(const DevMat &m, int dim, int N, int sv, mgh::Csr &out, bool drop_zero = false)
{
    out.nrows = m.n;
    out.rowptr.assign((size_t)m.n + 1, 0);
    out.col.clear();
    out.val.clear();
    if (m.fmt == MG_STORAGE_CSR) {
        out.rowptr.resize((size_t)m.n + 1);
        CK(cudaMemcpy(out.rowptr.data(), m.rowptr, (m.n + 1) * 8, cudaMemcpyDeviceToHost));
        out.col.resize((size_t)m.nnz);
        CK(cudaMemcpy(out.col.data(), m.col, m.nnz * 4, cudaMemcpyDeviceToHost));
        out.val = sv == 8 ? download_vals<double>(m, (size_t)m.nnz) : download_vals<float>(m, (size_t)m.nnz);
        return;
    }
    if (m.fmt == MG_STORAGE_SELL) {  // back to rows in DOF order, padding dropped
        std::vector<double> v = sv == 8 ? download_vals<double>(m, (size_t)m.padded) : download_vals<float>(m, (size_t)m.padded);
        std::vector<int32_t> c((size_t)m.padded), perm((size_t)m.n);
        std::vector<int64_t> sptr((size_t)m.nslices + 1);
        CK(cudaMemcpy(c.data(), m.col, c.size() * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(perm.data(), m.perm, perm.size() * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(sptr.data(), m.rowptr, sptr.size() * 8, cudaMemcpyDeviceToHost));
        std::vector<std::vector<std::pair<int32_t, double>>> rows((size_t)m.n);
        for (int64_t r = 0; r < m.n; r++) {
            int64_t sl = r / 32, Ks = (sptr[sl + 1] - sptr[sl]) / 32;
            int32_t prev = -1;
            for (int64_t k = 0; k < Ks; k++) {
                size_t e = (size_t)(sptr[sl] + 32 * k + r % 32);
                if (c[e] <= prev) break;  // padding (column i after larger columns)
                if (drop_zero && v[e] == 0.0) continue;
                prev = c[e];
                rows[perm[r]].push_back({c[e], v[e]});
            }
        }
        for (int64_t i = 0; i < m.n; i++) {
            for (auto &e : rows[i]) {
                out.col.push_back(e.first);
                out.val.push_back(e.second);
            }
            out.rowptr[i + 1] = (int64_t)out.col.size();
        }
        return;
    }
    if (m.fmt == MG_STORAGE_COEF) {  // the operator the sweep applies: sums of -kap_e, 4 sum kap_e
        int64_t n1 = N - 1, nc = N;
        std::vector<float> kap((size_t)(nc * nc * nc));
        CK(cudaMemcpy(kap.data(), m.val, kap.size() * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < m.n; i++) {
            int ci[3] = {0, 0, 0};
            mgh::q1_coords(3, N, i, ci);
            auto K = [&](int a, int b, int c) { return kap[(size_t)((ci[0] - 1 + a) + nc * ((ci[1] - 1 + b) + nc * (ci[2] - 1 + c)))]; };
            for (int p = 0; p < 27; p++) {
                int d[3] = {p % 3 - 1, (p / 3) % 3 - 1, p / 9 - 1};
                int nz = (d[0] != 0) + (d[1] != 0) + (d[2] != 0);
                bool inside = true;
                for (int a = 0; a < 3; a++)
                    if (ci[a] + d[a] < 1 || ci[a] + d[a] > N - 1) inside = false;
                if (!inside) continue;
                float v = 0.0f;
                if (nz == 0) {
                    float ks = ((K(0, 0, 0) + K(1, 0, 0)) + (K(0, 1, 0) + K(1, 1, 0))) +
                               ((K(0, 0, 1) + K(1, 0, 1)) + (K(0, 1, 1) + K(1, 1, 1)));
                    v = 4.0f * ks;
                } else if (nz >= 2) {  // the cells holding both corners: one per nonzero offset side
                    for (int a = 0; a < 2; a++)
                        for (int b = 0; b < 2; b++)
                            for (int c = 0; c < 2; c++) {
                                int side[3] = {a, b, c};
                                bool both = true;
                                for (int q = 0; q < 3; q++)
                                    if (d[q] != 0 && side[q] != (d[q] > 0 ? 1 : 0)) both = false;
                                if (both) v -= K(a, b, c);
                            }
                }
                out.col.push_back((int32_t)(i + d[0] + n1 * d[1] + n1 * n1 * d[2]));
                out.val.push_back((double)v);
            }
            out.rowptr[i + 1] = (int64_t)out.col.size();
        }
        return;
    }
    if (m.fmt == MG_STORAGE_STENCIL && m.elem == MG_RQ1) {  // the face stencil, columns ascending
        float hv = (float)m.sval[1];
        const double rv[3] = {(double)(6.0f * hv), (double)hv, -(double)hv};
        for (int64_t i = 0; i < m.n; i++) {
            int64_t col[11];
            int role[11];
            int cnt = rq1_neighbours(N, i, col, role);
            std::vector<std::pair<int64_t, double>> row;
            for (int k = 0; k < cnt; k++) row.push_back({col[k], rv[role[k]]});
            std::sort(row.begin(), row.end());
            for (auto &e : row) {
                out.col.push_back((int32_t)e.first);
                out.val.push_back(e.second);
            }
            out.rowptr[i + 1] = (int64_t)out.col.size();
        }
        return;
    }
    if (m.fmt == MG_STORAGE_STENCIL) {  // every in-grid neighbour with the stencil's value
        int slot_of[27];
        for (int p = 0; p < 27; p++) slot_of[p] = -1;
        for (int k = 0; k < m.K; k++) slot_of[m.full_of[k]] = k;
        int64_t n1 = N - 1;
        for (int64_t i = 0; i < m.n; i++) {
            int ci[3] = {0, 0, 0};
            mgh::q1_coords(dim, N, i, ci);
            for (int p = 0; p < (dim == 3 ? 27 : 9); p++) {
                int d[3] = {p % 3 - 1, (p / 3) % 3 - 1, dim == 3 ? p / 9 - 1 : 0};
                bool inside = true;
                for (int a = 0; a < dim; a++)
                    if (ci[a] + d[a] < 1 || ci[a] + d[a] > N - 1) inside = false;
                if (!inside) continue;
                out.col.push_back((int32_t)(i + d[0] + n1 * d[1] + n1 * n1 * d[2]));
                out.val.push_back(slot_of[p] >= 0 ? m.sval[slot_of[p]] : 0.0);
            }
            out.rowptr[i + 1] = (int64_t)out.col.size();
        }
        return;
    }
    size_t cnt = (size_t)m.K * m.ld;
    std::vector<double> v = sv == 8 ? download_vals<double>(m, cnt) : download_vals<float>(m, cnt);
    std::vector<int32_t> c;
    if (m.fmt == MG_STORAGE_ELL) {
        c.resize(cnt);
        CK(cudaMemcpy(c.data(), m.col, cnt * 4, cudaMemcpyDeviceToHost));
    }
    int slot_of[27];
    for (int p = 0; p < 27; p++) slot_of[p] = -1;
    if (m.fmt == MG_STORAGE_DIA)
        for (int k = 0; k < m.K; k++) slot_of[m.full_of[k]] = k;
    int64_t n1 = N - 1;
    for (int64_t i = 0; i < m.n; i++) {
        if (m.fmt == MG_STORAGE_DIA) {
            // every in-grid neighbour is a structural entry; dropped positions are zero
            int ci[3] = {0, 0, 0};
            mgh::q1_coords(dim, N, i, ci);
            for (int p = 0; p < (dim == 3 ? 27 : 9); p++) {
                int d[3] = {p % 3 - 1, (p / 3) % 3 - 1, dim == 3 ? p / 9 - 1 : 0};
                bool inside = true;
                for (int a = 0; a < dim; a++)
                    if (ci[a] + d[a] < 1 || ci[a] + d[a] > N - 1) inside = false;
                if (!inside) continue;
                out.col.push_back((int32_t)(i + d[0] + n1 * d[1] + n1 * n1 * d[2]));
                out.val.push_back(slot_of[p] >= 0 ? v[(size_t)slot_of[p] * m.ld + i] : 0.0);
            }
        } else {
            int32_t prev = -1;
            for (int k = 0; k < m.K; k++) {
                int32_t j = c[(size_t)k * m.ld + i];
                if (j <= prev) break;  // padding (column i after larger columns)
                prev = j;
                out.col.push_back(j);
                out.val.push_back(v[(size_t)k * m.ld + i]);
            }
        }
        out.rowptr[i + 1] = (int64_t)out.col.size();
    }
}

extern "C" mg_status mg_export_operator(const mg_hierarchy *hc, int level, int which, int precision, int64_t *nrows,
                                        int64_t *nnz, int64_t *rowptr, int32_t *col, double *val)
{
    mg_hierarchy *h = const_cast<mg_hierarchy *>(hc);
    return guarded(h, [&]() -> mg_status {
        if (level < 0 || level > h->Lf || which < 0 || which > 2 || (which > 0 && level < 1))
            throw Error(MG_EINVAL, "bad level/which");
        mgh::Csr m;
        const LevelD &L = h->lev[level];
        if (which == 0) {
            if (precision == MG_FP64 && h->mixed) {
                if (level != h->Lf) throw Error(MG_EINVAL, "FP64 copy exists on the finest level only");
                export_dev(h->A64, h->dim, L.N, 8, m);
            } else if (precision == MG_MIXED && !h->mixed) {
                throw Error(MG_EINVAL, "no FP32 copy in an FP64 hierarchy");
            } else {
                export_dev(L.A, h->dim, L.N, h->inner_size, m);
            }
        } else if (L.structured) {
            mgh::Csr P;
            mgh::prolongation(h->dim, h->elem, h->lev[level - 1].N, P);
            if (which == 1)
                m = P;
            else
                mgh::transpose(P, m);
        } else {
            export_dev(which == 1 ? L.P : L.R, h->dim, L.N, h->inner_size, m, true);
            if (which == 2) m.nrows = h->lev[level - 1].n;
        }
        if (which == 2 && L.structured) m.nrows = h->lev[level - 1].n;
        if (nrows) *nrows = m.nrows;
        if (nnz) *nnz = m.nnz();
        if (rowptr) {
            std::memcpy(rowptr, m.rowptr.data(), m.rowptr.size() * 8);
            if (col) std::memcpy(col, m.col.data(), m.col.size() * 4);
            if (val) std::memcpy(val, m.val.data(), m.val.size() * 8);
        }
        return MG_OK;
    });
}

extern "C" mg_status mg_profile_enable(mg_hierarchy *h, int enable, unsigned class_mask, unsigned level_mask)
{
    return guarded(h, [&]() -> mg_status {
        CK(cudaStreamSynchronize(h->s));
        destroy_graphs(h);
        h->prof.release(h->rec_eager);
        h->prof.reset();
        h->profiling = enable != 0;
        h->prof_class_mask = class_mask;
        h->prof_level_mask = level_mask;
        ensure_graphs(h);
        return MG_OK;
    });
}

extern "C" mg_status mg_profile_read(const mg_hierarchy *h, int kclass, int level, double *ms_total, int64_t *launches,
                                     double *bytes_per_launch, double *flops_per_launch)
{
    if (!h || kclass < 0 || kclass >= MG_K_COUNT || level < 0 || level >= MG_MAX_LEVELS) {
        g_err = "bad arguments";
        return MG_EINVAL;
    }
    int k = kclass * MG_MAX_LEVELS + level;
    if (ms_total) *ms_total = h->prof.ms_total[k];
    if (launches) *launches = h->prof.launches[k];
    if (bytes_per_launch) *bytes_per_launch = h->prof.launches[k] ? h->prof.bytes_total[k] / h->prof.launches[k] : 0.0;
    if (flops_per_launch) *flops_per_launch = h->prof.launches[k] ? h->prof.flops_total[k] / h->prof.launches[k] : 0.0;
    return MG_OK;
}

// ------------------------------------------------------------------------------------
// Residual and norm without any allocation
// ------------------------------------------------------------------------------------
// Some callers cannot allocate device memory when they need a residual: code running
// where cudaMalloc is not allowed or would stall (a memory pool that owns the whole
// device, an allocator that must not be re-entered from a callback, a latency-critical
// path that may not trigger allocation). mg_residual_norm_noalloc serves them: its
// block partial sums, completion ticket and result live in the fixed device array
// below (about 512 KiB, held by every GPU that loads the library until the process
// exits), so a call allocates nothing. The array is shared by all calls: overlapping
// calls on the GPU (different streams or threads) race on it.
#define MG_NOALLOC_MAX_BLOCKS 65536
#define MG_NOALLOC_MAX_ROWS ((int64_t)MG_NOALLOC_MAX_BLOCKS * 256)

struct NoallocScratch {
    double partial[MG_NOALLOC_MAX_BLOCKS];
    double result;
    unsigned ticket;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Same residual as the outer residual kernel, for x without the padding the DIA gathers
// need: neighbours outside [0, n) read as zero (their matrix entries are zero).
template <int FMT, int K>
__global__ void __launch_bounds__(256) k_residual_noalloc(MatView<double> A, int n, const double *__restrict__ x,
                                                          const double *__restrict__ b, double *__restrict__ r,
                                                          NoallocScratch *sc)
{
    int q = blockIdx.x * blockDim.x + threadIdx.x;  // storage position (the DOF but for SELL)
    double sq = 0.0;
    if (q < n) {
        int i = FMT == MG_STORAGE_SELL ? __ldg(A.perm + q) : q;
        double s = 0.0;
        if (FMT == MG_STORAGE_DIA) {
#pragma unroll
            for (int k = 0; k < K; k++) {
                int64_t j = (int64_t)i + A.offs.o[k];
                double xv = (j >= 0 && j < n) ? __ldg(x + j) : 0.0;
                s = __fma_rn(__ldcs(A.val + (int64_t)k * A.ld + i), xv, s);
            }
        } else if (FMT == MG_STORAGE_ELL) {
            for (int k = 0; k < A.K; k++) {
                int c = __ldcs(A.col + (int64_t)k * A.ld + i);
                s = __fma_rn(__ldcs(A.val + (int64_t)k * A.ld + i), __ldg(x + c), s);
            }
        } else if (FMT == MG_STORAGE_SELL) {
            int64_t base = A.rowptr[q >> 5];
            int Ks = (int)((A.rowptr[(q >> 5) + 1] - base) >> 5);
            int64_t e = base + (q & 31);
            for (int k = 0; k < Ks; k++, e += 32) s = __fma_rn(__ldcs(A.val + e), __ldg(x + __ldcs(A.col + e)), s);
        } else {
            for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; k++) s = __fma_rn(A.val[k], __ldg(x + A.col[k]), s);
        }
        double ri = __dsub_rn(b[i], s);
        r[i] = ri;
        sq = ri * ri;
    }
    finish_norm(sq, sc->partial, &sc->ticket, &sc->result);
}

// Device address of the scratch array, looked up once per device with that device
// current (the host-side name of a __device__ variable is not a device address).
static NoallocScratch *noalloc_scratch_address(int device)
{
    static std::mutex mu;
    static NoallocScratch *addr[256] = {};
    if (device < 0 || device >= 256) throw Error(MG_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw Error(MG_ECUDA, std::string("cudaGetSymbolAddress of the residual scratch: ") + cudaGetErrorString(e));
        addr[device] = (NoallocScratch *)p;
    }
    return addr[device];
}

extern "C" mg_status mg_residual_norm_noalloc(mg_hierarchy *h, const double *b_dev, const double *x_dev, double *r_dev,
                                              double *rnorm)
{
    return guarded(h, [&]() -> mg_status {
        if (!b_dev || !x_dev || !r_dev || !rnorm) throw Error(MG_EINVAL, "b, x, r or rnorm is NULL");
        const DevMat &A = h->A64;
        int64_t n = A.n;
        if (n > MG_NOALLOC_MAX_ROWS)
            throw Error(MG_EINVAL, "mg_residual_norm_noalloc: " + std::to_string(n) + " rows exceed its limit of " +
                                       std::to_string(MG_NOALLOC_MAX_ROWS));
        NoallocScratch *sc = noalloc_scratch_address(h->device);
        cudaStream_t s = h->caller;
        // the ticket must start at zero; the last block resets it, this covers an aborted call
        CK(cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned), s));
        MatView<double> v = view<double>(A);
        unsigned g = grid_for(n);
        int nn = (int)n;
        if (A.fmt == MG_STORAGE_DIA) {
            with_dia_k(A.K, [&](auto k) {
                k_residual_noalloc<MG_STORAGE_DIA, decltype(k)::value><<<g, 256, 0, s>>>(v, nn, x_dev, b_dev, r_dev, sc);
            });
        } else if (A.fmt == MG_STORAGE_ELL) {
            k_residual_noalloc<MG_STORAGE_ELL, 1><<<g, 256, 0, s>>>(v, nn, x_dev, b_dev, r_dev, sc);
        } else if (A.fmt == MG_STORAGE_SELL) {
            k_residual_noalloc<MG_STORAGE_SELL, 1><<<g, 256, 0, s>>>(v, nn, x_dev, b_dev, r_dev, sc);
        } else {
            k_residual_noalloc<MG_STORAGE_CSR, 1><<<g, 256, 0, s>>>(v, nn, x_dev, b_dev, r_dev, sc);
        }
        CKL();
        double nr2 = 0.0;
        CK(cudaMemcpyAsync(&nr2, &sc->result, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *rnorm = std::sqrt(nr2);
        return MG_OK;
    });
}
