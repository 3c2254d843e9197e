// mg_internal.h -- data structures shared by the library's translation units (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "mg.h"

namespace mgi {

struct Error {
    mg_status st;
    std::string msg;
    Error(mg_status s, std::string m) : st(s), msg(std::move(m)) {}
};

void set_error(const std::string &m);

// One device allocation per hierarchy, carved into 256-byte aligned pieces. A first
// pass only reserves (counts) so that the total is known before the allocation.
struct Slab {
    char *base = nullptr;
    size_t size = 0, used = 0;
    void reserve(size_t bytes);
    void *take(size_t bytes);
};

// A level operator in one device format (values of elem_size bytes).
struct DevMat {
    int fmt = 0;  // MG_STORAGE_*
    int64_t n = 0, ld = 0, nnz = 0;
    int K = 0;
    int elem_size = 8;
    mgk::DiaOffs offs{};
    int center = 0;      // DIA: stored slot of the diagonal
    int full_of[27] = {};// DIA: stencil position (dx+1) + 3(dy+1) + 9(dz+1) of each stored slot
    void *val = nullptr;
    int32_t *col = nullptr;
    int32_t *perm = nullptr;  // SELL: DOF of each storage position
    int64_t nslices = 0;      // SELL: slices of 32 rows
    int64_t padded = 0;       // SELL: stored slots (entries incl. padding)
    int64_t *rowptr = nullptr;
    void *dinv = nullptr;  // 1 / a_ii: FP64 levels; FP32 ELL/CSR/SELL levels
    // STENCIL (slots as DIA): the value of each slot and 1 / a_ii in the inner precision
    // (held as double), the grid (interior points per axis, dimension)
    double sval[27] = {};
    double sdinv = 0.0;
    int n1 = 0, dim = 3;
    int elem = MG_Q1;  // STENCIL: MG_RQ1 for the face stencil (sval[0..2]: diagonal, opposite, other)
};

struct LevelD {
    int N = 0;        // cells per axis
    int64_t n = 0;    // DOFs
    int64_t nnz = 0;  // structural nonzeros of A
    int fmt = 0;
    int64_t pad = 0;  // zero elements on each side of the x buffers (DIA gathers)
    int galerkin = 0;
    DevMat A;         // inner precision
    void *x[2] = {nullptr, nullptr};
    // 1 / a_ii of a per-cell-coefficient level, read by the kernel that takes the level's
    // first smoothing step with its right-hand side (zfuse)
    void *zdinv = nullptr;
    void *b = nullptr, *t = nullptr, *d = nullptr;
    bool structured = false;  // Q1 transfers computed from the grid
    DevMat P, R;              // explicit transfers to level-1 (SELL-32)
    // multicolour Gauss-Seidel: a copy of A with its rows stored colour by colour (row r
    // of G is DOF perm[r]; colour c owns rows coff[c] .. coff[c+1]); D^-1 in G.dinv
    DevMat G;
    int32_t *perm = nullptr;
    std::vector<int64_t> coff;
    std::vector<std::pair<int64_t, int64_t>> gs_groups;  // row ranges of one sweep's launches
    double omega = 0.8, lambda = 0.0, cheb_c0 = 0.0;
    std::vector<double> cheb_c1, cheb_c2;
};

struct Prof {
    struct Rec {
        int kclass, level;
        double bytes, flops;
        cudaEvent_t e0, e1;
    };
    double ms_total[MG_K_COUNT * MG_MAX_LEVELS] = {};
    int64_t launches[MG_K_COUNT * MG_MAX_LEVELS] = {};
    double bytes_total[MG_K_COUNT * MG_MAX_LEVELS] = {};
    double flops_total[MG_K_COUNT * MG_MAX_LEVELS] = {};
    void begin(cudaStream_t s, int kclass, int level, double bytes, double flops, std::vector<Rec> *sink,
               bool capturing);
    void end(cudaStream_t s, std::vector<Rec> *sink, bool capturing);
    void collect(std::vector<Rec> &recs);
    void release(std::vector<Rec> &recs);
    void reset()
    {
        for (int k = 0; k < MG_K_COUNT * MG_MAX_LEVELS; k++) {
            ms_total[k] = 0.0;
            launches[k] = 0;
            bytes_total[k] = 0.0;
            flops_total[k] = 0.0;
        }
    }
};

}  // namespace mgi

// A level hierarchy: device operators of every level, the coarsest LU factors, and
// (unless with_vectors is false) the vectors and CUDA graphs of the single-solve path.
struct mg_hierarchy {
    mg_problem prob{};
    mg_options opt{};
    int dim = 0, elem = 0, nlev = 0, Lf = 0;
    bool mixed = false;
    int inner_size = 8;  // bytes per inner-precision value
    mg_device dev{};
    bool own_alloc = false;
    cudaStream_t caller = nullptr, s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int device = 0;
    mgi::Slab slab;
    std::vector<mgi::LevelD> lev;
    mgi::DevMat A64;               // finest FP64 operator for the outer residual
    double *x64 = nullptr;      // interior pointer of the padded FP64 iterate
    double *b64 = nullptr;
    int64_t pad64 = 0;
    double *lu = nullptr;
    int *piv = nullptr;
    int *d_info = nullptr;
    int n0 = 0;
    double *partial = nullptr;
    unsigned *ticket = nullptr;
    double *norm2 = nullptr;
    double *h_norm2 = nullptr;  // pinned
    cudaGraphExec_t g_r = nullptr, g_v = nullptr;
    // preconditioned CG (mg_pcg): FP64 residual, search direction (padded like x64), A p,
    // the recurrence scalars; one graph for r_0, one per iteration
    double *pcg_r = nullptr, *pcg_p = nullptr, *pcg_q = nullptr, *pcg_scal = nullptr;
    cudaGraphExec_t g_pi = nullptr, g_pc = nullptr;
    // Crank-Nicolson (mg_heat): sigma, B = sigma M - A on the finest level (FP64), bF
    double mass = 0.0;
    mgi::DevMat B64;
    double *bF64 = nullptr;
    bool capturing = false;
    // profiling
    bool profiling = false;
    unsigned prof_class_mask = ~0u, prof_level_mask = ~0u;
    mgi::Prof prof;
    std::vector<mgi::Prof::Rec> rec_r, rec_v, rec_pi, rec_pc, rec_eager;
    std::vector<mgi::Prof::Rec> *sink = nullptr;
    int kernels_per_cycle = 0;
    int counting = 0;  // counts launches while > 0
    bool with_vectors = true;  // false: operators only (serving keeps vectors per request)
    // coarse-level tail: levels 0..tail_level run as one cluster launch (-1: none)
    int tail_level = -1;
    int tail_cluster = 8;
    bool tail_rec = false;
    // the V-cycle being enqueued is followed by x64 += c (enqueue_v); the finest level's last
    // post-smoothing sweep applied it (update_fused)
    bool fuse_update = false, update_fused = false;
    // zfuse: the restriction to level l - 1 >= 1 also takes that level's first smoothing
    // step (from x = 0); outer_z: the outer residual kernel takes the finest level's, and
    // the V-cycle that follows it (enqueue_v) starts after that step
    bool zfuse = false, outer_z = false;
    std::vector<mgk::TailOp> tail_ops;
    std::mutex mu;

    ~mg_hierarchy();
};

namespace mgi {
// Build h from the problem on the current device (host assembly, device formats, LU).
void build_hierarchy(mg_hierarchy *h, const mg_problem *p, const mg_options *o, const mg_device *dev,
                     bool with_vectors);
}  // namespace mgi

