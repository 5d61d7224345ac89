// fmm_internal.cuh -- internal declarations of the GB300 DTT-FMM library.
//
// Data layout in HBM (all owned by the handle):
//   particles  : float4 pos[N] in Morton order, (d_x, d_y, d_z, q) with d = u - X_frame
//                the offset of the normalised position u in (-1,1)^3 from the centre
//                of the parent of the particle's leaf, rounded once to FP32; perm[N]
//                int32 maps sorted slot -> caller index.
//   cells      : breadth-first order (level by level, Morton order inside a
//                level).  Structure-of-arrays: prefix (u64), level, pbeg,
//                pcnt, cbeg, ccnt, parent (int32), geom float4 (centre, radius).
//   lists      : int32 source cell ids grouped by target (CSR offsets per cell).
//   expansions : M and L, ncells x TP floats (TP = coefficients padded to 4).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fmm.h"

namespace fmm {

constexpr int kLevels = 21;     // 3 * 21 = 63 Morton bits (Sec. 2: 21 levels per 64-bit key)
constexpr int kPhases = FMM_NPHASES;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);

#define FMM_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ::fmm::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define FMM_CHECK_LAUNCH(what)                                                \
    do {                                                                      \
        cudaError_t e_ = cudaGetLastError();                                  \
        if (e_ != cudaSuccess) return ::fmm::cuda_fail(e_, what, __FILE__, __LINE__); \
    } while (0)

#define FMM_TRY(expr)                                                         \
    do {                                                                      \
        int r_ = (expr);                                                      \
        if (r_ != FMM_OK) return r_;                                          \
    } while (0)

// ---------------------------------------------------------------------------
// growable device buffer
// ---------------------------------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int reserve(size_t need);        // grows (contents discarded), never shrinks
    int reserve_keep(size_t need, cudaStream_t s);   // grows keeping contents
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Expansion orders compiled into the library.
inline bool supported_order(int P) { return P == 3 || P == 4 || P == 5 || P == 6 || P == 8; }

// Device-side counters of the traversal (one struct, zeroed per traversal).
struct TravCounters {
    unsigned long long n_m2l;     // pairs emitted to the M2L list
    unsigned long long n_p2p;     // pairs emitted to the P2P list
    unsigned long long pass_count[9];   // work-stack passes: seeds of pass p (spills of pass p - 1)
    unsigned long long pass_claim[8];   // work-stack pass p: next seed to claim
    unsigned long long p2p_pairs; // sum over P2P pairs of n_target * n_source
    unsigned int overflow;        // bit 0: m2l, bit 1: p2p, bit 2: frontier/spill
    unsigned int seg_long;        // list grouping: bit 0 / 1 when the m2l / p2p list repeats a (target, source) pair
    unsigned int reg_max[2];      // traversal: largest region count of the m2l / p2p list
    unsigned int nleaves;         // leaves found by the leaf-list kernel
    unsigned long long round_count[16];   // frontier size before each seeding round
};

// Page-locked host scratch of a handle (counters read back during a build).
struct PinnedScratch {
    TravCounters ctr;
    int2 root_kids;
    unsigned level_total;
    unsigned err;
};

struct Handle {
    // configuration
    int64_t N = 0;
    int P = 0, TP = 0, ncrit = 0;
    float theta = 0.f;
    int64_t hybrid_min_pairs = -1;   // M2L / P2P hybrid at the leaves (< 0: off)
    unsigned flags = 0;
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    PinnedScratch *pinned = nullptr;   // page-locked host scratch

    // build state
    const double *x_built = nullptr;
    bool built = false;
    bool evaluated = false;
    double norm_host[4] = {0, 0, 0, 1};   // centre xyz, h

    // normalisation / keys / sort
    DevBuf norm;          // double[4] + bbox partials
    DevBuf bbox_part;     // double[nblocks * 6]
    DevBuf err_flag;      // unsigned int: bit 0 = non-finite input, 1 = P2P staging wait, 2 = tensor-core wait, 3 = radix look-back wait
    DevBuf keys, keys_alt;        // u64[N]
    DevBuf idx, idx_alt;          // u32[N]
    DevBuf sort_hist;             // u32[256 * tiles]
    DevBuf scan_tmp;              // u32 scratch of the device-wide scan
    DevBuf pos_unsorted;          // float4[N]
    DevBuf u_unsorted, u_sorted;  // double[3][N]: normalised FP64 coordinates, input / Morton order
    DevBuf pos;                   // float4[N] sorted (u, q)
    DevBuf perm;                  // int32[N]

    // cells
    int64_t ncells = 0, nleaves = 0, cell_cap = 0;
    int nlevels = 0;
    std::vector<int64_t> level_off;   // host: first cell of each level, size nlevels + 1
    DevBuf c_prefix;      // u64
    DevBuf c_level, c_pbeg, c_pcnt, c_cbeg, c_ccnt, c_parent;   // int32
    DevBuf c_geom;        // float4 (centre, radius)
    DevBuf c_scale;       // float2 (1/h, 1/h^2) per cell: output units when cells of several systems share arrays
    DevBuf c_kids;        // int2 (first child, child count) for the traversal
    DevBuf c_r2bits;      // u32 max squared radius (bits) during the build
    DevBuf c_tmp;         // int32 per-cell scratch (child counts / offsets)
    DevBuf leaf_of;       // int32[N] leaf of each sorted particle

    // traversal
    DevBuf counters;      // TravCounters
    DevBuf front[2];      // int2 frontier / seed / spill arrays
    int64_t front_cap = 0;
    DevBuf m2l_raw, p2p_raw;   // int2 pairs as emitted
    int64_t m2l_cap = 0, p2p_cap = 0;   // per-region capacities of the traversal's list buffers
    DevBuf trav_reg;                    // unsigned[2 * regions]: region counts of the traversal
    DevBuf ldense;                      // int2[n]: a list compacted from its regions (radix regrouping only)
    int64_t n_m2l = 0, n_p2p = 0, p2p_pairs = 0;
    // grouped lists
    DevBuf lkeys, lkeys_alt;   // packed (target, source) keys of the radix grouping (long lists only)
    DevBuf lcnt;               // unsigned[ncells + 1]: per-target counts, then offsets, of the grouping
    // the M2L list is grouped on a second stream, beside the P2P list and the
    // mutual split (its own scratch; joined before the build returns)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool side_pending = false;
    DevBuf lcnt_side, lkeys_side, scan_tmp_side;
    DevBuf m2l_src, m2l_off;   // int32 sources, CSR offsets (ncells + 1)
    DevBuf p2p_src, p2p_off;
    DevBuf leaf_list;          // int32 leaf cell ids
    DevBuf p2p_items;          // int4 (leaf, first target, target count, leaf-list index) P2P work items
    DevBuf p2p_poff;           // u32 first source run of each leaf (leaf-list order), nleaves + 1
    DevBuf p2p_ent;            // float4 (X_frame(S) - X_frame(T), first particle) per source run
    DevBuf p2p_cnt;            // int end particle (exclusive) per source run
    int64_t n_pieces = 0;      // source runs over all target leaves
    int64_t n_items = 0;
    int p2p_g = 0;             // targets per P2P work item (0: the default, 16; 8 on request)
    DevBuf pairs_count;        // u64 scratch (P2P particle-pair count)
    // mutual schedule (FMM_FLAG_MUTUAL): the lists split into mutual entries
    // (B > A, mirrored) and one-sided ones (CSR by cell), their source runs, and
    // the accumulator of the mutual pass (float4 per sorted particle)
    bool mutual_ready = false;
    int mu_lanes = 2;               // staged sources per lane of the mutual pass: 2 (6 blocks / SM) or 4 (4 blocks / SM)
    bool full_runs_ready = false;   // the whole lists' runs (p2p_poff / ent / cnt) are built
    DevBuf mu_off, mu_src, os_off, os_src, mu_cnt_tmp;
    DevBuf mu_poff, mu_ent, mu_cnt, os_poff, os_ent, os_cnt;
    DevBuf racc;

    // expansions and outputs
    DevBuf M, L;          // float[ncells * TP]
    DevBuf Mf;            // folded multipoles of the harmonic M2L with centre and level, float4[ncells * (ceil(P^2 / 4) + 1)]

    // adjoint (fmm_backward): sorted upstream gradients, expansions of the
    // adjoint sources, work items of <= 8 targets
    DevBuf adj;           // float4[N] (dL/dphi, h^-1 dL/dgrad) in sorted order
    DevBuf Ma, La;        // float[ncells * TP]
    DevBuf adj_items;     // int4 work items
    int64_t n_adj_items = 0;
    bool adj_items_ready = false;

    // many charge vectors (fmm_evaluate_batch): charges [N][32] in sorted order
    // (FP32 and its BF16 hi / lo split), expansions [ncells][TP][32]
    DevBuf qb, qbh, qbl;
    DevBuf Mb, Lb;
    // the tensor-core P2P + L2P of the batched evaluation: work items of <= 32
    // targets, the leaves' local expansions split into BF16 hi / lo
    // [leaf][T][32], and the persistent CTAs' work counter
    DevBuf tc_items, lbh, lbl, tc_next;
    int64_t n_tc_items = 0;
    bool tc_items_ready = false;

    DevBuf phi_sorted;    // float[N] potential in sorted order (for the energy)
    DevBuf energy_part;   // double partials

    // host-side scratch for the host-buffer entry point
    DevBuf hx, hq, hphi, hgrad;

    // kernel launches issued by this handle (all phases, since creation)
    int64_t launches = 0;

    // timing
    cudaEvent_t ev[2 * kPhases + 8] = {};   // phases, build, evaluate, backward, batch
    bool events_ready = false;
    float ms_phase[kPhases] = {};
    float ms_build = 0.f, ms_eval = 0.f;
    bool backward_done = false;
    bool batch_done = false;
};

// ---------------------------------------------------------------------------
// phases (implemented in the .cu files)
// ---------------------------------------------------------------------------
int scan_exclusive_u32(Handle &h, const unsigned *in, unsigned *out, int64_t n, unsigned *total_dev);
int scan_exclusive_u32_on(Handle &h, cudaStream_t stream, DevBuf &tmp, const unsigned *in, unsigned *out, int64_t n,
                          unsigned *total_dev);
int radix_sort_pairs(Handle &h, uint64_t *&keys, uint64_t *&keys_alt, unsigned *&vals,
                     unsigned *&vals_alt, int64_t n, int begin_bit, int end_bit);
int radix_sort_keys(Handle &h, uint64_t *&keys, uint64_t *&keys_alt, int64_t n, int begin_bit,
                    int end_bit);
int radix_sort_keys32(Handle &h, uint32_t *&keys, uint32_t *&keys_alt, int64_t n, int begin_bit, int end_bit);

int build_keys(Handle &h, const double *x);       // bbox, normalise, Morton, sort, gather
int build_tree(Handle &h, const double *x);       // cells, geometry, leaf-local positions
int build_lists(Handle &h);                       // DTT + grouping (the M2L list on the second stream)
int join_lists_begin(Handle &h);                  // the handle's stream waits for the M2L list's grouping
int join_lists_end(Handle &h);                    // after a synchronisation: its repeated-pair check
int build_p2p_items(Handle &h);                   // P2P work items and source ranges
int build_work_items(Handle &h, int g, DevBuf &items, int64_t &n_items);   // items of <= g targets
int p2p_batch_tc(Handle &h, int nrhs, float *phi, float *grad);   // batched P2P + L2P, tensor cores
int build_runs(Handle &h, const int *off, const int *src, int64_t max_runs, DevBuf &roff, DevBuf &ent, DevBuf &cnt,
               int64_t *nruns);
int ensure_full_runs(Handle &h);   // the whole lists' runs (built on first use with the mutual schedule)
int build_mutual(Handle &h);   // split the P2P lists for the mutual schedule
int p2p_mutual(Handle &h);     // the mutual P2P pass (fills racc)

int evaluate_upward(Handle &h, const float *q);   // gather q, P2M, M2M
int evaluate_m2l(Handle &h, const float *M, float *L);
int evaluate_downward(Handle &h, float *L);       // L2L
int adjoint_upward(Handle &h, const float *dphi, const float *dgrad);   // gather (a, b / h), P2M, M2M into Ma
int adjoint_p2p(Handle &h, float *dq, float *dx); // adjoint P2P + L2P terms + scatter
int evaluate_batch(Handle &h, const float *q, int nrhs, float *phi, float *grad);   // many charge vectors
int evaluate_p2p(Handle &h, float *phi, float *grad);   // P2P + L2P + scatter
int energy_reduce(Handle &h, double *E);

// phase timing helpers
void phase_begin(Handle &h, int phase);
void phase_end(Handle &h, int phase);

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace fmm

struct fmm_handle {
    fmm::Handle h;
};
