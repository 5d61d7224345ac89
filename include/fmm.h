/*
 * fmm.h -- C ABI of the GB300 dual-tree-traversal FMM for the 3-D Laplace kernel.
 *
 * Method: R. Yokota, "An FMM Based on Dual Tree Traversal for Many-core
 * Architectures" (arXiv:1209.3516).  The library computes, for N particles
 * with positions x_i and charges q_i,
 *     phi_i  = sum_{j : r_ij != 0} q_j / r_ij                  (potential)
 *     grad_i = -sum_{j : r_ij != 0} q_j (x_i - x_j) / r_ij^3   (its gradient)
 * (the Laplace kernel of Sec. 3.2 and Table 3; no 1/(4 pi), no softening), with
 * an FMM whose interaction lists come from a dual tree traversal (Algorithms 3
 * and 4) under the multipole acceptance criterion theta * R > B_A + B_B
 * (Sec. 3.2), Cartesian Taylor expansions of order P (Sec. 3.1, Table 1), and
 * leaves of at most ncrit particles (Table 3).  Accuracy is controlled by both
 * P and theta (Sec. 3.2, Table 3).
 *
 * Conventions shared by every call:
 *   - Every call returns an int: FMM_OK (0) or a negative FMM_ERR_* code.  No
 *     exception or abort crosses the ABI.  fmm_last_error_string() returns a
 *     message for the last failing call of the calling thread.
 *   - Unless a call says "host", every pointer argument is a DEVICE pointer
 *     on the handle's device.  The caller owns all arrays it passes; the handle
 *     owns all of its internal device workspaces.
 *   - Work is issued asynchronously on the handle's stream (fmm_options.stream).
 *     Calls that return sizes or host data synchronise that stream.
 *   - A handle must not be used from two threads at the same time.
 *   - Layouts: positions x are N x 3 row-major FP64 (x0 y0 z0 x1 y1 z1 ...);
 *     charges q and potentials phi are N FP32; gradients grad are N x 3
 *     row-major FP32.  All outputs are in the caller's particle order.
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define FMM_OK 0
#define FMM_ERR_ARG (-1)          /* null pointer, size or parameter out of range */
#define FMM_ERR_UNSUPPORTED (-2)  /* expansion order P not compiled into the library */
#define FMM_ERR_INPUT (-3)        /* a coordinate is NaN or infinite */
#define FMM_ERR_CUDA (-4)         /* CUDA runtime error (see fmm_last_error_string) */
#define FMM_ERR_NOMEM (-5)        /* device allocation failed */
#define FMM_ERR_STATE (-6)        /* evaluate or query before a successful build */
#define FMM_ERR_CAPACITY (-7)     /* a traversal buffer overflowed again after regrowing */

/* Flags for fmm_options.flags. */
#define FMM_FLAG_KAHAN 1u         /* compensated (Kahan) P2P accumulation per target */
#define FMM_FLAG_TIMING 2u        /* record per-phase device times (adds events) */
#define FMM_FLAG_MUTUAL 4u        /* mutual near field: each unordered leaf pair of the P2P list once, both
                                     directions (Newton's third law, the falcON heritage of Sec. 2); the
                                     same lists and results to rounding, not bitwise (float reductions) */

/* Largest number of charge vectors of one fmm_evaluate_batch call. */
#define FMM_MAX_RHS 32

typedef struct fmm_handle fmm_handle;

typedef struct fmm_options {
    void *stream;      /* cudaStream_t to issue work on; NULL = the legacy default stream */
    int device;        /* CUDA device ordinal; -1 = the current device */
    unsigned flags;    /* FMM_FLAG_* */
} fmm_options;

/* Phase indices of fmm_stats.ms_phase (device times of the last build/evaluate). */
enum {
    FMM_PHASE_MORTON = 0,  /* bounding box, normalisation, Morton keys */
    FMM_PHASE_SORT,        /* radix sort of (key, index) */
    FMM_PHASE_TREE,        /* ncrit splitting, cell table, cell geometry */
    FMM_PHASE_TRAVERSE,    /* dual tree traversal (seeding rounds + work-stack kernel) */
    FMM_PHASE_LISTS,       /* grouping of the lists by target cell */
    FMM_PHASE_ITEMS,       /* P2P source runs, the mutual schedule's list split, work items */
    FMM_PHASE_UPWARD,      /* charge gather, P2M, M2M */
    FMM_PHASE_M2L,
    FMM_PHASE_DOWNWARD,    /* L2L */
    FMM_PHASE_P2P,         /* P2P + L2P + output scatter */
    FMM_NPHASES
};

/* Counters and timings (fmm_stats). */
struct fmm_stats {
    int64_t n;                  /* particles */
    int64_t ncells, nleaves;    /* cells of the octree, leaves among them */
    int32_t nlevels;            /* levels present (root = level 0) */
    int32_t P;                  /* expansion order */
    int64_t n_m2l, n_p2p;       /* cell pairs in the M2L and P2P lists */
    int64_t p2p_pairs;          /* particle pairs of the P2P list: sum n_target * n_source */
    double ms_build, ms_evaluate;          /* device time of the last build / evaluate */
    double ms_phase[FMM_NPHASES];          /* per phase, when FMM_FLAG_TIMING is set */
    int64_t kernel_launches;               /* CUDA kernels launched by this handle since creation */
    double ms_backward;                    /* device time of the last fmm_backward */
    double ms_batch;                       /* device time of the last fmm_evaluate_batch */
};

/*
 * fmm_create -- allocate a handle for N particles.
 *   N      >= 1 particles.
 *   P      expansion order: multipole and local expansions hold every Taylor
 *          coefficient of total degree <= P-1 (Sec. 3.1; the error of one M2L is
 *          of order ((B_A+B_B)/R)^P, Sec. 3.2).  Compiled orders: 3, 4, 5, 6, 8;
 *          others give FMM_ERR_UNSUPPORTED.
 *   theta  opening angle of the MAC, 0 <= theta < 1 (Sec. 3.2); theta = 0 accepts no
 *          pair, so every interaction is a direct P2P sum.
 *   ncrit  >= 1, the largest number of particles in a leaf (Table 3's N_crit);
 *          a cell at the deepest level (21) stays a leaf whatever its size.
 *   opt    may be NULL (default stream, current device, no flags).
 * On success *h holds a new handle; on error *h is set to NULL.
 */
int fmm_create(fmm_handle **h, int64_t N, int P, float theta, int ncrit, const fmm_options *opt);

/*
 * fmm_build -- tree and interaction lists for the positions x (device, N x 3 FP64).
 * Steps (each a GPU kernel, Sec. 3.3 and Table 2): bounding box and normalisation
 * to the cube (-1,1)^3 in FP64, 63-bit Morton keys, stable radix sort of
 * (key, index), level-by-level splitting of cells with more than ncrit particles
 * into their non-empty octants, cell centres and tight radii, then the dual tree
 * traversal (Algorithms 3 and 4) emitting the M2L and P2P cell-pair lists, which
 * are grouped by target cell.  x is only read during the call; the handle keeps
 * its own sorted copy.  Errors: FMM_ERR_INPUT for a NaN/Inf coordinate,
 * FMM_ERR_CAPACITY if a traversal buffer overflows after one regrowth.
 * Synchronises the stream (list sizes are read back).
 */
int fmm_build(fmm_handle *h, const double *x);

/*
 * fmm_evaluate -- potential and gradient at every particle.
 *   x     the positions (device); if x differs from the pointer passed to the
 *         last fmm_build, the tree is rebuilt first; NULL reuses the last build.
 *   q     charges, device, N FP32.
 *   phi   out, device, N FP32, or NULL if not wanted.
 *   grad  out, device, N x 3 FP32, or NULL if not wanted (not both NULL).
 * Steps: P2M, M2M (upward), M2L over the M2L list, L2L (downward), then one
 * kernel doing P2P over the P2P list, L2P, and the scatter to caller order and
 * physical units (phi / h, grad / h^2 for the normalisation scale h).
 * Asynchronous on the handle's stream.
 */
int fmm_evaluate(fmm_handle *h, const double *x, const float *q, float *phi, float *grad);

/*
 * fmm_evaluate_batch -- potentials and gradients of nrhs charge vectors on one
 * geometry in one call (the many-right-hand-side form of fmm_evaluate).
 *   x     as in fmm_evaluate (rebuild if it differs from the last build; NULL reuses it).
 *   q     device, nrhs x N FP32: vector r at q + r * N (caller order).
 *   nrhs  1 <= nrhs <= FMM_MAX_RHS.
 *   phi   out, device, nrhs x N FP32 (vector r at phi + r * N), or NULL.
 *   grad  out, device, nrhs x N x 3 FP32 (vector r at grad + 3 r N), or NULL.
 * The same tree, lists and operators as fmm_evaluate, with every operator a
 * contraction over the vectors: P2M, M2M, M2L and L2L apply each geometric
 * factor to all vectors (FP32); the P2P and the L2P are one dense product on
 * the 5th-generation tensor cores per work item of <= 32 targets: D = G Q + W L
 * with the kernel matrices G (1/r and e/r^3 of every target-source pair) and
 * the targets' Taylor monomials W generated in FP32 straight into tensor
 * memory, Q the charges and L the leaf's local expansions, every operand split
 * into BF16 high and low parts (three tcgen05.mma per K step, FP32
 * accumulation in tensor memory: about 2^-16 relative per term); the scatter
 * to caller order is fused.  Asynchronous (the first call after a build
 * synchronises once to size its work items).
 */
int fmm_evaluate_batch(fmm_handle *h, const double *x, const float *q, int nrhs, float *phi, float *grad);

/*
 * fmm_evaluate_host -- fmm_build + fmm_evaluate on HOST arrays: copies x (N x 3
 * FP64) and q (N FP32) to the device, builds, evaluates, copies phi (N) and grad
 * (N x 3) back.  phi or grad may be NULL.  Synchronous.
 */
int fmm_evaluate_host(fmm_handle *h, const double *x_host, const float *q_host, float *phi_host,
                      float *grad_host);

/*
 * fmm_energy -- E = 1/2 sum_i q_i phi_i of the last evaluate, reduced in FP64 on
 * the device.  E is a HOST pointer.  Synchronises the stream.
 */
int fmm_energy(fmm_handle *h, double *E);

/*
 * fmm_backward -- adjoint of the last fmm_evaluate on this handle (same x and q),
 * for the upstream gradients of a scalar loss L(phi, grad):
 *   dphi  device, N FP32, dL/dphi (caller order); NULL = zero.
 *   dgrad device, N x 3 FP32, dL/dgrad; NULL = zero.
 *   dq    out, device, N FP32, or NULL:  dL/dq_k = Psi(x_k), the potential at x_k of
 *         charges dphi_i and dipoles dgrad_i at the x_i:
 *         Psi(x) = sum_i dphi_i / |x - x_i| + sum_i dgrad_i . (x - x_i) / |x - x_i|^3.
 *   dx    out, device, N x 3 FP32, or NULL:
 *         dL/dx_k = dphi_k grad_k + H_k dgrad_k + q_k grad Psi(x_k),
 *         H_k the Hessian of the potential at x_k (pairs at distance 0 excluded).
 * dq and dx must not both be NULL.  The paper has no adjoint: these are the
 * derivatives of the sums of Sec. 3.2, evaluated with the same method: the
 * adjoint sources get a dipole P2M and the same M2M, M2L (same lists) and L2L;
 * one kernel then does the adjoint P2P over the P2P list, the L2P terms of both
 * local expansions (value, gradient and Hessian-vector product) and the
 * scatter.  The handle's forward local expansions and sorted charges are used,
 * so no evaluate may come between the fmm_evaluate being differentiated and
 * this call.  Asynchronous on the handle's stream (the first call after a build
 * synchronises once to size its work items).  FMM_ERR_STATE before an evaluate.
 */
int fmm_backward(fmm_handle *h, const float *dphi, const float *dgrad, float *dq, float *dx);

/*
 * fmm_measure_peaks -- the FP32 roofline denominators of the current GPU,
 * measured (the paper has no counterpart; it quotes its CPU's data-sheet
 * peak).  Three register-only kernels run one full wave on every SM: scalar
 * FFMA chains, packed FFMA2 chains and rsqrt.approx (SFU) chains; each is
 * launched 5 times on `stream` (NULL = legacy default stream) and the fastest
 * launch, timed with CUDA events, is kept.  Blocks until done (~0.3 s).
 * Allocates a small sink buffer (one float per resident thread) with
 * cudaMallocAsync on the stream.  FMA counts as 2 flops.
 *   out  HOST pointer, filled on success.
 */
typedef struct fmm_peaks {
    double ffma_tflops;     /* scalar FFMA, TFLOP/s */
    double ffma2_tflops;    /* packed FFMA2, TFLOP/s */
    double rsqrt_per_s;     /* SFU rsqrt.approx operations per second */
    double ms_ffma, ms_ffma2, ms_rsqrt;   /* fastest launch of each kernel */
    int32_t sms;
    int32_t reserved;
} fmm_peaks;
int fmm_measure_peaks(fmm_peaks *out, void *stream);

/*
 * fmm_energy_noalloc -- E = 1/2 sum_i q_i phi_i of caller arrays, reduced in FP64,
 * WITHOUT allocating any memory.  The paper has no counterpart: this entry point
 * exists for callers that cannot let a library call cudaMalloc, such as
 * applications that hand out all device memory from their own arena or a
 * framework's caching allocator and budget it up front.
 *   q, phi  device arrays of n FP32 values (any particle order, the same in both).
 *   n       1 <= n <= 16,777,216; larger n returns FMM_ERR_ARG.  The limit comes
 *           from the scratch: one FP64 partial per 2048 values in a fixed 64 KiB
 *           array of the library's device memory, which every GPU that loads the
 *           library holds until the process exits.
 *   E       out, DEVICE pointer to one double.
 *   stream  cudaStream_t to run on (NULL = legacy default stream); asynchronous.
 * q, phi and E must be device memory of the current GPU (or managed memory):
 * each pointer's kind is checked with cudaPointerGetAttributes before any
 * launch, and a host pointer (such as the host double that fmm_energy takes)
 * or another GPU's memory returns FMM_ERR_ARG.
 * The first call on a device (with that device current) looks up the scratch
 * array's device address and caches it with the current CUDA context (a new
 * context, e.g. after a device reset, is looked up again); make that first
 * call before any stream capture.  All calls share the scratch array, so calls
 * that overlap on the GPU (different streams or threads) race; the array keeps
 * the last call's contents, and each call writes every partial it reads.
 */
int fmm_energy_noalloc(const float *q, const float *phi, int64_t n, double *E, void *stream);

/*
 * Many independent systems in one evaluation.  Each system gets its own tree,
 * normalisation and lists; fmm_multi_build merges them into one set of
 * arrays (cells in (level, system) order, every index moved by its system's
 * offset, a per-cell unit scale), so that each evaluation operator runs as one
 * launch over all systems: one charge gather, one P2M, one M2M and one L2L per
 * level, one M2L and one P2P.  fmm_multi_evaluate captures that evaluation into
 * a CUDA graph on first use (after an eager run that sizes the buffers and an
 * autotuner that times the near field on the merged problem in four
 * configurations -- work items of 16 or 8 targets, one-sided or mutual -- and
 * keeps the fastest) and replays the graph afterwards; new q / phi / grad
 * pointers trigger a new capture.
 */
typedef struct fmm_multi fmm_multi;

struct fmm_multi_info {
    int64_t n_total;               /* particles over all systems */
    int64_t ncells, nleaves;       /* merged cells and leaves */
    int64_t n_m2l, p2p_pairs;      /* M2L cell pairs, P2P particle pairs over all systems */
    int64_t graph_nodes;           /* kernel nodes of the captured evaluation */
    int64_t kernel_launches;       /* kernels launched on the merged problem (merge, tuning, eager runs) */
    int32_t nsys, nlevels;
    int32_t p2p_targets_per_item;  /* the autotuner's choice (or the pinned one) */
    int32_t mutual;                /* 0: one-sided near field; 1 / 2: mutual with 2 / 4 staged sources per lane
                                      (the autotuner's choice or the pinned one) */
    double tune_ms[6];             /* near-field time with 16 / 8 targets per item: one-sided 16, 8; mutual
                                      (2 per lane) 16, 8; mutual (4 per lane) 16, 8 (best of 3 each) */
    double ms_evaluate;            /* device time of the last graph replay */
};

/*
 * fmm_multi_create -- nsys systems of N[s] particles (N: HOST array of nsys
 * sizes, each >= 1, total < 2^31), one P, theta, ncrit for all.  opt may be
 * NULL; opt->stream is the stream the calls are ordered after (the work runs
 * on a private stream of the handle); Kahan and timing flags are ignored.
 */
int fmm_multi_create(fmm_multi **m, int nsys, const int64_t *N, int P, float theta, int ncrit,
                     const fmm_options *opt);

/* fmm_multi_build -- x: device, (sum N) x 3 FP64, the systems back to back.  Synchronous. */
int fmm_multi_build(fmm_multi *m, const double *x);

/*
 * fmm_multi_evaluate -- q (device, sum N FP32, systems back to back) -> phi
 * (sum N) and grad ((sum N) x 3), either may be NULL but not both; each
 * system's particles interact only with each other.  Asynchronous with respect
 * to the host (ordered after and before the caller's stream).
 */
int fmm_multi_evaluate(fmm_multi *m, const float *q, float *phi, float *grad);

/* fmm_multi_set_hybrid -- fmm_set_hybrid for every system, for the next fmm_multi_build. */
int fmm_multi_set_hybrid(fmm_multi *m, int64_t min_pairs);

/*
 * fmm_multi_set_config -- pin the near-field configuration instead of letting
 * the autotuner choose: targets_per_item 0 (tune), 8 or 16; mutual -1 (tune),
 * 0 (one-sided), 1 (mutual, 2 staged sources per lane, 12 warps per SM) or 2
 * (mutual, 4 staged sources per lane, 8 warps per SM).  Applied at the next
 * fmm_multi_evaluate (the table is still timed and reported by fmm_multi_info).
 * FMM_ERR_ARG for any other value.
 */
int fmm_multi_set_config(fmm_multi *m, int targets_per_item, int mutual);

/* fmm_multi_info -- sizes, the autotuner's timings and choice, the last replay's time (HOST *info). */
int fmm_multi_info(fmm_multi *m, struct fmm_multi_info *info);

int fmm_multi_destroy(fmm_multi *m);

/*
 * fmm_set_hybrid -- the M2L / P2P hybrid at the leaves, for the next fmm_build.
 * Algorithm 4 sends a pair of leaves to P2P before looking at the MAC; with
 * min_pairs >= 0 a leaf pair that passes the MAC and holds at least min_pairs
 * particle pairs (n_A n_B) goes to M2L instead (the choice between the two
 * kernels at the leaves that the paper's exaFMM tunes, Sec. 2).  min_pairs < 0
 * (the default) keeps Algorithm 4 as printed.  The accuracy is still bounded by
 * the MAC; the lists change, so the oracle must be run with the same setting.
 */
int fmm_set_hybrid(fmm_handle *h, int64_t min_pairs);

/*
 * fmm_tune_hybrid -- like fmm_tune_ncrit, over candidate min_pairs values of the
 * hybrid (HOST array; a negative value is Algorithm 4 as printed) at one ncrit:
 * the fastest build + evaluate goes to *best, the medians to ms_out.
 */
int fmm_tune_hybrid(int64_t N, int P, float theta, int ncrit, const double *x, const float *q,
                    const int64_t *candidates, int ncand, int reps, const fmm_options *opt, int64_t *best,
                    double *ms_out);

/*
 * fmm_tune_ncrit -- the leaf size at which the evaluation is fastest for this
 * input: the balance between M2L (more, smaller cells) and P2P (fewer, larger
 * leaves) that the paper's auto-tuned hybrid selects by timing (Sec. 2, the
 * M2L / P2P choice of the leaf size).  For each of the ncand candidate ncrit
 * values (HOST array) a handle is built on x and evaluated with q (device
 * arrays, as in fmm_evaluate) `reps` times after one warm-up; the device time of
 * build + evaluate (median of reps) goes to ms_out[k] (HOST, ncand doubles, may
 * be NULL) and the fastest candidate to *best (HOST).  The accuracy is set by P
 * and theta (the MAC), not by ncrit.  Synchronous.
 */
int fmm_tune_ncrit(int64_t N, int P, float theta, const double *x, const float *q, const int *candidates,
                   int ncand, int reps, const fmm_options *opt, int *best, double *ms_out);

/* fmm_stats -- counters and timings of the last build/evaluate into *s (HOST). */
int fmm_stats(fmm_handle *h, struct fmm_stats *s);

/* fmm_destroy -- free the handle and all its device memory (NULL is a no-op). */
int fmm_destroy(fmm_handle *h);

/* Message for the last failing call on this thread (static storage; never NULL). */
const char *fmm_last_error_string(void);

/* ---- Introspection (synchronous device -> HOST copies, for tests and tools) ---- */

/*
 * fmm_get_norm -- normalisation of the last build: u = (x - centre) / h.
 * centre: HOST double[3]; h: HOST double.
 */
int fmm_get_norm(fmm_handle *h, double *centre, double *scale);

/*
 * fmm_get_sorted -- HOST arrays of length N: sorted Morton keys and perm
 * (perm[s] = caller index of the s-th particle in key order).  Either may be NULL.
 */
int fmm_get_sorted(fmm_handle *h, uint64_t *keys, int32_t *perm);

/* fmm_get_ncells -- number of cells of the last build (HOST out). */
int fmm_get_ncells(fmm_handle *h, int64_t *ncells);

/*
 * fmm_get_cells -- HOST arrays of length ncells (breadth-first order), any may be NULL:
 * canonical id (1 << 3*level) | Morton prefix, level, first sorted particle,
 * particle count, number of children (0 = leaf), parent index (-1 for the root),
 * centre (ncells x 3 FP32) and tight radius (FP32).
 */
int fmm_get_cells(fmm_handle *h, uint64_t *canon, int32_t *level, int32_t *pbeg, int32_t *pcnt,
                  int32_t *nchild, int32_t *parent, float *centre, float *radius);

/*
 * fmm_get_lists -- list sizes (HOST n_m2l, n_p2p; either may be NULL) and, if the
 * array pointers are non-NULL, the lists as HOST int32 (target, source) cell-index
 * pairs, 2 x n each, grouped by target and sorted by (target, source).
 */
int fmm_get_lists(fmm_handle *h, int64_t *n_m2l, int64_t *n_p2p, int32_t *m2l, int32_t *p2p);

#ifdef __cplusplus
}
#endif

#endif /* FMM_GB300_H */
