// tree.cu -- Morton-key octree on the device.
//
// Table 2 (FMM column) and Sec. 2: cubic cells, 64-bit Morton keys holding 21
// levels, leaves of at most N_crit particles (Table 3).  Steps:
//   1. FP64 bounding box and normalisation to the cube (-1,1)^3;
//   2. 63-bit keys from 21-bit integer coordinates;
//   3. stable radix sort of (key, index), gather of FP32 positions;
//   4. level-by-level split of every cell holding more than ncrit particles
//      into its non-empty octants (warp-parallel searches on the sorted keys);
//   5. cell geometry: geometric centre (exact in FP32) and tight radius
//      B = max |u_j - X_C| over the cell's particles (Sec. 3.2, B_max MAC),
//      computed in FP32 with one rounding per operation.
// Normalisation (not given by the paper): c = (min + max) / 2,
// h = (max extent / 2) (1 + 2^-20) (1 when all particles coincide),
// u = (x - c) / h, i_d = min(floor((u_d + 1) 2^20), 2^21 - 1).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "fmm_internal.cuh"

namespace fmm {

constexpr int kBBoxThreads = 256;

// ---------------------------------------------------------------------------
// 1. bounding box
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBBoxThreads) k_bbox_partial(const double *x, int64_t n, double *part,
                                                               unsigned *err)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v = x[3 * i + a];
            bad |= !isfinite(v);
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    }
    if (__any_sync(kFull, bad) && lane_id() == 0) atomicOr(err, 1u);
    __shared__ double s[kBBoxThreads / 32][6];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(kFull, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(kFull, hi[a], o));
        }
    }
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            s[w][a] = lo[a];
            s[w][3 + a] = hi[a];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = s[0][threadIdx.x];
        for (int k = 1; k < kBBoxThreads / 32; ++k)
            v = threadIdx.x < 3 ? fmin(v, s[k][threadIdx.x]) : fmax(v, s[k][threadIdx.x]);
        part[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

// One block: reduce the partial boxes and derive centre and scale.
__global__ void k_bbox_final(const double *part, int nb, double *norm)
{
    __shared__ double s[6][32];
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int a = 0; a < 6; ++a) v[a] = a < 3 ? fmin(v[a], part[b * 6 + a]) : fmax(v[a], part[b * 6 + a]);
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double t = __shfl_xor_sync(kFull, v[a], o);
            v[a] = a < 3 ? fmin(v[a], t) : fmax(v[a], t);
        }
    if (lane_id() == 0)
#pragma unroll
        for (int a = 0; a < 6; ++a) s[a][threadIdx.x >> 5] = v[a];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 1; k < nw; ++k)
            for (int a = 0; a < 6; ++a) s[a][0] = a < 3 ? fmin(s[a][0], s[a][k]) : fmax(s[a][0], s[a][k]);
        double ext = 0.0;
        for (int a = 0; a < 3; ++a) {
            norm[a] = __dmul_rn(__dadd_rn(s[a][0], s[3 + a][0]), 0.5);
            double e = __dsub_rn(s[3 + a][0], s[a][0]);
            ext = e > ext ? e : ext;
        }
        double h = __dmul_rn(ext, 0.5);
        h = __dmul_rn(h, 1.0 + 0x1p-20);
        if (h == 0.0) h = 1.0;
        norm[3] = h;
        norm[4] = __drcp_rn(h);
    }
}

// ---------------------------------------------------------------------------
// 2. Morton keys
// ---------------------------------------------------------------------------
// RN(d / h) for h > 0, given y = RN(1 / h).  The estimate q0 = RN(d y) is
// refined once with its remainder (Markstein, IBM J. Res. Develop. 34 (1990)),
// q1 = RN(q0 + (d - q0 h) y), and then proved: |d - q1 h| < h ulp(q1) / 2
// (tested with a 2^-20 margin, which also covers a rounded remainder) means
// that q1 is the double nearest to d / h when q1 is normal and not a power of
// two.  Otherwise the IEEE division decides.  The result is always RN(d / h).
__device__ __forceinline__ double div_rn_checked(double d, double h, double y)
{
    const double q0 = __dmul_rn(d, y);
    const double q1 = __fma_rn(__fma_rn(-q0, h, d), y, q0);
    const double r = __fma_rn(-q1, h, d);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(q1) & 0x7fffffffffffffffull;
    const int e = (int)(bits >> 52);
    if (e >= 54 && e < 2047 && (bits & 0xfffffffffffffull) != 0ull) {
        const double half_ulp = __longlong_as_double((long long)(e - 53) << 52);   // ulp(q1) / 2
        if (fabs(r) < __dmul_rn(__dmul_rn(half_ulp, h), 1.0 - 0x1p-20)) return q1;
    }
    return __ddiv_rn(d, h);
}

// u = (x - c) / h (FP64, correctly rounded), key = interleaved floor((u + 1) 2^20)
// per axis (clamped to 21 bits), u kept in FP64 (structure of arrays) and FP32.
__global__ void k_morton(const double *x, int64_t n, const double *norm, uint64_t *keys, unsigned *idx,
                         float4 *pos, double *u64)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double h = norm[3], y = norm[4];
    double u[3];
    uint64_t ic[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = div_rn_checked(__dsub_rn(x[3 * i + a], norm[a]), h, y);
        // RN((u + 1) 2^20) in one rounding, floored and clamped in integers
        const long long s = __double2ll_rd(__fma_rn(u[a], 0x1p20, 0x1p20));
        ic[a] = (uint64_t)min(max(s, 0ll), 2097151ll);
        u64[a * n + i] = u[a];
    }
    keys[i] = spread3(ic[0]) | (spread3(ic[1]) << 1) | (spread3(ic[2]) << 2);
    idx[i] = (unsigned)i;
    pos[i] = make_float4(__double2float_rn(u[0]), __double2float_rn(u[1]), __double2float_rn(u[2]), 0.0f);
}

__global__ void k_gather_sorted(const unsigned *idx, int64_t n, const float4 *pos_in, float4 *pos, int *perm,
                                const double *u_in, double *u_out)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const unsigned i = idx[s];
    pos[s] = pos_in[i];
    perm[s] = (int)i;
#pragma unroll
    for (int a = 0; a < 3; ++a) u_out[a * n + s] = u_in[a * n + i];
}

int build_keys(Handle &h, const double *x)
{
    const int64_t N = h.N;
    const int nb = std::min<int64_t>(ceil_div(N, kBBoxThreads), (int64_t)h.num_sms * 8);
    FMM_TRY(h.norm.reserve(5 * sizeof(double)));   // centre, h, RN(1 / h)
    FMM_TRY(h.bbox_part.reserve((size_t)nb * 6 * sizeof(double)));
    FMM_TRY(h.err_flag.reserve(sizeof(unsigned)));
    FMM_TRY(h.keys.reserve(N * sizeof(uint64_t)));
    FMM_TRY(h.keys_alt.reserve(N * sizeof(uint64_t)));
    FMM_TRY(h.idx.reserve(N * sizeof(unsigned)));
    FMM_TRY(h.idx_alt.reserve(N * sizeof(unsigned)));
    FMM_TRY(h.pos_unsorted.reserve(N * sizeof(float4)));
    FMM_TRY(h.u_unsorted.reserve(3 * N * sizeof(double)));
    FMM_TRY(h.u_sorted.reserve(3 * N * sizeof(double)));
    FMM_TRY(h.pos.reserve(N * sizeof(float4)));
    FMM_TRY(h.perm.reserve(N * sizeof(int)));

    phase_begin(h, FMM_PHASE_MORTON);
    FMM_CUDA(cudaMemsetAsync(h.err_flag.p, 0, sizeof(unsigned), h.stream));
    ++h.launches;
    k_bbox_partial<<<nb, kBBoxThreads, 0, h.stream>>>(x, N, h.bbox_part.as<double>(), h.err_flag.as<unsigned>());
    ++h.launches;
    k_bbox_final<<<1, 256, 0, h.stream>>>(h.bbox_part.as<double>(), nb, h.norm.as<double>());
    ++h.launches;
    k_morton<<<ceil_div(N, 256), 256, 0, h.stream>>>(x, N, h.norm.as<double>(), h.keys.as<uint64_t>(),
                                                     h.idx.as<unsigned>(), h.pos_unsorted.as<float4>(),
                                                     h.u_unsorted.as<double>());
    FMM_CHECK_LAUNCH("morton");
    phase_end(h, FMM_PHASE_MORTON);

    // non-finite input is an error of the call: check before going further
    FMM_CUDA(cudaMemcpyAsync(&h.pinned->err, h.err_flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaMemcpyAsync(h.norm_host, h.norm.p, 4 * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    if (h.pinned->err) {
        set_error("fmm_build: a coordinate is NaN or infinite");
        return FMM_ERR_INPUT;
    }

    phase_begin(h, FMM_PHASE_SORT);
    uint64_t *k = h.keys.as<uint64_t>(), *ka = h.keys_alt.as<uint64_t>();
    unsigned *v = h.idx.as<unsigned>(), *va = h.idx_alt.as<unsigned>();
    FMM_TRY(radix_sort_pairs(h, k, ka, v, va, N, 0, 3 * kLevels));
    // keep the sorted arrays in the primary buffers
    if (k != h.keys.as<uint64_t>()) {
        std::swap(h.keys, h.keys_alt);
        std::swap(h.idx, h.idx_alt);
    }
    ++h.launches;
    k_gather_sorted<<<ceil_div(N, 256), 256, 0, h.stream>>>(h.idx.as<unsigned>(), N, h.pos_unsorted.as<float4>(),
                                                            h.pos.as<float4>(), h.perm.as<int>(),
                                                            h.u_unsorted.as<double>(), h.u_sorted.as<double>());
    FMM_CHECK_LAUNCH("gather");
    phase_end(h, FMM_PHASE_SORT);
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// 4. ncrit splitting, level by level
// ---------------------------------------------------------------------------
// First index in [lo, hi) with keys[index] >= v (hi if none), searched by the
// whole warp: 32 samples per round narrow the range 32-fold, so a cell of a
// million particles needs 4 dependent rounds instead of 20.  All lanes return
// the same value.
__device__ __forceinline__ int warp_lower_bound(const uint64_t *keys, int lo, int hi, uint64_t v)
{
    const int lane = (int)lane_id();
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) / 32;
        const int p = lo + lane * step;
        const bool pred = p < hi && keys[p] < v;
        const int k = __popc(__ballot_sync(kFull, pred));
        // keys[p_(k-1)] < v <= keys[p_k]: the answer lies in [p_(k-1) + 1, p_k]
        const int nlo = k == 0 ? lo : lo + (k - 1) * step + 1;
        const int nhi = min(lo + k * step, hi);
        lo = nlo;
        hi = nhi;
    }
    const bool pred = lo + lane < hi && keys[lo + lane] < v;
    return lo + __popc(__ballot_sync(kFull, pred));
}

// One warp per cell of level l: the cell splits when it holds more than ncrit
// particles (and l < 21); its octant boundaries bnd[8 i + o] (first particle of
// octant o) come from warp searches on the sorted keys, and cnt[i] counts the
// non-empty octants.
__global__ void k_split_bounds(int l, int lo, int n, int ncrit, const uint64_t *keys, const uint64_t *prefix,
                               const int *pbeg, const int *pcnt, int *bnd, unsigned *cnt)
{
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    const int c = lo + i;
    const int b = pbeg[c], e = b + pcnt[c];
    unsigned nch = 0;
    if (e - b > ncrit && l < kLevels) {
        const int shift = 3 * (kLevels - (l + 1));
        const uint64_t p = prefix[c];
        int prev = b;
        for (int o = 1; o <= 8; ++o) {
            const int next = o < 8 ? warp_lower_bound(keys, prev, e, ((p << 3) | (uint64_t)o) << shift) : e;
            if (lane_id() == 0) bnd[8 * i + o - 1] = prev;
            nch += next > prev;
            prev = next;
        }
    }
    if (lane_id() == 0) cnt[i] = nch;
}

__global__ void k_split_write(int l, int lo, int n, int ncrit, int next_lo, const int *bnd, const unsigned *off,
                              uint64_t *prefix, int *level, int *pbeg, int *pcnt, int *cbeg, int *ccnt, int *parent)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = lo + i;
    const int e = pbeg[c] + pcnt[c];
    if (!(pcnt[c] > ncrit && l < kLevels)) return;
    const uint64_t p = prefix[c];
    int w = next_lo + (int)off[i];
    cbeg[c] = w;
    int nch = 0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
        const int b0 = bnd[8 * i + o], b1 = o < 7 ? bnd[8 * i + o + 1] : e;
        if (b1 > b0) {
            prefix[w] = (p << 3) | (uint64_t)o;
            level[w] = l + 1;
            pbeg[w] = b0;
            pcnt[w] = b1 - b0;
            cbeg[w] = 0;
            ccnt[w] = 0;
            parent[w] = c;
            ++w;
            ++nch;
        }
    }
    ccnt[c] = nch;
}

__global__ void k_root(int n, uint64_t *prefix, int *level, int *pbeg, int *pcnt, int *cbeg, int *ccnt, int *parent)
{
    prefix[0] = 0;
    level[0] = 0;
    pbeg[0] = 0;
    pcnt[0] = n;
    cbeg[0] = 0;
    ccnt[0] = 0;
    parent[0] = -1;
}

// ---------------------------------------------------------------------------
// 5. geometry
// ---------------------------------------------------------------------------
__global__ void k_centres(int nc, const uint64_t *prefix, const int *level, float4 *geom, unsigned *r2bits)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int l = level[c];
    const uint64_t p = prefix[c];
    const float s = ldexpf(1.0f, -l);
    // (2 i + 1) 2^-l - 1 is exact in FP32 for l <= 21
    const float cx = __fsub_rn(__fmul_rn((float)(2u * compact3(p) + 1u), s), 1.0f);
    const float cy = __fsub_rn(__fmul_rn((float)(2u * compact3(p >> 1) + 1u), s), 1.0f);
    const float cz = __fsub_rn(__fmul_rn((float)(2u * compact3(p >> 2) + 1u), s), 1.0f);
    geom[c] = make_float4(cx, cy, cz, 0.0f);
    r2bits[c] = 0u;
}

__global__ void k_mark_leaves(int nc, const int *pbeg, const int *pcnt, const int *ccnt, int *leaf_of)
{
    const int c = blockIdx.x;
    if (c >= nc || ccnt[c] != 0) return;
    for (int j = threadIdx.x; j < pcnt[c]; j += blockDim.x) leaf_of[pbeg[c] + j] = c;
}

constexpr int kRadThreads = 256;

// Tight radius: for each particle and each of its ancestors (levels 0..leaf), the
// FP32 squared distance to the cell centre, max-reduced per cell.  Consecutive
// particles share ancestors, so the max is taken per block when the whole block
// sits in one cell, else per run of equal cells inside a warp, then atomically.
__global__ void __launch_bounds__(kRadThreads) k_radius(int64_t n, const float4 *pos, const int *leaf_of,
                                                        const int *parent, const int *level, const float4 *geom,
                                                        unsigned *r2bits)
{
    __shared__ int s_cell0;
    __shared__ int s_maxd;
    __shared__ unsigned s_red[kRadThreads / 32];
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = s < n;
    int cur = valid ? leaf_of[s] : -1;
    const int depth = valid ? level[cur] : -1;
    if (threadIdx.x == 0) s_maxd = -1;
    __syncthreads();
    atomicMax(&s_maxd, depth);
    const float4 u = valid ? pos[s] : make_float4(0.f, 0.f, 0.f, 0.f);
    const unsigned lane = lane_id();
    __syncthreads();
    const int maxd = s_maxd;
    for (int l = maxd; l >= 0; --l) {
        const int cell = (valid && depth >= l) ? cur : -1;
        unsigned bits = 0u;
        if (cell >= 0) {
            const float4 X = geom[cell];
            const float dx = __fsub_rn(u.x, X.x), dy = __fsub_rn(u.y, X.y), dz = __fsub_rn(u.z, X.z);
            const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            bits = __float_as_uint(r2);
        }
        if (threadIdx.x == 0) s_cell0 = cell;
        __syncthreads();
        const bool uniform = __syncthreads_and(cell == s_cell0) != 0;
        if (uniform) {
            if (s_cell0 >= 0) {
                unsigned m = bits;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
                if (lane == 0) s_red[threadIdx.x >> 5] = m;
                __syncthreads();
                if (threadIdx.x == 0) {
                    unsigned mm = 0;
                    for (int k = 0; k < kRadThreads / 32; ++k) mm = max(mm, s_red[k]);
                    atomicMax(&r2bits[s_cell0], mm);
                }
            }
        } else {
            // segmented max over runs of equal cells (runs are contiguous)
            unsigned m = bits;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned om = __shfl_down_sync(kFull, m, o);
                int oc = __shfl_down_sync(kFull, cell, o);
                if ((int)lane + o < 32 && oc == cell) m = max(m, om);
            }
            int prev = __shfl_up_sync(kFull, cell, 1);
            if (cell >= 0 && (lane == 0 || prev != cell)) atomicMax(&r2bits[cell], m);
        }
        __syncthreads();
        if (cell >= 0 && l > 0) cur = parent[cur];
    }
}

__global__ void k_radius_final(int nc, const unsigned *r2bits, float4 *geom)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    geom[c].w = __fsqrt_rn(__uint_as_float(r2bits[c]));
}

// Particle positions are stored as FP32 offsets from the centre of their
// leaf's parent (the "frame" cell; the root frames itself), d = u - X_frame,
// rounded once from the FP64 coordinates u of the key computation.  Cell
// centres are exact in FP32, so kernels recover differences of nearby
// particles to ~2^-24 of the frame size instead of 2^-24 of the domain size;
// sibling leaves share a frame, so a run of consecutive siblings is one
// contiguous block of particles in one frame.
__global__ void k_local_positions(int64_t n, const double *u, const int *leaf_of, const int *parent,
                                  const float4 *geom, float4 *pos)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int lf = leaf_of[s];
    const int fr = parent[lf] >= 0 ? parent[lf] : lf;
    const float4 X = geom[fr];
    pos[s] = make_float4(__double2float_rn(u[s] - (double)X.x), __double2float_rn(u[n + s] - (double)X.y),
                         __double2float_rn(u[2 * n + s] - (double)X.z), 0.0f);
}

static int grow_cells(Handle &h, int64_t need)
{
    if (need <= h.cell_cap) return FMM_OK;
    int64_t cap = std::max<int64_t>(need, h.cell_cap * 2);
    FMM_TRY(h.c_prefix.reserve_keep(cap * sizeof(uint64_t), h.stream));
    FMM_TRY(h.c_level.reserve_keep(cap * sizeof(int), h.stream));
    FMM_TRY(h.c_pbeg.reserve_keep(cap * sizeof(int), h.stream));
    FMM_TRY(h.c_pcnt.reserve_keep(cap * sizeof(int), h.stream));
    FMM_TRY(h.c_cbeg.reserve_keep(cap * sizeof(int), h.stream));
    FMM_TRY(h.c_ccnt.reserve_keep(cap * sizeof(int), h.stream));
    FMM_TRY(h.c_parent.reserve_keep(cap * sizeof(int), h.stream));
    h.cell_cap = cap;
    return FMM_OK;
}

int build_tree(Handle &h, const double *x)
{
    const int64_t N = h.N;
    phase_begin(h, FMM_PHASE_TREE);
    FMM_TRY(grow_cells(h, std::max<int64_t>(1024, 4 * (N / std::max(1, h.ncrit)) + 64)));
    ++h.launches;
    k_root<<<1, 1, 0, h.stream>>>((int)N, h.c_prefix.as<uint64_t>(), h.c_level.as<int>(), h.c_pbeg.as<int>(),
                                  h.c_pcnt.as<int>(), h.c_cbeg.as<int>(), h.c_ccnt.as<int>(), h.c_parent.as<int>());
    FMM_CHECK_LAUNCH("root");
    h.level_off.assign(1, 0);
    h.level_off.push_back(1);
    unsigned *total_host = &h.pinned->level_total;
    int rc = FMM_OK;
    for (int l = 0; l < kLevels; ++l) {
        const int64_t lo = h.level_off[l], hi = h.level_off[l + 1], n = hi - lo;
        if (n == 0) break;
        rc = h.c_tmp.reserve((size_t)(10 * n + 1) * sizeof(unsigned));
        if (rc) break;
        unsigned *cnt = h.c_tmp.as<unsigned>(), *off = cnt + n, *tot = off + n;
        int *bnd = reinterpret_cast<int *>(tot + 1);
        ++h.launches;
        k_split_bounds<<<ceil_div(n * 32, 128), 128, 0, h.stream>>>(l, (int)lo, (int)n, h.ncrit, h.keys.as<uint64_t>(),
                                                                   h.c_prefix.as<uint64_t>(), h.c_pbeg.as<int>(),
                                                                   h.c_pcnt.as<int>(), bnd, cnt);
        rc = scan_exclusive_u32(h, cnt, off, n, tot);
        if (rc) break;
        cudaError_t e = cudaMemcpyAsync(total_host, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, h.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h.stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "tree level count", __FILE__, __LINE__);
            break;
        }
        const int64_t next = *total_host;
        if (next == 0) break;
        rc = grow_cells(h, hi + next);
        if (rc) break;
        ++h.launches;
        k_split_write<<<ceil_div(n, 128), 128, 0, h.stream>>>(
            l, (int)lo, (int)n, h.ncrit, (int)hi, bnd, off, h.c_prefix.as<uint64_t>(), h.c_level.as<int>(),
            h.c_pbeg.as<int>(), h.c_pcnt.as<int>(), h.c_cbeg.as<int>(), h.c_ccnt.as<int>(), h.c_parent.as<int>());
        h.level_off.push_back(hi + next);
    }
    if (rc) return rc;
    FMM_CHECK_LAUNCH("tree levels");
    h.nlevels = (int)h.level_off.size() - 1;
    h.ncells = h.level_off.back();
    const int nc = (int)h.ncells;

    // geometry
    FMM_TRY(h.c_geom.reserve(nc * sizeof(float4)));
    FMM_TRY(h.c_r2bits.reserve(nc * sizeof(unsigned)));
    FMM_TRY(h.leaf_of.reserve(N * sizeof(int)));
    ++h.launches;
    k_centres<<<ceil_div(nc, 256), 256, 0, h.stream>>>(nc, h.c_prefix.as<uint64_t>(), h.c_level.as<int>(),
                                                       h.c_geom.as<float4>(), h.c_r2bits.as<unsigned>());
    ++h.launches;
    k_mark_leaves<<<nc, 64, 0, h.stream>>>(nc, h.c_pbeg.as<int>(), h.c_pcnt.as<int>(), h.c_ccnt.as<int>(),
                                           h.leaf_of.as<int>());
    ++h.launches;
    k_radius<<<ceil_div(N, kRadThreads), kRadThreads, 0, h.stream>>>(
        N, h.pos.as<float4>(), h.leaf_of.as<int>(), h.c_parent.as<int>(), h.c_level.as<int>(), h.c_geom.as<float4>(),
        h.c_r2bits.as<unsigned>());
    ++h.launches;
    k_radius_final<<<ceil_div(nc, 256), 256, 0, h.stream>>>(nc, h.c_r2bits.as<unsigned>(), h.c_geom.as<float4>());
    // from here on particles are stored relative to the centre of their leaf's parent
    ++h.launches;
    k_local_positions<<<ceil_div(N, 256), 256, 0, h.stream>>>(N, h.u_sorted.as<double>(), h.leaf_of.as<int>(),
                                                              h.c_parent.as<int>(), h.c_geom.as<float4>(),
                                                              h.pos.as<float4>());
    FMM_CHECK_LAUNCH("geometry");
    phase_end(h, FMM_PHASE_TREE);
    return FMM_OK;
}

}  // namespace fmm
