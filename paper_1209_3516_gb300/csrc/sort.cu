// sort.cu -- device-wide exclusive scan and LSD radix sort (64-bit keys).
//
// The radix sort orders the Morton keys of the particles (stable, so equal keys
// keep the caller's order: the octree of Table 2 is "Morton key" based) and
// groups the interaction lists by target cell.  Each 8-bit pass is three
// kernels: a per-tile digit histogram, a device-wide exclusive scan of the
// histograms in digit-major order, and a stable scatter whose in-tile ranks
// come from __match_any_sync peer groups.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "fmm_internal.cuh"

namespace fmm {

// ---------------------------------------------------------------------------
// exclusive scan of uint32
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;   // 4096 values per block

// Exclusive scan across the block (blockDim.x a multiple of 32, at most 1024).
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned *total)
{
    __shared__ unsigned warp_tot[32];
    __shared__ unsigned block_tot;
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned t = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        unsigned w = (int)lane < nw ? warp_tot[lane] : 0u;
        unsigned wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned t = __shfl_up_sync(kFull, wi, o);
            if ((int)lane >= o) wi += t;
        }
        if ((int)lane < nw) warp_tot[lane] = wi - w;
        if (lane == 31) block_tot = wi;
    }
    __syncthreads();
    unsigned res = incl - v + warp_tot[warp];
    if (total) *total = block_tot;
    __syncthreads();
    return res;
}

__global__ void k_scan_reduce(const unsigned *in, int64_t n, unsigned *block_sums)
{
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    s = warp_sum(s);
    __shared__ unsigned ws[kScanThreads / 32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned t = threadIdx.x < kScanThreads / 32 ? ws[threadIdx.x] : 0u;
        t = warp_sum(t);
        if (threadIdx.x == 0) block_sums[blockIdx.x] = t;
    }
}

// Single block: exclusive scan of nb block sums in place, total to *total.
__global__ void k_scan_blocks(unsigned *sums, int nb, unsigned *total)
{
    unsigned carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        int i = base + threadIdx.x;
        unsigned v = i < nb ? sums[i] : 0u;
        unsigned tot;
        unsigned ex = block_exclusive_scan(v, &tot);
        if (i < nb) sums[i] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_apply(const unsigned *in, int64_t n, const unsigned *block_off, unsigned *out)
{
    __shared__ unsigned tile[kScanChunk];
    const int64_t base = (int64_t)blockIdx.x * kScanChunk;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        tile[k * kScanThreads + threadIdx.x] = i < n ? in[i] : 0u;
    }
    __syncthreads();
    unsigned loc[kScanItems];
    unsigned s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        loc[k] = s;
        s += tile[threadIdx.x * kScanItems + k];
    }
    unsigned ex = block_exclusive_scan(s, nullptr) + block_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) tile[threadIdx.x * kScanItems + k] = ex + loc[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = tile[k * kScanThreads + threadIdx.x];
    }
}

// One block for arrays of at most one tile (one launch instead of three);
// longer arrays take the three-kernel scan, which is faster from two tiles on.
constexpr int64_t kScanSingleMax = kScanChunk;

__global__ void __launch_bounds__(kScanThreads) k_scan_single(const unsigned *in, int64_t n, unsigned *out,
                                                              unsigned *total)
{
    __shared__ unsigned tile[kScanChunk];
    unsigned carry = 0;
    unsigned nxt[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t i = k * kScanThreads + threadIdx.x;
        nxt[k] = i < n ? in[i] : 0u;
    }
    for (int64_t base = 0; base < n; base += kScanChunk) {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) tile[k * kScanThreads + threadIdx.x] = nxt[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t i = base + kScanChunk + k * kScanThreads + threadIdx.x;
            nxt[k] = i < n ? in[i] : 0u;
        }
        unsigned loc[kScanItems];
        unsigned s = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            loc[k] = s;
            s += tile[threadIdx.x * kScanItems + k];
        }
        unsigned tot;
        const unsigned ex = block_exclusive_scan(s, &tot) + carry;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) tile[threadIdx.x * kScanItems + k] = ex + loc[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t i = base + k * kScanThreads + threadIdx.x;
            if (i < n) out[i] = tile[k * kScanThreads + threadIdx.x];
        }
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

int scan_exclusive_u32(Handle &h, const unsigned *in, unsigned *out, int64_t n, unsigned *total_dev)
{
    return scan_exclusive_u32_on(h, h.stream, h.scan_tmp, in, out, n, total_dev);
}

int scan_exclusive_u32_on(Handle &h, cudaStream_t stream, DevBuf &tmp, const unsigned *in, unsigned *out, int64_t n,
                          unsigned *total_dev)
{
    if (n <= 0) {
        if (total_dev) FMM_CUDA(cudaMemsetAsync(total_dev, 0, sizeof(unsigned), stream));
        return FMM_OK;
    }
    if (n <= kScanSingleMax) {
        ++h.launches;
        k_scan_single<<<1, kScanThreads, 0, stream>>>(in, n, out, total_dev);
        FMM_CHECK_LAUNCH("scan");
        return FMM_OK;
    }
    const int nb = ceil_div(n, kScanChunk);
    FMM_TRY(tmp.reserve((size_t)(nb + 1) * sizeof(unsigned)));
    unsigned *sums = tmp.as<unsigned>();
    ++h.launches;
    k_scan_reduce<<<nb, kScanThreads, 0, stream>>>(in, n, sums);
    ++h.launches;
    k_scan_blocks<<<1, kScanThreads, 0, stream>>>(sums, nb, total_dev);
    ++h.launches;
    k_scan_apply<<<nb, kScanThreads, 0, stream>>>(in, n, sums, out);
    FMM_CHECK_LAUNCH("scan");
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsMaxRounds = 16;   // a tile is kRsThreads x rounds keys, rounds <= 16 (4096 keys)

template <class K>
__global__ void __launch_bounds__(kRsThreads) k_rs_upsweep(const K *keys, int64_t n, int shift, int ntiles,
                                                           int rounds, unsigned *hist)
{
    __shared__ unsigned cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * rounds * kRsThreads;
#pragma unroll 4
    for (int r = 0; r < rounds; ++r) {
        int64_t i = base + r * kRsThreads + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(unsigned)(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

template <class K, bool kVals>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K *keys, const unsigned *vals, int64_t n,
                                                           int shift, int ntiles, int rounds,
                                                           const unsigned *offsets, K *keys_out, unsigned *vals_out)
{
    __shared__ unsigned s_base[256];
    __shared__ unsigned s_cnt[kRsWarps][256];
    const unsigned t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    s_base[t] = offsets[(int64_t)t * ntiles + blockIdx.x];
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) s_cnt[w][t] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * rounds * kRsThreads;
    for (int r = 0; r < rounds; ++r) {
        const int64_t i = base + r * kRsThreads + t;
        const bool valid = i < n;
        K key = valid ? keys[i] : (K)0;
        unsigned val = 0;
        if (kVals && valid) val = vals[i];
        const unsigned d = valid ? ((unsigned)(key >> shift) & 0xffu) : 256u;
        const unsigned peers = __match_any_sync(kFull, d);
        const unsigned rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) s_cnt[warp][d] = __popc(peers);
        __syncthreads();
        unsigned run = 0;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) {
            unsigned c = s_cnt[w][t];
            s_cnt[w][t] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            const unsigned pos = s_base[d] + s_cnt[warp][d] + rank;
            keys_out[pos] = key;
            if (kVals) vals_out[pos] = val;
        }
        __syncthreads();
        s_base[t] += run;
#pragma unroll
        for (int w = 0; w < kRsWarps; ++w) s_cnt[w][t] = 0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// One-sweep LSD radix sort (one kernel per 8-bit pass): the digit totals of
// every pass come from one histogram kernel; in a pass, each block claims the
// next tile in order, ranks its keys stably per warp (peer groups of equal
// digits, warp-private running counts), publishes the tile's digit counts and
// finds the count of each digit in all earlier tiles by looking back over
// their published counts (decoupled look-back: a tile whose prefix is known
// publishes the inclusive prefix, so a look-back stops there), then scatters.
// Every wait of the look-back is bounded; a wait that gives up sets bit 8 of
// the error word (the build then fails instead of hanging).
// ---------------------------------------------------------------------------
// Tile shape (N = 1M, Morton sort phase): 256 x 16 keys 0.276 ms, 512 x 8 0.266,
// 512 x 16 (spills) 0.259, 1024 x 8 0.252: fewer, larger tiles shorten the
// look-back chain.
#ifndef FMM_OS_THREADS
#define FMM_OS_THREADS 1024
#endif
constexpr int kOsThreads = FMM_OS_THREADS;              // threads 0..255 also own one digit each
constexpr int kOsWarps = kOsThreads / 32;
#ifndef FMM_OS_PER_THREAD
#define FMM_OS_PER_THREAD 8
#endif
constexpr int kOsPerThread = FMM_OS_PER_THREAD;         // keys per thread
// Peer groups (lanes holding the same digit) from nine ballots, one per bit
// of the 9-bit value, instead of __match_any_sync: sort phase at N = 1M
// 0.253 -> 0.230 ms.
#ifndef FMM_OS_BALLOT
#define FMM_OS_BALLOT 1
#endif
constexpr bool kOsBallotPeers = FMM_OS_BALLOT != 0;
constexpr int kOsTile = kOsThreads * kOsPerThread;      // keys per tile (8192)
constexpr unsigned kOsAgg = 1u << 30, kOsPrefix = 2u << 30, kOsValue = (1u << 30) - 1u;
constexpr int kOsSpinMax = 1 << 20;   // look-back windows without progress before giving up
constexpr int kOsWindow = 16;          // predecessors read per look-back window

// A status word holds its own flag and count in one 32-bit store, and nothing
// else is read through it, so relaxed device-scope accesses suffice.
__device__ __forceinline__ void st_status(unsigned *p, unsigned v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_status(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ghist[pass][digit] += count of keys with that digit, for every pass.
template <class K>
__global__ void __launch_bounds__(kOsThreads) k_os_hist(const K *keys, int64_t n, int begin_bit, int npass,
                                                        unsigned *ghist)
{
    __shared__ unsigned h[8][256];
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) (&h[0][0])[i] = 0u;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const K k = keys[i];
        for (int p = 0; p < npass; ++p) atomicAdd(&h[p][(unsigned)(k >> (begin_bit + 8 * p)) & 0xffu], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * 256; i += blockDim.x) {
        const unsigned c = (&h[0][0])[i];
        if (c) atomicAdd(&ghist[i], c);
    }
}

template <class K, bool kVals>
__global__ void __launch_bounds__(kOsThreads, 1024 / kOsThreads) k_os_pass(const K *keys, const unsigned *vals, int64_t n, int shift,
                                                        const unsigned *ghist, unsigned *status, unsigned *tile_ctr,
                                                        K *keys_out, unsigned *vals_out, unsigned *err)
{
    __shared__ unsigned s_tile;
    __shared__ unsigned s_wcnt[kOsWarps][256];   // per-warp running digit counts, then warp offsets
    __shared__ unsigned s_base[256];             // global position of the tile's first key of each digit
    const unsigned t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    if (t == 0) s_tile = atomicAdd(tile_ctr, 1u);
    for (int i = t; i < kOsWarps * 256; i += kOsThreads) (&s_wcnt[0][0])[i] = 0u;
    __syncthreads();
    const unsigned tile = s_tile;
    // digit start over all keys (exclusive scan of this pass's totals)
    const unsigned dstart = block_exclusive_scan(t < 256u ? ghist[t] : 0u, nullptr);
    // warp w ranks its keys [w 32 R, (w + 1) 32 R) of the tile, 32 per round in order
    const int64_t base = (int64_t)tile * kOsTile + (int64_t)warp * 32 * kOsPerThread;
    K key[kOsPerThread];
    unsigned val[kOsPerThread], dig[kOsPerThread], rank[kOsPerThread];
#pragma unroll
    for (int r = 0; r < kOsPerThread; ++r) {
        const int64_t i = base + 32 * r + lane;
        const bool valid = i < n;
        key[r] = valid ? keys[i] : (K)0;
        val[r] = (kVals && valid) ? vals[i] : 0u;
        dig[r] = valid ? ((unsigned)(key[r] >> shift) & 0xffu) : 256u;
    }
#pragma unroll
    for (int r = 0; r < kOsPerThread; ++r) {
        const unsigned d = dig[r];
        unsigned peers;
        if constexpr (kOsBallotPeers) {
            // lanes with the same 9-bit value (digit, or 256 past the end): one ballot per bit
            peers = kFull;
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                const unsigned m = __ballot_sync(kFull, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? m : ~m;
            }
        } else {
            peers = __match_any_sync(kFull, d);
        }
        const unsigned before = d < 256u ? s_wcnt[warp][d] : 0u;
        rank[r] = before + __popc(peers & lanemask_lt());
        __syncwarp();
        if (d < 256u && lane == (unsigned)(__ffs(peers) - 1)) s_wcnt[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread t < 256 = digit t: the tile's count and each warp's offset within
    // the tile, then the count in all earlier tiles
    if (t < 256u) {
    unsigned cnt = 0;
#pragma unroll
    for (int w = 0; w < kOsWarps; ++w) {
        const unsigned c = s_wcnt[w][t];
        s_wcnt[w][t] = cnt;
        cnt += c;
    }
    // publish, then look back for the count of digit t in all earlier tiles
    unsigned *st = status + (size_t)tile * 256;
    unsigned excl = 0;
    if (tile == 0) {
        st_status(st + t, kOsPrefix | cnt);
    } else {
        st_status(st + t, kOsAgg | cnt);
        // windows of kOsWindow predecessors: their words are read together, then
        // consumed nearest first up to the first word not yet published (read
        // again in the next window) or the first inclusive prefix
        int64_t j = (int64_t)tile - 1;
        int idle = 0;
        for (;;) {
            unsigned v[kOsWindow];
#pragma unroll
            for (int q = 0; q < kOsWindow; ++q)
                v[q] = j - q >= 0 ? ld_status(status + (size_t)(j - q) * 256 + t) : kOsPrefix;
            int used = 0;
            bool found = false;
#pragma unroll
            for (int q = 0; q < kOsWindow; ++q) {
                if (found || used < q || !(v[q] & (kOsAgg | kOsPrefix))) continue;
                excl += v[q] & kOsValue;
                used = q + 1;
                found = (v[q] & kOsPrefix) != 0;
            }
            if (found) break;
            j -= used;
            if (used == 0 && ++idle >= kOsSpinMax) {
                atomicOr(err, 8u);
                break;
            }
        }
        st_status(st + t, kOsPrefix | (excl + cnt));
    }
    s_base[t] = dstart + excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kOsPerThread; ++r) {
        const unsigned d = dig[r];
        if (d < 256u) {
            const unsigned pos = s_base[d] + s_wcnt[warp][d] + rank[r];
            keys_out[pos] = key[r];
            if (kVals) vals_out[pos] = val[r];
        }
    }
}

template <class K>
static int radix_sort_impl(Handle &h, K *&keys, K *&keys_alt, unsigned *&vals, unsigned *&vals_alt, bool with_vals,
                           int64_t n, int begin_bit, int end_bit)
{
    if (n <= 1 || end_bit <= begin_bit) return FMM_OK;
    if (n > 0xffffffffll) {
        set_error("radix sort: more than 2^32 keys");
        return FMM_ERR_ARG;
    }
    const int npass = (end_bit - begin_bit + 7) / 8;
    if (n < (int64_t)kOsValue && npass <= 8) {
        // one-sweep passes
        const int ntiles = ceil_div(n, (int64_t)kOsTile);
        const size_t words = (size_t)npass * 256 + (size_t)npass * 32 + (size_t)npass * ntiles * 256;
        FMM_TRY(h.sort_hist.reserve(words * sizeof(unsigned)));
        FMM_TRY(h.err_flag.reserve(sizeof(unsigned)));
        unsigned *ghist = h.sort_hist.as<unsigned>();
        unsigned *ctrs = ghist + (size_t)npass * 256;   // one tile counter per pass (32-word stride)
        unsigned *status = ctrs + (size_t)npass * 32;
        FMM_CUDA(cudaMemsetAsync(ghist, 0, words * sizeof(unsigned), h.stream));
        ++h.launches;
        k_os_hist<K><<<std::min<int64_t>(ceil_div(n, (int64_t)kOsThreads * 8), (int64_t)h.num_sms * 8), kOsThreads,
                       0, h.stream>>>(keys, n, begin_bit, npass, ghist);
        for (int p = 0; p < npass; ++p) {
            const int shift = begin_bit + 8 * p;
            unsigned *stp = status + (size_t)p * ntiles * 256;
            ++h.launches;
            if (with_vals)
                k_os_pass<K, true><<<ntiles, kOsThreads, 0, h.stream>>>(keys, vals, n, shift, ghist + 256 * p, stp,
                                                                       ctrs + 32 * p, keys_alt, vals_alt,
                                                                       h.err_flag.as<unsigned>());
            else
                k_os_pass<K, false><<<ntiles, kOsThreads, 0, h.stream>>>(keys, nullptr, n, shift, ghist + 256 * p,
                                                                        stp, ctrs + 32 * p, keys_alt, nullptr,
                                                                        h.err_flag.as<unsigned>());
            FMM_CHECK_LAUNCH("radix pass");
            std::swap(keys, keys_alt);
            if (with_vals) std::swap(vals, vals_alt);
        }
        return FMM_OK;
    }
    // tiles small enough that the grid covers the SMs about four times over
    // (latency-bound kernels), at most 16 rounds of 256 keys
    const int rounds = (int)std::max<int64_t>(1, std::min<int64_t>(kRsMaxRounds, n / ((int64_t)kRsThreads * 4 * h.num_sms)));
    const int ntiles = ceil_div(n, (int64_t)rounds * kRsThreads);
    const int64_t nh = (int64_t)256 * ntiles;
    FMM_TRY(h.sort_hist.reserve((size_t)nh * 2 * sizeof(unsigned)));
    unsigned *hist = h.sort_hist.as<unsigned>();
    unsigned *offs = hist + nh;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        ++h.launches;
        k_rs_upsweep<K><<<ntiles, kRsThreads, 0, h.stream>>>(keys, n, shift, ntiles, rounds, hist);
        FMM_CHECK_LAUNCH("radix upsweep");
        FMM_TRY(scan_exclusive_u32(h, hist, offs, nh, nullptr));
        if (with_vals) {
            ++h.launches;
            k_rs_scatter<K, true><<<ntiles, kRsThreads, 0, h.stream>>>(keys, vals, n, shift, ntiles, rounds, offs,
                                                                     keys_alt, vals_alt);
        } else {
            ++h.launches;
            k_rs_scatter<K, false><<<ntiles, kRsThreads, 0, h.stream>>>(keys, nullptr, n, shift, ntiles, rounds,
                                                                      offs, keys_alt, nullptr);
        }
        FMM_CHECK_LAUNCH("radix scatter");
        K *tk = keys;
        keys = keys_alt;
        keys_alt = tk;
        if (with_vals) {
            unsigned *tv = vals;
            vals = vals_alt;
            vals_alt = tv;
        }
    }
    return FMM_OK;
}

int radix_sort_pairs(Handle &h, uint64_t *&keys, uint64_t *&keys_alt, unsigned *&vals, unsigned *&vals_alt,
                     int64_t n, int begin_bit, int end_bit)
{
    return radix_sort_impl<uint64_t>(h, keys, keys_alt, vals, vals_alt, true, n, begin_bit, end_bit);
}

int radix_sort_keys(Handle &h, uint64_t *&keys, uint64_t *&keys_alt, int64_t n, int begin_bit, int end_bit)
{
    unsigned *a = nullptr, *b = nullptr;
    return radix_sort_impl<uint64_t>(h, keys, keys_alt, a, b, false, n, begin_bit, end_bit);
}

int radix_sort_keys32(Handle &h, uint32_t *&keys, uint32_t *&keys_alt, int64_t n, int begin_bit, int end_bit)
{
    unsigned *a = nullptr, *b = nullptr;
    return radix_sort_impl<uint32_t>(h, keys, keys_alt, a, b, false, n, begin_bit, end_bit);
}

}  // namespace fmm
