// batch_tc.cu -- many charge vectors: P2P + L2P on the 5th-generation tensor cores.
//
// For a work item of <= 32 targets of one leaf and 32 charge vectors, the near
// field (Sec. 3.3, the P2P kernel) and the leaf's local expansion (the L2P of
// the downward pass) are one accumulation into a 128 x 32 FP32 tile D in
// tensor memory (TMEM):
//     D[(k, t), r] = sum_s G_k(t, s) Q[s, r]  +  sum_n W_k(t, n) Lb[n, r]
// with rows (kernel k, target t), k = 0 for 1/r and k = 1..3 for the components
// of e/r^3 (e = u_s - u_t), columns r = charge vector; W_0(t, n) = w_n(v_t) are
// the target's Taylor monomials and W_d(t, n) = w_{n - e_d}(v_t) / s their
// derivatives, so that the potential and the gradient of the local expansion
// (phi = sum_n Lb_n w_n, d phi / dx_d = (1/s) sum_m Lb_{m + e_d} w_m) come out
// of the same product.  The source (or expansion-row) axis is walked in
// chunks of 32:
//   - warp 0 stages a chunk: the sources' positions moved into the target
//     frame, and their 32 charges (or the leaf's 32 expansion rows), split into
//     BF16 high and low parts, copied by cp.async into the MN-major B layout;
//   - every thread computes its share of the A operand on the CUDA cores
//     (thread (g, j) of warp w: target 8 w' + g, the 4 sources 4 j .. 4 j + 3
//     of a K = 16 step) and writes it, split into BF16 high and low parts,
//     straight into TMEM with tcgen05.st (16x256b: the lanes of the warp's
//     quarter, two BF16 per column);
//   - one thread issues tcgen05.mma kind::f16 (A from TMEM, B from shared
//     memory, FP32 accumulate) three times per K step: hi*hi, hi*lo and lo*hi,
//     which keeps each product to ~2^-16 relative, and commits the chunk to an
//     mbarrier; A and B are double-buffered, so the next chunk is generated and
//     staged while the tensor core works on this one.
// Items of <= 16 targets occupy two warp quarters only; the other two quarters
// then hold the same targets and take the odd K steps (their rows of the even
// steps are zero and vice versa), so that all four warps generate, and the two
// halves of D are added in the epilogue.  The epilogue reads D from TMEM
// (tcgen05.ld), restores the units and writes the results in caller order.
// The CTA is persistent (4 per SM, 128 TMEM columns each: all 512 columns of
// an SM) and claims work items from a counter.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "fmm_internal.cuh"
#include "mi.cuh"
#include "p2p_common.cuh"
#include "tc.cuh"

namespace fmm {

constexpr int kTcGenWarps = 4;    // warps 0-3 generate A: warp w writes TMEM lane quarter w
constexpr int kTcThreads = 32 * (kTcGenWarps + 1);   // warp 4 stages chunks and issues the MMAs
constexpr int kTcTargets = 32;    // targets per work item
constexpr int kTcChunk = 32;      // sources (or expansion rows) per staged chunk: two K = 16 steps
constexpr int kTcSlots = kTcChunk / 32;   // staged rows per producer lane
constexpr int kTcABufs = 3;       // A operands in TMEM (one chunk each)
constexpr int kTcStages = 4;      // staged chunks in shared memory (ring)
constexpr int kTcCols = 128;      // TMEM columns per CTA: D [0, 32), A buffer a at 32 + 32 a (hi / lo per K step)
constexpr int kTcCtasPerSM = 4;   // 4 x 128 columns = the SM's 512
constexpr int kTcRhs = 32;
constexpr unsigned kTcIdesc = tc::idesc_bf16(128, kTcRhs);
// B layout of one chunk (MN-major, no swizzle): k-step s at s * 1024, its two
// 8-row core-matrix groups along K at 512 bytes, the four 8-column groups
// along N at 128 bytes, one 16-byte row per k.
constexpr unsigned kTcLbo = 512, kTcSbo = 128;

struct TcSmem {
    unsigned char bq[kTcStages][2][kTcChunk * 64];   // [stage][hi, lo] charges or expansion rows, BF16, MN-major
    float4 spos[kTcStages][kTcChunk];       // [stage] staged source positions in the target frame
    float xch[64][kTcRhs + 1];              // epilogue: the replicated half of D
    float pw[kTcGenWarps][8][3][8];         // per generating warp and target: v_d^a / a!, a < P (L2P)
    unsigned long long staged[kTcStages];   // per stage: the producer has staged a chunk
    unsigned long long full[kTcABufs];      // per A buffer: the generating warps have written A
    unsigned long long empty[kTcABufs];     // per A buffer: the chunk's MMAs have completed
    unsigned long long dfree;               // the epilogue warps have read D
    unsigned long long xbar;                // warps 2 and 3 have written their half of D to xch
    unsigned long long fin;                 // every MMA of the CTA has completed
    int meta[kTcStages][8];                 // per stage: rows, self, kind, first row, item (-1: end), first, last
    unsigned tmem_base;
};
// Dynamic shared memory requested per CTA: more than the structure, so that no
// more than four CTAs (the TMEM budget) can be resident on one SM.
constexpr int kTcSmemBytes = 50 * 1024;
static_assert(sizeof(TcSmem) + 1024 <= kTcSmemBytes, "shared memory layout");
// TMEM column of the high parts of K step s of A buffer a (low parts 8 columns on)
__host__ __device__ constexpr unsigned tc_acol(int a, int s) { return 32u + 32u * (unsigned)a + 16u * (unsigned)s; }
static_assert(tc_acol(kTcABufs - 1, kTcChunk / 16 - 1) + 16 <= kTcCols, "TMEM columns");

// Multi-index table (a | b << 4 | c << 8) by storage index, 0xFFFF past T.
template <int P> struct TcMI {
    unsigned short v[128];
};
template <int P> __host__ __device__ constexpr TcMI<P> make_tc_mi()
{
    TcMI<P> t{};
    for (int i = 0; i < 128; ++i) t.v[i] = 0xFFFF;
    for (int n = 0; n < P; ++n)
        for (int a = n; a >= 0; --a)
            for (int b = n - a; b >= 0; --b) {
                const int c = n - a - b;
                t.v[MI<P>::idx(a, b, c)] = (unsigned short)(a | (b << 4) | (c << 8));
            }
    return t;
}
__constant__ TcMI<3> c_tc_mi3 = make_tc_mi<3>();
__constant__ TcMI<4> c_tc_mi4 = make_tc_mi<4>();
__constant__ TcMI<5> c_tc_mi5 = make_tc_mi<5>();
__constant__ TcMI<6> c_tc_mi6 = make_tc_mi<6>();
__constant__ TcMI<8> c_tc_mi8 = make_tc_mi<8>();
template <int P> __device__ __forceinline__ unsigned tc_mi(int n);
template <> __device__ __forceinline__ unsigned tc_mi<3>(int n) { return c_tc_mi3.v[n]; }
template <> __device__ __forceinline__ unsigned tc_mi<4>(int n) { return c_tc_mi4.v[n]; }
template <> __device__ __forceinline__ unsigned tc_mi<5>(int n) { return c_tc_mi5.v[n]; }
template <> __device__ __forceinline__ unsigned tc_mi<6>(int n) { return c_tc_mi6.v[n]; }
template <> __device__ __forceinline__ unsigned tc_mi<8>(int n) { return c_tc_mi8.v[n]; }

// v = hi + lo for two values: hi = bf16(v) (round to nearest), lo = bf16(v - hi),
// each packed two per register (the first value in the low half).
__device__ __forceinline__ void tc_split(float2 v, unsigned &hi, unsigned &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    hi = *reinterpret_cast<const unsigned *>(&h);
    const float2 r = __fadd2_rn(v, make_float2(-__uint_as_float(hi << 16), -__uint_as_float(hi & 0xffff0000u)));
    const __nv_bfloat162 l = __floats2bfloat162_rn(r.x, r.y);
    lo = *reinterpret_cast<const unsigned *>(&l);
}

// The four kernel values of one target (negated position nt) with two sources
// (positions in the target frame): 1/r and e/r^3, e = u_s - u_t, each as
// (first source, second source).  kExact: a pair at distance 0 gives 0.
template <bool kExact>
__device__ __forceinline__ void tc_kernel2(float4 s0, float4 s1, float2 ntx, float2 nty, float2 ntz, float2 *kv)
{
    constexpr float kEps = 1.17549435e-38f;
    const float2 ex = __fadd2_rn(make_float2(s0.x, s1.x), ntx);
    const float2 ey = __fadd2_rn(make_float2(s0.y, s1.y), nty);
    const float2 ez = __fadd2_rn(make_float2(s0.z, s1.z), ntz);
    const float2 r2 = __ffma2_rn(ez, ez, __ffma2_rn(ey, ey, __ffma2_rn(ex, ex, make_float2(kEps, kEps))));
    float2 rinv;
    if (kExact) {
        rinv.x = r2.x > kEps ? rsqrt_approx(r2.x) : 0.0f;
        rinv.y = r2.y > kEps ? rsqrt_approx(r2.y) : 0.0f;
    } else {
        rinv.x = rsqrt_approx(r2.x);
        rinv.y = rsqrt_approx(r2.y);
    }
    const float2 rinv3 = __fmul2_rn(__fmul2_rn(rinv, rinv), rinv);
    kv[0] = rinv;
    kv[1] = __fmul2_rn(ex, rinv3);
    kv[2] = __fmul2_rn(ey, rinv3);
    kv[3] = __fmul2_rn(ez, rinv3);
}

// Write the A values of one K step of a thread (kernel k, its 4 k-columns as two
// pairs: v[k][0] = columns 4j, 4j+1, v[k][1] = 4j+2, 4j+3) into TMEM, high parts
// at column ahi, low parts at ahi + 8; q is the TMEM address of the warp quarter.
__device__ __forceinline__ void tc_store_step(unsigned q, unsigned ahi, const float2 (*v)[2])
{
    unsigned h[4][2], l[4][2];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int p = 0; p < 2; ++p) tc_split(v[k][p], h[k][p], l[k][p]);
    tc::st_16x256b(q + ahi, h[0][0], h[0][1], h[1][0], h[1][1]);
    tc::st_16x256b(q + (16u << 16) + ahi, h[2][0], h[2][1], h[3][0], h[3][1]);
    tc::st_16x256b(q + ahi + 8, l[0][0], l[0][1], l[1][0], l[1][1]);
    tc::st_16x256b(q + (16u << 16) + ahi + 8, l[2][0], l[2][1], l[3][0], l[3][1]);
}
__device__ __forceinline__ void tc_store_zero(unsigned q, unsigned ahi)
{
    tc::st_16x256b(q + ahi, 0u, 0u, 0u, 0u);
    tc::st_16x256b(q + (16u << 16) + ahi, 0u, 0u, 0u, 0u);
    tc::st_16x256b(q + ahi + 8, 0u, 0u, 0u, 0u);
    tc::st_16x256b(q + (16u << 16) + ahi + 8, 0u, 0u, 0u, 0u);
}

// The producer's cursor over an item's source runs.  The run records are held
// in a register window (lane k: run wbase + k, loaded 32 at a time with one
// coalesced load) and handed out by shuffles, so that crossing into the next
// run costs no dependent global load.
struct TcRuns {
    int e, e1, wbase, o;   // current run, end of the item's runs, first run of the window, taken of run e
    float4 rec;            // lane k: record of run wbase + k (frame shift, first particle)
    int rend;              // lane k: end particle of run wbase + k
    int pb, cnt;           // run e: first particle, count (warp-uniform)
    float shx, shy, shz;   // run e: frame shift
    __device__ __forceinline__ void window(const float4 *run, const int *run_end)
    {
        const int k = e + (int)lane_id();
        wbase = e;
        if (k < e1) {
            rec = run[k];
            rend = run_end[k];
        }
    }
    __device__ __forceinline__ void fetch()
    {
        const int src = e - wbase;
        shx = __shfl_sync(kFull, rec.x, src);
        shy = __shfl_sync(kFull, rec.y, src);
        shz = __shfl_sync(kFull, rec.z, src);
        pb = __float_as_int(__shfl_sync(kFull, rec.w, src));
        cnt = __shfl_sync(kFull, rend, src) - pb;
    }
    __device__ __forceinline__ void init(const unsigned *roff, int li, const float4 *run, const int *run_end)
    {
        e = (int)roff[li];
        e1 = (int)roff[li + 1];
        o = 0;
        if (e < e1) {
            window(run, run_end);
            fetch();
        }
    }
    __device__ __forceinline__ void advance(const float4 *run, const int *run_end)
    {
        ++e;
        o = 0;
        if (e < e1) {
            if (e - wbase >= 32) window(run, run_end);
            fetch();
        }
    }
};

// The producer's view of the chunk it is staging: lane k holds slots k, k + 32, ...
struct TcStage {
    int row[kTcSlots];     // global row (sorted particle, or leaf-list row li * T + n); -1 past the count
    float4 p[kTcSlots];    // the particles' positions (P2P), loaded at pick time
    float sh[kTcSlots][3]; // their frame shifts
    int count, self, kind, base;
    int item, first, last;   // work item (-1: no more work), first / last chunk of the item
};

// Pick the next chunk of an item: up to kTcChunk sources of its runs
// (warp-uniform cursor), then the leaf's expansion rows kTcChunk at a time.  False when none is left.
template <int P>
__device__ __forceinline__ bool tc_pick(TcRuns &cur, const float4 *run, const int *run_end, const float4 *pos,
                                        int lb0, int lb1, int li, int &lchunk, TcStage &st)
{
    constexpr int T = MI<P>::T;
    const int lane = (int)lane_id();
#pragma unroll
    for (int h = 0; h < kTcSlots; ++h) {
        st.row[h] = -1;
        st.sh[h][0] = st.sh[h][1] = st.sh[h][2] = 0.0f;
    }
    if (cur.e < cur.e1) {
        int slots = 0;
        bool sf = false;
        while (slots < kTcChunk && cur.e < cur.e1) {
            const int m = min(cur.cnt - cur.o, kTcChunk - slots);
            const int begin = cur.pb + cur.o;
            sf |= begin < lb1 && begin + m > lb0;
#pragma unroll
            for (int h = 0; h < kTcSlots; ++h) {
                const int k = lane + 32 * h;
                if (k >= slots && k < slots + m) {
                    st.row[h] = begin + k - slots;
                    st.sh[h][0] = cur.shx;
                    st.sh[h][1] = cur.shy;
                    st.sh[h][2] = cur.shz;
                }
            }
            slots += m;
            cur.o += m;
            if (cur.o == cur.cnt) cur.advance(run, run_end);
        }
        st.count = slots;
        st.self = sf ? 1 : 0;
        st.kind = 0;
        st.base = 0;
        st.last = 0;   // the expansion rows follow
#pragma unroll
        for (int h = 0; h < kTcSlots; ++h)
            if (st.row[h] >= 0) st.p[h] = pos[st.row[h]];   // in flight until the chunk is staged
        return true;
    }
    const int base = lchunk * kTcChunk;
    if (base >= T) return false;
    ++lchunk;
#pragma unroll
    for (int h = 0; h < kTcSlots; ++h) {
        const int nn = base + lane + 32 * h;
        st.row[h] = nn < T ? li * T + nn : -1;
    }
    st.count = min(kTcChunk, T - base);
    st.self = 0;
    st.kind = 1;
    st.base = base;
    st.last = lchunk * kTcChunk >= T ? 1 : 0;
    return true;
}

// Stage the picked chunk into ring slot sl (its previous MMAs have completed):
// the 32 BF16 values of each row, high and low parts, by cp.async into the
// MN-major layout (zeros past the count), the positions moved into the target
// frame (far away past the count, where every kernel value is 0), and the
// chunk's metadata.
__device__ __forceinline__ void tc_stage(TcSmem &S, int sl, const TcStage &st, const __nv_bfloat16 *qh,
                                         const __nv_bfloat16 *ql, const __nv_bfloat16 *lh, const __nv_bfloat16 *ll)
{
    const int lane = (int)lane_id();
    const __nv_bfloat16 *sh = st.kind ? lh : qh, *slo = st.kind ? ll : ql;
#pragma unroll
    for (int h = 0; h < kTcSlots; ++h) {
        const int k = lane + 32 * h;
        const int off = (k >> 4) * 1024 + ((k >> 3) & 1) * 512 + (k & 7) * 16;
        unsigned char *dh = S.bq[sl][0] + off, *dl = S.bq[sl][1] + off;
        if (st.row[h] >= 0) {
            const __nv_bfloat16 *gh = sh + (size_t)st.row[h] * kTcRhs, *gl = slo + (size_t)st.row[h] * kTcRhs;
#pragma unroll
            for (int ng = 0; ng < 4; ++ng) {
                cp_async16(dh + ng * 128, gh + ng * 8);
                cp_async16(dl + ng * 128, gl + ng * 8);
            }
        } else {
#pragma unroll
            for (int ng = 0; ng < 4; ++ng) {
                *reinterpret_cast<uint4 *>(dh + ng * 128) = make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(dl + ng * 128) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        S.spos[sl][k] = (st.kind == 0 && st.row[h] >= 0)
                            ? make_float4(st.p[h].x + st.sh[h][0], st.p[h].y + st.sh[h][1], st.p[h].z + st.sh[h][2], 0.0f)
                            : make_float4(1e20f, 1e20f, 1e20f, 0.0f);
    }
    if (lane == 0) {
        S.meta[sl][0] = st.count;
        S.meta[sl][1] = st.self;
        S.meta[sl][2] = st.kind;
        S.meta[sl][3] = st.base;
        S.meta[sl][4] = st.item;
        S.meta[sl][5] = st.first;
        S.meta[sl][6] = st.last;
    }
}

// Wait (bounded) for the given number of completions of an MMA mbarrier.
__device__ __forceinline__ bool tc_wait(unsigned long long *bar, unsigned completions)
{
    const unsigned parity = (completions - 1u) & 1u;
    for (unsigned i = 0; i < kMbarPolls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// A values of one K step of an L2P chunk for target factors pw (v_d^a / a!):
// rows 1/r -> w_n, e_d/r^3 -> w_{n - e_d} / s, for n = n0 .. n0 + 3.
template <int P>
__device__ __forceinline__ void tc_l2p_values(const float (*pw)[8], int n0, float inv_s, float2 (*v)[2])
{
    constexpr int T = MI<P>::T;
    float x[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int n = n0 + i;
        x[0][i] = x[1][i] = x[2][i] = x[3][i] = 0.0f;
        if (n < T) {
            const unsigned code = tc_mi<P>(n);
            const int a = code & 15, b = (code >> 4) & 15, c = code >> 8;
            const float fx = pw[0][a], fy = pw[1][b], fz = pw[2][c];
            const float fyz = fy * fz;
            x[0][i] = fx * fyz;
            if (a) x[1][i] = pw[0][a - 1] * fyz * inv_s;
            if (b) x[2][i] = fx * pw[1][b - 1] * fz * inv_s;
            if (c) x[3][i] = fx * fy * pw[2][c - 1] * inv_s;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k][0] = make_float2(x[k][0], x[k][1]);
        v[k][1] = make_float2(x[k][2], x[k][3]);
    }
}

// One K step of a P2P chunk: the thread's target (negated position) with the
// staged sources k0 .. k0 + 3.
template <bool kExact>
__device__ __forceinline__ void tc_p2p_values(const float4 *sp, int k0, float2 ntx, float2 nty, float2 ntz,
                                              float2 (*v)[2])
{
    float2 a[4], b[4];
    tc_kernel2<kExact>(sp[k0], sp[k0 + 1], ntx, nty, ntz, a);
    tc_kernel2<kExact>(sp[k0 + 2], sp[k0 + 3], ntx, nty, ntz, b);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k][0] = a[k];
        v[k][1] = b[k];
    }
}

__device__ __forceinline__ void mbar_arrive_one(unsigned long long *bar) { mbar_arrive(bar); }

// Producer (warp 8): claim items, pick and stage chunks two ahead of the
// generating warps into a ring of kTcStages shared-memory slots, and issue each
// chunk's MMAs once its A operand is complete.  A chunk's positions are loaded
// one iteration before they are staged, and its copies are waited for one
// iteration after they are issued, so no memory latency sits on the per-chunk
// path.  The chunk sequence ends with one marker chunk (item -1).
template <int P>
__device__ __forceinline__ bool tc_producer(TcSmem &S, unsigned tbase, int nitems, const int4 *items,
                                            unsigned *next_item, const unsigned *roff, const float4 *run,
                                            const int *run_end, const float4 *pos, const __nv_bfloat16 *qh,
                                            const __nv_bfloat16 *ql, const __nv_bfloat16 *lh,
                                            const __nv_bfloat16 *ll, const int *pbeg, const int *pcnt)
{
    const int lane = (int)lane_id();
    bool ok = true;
    TcRuns cur;
    int lchunk = 0, lb0 = 0, lb1 = 0, li = 0, item = -1;
    bool need_claim = true, done = false;
    auto pick = [&](TcStage &st) -> bool {
        if (done) return false;
        if (need_claim) {
            unsigned v = 0;
            if (lane == 0) v = atomicAdd(next_item, 1u);
            const int ii = (int)__shfl_sync(kFull, v, 0);
            if (ii >= nitems) {   // the end marker
                st.item = -1;
#pragma unroll
                for (int h = 0; h < kTcSlots; ++h) st.row[h] = -1;
                st.count = 0;
                st.self = st.kind = st.base = st.first = st.last = 0;
                done = true;
                return true;
            }
            const int4 it = items[ii];
            item = ii;
            li = it.w;
            lb0 = pbeg[it.x];
            lb1 = lb0 + pcnt[it.x];
            lchunk = 0;
            cur.init(roff, li, run, run_end);
            tc_pick<P>(cur, run, run_end, pos, lb0, lb1, li, lchunk, st);
            st.first = 1;
        } else {
            tc_pick<P>(cur, run, run_end, pos, lb0, lb1, li, lchunk, st);
            st.first = 0;
        }
        st.item = item;
        need_claim = st.last != 0;
        return true;
    };
    auto stage = [&](const TcStage &st, int c) {
        tc_stage(S, c % kTcStages, st, qh, ql, lh, ll);
        cp_async_commit();
    };
    auto signal = [&](int c) {   // every copy issued so far has landed: chunk c is complete
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive_one(&S.staged[c % kTcStages]);
    };

    TcStage a;
    pick(a);
    stage(a, 0);
    signal(0);
    bool h1 = pick(a);
    if (h1) stage(a, 1);
    bool h2 = pick(a);
    int items_started = 0;
    for (int c = 0;; ++c) {
        const int ab = c % kTcABufs, sl = c % kTcStages;
        if (h1) signal(c + 1);   // its copies were issued one iteration ago
        if (h2) {   // stage chunk c + 2 (its ring slot was last used by chunk c - 2)
            if (c >= 2) ok &= tc_wait(&S.empty[(c - 2) % kTcABufs], (unsigned)((c - 2) / kTcABufs) + 1u);
            stage(a, c + 2);
        }
        const bool h3 = h2 ? pick(a) : false;
        const int item_c = S.meta[sl][4];
        if (item_c < 0) break;
        const int cnt = S.meta[sl][0], first = S.meta[sl][5];
        ok &= tc_wait(&S.full[ab], (unsigned)(c / kTcABufs) + 1u);
        if (first) {
            if (items_started > 0) ok &= tc_wait(&S.dfree, (unsigned)items_started);   // D read out
            ++items_started;
        }
        if (!ok) break;   // a wait gave up: stop issuing (the host sees the error flag)
        if (lane == 0) {
            tc::fence_after();
            const int nsteps = (cnt + 15) >> 4;
#pragma unroll
            for (int s = 0; s < kTcChunk / 16; ++s) {
                if (s >= nsteps) break;
                const unsigned ahi = tbase + tc_acol(ab, s);
                const uint64_t dh = tc::smem_desc(S.bq[sl][0] + s * 1024, kTcLbo, kTcSbo);
                const uint64_t dl = tc::smem_desc(S.bq[sl][1] + s * 1024, kTcLbo, kTcSbo);
                tc::mma_ts(tbase, ahi, dh, kTcIdesc, !(first && s == 0));
                tc::mma_ts(tbase, ahi, dl, kTcIdesc, true);
                tc::mma_ts(tbase, ahi + 8u, dh, kTcIdesc, true);
            }
            tc::commit(&S.empty[ab]);
        }
        __syncwarp();
        h1 = h2;
        h2 = h3;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    // every MMA issued by this warp has completed before TMEM is released
    if (lane == 0) tc::commit(&S.fin);
    __syncwarp();
    ok &= tc_wait(&S.fin, 1u);
    return ok;
}

// Generating warps 0-7: warp w writes the A operand of TMEM lane quarter w % 4
// for half of each chunk's K steps; after an item's last chunk, warps 0-3 read
// D and write the results.
template <int P>
__device__ __forceinline__ bool tc_consumer(TcSmem &S, unsigned tbase, const int4 *items, const float4 *pos,
                                            const int *level, const int *parent, const float4 *geom,
                                            const int *perm, int64_t n, int nrhs, float phi_scale,
                                            float grad_scale, float *phi, float *grad)
{
    const int w = (int)(threadIdx.x >> 5), lane = (int)lane_id(), g = lane >> 2, j = lane & 3;
    const int q = w & 3, half = w >> 2;
    const unsigned qaddr = tbase + ((unsigned)(32 * q) << 16);   // this warp's lane quarter
    bool ok = true;
    int tb = 0, tcnt = 1, tq = 0, tt = 0;
    unsigned xcount = 0;   // epilogues that exchanged halves of D
    bool rep2 = false, active = false;
    float inv_s = 1.0f;
    float2 ntx = make_float2(0.f, 0.f), nty = ntx, ntz = ntx;
    for (int c = 0;; ++c) {
        const int ab = c % kTcABufs, sl = c % kTcStages;
        ok &= tc_wait(&S.staged[sl], (unsigned)(c / kTcStages) + 1u);
        if (!ok) break;
        const int cnt = S.meta[sl][0], self = S.meta[sl][1], kind = S.meta[sl][2], base = S.meta[sl][3];
        const int item = S.meta[sl][4], first = S.meta[sl][5], last = S.meta[sl][6];
        if (item < 0) break;
        if (first) {   // the item's targets
            const int4 it = items[item];
            const int leaf = it.x;
            tb = it.y;
            tcnt = it.z;
            rep2 = tcnt <= 16;
            tq = rep2 ? (q & 1) : q;
            tt = min(8 * tq + g, tcnt - 1);
            active = 8 * tq < tcnt;
            const float4 tp = pos[tb + tt];
            ntx = make_float2(-tp.x, -tp.x);
            nty = make_float2(-tp.y, -tp.y);
            ntz = make_float2(-tp.z, -tp.z);
            inv_s = ldexpf(1.0f, level[leaf]);
            if (active && j == 0) {   // L2P factors of this lane's target
                const float4 Xc = geom[leaf], Xf = geom[frame_of(parent, leaf)];
                const float vv[3] = {fmaf(tp.x, inv_s, -(Xc.x - Xf.x) * inv_s),
                                     fmaf(tp.y, inv_s, -(Xc.y - Xf.y) * inv_s),
                                     fmaf(tp.z, inv_s, -(Xc.z - Xf.z) * inv_s)};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    float f = 1.0f;
                    S.pw[w][g][d][0] = 1.0f;
#pragma unroll
                    for (int a = 1; a < P; ++a) {
                        f = f * (vv[d] * (1.0f / a));
                        S.pw[w][g][d][a] = f;
                    }
                }
            }
            __syncwarp();
        }
        if (c >= kTcABufs) ok &= tc_wait(&S.empty[ab], (unsigned)(c / kTcABufs));   // A[ab] free (chunk c - 3)
        tc::fence_after();
        const int nsteps = (cnt + 15) >> 4;
        if (active) {
            // the two K steps of this warp: (computed, computed) or, with replicated
            // quarters, (computed, zero) in the order of the step index
            const int s0 = rep2 ? 2 * half : 2 * half, s1 = s0 + 1;
            const int sc = rep2 ? (q >> 1) + 2 * half : -1;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int s = u ? s1 : s0;
                if (s >= nsteps) continue;
                const unsigned ahi = tc_acol(ab, s);
                if (rep2 && s != sc) {
                    tc_store_zero(qaddr, ahi);
                    continue;
                }
                float2 v[4][2];
                if (kind == 0) {
                    if (self) tc_p2p_values<true>(S.spos[sl], 16 * s + 4 * j, ntx, nty, ntz, v);
                    else tc_p2p_values<false>(S.spos[sl], 16 * s + 4 * j, ntx, nty, ntz, v);
                } else {
                    tc_l2p_values<P>(S.pw[w][tt - 8 * tq], base + 16 * s + 4 * j, inv_s, v);
                }
                tc_store_step(qaddr, ahi, v);
            }
        }
        tc::wait_st();
        tc::fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_one(&S.full[ab]);
        if (!last || half) continue;

        // epilogue (warps 0-3): D row 32 q + lane = kernel lane / 8 of target 8 tq + lane % 8
        ok &= tc_wait(&S.empty[ab], (unsigned)(c / kTcABufs) + 1u);
        tc::fence_after();
        float v[kTcRhs];
        tc::ld_32x32b_x16(qaddr, v);
        tc::ld_32x32b_x16(qaddr + 16u, v + 16);
        tc::wait_ld();
        tc::fence_before();
        __syncwarp();
        if (rep2) {   // warps 2, 3 hand their half of D to warps 0, 1
            ++xcount;
            if (w >= 2) {
#pragma unroll
                for (int r = 0; r < kTcRhs; ++r) S.xch[32 * (w - 2) + lane][r] = v[r];
                __syncwarp();
                if (lane == 0) mbar_arrive_one(&S.xbar);
            } else {
                ok &= tc_wait(&S.xbar, xcount);
#pragma unroll
                for (int r = 0; r < kTcRhs; ++r) v[r] += S.xch[32 * w + lane][r];
            }
        }
        if (lane == 0) mbar_arrive_one(&S.dfree);   // D may be overwritten by the next item
        const int kk = lane >> 3, t = 8 * tq + (lane & 7);
        if ((!rep2 || w < 2) && t < tcnt) {
            const int64_t dst = perm[tb + t];
            if (kk == 0) {
                if (phi) {
#pragma unroll
                    for (int r = 0; r < kTcRhs; ++r)
                        if (r < nrhs) phi[(int64_t)r * n + dst] = v[r] * phi_scale;
                }
            } else if (grad) {
#pragma unroll
                for (int r = 0; r < kTcRhs; ++r)
                    if (r < nrhs) grad[((int64_t)r * n + dst) * 3 + kk - 1] = v[r] * grad_scale;
            }
        }
    }
    return ok;
}

template <int P>
__global__ void __launch_bounds__(kTcThreads, kTcCtasPerSM)
    k_p2p_tc(int nitems, const int4 *items, unsigned *next_item, const unsigned *roff, const float4 *run,
             const int *run_end, const float4 *pos, const __nv_bfloat16 *qh, const __nv_bfloat16 *ql,
             const __nv_bfloat16 *lh, const __nv_bfloat16 *ll, const int *pbeg, const int *pcnt, const int *level,
             const int *parent, const float4 *geom, const int *perm, int64_t n, int nrhs, float phi_scale,
             float grad_scale, float *phi, float *grad, unsigned *err)
{
    extern __shared__ __align__(16) unsigned char tc_smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(tc_smem_raw);
    const int w = (int)(threadIdx.x >> 5);
    if (w == 0) {
        tc::alloc(&S.tmem_base, kTcCols);
        tc::relinquish();
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < kTcStages; ++b) mbar_init(&S.staged[b], 1);
        for (int b = 0; b < kTcABufs; ++b) {
            mbar_init(&S.full[b], kTcGenWarps);
            mbar_init(&S.empty[b], 1);
        }
        mbar_init(&S.dfree, 4);
        mbar_init(&S.xbar, 2);
        mbar_init(&S.fin, 1);
        fence_mbar_init();
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const unsigned tbase = S.tmem_base;
    bool ok;
    if (w == kTcGenWarps)
        ok = tc_producer<P>(S, tbase, nitems, items, next_item, roff, run, run_end, pos, qh, ql, lh, ll, pbeg, pcnt);
    else
        ok = tc_consumer<P>(S, tbase, items, pos, level, parent, geom, perm, n, nrhs, phi_scale, grad_scale, phi,
                            grad);
    if (!ok && lane_id() == 0) atomicOr(err, 4u);
    tc::fence_before();
    __syncthreads();
    if (w == 0) {
        tc::fence_after();
        tc::dealloc(tbase, kTcCols);
    }
}

// The local expansions of the leaves, BF16 high and low parts, in leaf-list
// order: lh[li][n][r] = bf16(Lb[leaf li][n][r]), ll = bf16(remainder), n < T.
template <int P>
__global__ void k_split_leaf_locals(int nleaves, const int *leaf_list, const float *Lb, __nv_bfloat16 *lh,
                                    __nv_bfloat16 *ll)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nleaves * T * kTcRhs) return;
    const int r = (int)(i % kTcRhs);
    const int64_t rest = i / kTcRhs;
    const int nn = (int)(rest % T);
    const int li = (int)(rest / T);
    const float v = Lb[((int64_t)leaf_list[li] * TP + nn) * kTcRhs + r];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    lh[i] = h;
    ll[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}

template <int P> static int p2p_batch_tc_impl(Handle &h, int nrhs, float *phi, float *grad)
{
    constexpr int T = MI<P>::T;
    const int nl = (int)h.nleaves;
    FMM_TRY(ensure_full_runs(h));
    if (!h.tc_items_ready) {
        FMM_TRY(build_work_items(h, kTcTargets, h.tc_items, h.n_tc_items));
        h.tc_items_ready = true;
    }
    FMM_TRY(h.lbh.reserve((size_t)nl * T * kTcRhs * sizeof(__nv_bfloat16)));
    FMM_TRY(h.lbl.reserve((size_t)nl * T * kTcRhs * sizeof(__nv_bfloat16)));
    FMM_TRY(h.tc_next.reserve(sizeof(unsigned)));
    FMM_TRY(h.err_flag.reserve(sizeof(unsigned)));
    ++h.launches;
    k_split_leaf_locals<P><<<ceil_div((int64_t)nl * T * kTcRhs, 256), 256, 0, h.stream>>>(
        nl, h.leaf_list.as<int>(), h.Lb.as<float>(), h.lbh.as<__nv_bfloat16>(), h.lbl.as<__nv_bfloat16>());
    FMM_CUDA(cudaMemsetAsync(h.tc_next.p, 0, sizeof(unsigned), h.stream));
    static bool configured[64][9] = {};
    if (h.device >= 0 && h.device < 64 && !configured[h.device][P]) {
        FMM_CUDA(cudaFuncSetAttribute(k_p2p_tc<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes));
        configured[h.device][P] = true;
    }
    const int grid = (int)std::min<int64_t>(h.n_tc_items, (int64_t)h.num_sms * kTcCtasPerSM);
    const double ih = 1.0 / h.norm_host[3];
    ++h.launches;
    k_p2p_tc<P><<<std::max(grid, 1), kTcThreads, kTcSmemBytes, h.stream>>>(
        (int)h.n_tc_items, h.tc_items.as<int4>(), h.tc_next.as<unsigned>(), h.p2p_poff.as<unsigned>(),
        h.p2p_ent.as<float4>(), h.p2p_cnt.as<int>(), h.pos.as<float4>(), h.qbh.as<__nv_bfloat16>(),
        h.qbl.as<__nv_bfloat16>(), h.lbh.as<__nv_bfloat16>(), h.lbl.as<__nv_bfloat16>(), h.c_pbeg.as<int>(),
        h.c_pcnt.as<int>(), h.c_level.as<int>(), h.c_parent.as<int>(), h.c_geom.as<float4>(), h.perm.as<int>(), h.N,
        nrhs, (float)ih, (float)(ih * ih), phi, grad, h.err_flag.as<unsigned>());
    FMM_CHECK_LAUNCH("batched p2p (tensor cores)");
    return FMM_OK;
}

// P2P + L2P of the batched evaluation on the tensor cores (after the far field
// has filled Lb and the charges have been gathered into qbh / qbl).
int p2p_batch_tc(Handle &h, int nrhs, float *phi, float *grad)
{
    switch (h.P) {
    case 3: return p2p_batch_tc_impl<3>(h, nrhs, phi, grad);
    case 4: return p2p_batch_tc_impl<4>(h, nrhs, phi, grad);
    case 5: return p2p_batch_tc_impl<5>(h, nrhs, phi, grad);
    case 6: return p2p_batch_tc_impl<6>(h, nrhs, phi, grad);
    case 8: return p2p_batch_tc_impl<8>(h, nrhs, phi, grad);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

}  // namespace fmm
