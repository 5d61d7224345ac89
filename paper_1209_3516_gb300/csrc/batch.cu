// batch.cu -- many charge vectors on one geometry (fmm_evaluate_batch).
//
// With nrhs <= 32 charge vectors on a fixed tree, every operator of the
// evaluation becomes a contraction over the right-hand sides:
//   P2M, M2M, M2L, L2L  one warp per cell, lane r = right-hand side r: the
//        geometric factors (monomials, kernel derivatives D) are computed once
//        and applied to 32 expansion vectors; expansions are stored
//        Mb[cell][TP][32] so that lanes read consecutive words;
//   P2P  a dense product on the tensor cores: for a target leaf slice of 8
//        targets and 16 staged sources, Phi[4 x 8 targets, 32 rhs] +=
//        G[4 x 8, 16] Q[16, 32] with the four kernel matrices (1/r and the three
//        components of e/r^3, e = u_s - u_t) generated in FP32 on the CUDA
//        cores.  G and Q are each split into BF16 high and low parts
//        (v = hi + lo to ~2^-16) and three MMAs (hi*hi + hi*lo + lo*hi,
//        mma.sync m16n8k16, FP32 accumulate) give the product to ~2^-16
//        relative per term.  The target's L2P of all 32 local expansions and the
//        scatter to caller order follow in the same kernel.
// The tree, lists and P2P source runs are those of the last build.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "fmm_internal.cuh"
#include "mi.cuh"
#include "p2p_common.cuh"

namespace fmm {

constexpr int kB = 32;              // right-hand sides per batch (lanes)
constexpr int kBT = 8;              // targets per tensor-core work item (one warp)
constexpr int kBThreads = 128;
constexpr int kBChunk = 32;         // staged sources per buffer
constexpr int kQStride = 40;        // bf16 per staged charge row (32 + 8 padding: conflict-free ldmatrix)
// per warp and buffer: positions, shifts (float4 each) and the hi / lo charge rows
constexpr int kBBufBytes = kBChunk * 16 * 2 + kBChunk * kQStride * 2 * 2;
constexpr int kBSmem = (kBThreads / 32) * 2 * kBBufBytes;

// ---------------------------------------------------------------------------
// gather: qb[s][r] = q[r][perm[s]] (FP32) and its BF16 split (hi, lo)
// ---------------------------------------------------------------------------
__global__ void k_gather_qbatch(int64_t n, int nrhs, const int *perm, const float *q, float *qb,
                                __nv_bfloat16 *qh, __nv_bfloat16 *ql)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * kB) return;
    const int64_t s = i / kB;
    const int r = (int)(i % kB);
    const float v = r < nrhs ? q[(int64_t)r * n + perm[s]] : 0.0f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    qb[i] = v;
    qh[i] = hi;
    ql[i] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// ---------------------------------------------------------------------------
// far field, lanes over right-hand sides
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_p2m_batch(int nleaves, const int *leaf_list, const int *pbeg, const int *pcnt, const int *level,
                            const int *parent, const float4 *geom, const float4 *pos, const float *qb, float *Mb)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= nleaves) return;
    const int r = (int)lane_id();
    const int c = leaf_list[warp];
    const float inv_s = ldexpf(1.0f, level[c]);
    const int fr = parent[c] >= 0 ? parent[c] : c;
    const float4 Xc = geom[c], Xf = geom[fr];
    const float ox = (Xc.x - Xf.x) * inv_s, oy = (Xc.y - Xf.y) * inv_s, oz = (Xc.z - Xf.z) * inv_s;
    float acc[T];
#pragma unroll
    for (int i = 0; i < T; ++i) acc[i] = 0.0f;
    const int b = pbeg[c], e = b + pcnt[c];
    for (int j = b; j < e; ++j) {
        const float4 p = pos[j];
        float w[T];
        taylor_monomials<P>(fmaf(-p.x, inv_s, ox), fmaf(-p.y, inv_s, oy), fmaf(-p.z, inv_s, oz), w);
        const float q = qb[(size_t)j * kB + r];
#pragma unroll
        for (int i = 0; i < T; ++i) acc[i] = fmaf(q, w[i], acc[i]);
    }
    float *dst = Mb + (size_t)c * TP * kB + r;
#pragma unroll
    for (int i = 0; i < TP; ++i) dst[i * kB] = i < T ? acc[i] : 0.0f;
}

template <int P>
__global__ void k_m2m_batch(int lo, int n, const int *cbeg, const int *ccnt, const float4 *geom, float *Mb)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= n) return;
    const int r = (int)lane_id();
    const int c = lo + warp;
    const int nch = ccnt[c];
    if (nch == 0) return;   // leaf: its multipole comes from P2M
    const float4 Xp = geom[c];
    float acc[T];
#pragma unroll
    for (int t = 0; t < T; ++t) acc[t] = 0.0f;
    for (int k = 0; k < nch; ++k) {
        const int ch = cbeg[c] + k;
        const float4 Xc = geom[ch];
        // child multipole, scaled to the parent's cell size: 2^-|m| Mb_m(C)
        float mc[T];
        const float *src = Mb + (size_t)ch * TP * kB + r;
#pragma unroll
        for (int na = 0; na < P; ++na)
#pragma unroll
            for (int a = na; a >= 0; --a)
#pragma unroll
                for (int b = na - a; b >= 0; --b) {
                    const int i = MI<P>::idx(a, b, na - a - b);
                    mc[i] = src[i * kB] * (1.0f / (float)(1 << na));
                }
        // separable shift by (X_P - X_C) / s_P = -+1/2 per axis, one axis at a time:
        // m'_(a,b,c) = sum_{a' <= a} m_(a',b,c) dx^(a-a') / (a-a')!
        const float d[3] = {Xc.x > Xp.x ? -0.5f : 0.5f, Xc.y > Xp.y ? -0.5f : 0.5f, Xc.z > Xp.z ? -0.5f : 0.5f};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            float pw[P];   // d^j / j!
            pw[0] = 1.0f;
#pragma unroll
            for (int j = 1; j < P; ++j) pw[j] = pw[j - 1] * d[ax] * (1.0f / j);
            // in place, highest power first along the axis so sources are still unshifted
#pragma unroll
            for (int na = P - 1; na >= 0; --na)
#pragma unroll
                for (int a = na; a >= 0; --a)
#pragma unroll
                    for (int b = na - a; b >= 0; --b) {
                        const int cc = na - a - b;
                        const int e[3] = {a, b, cc};
                        const int i = MI<P>::idx(a, b, cc);
                        float s = mc[i];
#pragma unroll
                        for (int j = 1; j <= e[ax]; ++j) {
                            int f[3] = {a, b, cc};
                            f[ax] -= j;
                            s = fmaf(mc[MI<P>::idx(f[0], f[1], f[2])], pw[j], s);
                        }
                        mc[i] = s;
                    }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) acc[t] += mc[t];
    }
    float *dst = Mb + (size_t)c * TP * kB + r;
#pragma unroll
    for (int t = 0; t < TP; ++t) dst[t * kB] = t < T ? acc[t] : 0.0f;
}

// M2L: one warp per target cell; per chunk of 32 sources each lane computes the
// kernel derivatives of one pair into shared memory, then lane r contracts
// every pair of the chunk with its multipole vector r.
constexpr int kM2LBatchThreads = 64;   // two warps: 2 x 32 x (T + 1) floats of D fit static shared memory

// Outputs N0 <= idx(n) < N1 only (at P = 8 two launches split them, as for the
// single-vector M2L: half the accumulators, no spills; multipole coefficients
// that no output of the slice uses are not loaded).
template <int P, int N0, int N1>
__global__ void __launch_bounds__(kM2LBatchThreads) k_m2l_batch(int ncells, const int *off, const int *src,
                                                                const int *level, const float4 *geom, const float *Mb,
                                                                float *Lb)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP, NO = N1 - N0;
    constexpr int W = kM2LBatchThreads / 32;
    __shared__ float Ds[W][32][T + 1];
    __shared__ float Rho[W][32];
    __shared__ int Src[W][32];
    const int w = threadIdx.x >> 5;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= ncells) return;
    const int lane = (int)lane_id();
    const float4 Xt = geom[t];
    const int lt = level[t];
    const float inv_st = ldexpf(1.0f, lt);
    float acc[NO];
#pragma unroll
    for (int i = 0; i < NO; ++i) acc[i] = 0.0f;
    const int b = off[t], e = off[t + 1];
    for (int k0 = b; k0 < e; k0 += 32) {
        const int k = k0 + lane;
        if (k < e) {
            const int s = src[k];
            const float4 Xs = geom[s];
            float D[T];
            laplace_derivatives<P>((Xt.x - Xs.x) * inv_st, (Xt.y - Xs.y) * inv_st, (Xt.z - Xs.z) * inv_st, D);
#pragma unroll
            for (int i = 0; i < T; ++i) Ds[w][lane][i] = D[i];
            Rho[w][lane] = ldexpf(1.0f, lt - level[s]);
            Src[w][lane] = s;
        }
        __syncwarp();
        const int np = min(32, e - k0);
        for (int j = 0; j < np; ++j) {
            const float *Mj = Mb + (size_t)Src[w][j] * TP * kB + lane;
            const float *D = Ds[w][j];
            const float rho = Rho[w][j];
            float rp = 1.0f;
#pragma unroll
            for (int nk = 0; nk < P; ++nk) {
#pragma unroll
                for (int ka = nk; ka >= 0; --ka)
#pragma unroll
                    for (int kb = nk - ka; kb >= 0; --kb) {
                        const int kc = nk - ka - kb;
                        // the outputs of this slice that k reaches: degrees 0 .. P-1-nk
                        if (N0 >= MI<P>::idx(P - nk, 0, 0)) continue;
                        const float m = Mj[MI<P>::idx(ka, kb, kc) * kB] * rp;
#pragma unroll
                        for (int nn = 0; nn + nk < P; ++nn)
#pragma unroll
                            for (int na = nn; na >= 0; --na)
#pragma unroll
                                for (int nb = nn - na; nb >= 0; --nb) {
                                    const int nc = nn - na - nb;
                                    const int in = MI<P>::idx(na, nb, nc);
                                    if (in >= N0 && in < N1)
                                        acc[in - N0] = fmaf(m, D[MI<P>::idx(na + ka, nb + kb, nc + kc)], acc[in - N0]);
                                }
                    }
                rp *= rho;
            }
        }
        __syncwarp();
    }
    float *dst = Lb + (size_t)t * TP * kB + lane;
#pragma unroll
    for (int i = 0; i < NO; ++i) dst[(N0 + i) * kB] = acc[i] * inv_st;
    if (N1 == T)
#pragma unroll
        for (int i = T; i < TP; ++i) dst[i * kB] = 0.0f;
}

template <int P>
__global__ void k_l2l_batch(int lo, int n, const int *parent, const float4 *geom, float *Lb)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= n) return;
    const int r = (int)lane_id();
    const int c = lo + warp;
    const int p = parent[c];
    const float4 Xc = geom[c], Xp = geom[p];
    float w[T];
    taylor_monomials<P>(Xc.x > Xp.x ? 0.5f : -0.5f, Xc.y > Xp.y ? 0.5f : -0.5f, Xc.z > Xp.z ? 0.5f : -0.5f, w);
    float lp[T];
    const float *sp = Lb + (size_t)p * TP * kB + r;
#pragma unroll
    for (int t = 0; t < T; ++t) lp[t] = sp[t * kB];
    float *dst = Lb + (size_t)c * TP * kB + r;
#pragma unroll
    for (int nk = 0; nk < P; ++nk)
#pragma unroll
        for (int ka = nk; ka >= 0; --ka)
#pragma unroll
            for (int kb = nk - ka; kb >= 0; --kb) {
                const int kc = nk - ka - kb;
                float s = 0.0f;
#pragma unroll
                for (int nm = 0; nm + nk < P; ++nm)
#pragma unroll
                    for (int ma = nm; ma >= 0; --ma)
#pragma unroll
                        for (int mb = nm - ma; mb >= 0; --mb) {
                            const int mc = nm - ma - mb;
                            s = fmaf(lp[MI<P>::idx(ka + ma, kb + mb, kc + mc)], w[MI<P>::idx(ma, mb, mc)], s);
                        }
                const int id = MI<P>::idx(ka, kb, kc);
                dst[id * kB] += s * (1.0f / (float)(1 << nk));
            }
}

// ---------------------------------------------------------------------------
// P2P on the tensor cores
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned pack_bf16(float lo_col, float hi_col)
{
    // lower 16 bits: the element of the lower column index
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_col, hi_col);
    return *reinterpret_cast<const unsigned *>(&v);
}

// v = hi + lo: hi = bf16(v), lo = bf16(v - hi), two values per register
__device__ __forceinline__ void split_bf16(float v0, float v1, unsigned &hi, unsigned &lo)
{
    hi = pack_bf16(v0, v1);
    const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&hi);
    const float2 hf = __bfloat1622float2(h);
    lo = pack_bf16(v0 - hf.x, v1 - hf.y);
}

// (not volatile: a pure function of its operands, so the compiler may interleave
// independent accumulators)
__device__ __forceinline__ void mma_bf16(float *c, const unsigned *a, unsigned b0, unsigned b1)
{
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4_trans(unsigned *r, const void *smem_row)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s)
                 : "memory");
}

struct BatchBuf {   // one staging buffer of a warp
    float4 *pos, *shift;
    __nv_bfloat16 *qh, *ql;   // [kBChunk][kQStride]
};

__device__ __forceinline__ BatchBuf batch_buf(unsigned char *base)
{
    BatchBuf b;
    b.pos = reinterpret_cast<float4 *>(base);
    b.shift = b.pos + kBChunk;
    b.qh = reinterpret_cast<__nv_bfloat16 *>(b.shift + kBChunk);
    b.ql = b.qh + kBChunk * kQStride;
    return b;
}

// Stage up to kBChunk sources of the item's runs: positions and charge rows by
// cp.async, shifts by plain stores; rows past the count are zero charges at a
// far position (every product term an exact 0).
__device__ __forceinline__ int batch_stage(RunCursor &cur, const float4 *run, const int *run_end, const float4 *pos,
                                           const __nv_bfloat16 *qh, const __nv_bfloat16 *ql, const BatchBuf &b,
                                           int tb0, int tb1, bool *self)
{
    const int lane = (int)lane_id();
    int slots = 0;
    bool sf = false;
    while (slots < kBChunk && cur.e < cur.e1) {
        const int m = min(cur.cnt - cur.o, kBChunk - slots);
        const int begin = cur.pb + cur.o;
        sf |= begin < tb1 && begin + m > tb0;
        const float4 sh = make_float4(cur.shx, cur.shy, cur.shz, 0.0f);
        for (int i = lane; i < m; i += 32) {
            cp_async16(b.pos + slots + i, pos + begin + i);
            b.shift[slots + i] = sh;
        }
        // charge rows: 4 x 16 bytes of hi and of lo per source
        for (int i = lane; i < m * 8; i += 32) {
            const int row = i >> 3, part = i & 7;
            const __nv_bfloat16 *g = (part < 4 ? qh : ql) + (size_t)(begin + row) * kB + (part & 3) * 8;
            __nv_bfloat16 *d = (part < 4 ? b.qh : b.ql) + (slots + row) * kQStride + (part & 3) * 8;
            cp_async16(d, g);
        }
        slots += m;
        cur.o += m;
        if (cur.o == cur.cnt) {
            ++cur.e;
            cur.o = 0;
            cur.load(run, run_end);
        }
    }
    // pad to a multiple of 16 sources
    const int padded = (slots + 15) & ~15;
    for (int i = slots + lane; i < padded; i += 32) {
        b.pos[i] = make_float4(1e20f, 1e20f, 1e20f, 0.0f);
        b.shift[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int i = lane; i < (padded - slots) * 8; i += 32) {
        const int row = slots + (i >> 3), part = i & 7;
        __nv_bfloat16 *d = (part < 4 ? b.qh : b.ql) + row * kQStride + (part & 3) * 8;
        *reinterpret_cast<uint4 *>(d) = make_uint4(0u, 0u, 0u, 0u);
    }
    *self = sf;
    return padded;
}

// Kernel values of one target (ntx, nty, ntz: negated) with the two staged
// sources j and j + 1 (positions already moved into the target frame), packed
// FP32 (two pairs per instruction): 1/r and e/r^3, e = u_s - u_t, each as
// (source j, source j + 1).
template <bool kExact>
__device__ __forceinline__ void kernel_values2(const BatchBuf &b, int j, float2 ntx, float2 nty, float2 ntz,
                                               float2 &k1, float2 &kx, float2 &ky, float2 &kz)
{
    constexpr float kEps = 1.17549435e-38f;
    const float4 s0 = b.pos[j], s1 = b.pos[j + 1];
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
    k1 = rinv;
    kx = __fmul2_rn(ex, rinv3);
    ky = __fmul2_rn(ey, rinv3);
    kz = __fmul2_rn(ez, rinv3);
}

// v = hi + lo for a pair of values: hi = bf16(v), lo = bf16(v - hi), packed
// two per register (lower half: the first value)
__device__ __forceinline__ void split_bf16x2(float2 v, unsigned &hi, unsigned &lo)
{
    hi = pack_bf16(v.x, v.y);
    const float2 hf = make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
    const float2 r = __fadd2_rn(v, make_float2(-hf.x, -hf.y));
    lo = pack_bf16(r.x, r.y);
}

// One k16 step: 16 staged sources from k0.  Thread (g = lane / 4, t = lane % 4)
// computes target g with sources k0 + {2t, 2t+1, 2t+8, 2t+9}: the A fragments
// of two m16 tiles (rows g / g+8: phi / gx in tile 0, gy / gz in tile 1).
template <bool kExact>
__device__ __forceinline__ void batch_kstep(const BatchBuf &b, int k0, float2 ntx, float2 nty, float2 ntz,
                                            float (*acc)[4][4])
{
    const int lane = (int)lane_id();
    const int t = lane & 3;
    float2 p01, x01, y01, z01, p89, x89, y89, z89;
    kernel_values2<kExact>(b, k0 + 2 * t, ntx, nty, ntz, p01, x01, y01, z01);
    kernel_values2<kExact>(b, k0 + 2 * t + 8, ntx, nty, ntz, p89, x89, y89, z89);
    unsigned ah[2][4], al[2][4];
    split_bf16x2(p01, ah[0][0], al[0][0]);   // tile 0 row g: phi, cols 2t, 2t+1
    split_bf16x2(x01, ah[0][1], al[0][1]);   // tile 0 row g+8: gx
    split_bf16x2(p89, ah[0][2], al[0][2]);   // cols 2t+8, 2t+9
    split_bf16x2(x89, ah[0][3], al[0][3]);
    split_bf16x2(y01, ah[1][0], al[1][0]);   // tile 1 row g: gy
    split_bf16x2(z01, ah[1][1], al[1][1]);   // tile 1 row g+8: gz
    split_bf16x2(y89, ah[1][2], al[1][2]);
    split_bf16x2(z89, ah[1][3], al[1][3]);
    // B fragments (charges) of the 4 n8 tiles, by transposing loads: lanes 0-7 give
    // rows k0..k0+7 (n 0-7), 8-15 rows k0+8.. (n 0-7), 16-23 / 24-31 the same rows at n + 8
    const int row = k0 + (lane & 7) + ((lane >> 3) & 1) * 8;
    const int coff = (lane >> 4) * 8;
    // bh[n], bl[n]: the two B registers of n tile n (hi and lo parts)
    unsigned bh[4][2], bl[4][2];
#pragma unroll
    for (int half = 0; half < 2; ++half) {   // n tiles {0,1} then {2,3}
        unsigned rh[4], rl[4];
        ldmatrix_x4_trans(rh, b.qh + row * kQStride + half * 16 + coff);
        ldmatrix_x4_trans(rl, b.ql + row * kQStride + half * 16 + coff);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            bh[2 * half + nt][0] = rh[2 * nt];
            bh[2 * half + nt][1] = rh[2 * nt + 1];
            bl[2 * half + nt][0] = rl[2 * nt];
            bl[2 * half + nt][1] = rl[2 * nt + 1];
        }
    }
    // three passes over the 8 accumulators (hi*hi, hi*lo, lo*hi), so that
    // consecutive MMAs are independent
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 4; ++n) mma_bf16(acc[m][n], ah[m], bh[n][0], bh[n][1]);
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 4; ++n) mma_bf16(acc[m][n], ah[m], bl[n][0], bl[n][1]);
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 4; ++n) mma_bf16(acc[m][n], al[m], bh[n][0], bh[n][1]);
}

#ifndef FMM_BATCH_MIN_BLOCKS
#define FMM_BATCH_MIN_BLOCKS 4
#endif

template <int P>
__global__ void __launch_bounds__(kBThreads, FMM_BATCH_MIN_BLOCKS) k_p2p_batch(int nitems, const int4 *items, const unsigned *roff,
                                                         const float4 *run, const int *run_end, const float4 *pos,
                                                         const __nv_bfloat16 *qh, const __nv_bfloat16 *ql,
                                                         const int *pbeg, const int *pcnt, const int *level,
                                                         const int *parent, const float4 *geom, const float *Lb,
                                                         const int *perm, int64_t n, int nrhs, float phi_scale,
                                                         float grad_scale, float *phi, float *grad)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    extern __shared__ __align__(16) unsigned char batch_smem[];
    const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= nitems) return;
    const int lane = (int)lane_id();
    unsigned char *wbase = batch_smem + (threadIdx.x >> 5) * 2 * kBBufBytes;
    const int4 it = items[item];
    const int leaf = it.x, tb = it.y, tc = it.z;
    const int lb0 = pbeg[leaf], lb1 = lb0 + pcnt[leaf];
    const int g = lane >> 2, t = lane & 3;
    const float4 tp = pos[tb + min(g, tc - 1)];   // extra rows repeat the last target
    const float2 ntx = make_float2(-tp.x, -tp.x), nty = make_float2(-tp.y, -tp.y), ntz = make_float2(-tp.z, -tp.z);

    float acc[2][4][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int nn = 0; nn < 4; ++nn)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[m][nn][k] = 0.0f;

    RunCursor cur;
    cur.init(roff, it.w, run, run_end);
    bool self_cur = false, self_next = false;
    int n_cur = batch_stage(cur, run, run_end, pos, qh, ql, batch_buf(wbase), lb0, lb1, &self_cur);
    cp_async_commit();
    for (int c = 0; n_cur > 0; ++c) {
        const BatchBuf bc = batch_buf(wbase + (c & 1) * kBBufBytes);
        const int n_next =
            batch_stage(cur, run, run_end, pos, qh, ql, batch_buf(wbase + ((c + 1) & 1) * kBBufBytes), lb0, lb1,
                        &self_next);
        cp_async_commit();
        cp_async_wait_1();
        __syncwarp();
        {   // move this chunk's sources into the target frame once (one source per lane)
            float4 sp = bc.pos[lane];
            const float4 d = bc.shift[lane];
            sp.x += d.x;
            sp.y += d.y;
            sp.z += d.z;
            bc.pos[lane] = sp;
        }
        __syncwarp();
        for (int k0 = 0; k0 < n_cur; k0 += 16) {
            if (self_cur) batch_kstep<true>(bc, k0, ntx, nty, ntz, acc);
            else batch_kstep<false>(bc, k0, ntx, nty, ntz, acc);
        }
        __syncwarp();
        n_cur = n_next;
        self_cur = self_next;
    }

    // epilogue, through the warp's (now idle) staging memory so that few values
    // stay live: (1) thread (g, t) holds target g, right-hand sides
    // 8 nt + 2t + {0, 1}: acc[0][nt] = (phi, phi, gx, gx), acc[1][nt] = (gy, gy, gz, gz);
    // they go to Acc[g][r][4]; (2) lanes g < tc write the Taylor monomials of
    // their target to W[g][T]; (3) lane r adds the L2P of local expansion r to
    // each target and writes the results.
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();
    float *Acc = reinterpret_cast<float *>(wbase);   // [kBT][kB][4]
    float *W = Acc + kBT * kB * 4;                    // [kBT][T]
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = 8 * nt + 2 * t + h;
            *reinterpret_cast<float4 *>(Acc + (g * kB + r) * 4) =
                make_float4(acc[0][nt][h], acc[0][nt][2 + h], acc[1][nt][h], acc[1][nt][2 + h]);
        }
    const float inv_s = ldexpf(1.0f, level[leaf]);
    const float4 Xc = geom[leaf], Xf = geom[frame_of(parent, leaf)];
    if (lane < tc) {
        const float4 p = pos[tb + lane];
        const float vx = fmaf(p.x, inv_s, -(Xc.x - Xf.x) * inv_s), vy = fmaf(p.y, inv_s, -(Xc.y - Xf.y) * inv_s),
                    vz = fmaf(p.z, inv_s, -(Xc.z - Xf.z) * inv_s);
        float *Wg = W + lane * T;
        Wg[0] = 1.0f;
#pragma unroll
        for (int nm = 1; nm < P; ++nm)
#pragma unroll
            for (int a = nm; a >= 0; --a)
#pragma unroll
                for (int bb = nm - a; bb >= 0; --bb) {
                    const int cc = nm - a - bb;
                    const int i = MI<P>::idx(a, bb, cc);
                    if (a > 0) Wg[i] = Wg[MI<P>::idx(a - 1, bb, cc)] * (vx * (1.0f / a));
                    else if (bb > 0) Wg[i] = Wg[MI<P>::idx(a, bb - 1, cc)] * (vy * (1.0f / bb));
                    else Wg[i] = Wg[MI<P>::idx(a, bb, cc - 1)] * (vz * (1.0f / cc));
                }
    }
    __syncwarp();
    const int r = lane;
    if (r >= nrhs) return;
    const float *Lc = Lb + (size_t)leaf * TP * kB + r;
    for (int gg = 0; gg < tc; ++gg) {
        const float *Wg = W + gg * T;
        const float4 pa = *reinterpret_cast<const float4 *>(Acc + (gg * kB + r) * 4);
        float lp = 0.0f, lx = 0.0f, ly = 0.0f, lz = 0.0f;
#pragma unroll
        for (int nm = 0; nm < P; ++nm)
#pragma unroll
            for (int a = nm; a >= 0; --a)
#pragma unroll
                for (int bb = nm - a; bb >= 0; --bb) {
                    const int cc = nm - a - bb;
                    const float wm = Wg[MI<P>::idx(a, bb, cc)];
                    lp = fmaf(Lc[MI<P>::idx(a, bb, cc) * kB], wm, lp);
                    if (nm + 1 < P) {
                        lx = fmaf(Lc[MI<P>::idx(a + 1, bb, cc) * kB], wm, lx);
                        ly = fmaf(Lc[MI<P>::idx(a, bb + 1, cc) * kB], wm, ly);
                        lz = fmaf(Lc[MI<P>::idx(a, bb, cc + 1) * kB], wm, lz);
                    }
                }
        const int dst = perm[tb + gg];
        if (phi) phi[(int64_t)r * n + dst] = (pa.x + lp) * phi_scale;
        if (grad) {
            float *gp = grad + ((int64_t)r * n + dst) * 3;
            gp[0] = fmaf(lx, inv_s, pa.y) * grad_scale;
            gp[1] = fmaf(ly, inv_s, pa.z) * grad_scale;
            gp[2] = fmaf(lz, inv_s, pa.w) * grad_scale;
        }
    }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
template <int P> static int batch_impl(Handle &h, const float *q, int nrhs, float *phi, float *grad)
{
    const int64_t N = h.N;
    const int nl = (int)h.nleaves, nc = (int)h.ncells;
    constexpr int TP = MI<P>::TP;
    FMM_TRY(h.qb.reserve((size_t)N * kB * sizeof(float)));
    FMM_TRY(h.qbh.reserve((size_t)N * kB * sizeof(__nv_bfloat16)));
    FMM_TRY(h.qbl.reserve((size_t)N * kB * sizeof(__nv_bfloat16)));
    FMM_TRY(h.Mb.reserve((size_t)nc * TP * kB * sizeof(float)));
    FMM_TRY(h.Lb.reserve((size_t)nc * TP * kB * sizeof(float)));
    if (!h.batch_items_ready) {
        FMM_TRY(build_work_items(h, kBT, h.batch_items, h.n_batch_items));
        h.batch_items_ready = true;
    }
    float *Mb = h.Mb.as<float>(), *Lb = h.Lb.as<float>();
    phase_begin(h, FMM_PHASE_UPWARD);
    ++h.launches;
    k_gather_qbatch<<<ceil_div(N * kB, 256), 256, 0, h.stream>>>(N, nrhs, h.perm.as<int>(), q, h.qb.as<float>(),
                                                                h.qbh.as<__nv_bfloat16>(), h.qbl.as<__nv_bfloat16>());
    ++h.launches;
    k_p2m_batch<P><<<ceil_div((int64_t)nl * 32, 128), 128, 0, h.stream>>>(
        nl, h.leaf_list.as<int>(), h.c_pbeg.as<int>(), h.c_pcnt.as<int>(), h.c_level.as<int>(), h.c_parent.as<int>(),
        h.c_geom.as<float4>(), h.pos.as<float4>(), h.qb.as<float>(), Mb);
    for (int l = h.nlevels - 2; l >= 0; --l) {
        const int lo = (int)h.level_off[l], n = (int)(h.level_off[l + 1] - h.level_off[l]);
        ++h.launches;
        k_m2m_batch<P><<<ceil_div((int64_t)n * 32, 128), 128, 0, h.stream>>>(lo, n, h.c_cbeg.as<int>(),
                                                                             h.c_ccnt.as<int>(), h.c_geom.as<float4>(), Mb);
    }
    phase_end(h, FMM_PHASE_UPWARD);
    phase_begin(h, FMM_PHASE_M2L);
    ++h.launches;
    {
        constexpr int T = MI<P>::T;
        constexpr int H = P >= 8 ? ((T / 2 + 3) & ~3) : T;   // two launches at P = 8
        const int mb = ceil_div((int64_t)nc * 32, kM2LBatchThreads);
        k_m2l_batch<P, 0, H><<<mb, kM2LBatchThreads, 0, h.stream>>>(
            nc, h.m2l_off.as<int>(), h.m2l_src.as<int>(), h.c_level.as<int>(), h.c_geom.as<float4>(), Mb, Lb);
        if constexpr (H < T) {
            ++h.launches;
            k_m2l_batch<P, H, T><<<mb, kM2LBatchThreads, 0, h.stream>>>(
                nc, h.m2l_off.as<int>(), h.m2l_src.as<int>(), h.c_level.as<int>(), h.c_geom.as<float4>(), Mb, Lb);
        }
    }
    phase_end(h, FMM_PHASE_M2L);
    phase_begin(h, FMM_PHASE_DOWNWARD);
    for (int l = 1; l < h.nlevels; ++l) {
        const int lo = (int)h.level_off[l], n = (int)(h.level_off[l + 1] - h.level_off[l]);
        ++h.launches;
        k_l2l_batch<P><<<ceil_div((int64_t)n * 32, 128), 128, 0, h.stream>>>(lo, n, h.c_parent.as<int>(),
                                                                             h.c_geom.as<float4>(), Lb);
    }
    phase_end(h, FMM_PHASE_DOWNWARD);
    FMM_CHECK_LAUNCH("batched far field");
    phase_begin(h, FMM_PHASE_P2P);
    FMM_TRY(p2p_batch_tc(h, nrhs, phi, grad));
    phase_end(h, FMM_PHASE_P2P);
    FMM_CHECK_LAUNCH("batched p2p");
    return FMM_OK;
}

int evaluate_batch(Handle &h, const float *q, int nrhs, float *phi, float *grad)
{
    switch (h.P) {
    case 3: return batch_impl<3>(h, q, nrhs, phi, grad);
    case 4: return batch_impl<4>(h, q, nrhs, phi, grad);
    case 5: return batch_impl<5>(h, q, nrhs, phi, grad);
    case 6: return batch_impl<6>(h, q, nrhs, phi, grad);
    case 8: return batch_impl<8>(h, q, nrhs, phi, grad);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

}  // namespace fmm
