// p2p.cu -- near field: P2P over the P2P list, fused with L2P and the output scatter.
//
// P2P (Sec. 3.3, Table 4): phi_i += sum_j q_j / r_ij, grad_i += sum_j q_j (x_j - x_i) / r_ij^3
// over the particles j of every source leaf listed for the target leaf of i
// (pairs at distance 0 contribute nothing).  The paper's kernel is AVX with
// rsqrt_ps (Sec. 3.3); here:
//   - work item = (target leaf, slice of <= 16 of its targets); one warp per item;
//   - the 16 target positions sit in registers (warp-uniform), the warp's 32
//     lanes stream the source particles of all listed leaves as one
//     concatenated sequence (float4 (x, y, z, q) loads, coalesced inside each
//     leaf), each lane computing 16 pair interactions per source with one SFU
//     rsqrt each;
//   - positions are FP32 offsets from the leaf centre; a source is moved into
//     the target leaf's frame by the exact (dyadic) shift X_S - X_T, so close
//     pairs keep ~2^-24 of the leaf size in absolute precision;
//   - the 4 x 16 accumulators are reduce-scattered across the warp (62
//     shuffles), then lanes 2g / 2g+1 own target g: L2P of the leaf's local
//     expansion is added, units restored (phi / h, grad / h^2) and the result
//     written at the caller's index.
// With FMM_FLAG_KAHAN each lane keeps its per-target sums as (sum, compensation)
// pairs updated once per 8 sources (plain FP32 inside the block of 8).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "fmm_internal.cuh"
#include "mi.cuh"

namespace fmm {

constexpr int kP2PG = 16;          // targets per work item
constexpr int kP2PThreads = 128;

// Work items: one per slice of <= 16 targets of a leaf, slices balanced in size.
__global__ void k_p2p_item_count(int nleaves, const int *leaf_list, const int *pcnt, unsigned *cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaves) return;
    const int nt = pcnt[leaf_list[i]];
    cnt[i] = (unsigned)((nt + kP2PG - 1) / kP2PG);
}

__global__ void k_p2p_item_write(int nleaves, const int *leaf_list, const int *pbeg, const int *pcnt,
                                 const unsigned *off, int4 *items)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaves) return;
    const int c = leaf_list[i];
    const int nt = pcnt[c], b = pbeg[c];
    const int ns = (nt + kP2PG - 1) / kP2PG;
    for (int k = 0; k < ns; ++k) {
        const int t0 = (int)((int64_t)nt * k / ns), t1 = (int)((int64_t)nt * (k + 1) / ns);
        items[off[i] + k] = make_int4(c, b + t0, t1 - t0, 0);
    }
}

// Source ranges (first particle, count, source leaf) of every P2P list entry.
__global__ void k_p2p_ranges(int64_t n, const int *src, const int *pbeg, const int *pcnt, int4 *rng)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int s = src[e];
    rng[e] = make_int4(pbeg[s], pcnt[s], s, 0);
}

// Reduce-scatter 2 * NV values across the warp by recursive halving.
// On return lane l holds entries 2l and 2l+1 of the warp-wide sums (NV = 32).
__device__ __forceinline__ void warp_reduce_scatter64(float *v)
{
    const unsigned lane = lane_id();
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int half = 32 >> step;          // values kept after this step
        const unsigned mask = 16u >> step;
        const bool upper = (lane & mask) != 0u;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, mask);
        }
    }
}

template <int P, bool kKahan>
__global__ void __launch_bounds__(kP2PThreads) k_p2p(int nitems, const int4 *items, const int *off, const int4 *rng,
                                                     const float4 *pos, const float4 *geom, const int *level,
                                                     const float *L, const int *perm, float phi_scale,
                                                     float grad_scale, float *phi, float *grad, float *phi_sorted)
{
    constexpr int G = kP2PG;
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= nitems) return;
    const unsigned lane = lane_id();
    const int4 it = items[item];
    const int leaf = it.x, tb = it.y, tc = it.z;

    // targets and sources are offsets from their leaf centres; a source of leaf S
    // is moved into the target leaf's frame by the exact shift X_S - X_T
    const float4 Xt = geom[leaf];
    float tx[G], ty[G], tz[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const float4 p = pos[tb + min(g, tc - 1)];
        tx[g] = p.x;
        ty[g] = p.y;
        tz[g] = p.z;
    }
    // acc layout: v[4 g + 0] potential, v[4 g + 1..3] gradient
    float v[4 * G];
#pragma unroll
    for (int i = 0; i < 4 * G; ++i) v[i] = 0.0f;
    float comp[kKahan ? 4 * G : 1];
    float blk[kKahan ? 4 * G : 1];
    if (kKahan) {
#pragma unroll
        for (int i = 0; i < 4 * G; ++i) comp[i] = blk[i] = 0.0f;
    }

    // per-lane cursor over the concatenated source particles of the item's list:
    // entry e, offset o inside it, its range r and its frame shift
    const int e1 = off[leaf + 1];
    int e = off[leaf];
    int o = (int)lane;
    int4 r = make_int4(0, 0, 0, 0);
    float shx = 0.f, shy = 0.f, shz = 0.f;
    bool fresh = true;
    for (;;) {
        if (fresh) r = e < e1 ? rng[e] : make_int4(0, 0, 0, 0);
        if (e < e1 && o >= r.y) {
            o -= r.y;
            ++e;
            fresh = true;
            continue;
        }
        break;
    }
    if (e < e1) {
        const float4 Xs = geom[r.z];
        shx = Xs.x - Xt.x;
        shy = Xs.y - Xt.y;
        shz = Xs.z - Xt.z;
    }
    int nsub = 0;
    while (__any_sync(kFull, e < e1)) {
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < e1) {
            s = pos[r.x + o];
            s.x += shx;
            s.y += shy;
            s.z += shz;
        }
#pragma unroll
        for (int sb = 0; sb < G / 4; ++sb) {
            if (4 * sb < tc) {
#pragma unroll
                for (int gg = 0; gg < 4; ++gg) {
                    const int g = 4 * sb + gg;
                    const float dx = s.x - tx[g], dy = s.y - ty[g], dz = s.z - tz[g];
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    float rinv = rsqrtf(r2);
                    rinv = r2 > 0.0f ? rinv : 0.0f;
                    const float qr = s.w * rinv;
                    const float qr3 = qr * rinv * rinv;
                    float *acc = kKahan ? blk : v;
                    acc[4 * g + 0] += qr;
                    acc[4 * g + 1] = fmaf(qr3, dx, acc[4 * g + 1]);
                    acc[4 * g + 2] = fmaf(qr3, dy, acc[4 * g + 2]);
                    acc[4 * g + 3] = fmaf(qr3, dz, acc[4 * g + 3]);
                }
            }
        }
        if (kKahan && ++nsub == 8) {
            nsub = 0;
#pragma unroll
            for (int i = 0; i < 4 * G; ++i) {
                const float y = blk[i] - comp[i];
                const float t = v[i] + y;
                comp[i] = (t - v[i]) - y;
                v[i] = t;
                blk[i] = 0.0f;
            }
        }
        o += 32;
        if (e < e1 && o >= r.y) {
            do {
                o -= r.y;
                ++e;
                r = e < e1 ? rng[e] : make_int4(0, 0, 0, 0);
            } while (e < e1 && o >= r.y);
            if (e < e1) {
                const float4 Xs = geom[r.z];
                shx = Xs.x - Xt.x;
                shy = Xs.y - Xt.y;
                shz = Xs.z - Xt.z;
            }
        }
    }
    if (kKahan) {
#pragma unroll
        for (int i = 0; i < 4 * G; ++i) {
            const float y = blk[i] - comp[i];
            v[i] = v[i] + y;
        }
    }

    warp_reduce_scatter64(v);
    // lane 2g holds (phi, gx) of target g, lane 2g+1 holds (gy, gz)
    const float o0 = __shfl_down_sync(kFull, v[0], 1);
    const float o1 = __shfl_down_sync(kFull, v[1], 1);
    const int g = (int)(lane >> 1);
    if ((lane & 1u) || g >= tc) return;
    const int sidx = tb + g;
    const float4 p = pos[sidx];
    float pot = v[0], gx = v[1], gy = o0, gz = o1;

    // L2P: phi += sum_n Lb_n w_n(r / s), grad += (1/s) sum_m Lb_{m + e_d} w_m(r / s), r = p (leaf offset)
    {
        const float inv_s = ldexpf(1.0f, level[leaf]);
        float w[T];
        taylor_monomials<P>(p.x * inv_s, p.y * inv_s, p.z * inv_s, w);
        const float *Lc = L + (size_t)leaf * TP;
        float lp = 0.0f, lx = 0.0f, ly = 0.0f, lz = 0.0f;
#pragma unroll
        for (int nm = 0; nm < P; ++nm)
#pragma unroll
            for (int a = nm; a >= 0; --a)
#pragma unroll
                for (int b = nm - a; b >= 0; --b) {
                    const int c = nm - a - b;
                    const float wm = w[MI<P>::idx(a, b, c)];
                    lp = fmaf(Lc[MI<P>::idx(a, b, c)], wm, lp);
                    if (nm + 1 < P) {
                        lx = fmaf(Lc[MI<P>::idx(a + 1, b, c)], wm, lx);
                        ly = fmaf(Lc[MI<P>::idx(a, b + 1, c)], wm, ly);
                        lz = fmaf(Lc[MI<P>::idx(a, b, c + 1)], wm, lz);
                    }
                }
        pot += lp;
        gx = fmaf(lx, inv_s, gx);
        gy = fmaf(ly, inv_s, gy);
        gz = fmaf(lz, inv_s, gz);
    }
    const int dst = perm[sidx];
    const float ph = pot * phi_scale;
    if (phi) phi[dst] = ph;
    if (phi_sorted) phi_sorted[sidx] = ph;
    if (grad) {
        grad[3 * (int64_t)dst + 0] = gx * grad_scale;
        grad[3 * (int64_t)dst + 1] = gy * grad_scale;
        grad[3 * (int64_t)dst + 2] = gz * grad_scale;
    }
}

int build_p2p_items(Handle &h)
{
    const int nl = (int)h.nleaves;
    FMM_TRY(h.c_tmp.reserve((size_t)(2 * nl + 1) * sizeof(unsigned)));
    unsigned *cnt = h.c_tmp.as<unsigned>(), *off = cnt + nl, *tot = off + nl;
    ++h.launches;
    k_p2p_item_count<<<ceil_div(nl, 256), 256, 0, h.stream>>>(nl, h.leaf_list.as<int>(), h.c_pcnt.as<int>(), cnt);
    FMM_TRY(scan_exclusive_u32(h, cnt, off, nl, tot));
    FMM_CUDA(cudaMemcpyAsync(&h.pinned->level_total, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    h.n_items = h.pinned->level_total;
    FMM_TRY(h.p2p_items.reserve(std::max<int64_t>(h.n_items, 1) * sizeof(int4)));
    ++h.launches;
    k_p2p_item_write<<<ceil_div(nl, 256), 256, 0, h.stream>>>(nl, h.leaf_list.as<int>(), h.c_pbeg.as<int>(),
                                                              h.c_pcnt.as<int>(), off, h.p2p_items.as<int4>());
    FMM_TRY(h.p2p_rng.reserve(std::max<int64_t>(h.n_p2p, 1) * sizeof(int4)));
    if (h.n_p2p > 0) {
        ++h.launches;
        k_p2p_ranges<<<ceil_div(h.n_p2p, 256), 256, 0, h.stream>>>(h.n_p2p, h.p2p_src.as<int>(), h.c_pbeg.as<int>(),
                                                                 h.c_pcnt.as<int>(), h.p2p_rng.as<int4>());
    }
    FMM_CHECK_LAUNCH("p2p items");
    return FMM_OK;
}

template <int P> static int p2p_impl(Handle &h, float *phi, float *grad)
{
    const float phi_scale = (float)(1.0 / h.norm_host[3]);
    const float grad_scale = (float)(1.0 / (h.norm_host[3] * h.norm_host[3]));
    const int blocks = ceil_div((int64_t)h.n_items * 32, kP2PThreads);
    if (h.flags & FMM_FLAG_KAHAN) {
        ++h.launches;
        k_p2p<P, true><<<blocks, kP2PThreads, 0, h.stream>>>(
            (int)h.n_items, h.p2p_items.as<int4>(), h.p2p_off.as<int>(), h.p2p_rng.as<int4>(), h.pos.as<float4>(),
            h.c_geom.as<float4>(), h.c_level.as<int>(), h.L.as<float>(), h.perm.as<int>(), phi_scale, grad_scale, phi,
            grad, h.phi_sorted.as<float>());
    } else {
        ++h.launches;
        k_p2p<P, false><<<blocks, kP2PThreads, 0, h.stream>>>(
            (int)h.n_items, h.p2p_items.as<int4>(), h.p2p_off.as<int>(), h.p2p_rng.as<int4>(), h.pos.as<float4>(),
            h.c_geom.as<float4>(), h.c_level.as<int>(), h.L.as<float>(), h.perm.as<int>(), phi_scale, grad_scale, phi,
            grad, h.phi_sorted.as<float>());
    }
    FMM_CHECK_LAUNCH("p2p");
    return FMM_OK;
}

int evaluate_p2p(Handle &h, float *phi, float *grad)
{
    FMM_TRY(h.phi_sorted.reserve(h.N * sizeof(float)));
    switch (h.P) {
    case 3: return p2p_impl<3>(h, phi, grad);
    case 4: return p2p_impl<4>(h, phi, grad);
    case 5: return p2p_impl<5>(h, phi, grad);
    case 6: return p2p_impl<6>(h, phi, grad);
    case 8: return p2p_impl<8>(h, phi, grad);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

// ---------------------------------------------------------------------------
// energy E = 1/2 sum_i q_i phi_i, reduced in FP64
// ---------------------------------------------------------------------------
constexpr int kEnergyThreads = 256;

__global__ void __launch_bounds__(kEnergyThreads) k_energy_partial(int64_t n, const float4 *pos, const float *phi,
                                                                   double *part)
{
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)pos[i].w * (double)phi[i];
    s = warp_sum(s);
    __shared__ double ws[kEnergyThreads / 32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kEnergyThreads / 32; ++k) t += ws[k];
        part[blockIdx.x] = t;
    }
}

__global__ void k_energy_final(int nb, const double *part, double *E)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
    s = warp_sum(s);
    __shared__ double ws[32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws[k];
        *E = 0.5 * t;
    }
}

int energy_reduce(Handle &h, double *E)
{
    const int nb = std::min(ceil_div(h.N, kEnergyThreads), h.num_sms * 4);
    FMM_TRY(h.energy_part.reserve((size_t)(nb + 1) * sizeof(double)));
    double *part = h.energy_part.as<double>();
    ++h.launches;
    k_energy_partial<<<nb, kEnergyThreads, 0, h.stream>>>(h.N, h.pos.as<float4>(), h.phi_sorted.as<float>(), part);
    ++h.launches;
    k_energy_final<<<1, 256, 0, h.stream>>>(nb, part, part + nb);
    FMM_CHECK_LAUNCH("energy");
    FMM_CUDA(cudaMemcpyAsync(E, part + nb, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    return FMM_OK;
}

}  // namespace fmm
