// multi.cu -- many independent systems in one evaluation (fmm_multi_*).
//
// Each system gets its own tree and traversal lists (an ordinary handle, with
// its own normalisation).  The trees are then merged into one set of arrays:
// cells ordered by (level, system, cell), particles and source runs back to
// back, every index moved by its system's offset, and a per-cell unit scale
// (1/h, 1/h^2 of the cell's system).  Interactions never cross systems because
// no list entry does, so the ordinary evaluation kernels run once over all
// systems: one charge gather, one P2M, one M2M and one L2L launch per level,
// one M2L and one P2P launch in total, whatever the number of systems.
// That evaluation is captured into a CUDA graph once and replayed, so a call
// costs one graph launch.  Before capture an autotuner times the near field on
// the merged problem in six configurations -- work items of 16 or 8 targets;
// one-sided, or mutual (each unordered leaf pair once, both directions) with 2
// or 4 staged sources per lane -- and keeps the fastest (fmm_multi_set_config
// can pin any choice).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "device_util.cuh"
#include "fmm_internal.cuh"

namespace fmm {

__global__ void k_merge_cells(int nc, const int *level, const int *pbeg, const int *pcnt, const int *cbeg,
                              const int *ccnt, const int *parent, const float4 *geom, const int *m2l_off,
                              const int *map_base, int pbase, float2 scale, int *m_level, int *m_pbeg, int *m_pcnt,
                              int *m_cbeg, int *m_ccnt, int *m_parent, float4 *m_geom, float2 *m_scale,
                              unsigned *m_m2l_count)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int l = level[c];
    const int nw = c + map_base[l];
    m_level[nw] = l;
    m_pbeg[nw] = pbeg[c] + pbase;
    m_pcnt[nw] = pcnt[c];
    m_ccnt[nw] = ccnt[c];
    m_cbeg[nw] = ccnt[c] > 0 ? cbeg[c] + map_base[l + 1] : 0;
    m_parent[nw] = parent[c] >= 0 ? parent[c] + map_base[l - 1] : -1;
    m_geom[nw] = geom[c];
    m_scale[nw] = scale;
    m_m2l_count[nw] = (unsigned)(m2l_off[c + 1] - m2l_off[c]);
}

// per cell: its list length (cell-indexed CSR offsets) at its merged index
__global__ void k_merge_count(int nc, const int *level, const int *map_base, const int *off, unsigned *m_count)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    m_count[c + map_base[level[c]]] = (unsigned)(off[c + 1] - off[c]);
}

// warp per cell: copy its list (M2L or P2P sources) to the merged list, renumbered
__global__ void k_merge_m2l(int nc, const int *level, const int *map_base, const int *m2l_off, const int *m2l_src,
                            const unsigned *m_off, int *m_src)
{
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= nc) return;
    const int nw = c + map_base[level[c]];
    const int b = m2l_off[c], e = m2l_off[c + 1];
    const unsigned o = m_off[nw];
    for (int k = b + (int)lane_id(); k < e; k += 32) {
        const int s = m2l_src[k];
        m_src[o + (k - b)] = s + map_base[level[s]];
    }
}

__global__ void k_merge_leaves(int nl, const int *leaf_list, const int *level, const int *map_base,
                               const unsigned *poff, int llbase, unsigned runbase, int *m_leaf_list, unsigned *m_poff)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    const int c = leaf_list[i];
    m_leaf_list[llbase + i] = c + map_base[level[c]];
    m_poff[llbase + i] = poff[i] + runbase;
}

__global__ void k_merge_runs(int nr, const float4 *ent, const int *end, int pbase, int runbase, float4 *m_ent,
                             int *m_end)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nr) return;
    const float4 e = ent[i];
    m_ent[runbase + i] = make_float4(e.x, e.y, e.z, __int_as_float(__float_as_int(e.w) + pbase));
    m_end[runbase + i] = end[i] + pbase;
}

__global__ void k_merge_particles(int n, const float4 *pos, const int *perm, int pbase, float4 *m_pos, int *m_perm)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    m_pos[pbase + i] = pos[i];
    m_perm[pbase + i] = perm[i] + pbase;
}

struct Multi {
    int nsys = 0;
    std::vector<fmm_handle *> sys;
    std::vector<int64_t> N, pbase;
    int64_t Ntot = 0;
    Handle hm;                       // the merged problem
    cudaStream_t user_stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t graph_nodes = 0;
    const float *g_q = nullptr;
    float *g_phi = nullptr, *g_grad = nullptr;
    bool merged = false, tuned = false, timed = false;
    // P2P phase time per configuration: one-sided with 16 / 8 targets per item,
    // mutual (2 sources per lane) with 16 / 8, mutual (4 sources per lane) with 16 / 8 (the autotuner's table)
    float tune_ms[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int pin_g = 0, pin_mutual = -1;   // fmm_multi_set_config (0 / -1: tune)
    int64_t n_m2l = 0, p2p_pairs = 0;
};

static void release_merged(Handle &h)
{
    DevBuf *bufs[] = {&h.pos, &h.perm, &h.c_level, &h.c_pbeg, &h.c_pcnt, &h.c_cbeg, &h.c_ccnt, &h.c_parent,
                      &h.c_geom, &h.c_scale, &h.m2l_off, &h.m2l_src, &h.leaf_list, &h.p2p_poff, &h.p2p_ent,
                      &h.p2p_cnt, &h.p2p_items, &h.M, &h.L, &h.phi_sorted, &h.c_tmp, &h.scan_tmp,
                      &h.p2p_off, &h.p2p_src, &h.mu_off, &h.mu_src, &h.os_off, &h.os_src, &h.mu_cnt_tmp,
                      &h.mu_poff, &h.mu_ent, &h.mu_cnt, &h.os_poff, &h.os_ent, &h.os_cnt, &h.racc, &h.Mf};
    for (DevBuf *b : bufs) b->release();
}

static int merge_systems(Multi &m)
{
    Handle &hm = m.hm;
    const int S = m.nsys;
    int L = 0;
    int64_t C = 0, NL = 0, NR = 0;
    for (int s = 0; s < S; ++s) {
        const Handle &h = m.sys[s]->h;
        L = std::max(L, h.nlevels);
        C += h.ncells;
        NL += h.nleaves;
        NR += h.n_pieces;
    }
    // cell order (level, system, cell): level bases, then each system's offset in each level
    std::vector<int64_t> level_n(L, 0);
    for (int s = 0; s < S; ++s) {
        const Handle &h = m.sys[s]->h;
        for (int l = 0; l < h.nlevels; ++l) level_n[l] += h.level_off[l + 1] - h.level_off[l];
    }
    hm.level_off.assign(L + 1, 0);
    for (int l = 0; l < L; ++l) hm.level_off[l + 1] = hm.level_off[l] + level_n[l];
    // map_base[s][l] = merged index - local index for a level-l cell of system s (levels -1 .. L as padding)
    std::vector<int> map_base((size_t)S * (L + 2), 0);
    std::vector<int64_t> fill(hm.level_off.begin(), hm.level_off.end() - 1);
    for (int s = 0; s < S; ++s) {
        const Handle &h = m.sys[s]->h;
        for (int l = 0; l < h.nlevels; ++l) {
            map_base[(size_t)s * (L + 2) + 1 + l] = (int)(fill[l] - h.level_off[l]);
            fill[l] += h.level_off[l + 1] - h.level_off[l];
        }
    }
    hm.N = m.Ntot;
    hm.ncells = C;
    hm.nleaves = NL;
    hm.nlevels = L;
    hm.n_pieces = NR;
    FMM_TRY(hm.pos.reserve(m.Ntot * sizeof(float4)));
    FMM_TRY(hm.perm.reserve(m.Ntot * sizeof(int)));
    for (DevBuf *b : {&hm.c_level, &hm.c_pbeg, &hm.c_pcnt, &hm.c_cbeg, &hm.c_ccnt, &hm.c_parent})
        FMM_TRY(b->reserve(C * sizeof(int)));
    FMM_TRY(hm.c_geom.reserve(C * sizeof(float4)));
    FMM_TRY(hm.c_scale.reserve(C * sizeof(float2)));
    FMM_TRY(hm.m2l_off.reserve((C + 1) * sizeof(unsigned)));
    FMM_TRY(hm.c_tmp.reserve((C + 1) * sizeof(unsigned)));
    FMM_TRY(hm.leaf_list.reserve(NL * sizeof(int)));
    FMM_TRY(hm.p2p_poff.reserve((NL + 1) * sizeof(unsigned)));
    FMM_TRY(hm.p2p_ent.reserve(std::max<int64_t>(NR, 1) * sizeof(float4)));
    FMM_TRY(hm.p2p_cnt.reserve(std::max<int64_t>(NR, 1) * sizeof(int)));
    DevBuf map_dev;
    FMM_TRY(map_dev.reserve(map_base.size() * sizeof(int)));
    FMM_CUDA(cudaMemcpyAsync(map_dev.p, map_base.data(), map_base.size() * sizeof(int), cudaMemcpyHostToDevice,
                             hm.stream));
    unsigned *mcount = hm.c_tmp.as<unsigned>();
    int64_t llbase = 0, runbase = 0, nm2l = 0, pairs = 0;
    for (int s = 0; s < S; ++s) {
        Handle &h = m.sys[s]->h;
        const int *mb = map_dev.as<int>() + (size_t)s * (L + 2) + 1;   // mb[l], l = -1 .. L
        const int nc = (int)h.ncells, nl = (int)h.nleaves, nr = (int)h.n_pieces, n = (int)h.N;
        const float2 scale = make_float2((float)(1.0 / h.norm_host[3]), (float)(1.0 / (h.norm_host[3] * h.norm_host[3])));
        ++hm.launches;
        k_merge_cells<<<ceil_div(nc, 256), 256, 0, hm.stream>>>(
            nc, h.c_level.as<int>(), h.c_pbeg.as<int>(), h.c_pcnt.as<int>(), h.c_cbeg.as<int>(), h.c_ccnt.as<int>(),
            h.c_parent.as<int>(), h.c_geom.as<float4>(), h.m2l_off.as<int>(), mb, (int)m.pbase[s], scale,
            hm.c_level.as<int>(), hm.c_pbeg.as<int>(), hm.c_pcnt.as<int>(), hm.c_cbeg.as<int>(), hm.c_ccnt.as<int>(),
            hm.c_parent.as<int>(), hm.c_geom.as<float4>(), hm.c_scale.as<float2>(), mcount);
        ++hm.launches;
        k_merge_leaves<<<ceil_div(nl, 256), 256, 0, hm.stream>>>(nl, h.leaf_list.as<int>(), h.c_level.as<int>(), mb,
                                                                 h.p2p_poff.as<unsigned>(), (int)llbase,
                                                                 (unsigned)runbase, hm.leaf_list.as<int>(),
                                                                 hm.p2p_poff.as<unsigned>());
        if (nr > 0) {
            ++hm.launches;
            k_merge_runs<<<ceil_div(nr, 256), 256, 0, hm.stream>>>(nr, h.p2p_ent.as<float4>(), h.p2p_cnt.as<int>(),
                                                                   (int)m.pbase[s], (int)runbase, hm.p2p_ent.as<float4>(),
                                                                   hm.p2p_cnt.as<int>());
        }
        ++hm.launches;
        k_merge_particles<<<ceil_div(n, 256), 256, 0, hm.stream>>>(n, h.pos.as<float4>(), h.perm.as<int>(),
                                                                   (int)m.pbase[s], hm.pos.as<float4>(),
                                                                   hm.perm.as<int>());
        llbase += nl;
        runbase += nr;
        nm2l += h.n_m2l;
        pairs += h.p2p_pairs;
    }
    unsigned total_runs = (unsigned)runbase;
    FMM_CUDA(cudaMemcpyAsync(hm.p2p_poff.as<unsigned>() + NL, &total_runs, sizeof(unsigned), cudaMemcpyHostToDevice,
                             hm.stream));
    // merged M2L CSR: offsets by a scan of the per-cell counts, then the renumbered sources
    FMM_TRY(scan_exclusive_u32(hm, mcount, hm.m2l_off.as<unsigned>(), C, hm.m2l_off.as<unsigned>() + C));
    FMM_TRY(hm.m2l_src.reserve(std::max<int64_t>(nm2l, 1) * sizeof(int)));
    for (int s = 0; s < S; ++s) {
        Handle &h = m.sys[s]->h;
        const int *mb = map_dev.as<int>() + (size_t)s * (L + 2) + 1;
        const int nc = (int)h.ncells;
        ++hm.launches;
        k_merge_m2l<<<ceil_div((int64_t)nc * 32, 256), 256, 0, hm.stream>>>(nc, h.c_level.as<int>(), mb,
                                                                            h.m2l_off.as<int>(), h.m2l_src.as<int>(),
                                                                            hm.m2l_off.as<unsigned>(),
                                                                            hm.m2l_src.as<int>());
    }
    // merged P2P CSR (the mutual schedule splits it), the same way
    FMM_TRY(hm.p2p_off.reserve((C + 1) * sizeof(unsigned)));
    int64_t np2p = 0;
    for (int s = 0; s < S; ++s) {
        Handle &h = m.sys[s]->h;
        const int *mb = map_dev.as<int>() + (size_t)s * (L + 2) + 1;
        const int nc = (int)h.ncells;
        ++hm.launches;
        k_merge_count<<<ceil_div(nc, 256), 256, 0, hm.stream>>>(nc, h.c_level.as<int>(), mb, h.p2p_off.as<int>(),
                                                                mcount);
        np2p += h.n_p2p;
    }
    FMM_TRY(scan_exclusive_u32(hm, mcount, hm.p2p_off.as<unsigned>(), C, hm.p2p_off.as<unsigned>() + C));
    FMM_TRY(hm.p2p_src.reserve(std::max<int64_t>(np2p, 1) * sizeof(int)));
    for (int s = 0; s < S; ++s) {
        Handle &h = m.sys[s]->h;
        const int *mb = map_dev.as<int>() + (size_t)s * (L + 2) + 1;
        const int nc = (int)h.ncells;
        ++hm.launches;
        k_merge_m2l<<<ceil_div((int64_t)nc * 32, 256), 256, 0, hm.stream>>>(nc, h.c_level.as<int>(), mb,
                                                                            h.p2p_off.as<int>(), h.p2p_src.as<int>(),
                                                                            hm.p2p_off.as<unsigned>(),
                                                                            hm.p2p_src.as<int>());
    }
    hm.n_p2p = np2p;
    hm.mutual_ready = false;
    FMM_CHECK_LAUNCH("merge systems");
    FMM_CUDA(cudaStreamSynchronize(hm.stream));
    map_dev.release();
    m.n_m2l = nm2l;
    m.p2p_pairs = pairs;
    hm.n_m2l = nm2l;
    hm.p2p_pairs = pairs;
    hm.p2p_g = 0;
    FMM_TRY(build_work_items(hm, 16, hm.p2p_items, hm.n_items));
    hm.built = true;
    hm.full_runs_ready = true;   // the merged runs
    m.merged = true;
    m.tuned = false;
    if (m.exec) {
        cudaGraphExecDestroy(m.exec);
        m.exec = nullptr;
    }
    return FMM_OK;
}

static int merged_evaluate(Handle &hm, const float *q, float *phi, float *grad)
{
    FMM_TRY(evaluate_upward(hm, q));
    FMM_TRY(hm.L.reserve((size_t)hm.ncells * hm.TP * sizeof(float)));
    FMM_TRY(evaluate_m2l(hm, hm.M.as<float>(), hm.L.as<float>()));
    FMM_TRY(evaluate_downward(hm, hm.L.as<float>()));
    return evaluate_p2p(hm, phi, grad);
}

// Best of 3 timed P2P phases (after one warm-up) of the current configuration.
static int time_p2p(Multi &m, float *phi, float *grad, float *best_ms)
{
    Handle &hm = m.hm;
    FMM_TRY(evaluate_p2p(hm, phi, grad));   // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        FMM_CUDA(cudaEventRecord(m.ev_t0, hm.stream));
        FMM_TRY(evaluate_p2p(hm, phi, grad));
        FMM_CUDA(cudaEventRecord(m.ev_t1, hm.stream));
        FMM_CUDA(cudaEventSynchronize(m.ev_t1));
        float ms = 0.f;
        FMM_CUDA(cudaEventElapsedTime(&ms, m.ev_t0, m.ev_t1));
        best = std::min(best, ms);
    }
    *best_ms = best;
    return FMM_OK;
}

// The tile autotuner of the merged problem (the far field of this call is in
// place): the near field with work items of 16 and of 8 targets, one-sided,
// mutual with 2 staged sources per lane (12 warps per SM) and mutual with 4
// (8 warps per SM), each timed on the merged problem; the fastest is kept,
// unless fmm_multi_set_config pinned a choice.
static int autotune(Multi &m, float *phi, float *grad)
{
    Handle &hm = m.hm;
    const int gs[2] = {16, 8};
    const int lanes[3] = {0, 2, 4};   // mode 0 one-sided, 1 / 2 mutual with that many sources per lane
    for (int mu = 0; mu < 3; ++mu) {
        if (mu == 1) FMM_TRY(build_mutual(hm));
        hm.mutual_ready = mu != 0;
        if (mu) hm.mu_lanes = lanes[mu];
        for (int k = 0; k < 2; ++k) {
            hm.p2p_g = gs[k];
            FMM_TRY(build_work_items(hm, gs[k], hm.p2p_items, hm.n_items));
            FMM_TRY(time_p2p(m, phi, grad, &m.tune_ms[2 * mu + k]));
        }
    }
    int best = 0;
    for (int i = 1; i < 6; ++i)
        if (m.tune_ms[i] < m.tune_ms[best]) best = i;
    int mu = best >> 1, g = gs[best & 1];
    if (m.pin_mutual >= 0) mu = m.pin_mutual;
    if (m.pin_g) g = m.pin_g;
    hm.mutual_ready = mu != 0;
    if (mu) hm.mu_lanes = lanes[mu];
    hm.p2p_g = g;
    FMM_TRY(build_work_items(hm, g, hm.p2p_items, hm.n_items));
    m.tuned = true;
    return FMM_OK;
}

static int capture(Multi &m, const float *q, float *phi, float *grad)
{
    Handle &hm = m.hm;
    if (m.exec) {
        cudaGraphExecDestroy(m.exec);
        m.exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    FMM_CUDA(cudaStreamBeginCapture(hm.stream, cudaStreamCaptureModeThreadLocal));
    const int rc = merged_evaluate(hm, q, phi, grad);
    const cudaError_t e = cudaStreamEndCapture(hm.stream, &graph);
    if (rc != FMM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    FMM_CUDA(e);
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    const cudaError_t ei = cudaGraphInstantiate(&m.exec, graph, 0);
    cudaGraphDestroy(graph);
    FMM_CUDA(ei);
    m.graph_nodes = nodes;
    m.g_q = q;
    m.g_phi = phi;
    m.g_grad = grad;
    return FMM_OK;
}

}  // namespace fmm

struct fmm_multi {
    fmm::Multi m;
};

using namespace fmm;

extern "C" {

int fmm_multi_create(fmm_multi **mp, int nsys, const int64_t *N, int P, float theta, int ncrit, const fmm_options *opt)
{
    if (!mp) {
        set_error("fmm_multi_create: null handle pointer");
        return FMM_ERR_ARG;
    }
    *mp = nullptr;
    if (nsys < 1 || !N) {
        set_error("fmm_multi_create: need nsys >= 1 and the system sizes");
        return FMM_ERR_ARG;
    }
    int64_t tot = 0;
    for (int s = 0; s < nsys; ++s) {
        if (N[s] < 1) {
            set_error("fmm_multi_create: every system needs N >= 1");
            return FMM_ERR_ARG;
        }
        tot += N[s];
    }
    if (tot > 0x7fffffffll) {
        set_error("fmm_multi_create: total N must be below 2^31");
        return FMM_ERR_ARG;
    }
    // the per-system checks of fmm_create, before any device call
    if (!(theta >= 0.0f && theta < 1.0f) || ncrit < 1) {
        set_error("fmm_multi_create: theta must be in [0, 1) and ncrit >= 1");
        return FMM_ERR_ARG;
    }
    if (!supported_order(P)) {
        set_error("fmm_multi_create: expansion order P must be one of 3, 4, 5, 6, 8");
        return FMM_ERR_UNSUPPORTED;
    }
    fmm_multi *w = new (std::nothrow) fmm_multi;
    if (!w) {
        set_error("fmm_multi_create: out of host memory");
        return FMM_ERR_NOMEM;
    }
    Multi &m = w->m;
    int dev = opt && opt->device >= 0 ? opt->device : -1;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    m.user_stream = opt ? static_cast<cudaStream_t>(opt->stream) : nullptr;
    cudaStream_t priv = nullptr;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(dev);
    cudaError_t e = cudaStreamCreateWithFlags(&priv, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m.ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m.ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&m.ev_t0);
    if (e == cudaSuccess) e = cudaEventCreate(&m.ev_t1);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "fmm_multi_create", __FILE__, __LINE__);
        delete w;
        return rc;
    }
    // every system (and the merged problem) runs on the private stream, which
    // the graph is captured on; calls order it after the caller's stream
    fmm_options so = {priv, dev, opt ? (opt->flags & ~FMM_FLAG_KAHAN & ~FMM_FLAG_TIMING & ~FMM_FLAG_MUTUAL) : 0u};
    m.nsys = nsys;
    m.N.assign(N, N + nsys);
    m.pbase.assign(nsys, 0);
    for (int s = 0; s < nsys; ++s) {
        m.pbase[s] = m.Ntot;
        m.Ntot += N[s];
        fmm_handle *h = nullptr;
        const int rc = fmm_create(&h, N[s], P, theta, ncrit, &so);
        if (rc != FMM_OK) {
            fmm_multi_destroy(w);
            return rc;
        }
        m.sys.push_back(h);
    }
    Handle &hm = m.hm;
    hm.P = P;
    hm.TP = ((P * (P + 1) * (P + 2) / 6) + 3) & ~3;
    hm.theta = theta;
    hm.ncrit = ncrit;
    hm.flags = 0;
    hm.device = dev;
    hm.stream = priv;
    hm.num_sms = m.sys[0]->h.num_sms;
    if (cudaMallocHost(reinterpret_cast<void **>(&hm.pinned), sizeof(PinnedScratch)) != cudaSuccess) {
        hm.pinned = nullptr;
        fmm_multi_destroy(w);
        set_error("fmm_multi_create: pinned scratch allocation failed");
        return FMM_ERR_NOMEM;
    }
    *mp = w;
    return FMM_OK;
}

int fmm_multi_destroy(fmm_multi *w)
{
    if (!w) return FMM_OK;
    Multi &m = w->m;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(m.hm.device);
    if (m.hm.stream) cudaStreamSynchronize(m.hm.stream);
    if (m.exec) cudaGraphExecDestroy(m.exec);
    for (fmm_handle *h : m.sys) fmm_destroy(h);
    release_merged(m.hm);
    if (m.hm.pinned) cudaFreeHost(m.hm.pinned);
    for (cudaEvent_t ev : {m.ev_in, m.ev_out, m.ev_t0, m.ev_t1})
        if (ev) cudaEventDestroy(ev);
    if (m.hm.stream) cudaStreamDestroy(m.hm.stream);
    if (prev >= 0) cudaSetDevice(prev);
    delete w;
    return FMM_OK;
}

int fmm_multi_build(fmm_multi *w, const double *x)
{
    if (!w || !x) {
        set_error("fmm_multi_build: null argument");
        return FMM_ERR_ARG;
    }
    Multi &m = w->m;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(m.hm.device);
    int rc = FMM_OK;
    // the caller's work on x comes first
    cudaEventRecord(m.ev_in, m.user_stream);
    cudaStreamWaitEvent(m.hm.stream, m.ev_in, 0);
    for (int s = 0; s < m.nsys && rc == FMM_OK; ++s) rc = fmm_build(m.sys[s], x + 3 * m.pbase[s]);
    if (rc == FMM_OK) rc = merge_systems(m);
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}

int fmm_multi_evaluate(fmm_multi *w, const float *q, float *phi, float *grad)
{
    if (!w || !q || (!phi && !grad)) {
        set_error("fmm_multi_evaluate: null argument");
        return FMM_ERR_ARG;
    }
    Multi &m = w->m;
    if (!m.merged) {
        set_error("fmm_multi_evaluate: no build");
        return FMM_ERR_STATE;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(m.hm.device);
    struct Restore {
        int d;
        ~Restore()
        {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{prev};
    Handle &hm = m.hm;
    FMM_CUDA(cudaEventRecord(m.ev_in, m.user_stream));
    FMM_CUDA(cudaStreamWaitEvent(hm.stream, m.ev_in, 0));
    if (!m.tuned || !m.exec || q != m.g_q || phi != m.g_phi || grad != m.g_grad) {
        // an eager evaluation sizes every buffer (nothing may allocate during
        // capture), the autotuner picks the P2P item size, then the capture
        FMM_TRY(merged_evaluate(hm, q, phi, grad));
        if (!m.tuned) FMM_TRY(autotune(m, phi, grad));
        FMM_TRY(capture(m, q, phi, grad));
    }
    FMM_CUDA(cudaEventRecord(m.ev_t0, hm.stream));
    FMM_CUDA(cudaGraphLaunch(m.exec, hm.stream));
    FMM_CUDA(cudaEventRecord(m.ev_t1, hm.stream));
    m.timed = true;
    FMM_CUDA(cudaEventRecord(m.ev_out, hm.stream));
    FMM_CUDA(cudaStreamWaitEvent(m.user_stream, m.ev_out, 0));
    return FMM_OK;
}

int fmm_multi_set_hybrid(fmm_multi *w, int64_t min_pairs)
{
    if (!w) {
        set_error("fmm_multi_set_hybrid: null handle");
        return FMM_ERR_ARG;
    }
    for (fmm_handle *h : w->m.sys) FMM_TRY(fmm_set_hybrid(h, min_pairs));
    w->m.merged = false;   // the lists change: build again
    return FMM_OK;
}

int fmm_multi_set_config(fmm_multi *w, int targets_per_item, int mutual)
{
    if (!w) {
        set_error("fmm_multi_set_config: null handle");
        return FMM_ERR_ARG;
    }
    if (targets_per_item != 0 && targets_per_item != 8 && targets_per_item != 16) {
        set_error("fmm_multi_set_config: targets_per_item must be 0 (tune), 8 or 16");
        return FMM_ERR_ARG;
    }
    if (mutual < -1 || mutual > 2) {
        set_error("fmm_multi_set_config: mutual must be -1 (tune), 0, 1 or 2");
        return FMM_ERR_ARG;
    }
    w->m.pin_g = targets_per_item;
    w->m.pin_mutual = mutual;
    w->m.tuned = false;   // applied (and the table timed again) at the next evaluation
    return FMM_OK;
}

int fmm_multi_info(fmm_multi *w, struct fmm_multi_info *info)
{
    if (!w || !info) {
        set_error("fmm_multi_info: null argument");
        return FMM_ERR_ARG;
    }
    Multi &m = w->m;
    std::memset(info, 0, sizeof(*info));
    info->nsys = m.nsys;
    info->n_total = m.Ntot;
    info->ncells = m.hm.ncells;
    info->nleaves = m.hm.nleaves;
    info->nlevels = m.hm.nlevels;
    info->n_m2l = m.n_m2l;
    info->p2p_pairs = m.p2p_pairs;
    info->p2p_targets_per_item = m.hm.p2p_g ? m.hm.p2p_g : 16;
    info->mutual = m.hm.mutual_ready ? (m.hm.mu_lanes == 4 ? 2 : 1) : 0;
    for (int i = 0; i < 6; ++i) info->tune_ms[i] = m.tune_ms[i];
    info->graph_nodes = (int64_t)m.graph_nodes;
    info->kernel_launches = m.hm.launches;
    if (m.timed) {
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(m.hm.device);
        float ms = 0.f;
        if (cudaEventSynchronize(m.ev_t1) == cudaSuccess && cudaEventElapsedTime(&ms, m.ev_t0, m.ev_t1) == cudaSuccess)
            info->ms_evaluate = ms;
        if (prev >= 0) cudaSetDevice(prev);
    }
    return FMM_OK;
}

}  // extern "C"
