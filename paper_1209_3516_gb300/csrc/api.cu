// api.cu -- the C ABI (include/fmm.h): handles, build / evaluate orchestration,
// host-buffer entry point, energy, counters and introspection.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    g_last_error = buf;
    return e == cudaErrorMemoryAllocation ? FMM_ERR_NOMEM : FMM_ERR_CUDA;
}

int DevBuf::reserve(size_t need)
{
    if (need <= bytes && p) return FMM_OK;
    release();
    size_t sz = std::max<size_t>(need, 256);
    cudaError_t e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) {
        p = nullptr;
        return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    }
    bytes = sz;
    return FMM_OK;
}

int DevBuf::reserve_keep(size_t need, cudaStream_t s)
{
    if (need <= bytes && p) return FMM_OK;
    void *np = nullptr;
    size_t sz = std::max<size_t>(need, 256);
    cudaError_t e = cudaMalloc(&np, sz);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    if (p) {
        e = cudaMemcpyAsync(np, p, bytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(np);
            return cuda_fail(e, "regrow copy", __FILE__, __LINE__);
        }
        cudaFree(p);
    }
    p = np;
    bytes = sz;
    return FMM_OK;
}

void DevBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

void phase_begin(Handle &h, int phase)
{
    if (h.events_ready && (h.flags & FMM_FLAG_TIMING)) cudaEventRecord(h.ev[2 * phase], h.stream);
}

void phase_end(Handle &h, int phase)
{
    if (h.events_ready && (h.flags & FMM_FLAG_TIMING)) cudaEventRecord(h.ev[2 * phase + 1], h.stream);
}


// Pins the handle's device for the duration of a call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Errors that kernels record asynchronously (bit 3 of err_flag, a radix-sort
// look-back wait, is checked at the end of every build; bit 1: a bounded wait of
// the P2P staging gave up); read at the synchronising entry points.
static int check_async_errors(Handle &h)
{
    if (!h.err_flag.p) return FMM_OK;
    FMM_CUDA(cudaMemcpyAsync(&h.pinned->err, h.err_flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    if (h.pinned->err & 2u) {
        FMM_CUDA(cudaMemsetAsync(h.err_flag.p, 0, sizeof(unsigned), h.stream));
        set_error("P2P staging: a bulk-copy wait gave up; the last evaluation is incomplete");
        return FMM_ERR_CUDA;
    }
    if (h.pinned->err & 4u) {
        FMM_CUDA(cudaMemsetAsync(h.err_flag.p, 0, sizeof(unsigned), h.stream));
        set_error("batched P2P: a tensor-core completion wait gave up; the last batched evaluation is incomplete");
        return FMM_ERR_CUDA;
    }
    return FMM_OK;
}

static int do_build(Handle &h, const double *x)
{
    if (h.side_pending) {
        // a build that failed after forking the M2L grouping: let it finish
        h.side_pending = false;
        FMM_CUDA(cudaStreamSynchronize(h.side));
    }
    h.built = false;
    h.evaluated = false;
    h.backward_done = false;
    h.batch_done = false;
    const int ev0 = 2 * kPhases, ev1 = 2 * kPhases + 1;
    if (h.events_ready) cudaEventRecord(h.ev[ev0], h.stream);
    FMM_TRY(build_keys(h, x));
    FMM_TRY(build_tree(h, x));
    FMM_TRY(build_lists(h));
    phase_begin(h, FMM_PHASE_ITEMS);
    FMM_TRY(build_p2p_items(h));
    phase_end(h, FMM_PHASE_ITEMS);
    FMM_TRY(join_lists_begin(h));
    if (h.events_ready) cudaEventRecord(h.ev[ev1], h.stream);
    FMM_CUDA(cudaMemcpyAsync(&h.pinned->err, h.err_flag.p, sizeof(unsigned), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    FMM_TRY(join_lists_end(h));
    if (h.pinned->err & 8u) {
        FMM_CUDA(cudaMemsetAsync(h.err_flag.p, 0, sizeof(unsigned), h.stream));
        set_error("fmm_build: a radix-sort look-back wait gave up; the build is invalid");
        return FMM_ERR_CUDA;
    }
    if (h.events_ready) cudaEventElapsedTime(&h.ms_build, h.ev[ev0], h.ev[ev1]);
    h.x_built = x;
    h.built = true;
    return FMM_OK;
}

static int do_evaluate(Handle &h, const float *q, float *phi, float *grad)
{
    const int ev0 = 2 * kPhases + 2, ev1 = 2 * kPhases + 3;
    if (h.events_ready) cudaEventRecord(h.ev[ev0], h.stream);
    phase_begin(h, FMM_PHASE_UPWARD);
    FMM_TRY(evaluate_upward(h, q));
    phase_end(h, FMM_PHASE_UPWARD);
    phase_begin(h, FMM_PHASE_M2L);
    FMM_TRY(h.L.reserve((size_t)h.ncells * h.TP * sizeof(float)));
    FMM_TRY(evaluate_m2l(h, h.M.as<float>(), h.L.as<float>()));
    phase_end(h, FMM_PHASE_M2L);
    phase_begin(h, FMM_PHASE_DOWNWARD);
    FMM_TRY(evaluate_downward(h, h.L.as<float>()));
    phase_end(h, FMM_PHASE_DOWNWARD);
    phase_begin(h, FMM_PHASE_P2P);
    FMM_TRY(evaluate_p2p(h, phi, grad));
    phase_end(h, FMM_PHASE_P2P);
    if (h.events_ready) cudaEventRecord(h.ev[ev1], h.stream);
    h.evaluated = true;
    return FMM_OK;
}

}  // namespace fmm

using namespace fmm;

extern "C" {

const char *fmm_last_error_string(void) { return g_last_error.c_str(); }

int fmm_create(fmm_handle **hp, int64_t N, int P, float theta, int ncrit, const fmm_options *opt)
{
    if (!hp) {
        set_error("fmm_create: null handle pointer");
        return FMM_ERR_ARG;
    }
    *hp = nullptr;
    if (N < 1 || N > 0x7fffffffll) {
        set_error("fmm_create: N must be in [1, 2^31 - 1]");
        return FMM_ERR_ARG;
    }
    if (!(theta >= 0.0f && theta < 1.0f)) {
        set_error("fmm_create: theta must be in [0, 1)");
        return FMM_ERR_ARG;
    }
    if (ncrit < 1) {
        set_error("fmm_create: ncrit must be >= 1");
        return FMM_ERR_ARG;
    }
    if (!supported_order(P)) {
        set_error("fmm_create: expansion order P must be one of 3, 4, 5, 6, 8");
        return FMM_ERR_UNSUPPORTED;
    }
    int dev = opt && opt->device >= 0 ? opt->device : -1;
    if (dev < 0) FMM_CUDA(cudaGetDevice(&dev));
    DeviceGuard guard(dev);
    fmm_handle *w = new (std::nothrow) fmm_handle;
    if (!w) {
        set_error("fmm_create: out of host memory");
        return FMM_ERR_NOMEM;
    }
    Handle &h = w->h;
    h.N = N;
    h.P = P;
    h.TP = ((P * (P + 1) * (P + 2) / 6) + 3) & ~3;
    h.theta = theta;
    h.ncrit = ncrit;
    h.flags = opt ? opt->flags : 0u;
    h.device = dev;
    h.stream = opt ? static_cast<cudaStream_t>(opt->stream) : nullptr;
    cudaError_t e = cudaDeviceGetAttribute(&h.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&h.pinned), sizeof(PinnedScratch));
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "fmm_create", __FILE__, __LINE__);
        delete w;
        return rc;
    }
    std::memset(h.pinned, 0, sizeof(PinnedScratch));
    bool ok = true;
    for (auto &ev : h.ev) ok = ok && cudaEventCreate(&ev) == cudaSuccess;
    h.events_ready = ok;
    *hp = w;
    return FMM_OK;
}

int fmm_destroy(fmm_handle *w)
{
    if (!w) return FMM_OK;
    Handle &h = w->h;
    DeviceGuard guard(h.device);
    if (h.stream) cudaStreamSynchronize(h.stream);
    else cudaDeviceSynchronize();
    DevBuf *bufs[] = {&h.norm, &h.bbox_part, &h.err_flag, &h.keys, &h.keys_alt, &h.idx, &h.idx_alt, &h.sort_hist,
                      &h.scan_tmp, &h.pos_unsorted, &h.u_unsorted, &h.u_sorted, &h.pos, &h.perm, &h.c_prefix, &h.c_level, &h.c_pbeg, &h.c_pcnt,
                      &h.c_cbeg, &h.c_ccnt, &h.c_parent, &h.c_geom, &h.c_kids, &h.c_r2bits, &h.c_tmp, &h.leaf_of,
                      &h.counters, &h.front[0], &h.front[1], &h.m2l_raw, &h.p2p_raw, &h.lkeys, &h.lkeys_alt, &h.lcnt,
                      &h.m2l_src, &h.m2l_off, &h.p2p_src, &h.p2p_off, &h.leaf_list, &h.p2p_items, &h.p2p_poff, &h.p2p_ent, &h.p2p_cnt,
                      &h.pairs_count, &h.M, &h.L, &h.phi_sorted, &h.energy_part, &h.hx, &h.hq, &h.hphi, &h.hgrad,
                      &h.adj, &h.Ma, &h.La, &h.adj_items, &h.qb, &h.qbh, &h.qbl, &h.Mb, &h.Lb,
                      &h.c_scale, &h.tc_items, &h.lbh, &h.lbl, &h.tc_next, &h.mu_off, &h.mu_src,
                      &h.os_off, &h.os_src, &h.mu_cnt_tmp, &h.mu_poff, &h.mu_ent, &h.mu_cnt, &h.os_poff, &h.os_ent,
                      &h.os_cnt, &h.racc, &h.Mf};
    for (DevBuf *b : bufs) b->release();
    h.lcnt_side.release();
    h.lkeys_side.release();
    h.scan_tmp_side.release();
    if (h.side) {
        cudaStreamSynchronize(h.side);
        cudaStreamDestroy(h.side);
        cudaEventDestroy(h.ev_fork);
        cudaEventDestroy(h.ev_join);
    }
    if (h.events_ready)
        for (auto &ev : h.ev) cudaEventDestroy(ev);
    if (h.pinned) cudaFreeHost(h.pinned);
    delete w;
    return FMM_OK;
}

int fmm_build(fmm_handle *w, const double *x)
{
    if (!w || !x) {
        set_error("fmm_build: null argument");
        return FMM_ERR_ARG;
    }
    DeviceGuard guard(w->h.device);
    return do_build(w->h, x);
}

int fmm_evaluate(fmm_handle *w, const double *x, const float *q, float *phi, float *grad)
{
    if (!w || !q || (!phi && !grad)) {
        set_error("fmm_evaluate: null argument");
        return FMM_ERR_ARG;
    }
    Handle &h = w->h;
    DeviceGuard guard(h.device);
    if (x && (!h.built || x != h.x_built)) FMM_TRY(do_build(h, x));
    if (!h.built) {
        set_error("fmm_evaluate: no tree (call fmm_build or pass x)");
        return FMM_ERR_STATE;
    }
    return do_evaluate(h, q, phi, grad);
}

int fmm_evaluate_batch(fmm_handle *w, const double *x, const float *q, int nrhs, float *phi, float *grad)
{
    if (!w || !q || (!phi && !grad)) {
        set_error("fmm_evaluate_batch: null argument");
        return FMM_ERR_ARG;
    }
    if (nrhs < 1 || nrhs > FMM_MAX_RHS) {
        set_error("fmm_evaluate_batch: nrhs must be in [1, FMM_MAX_RHS]");
        return FMM_ERR_ARG;
    }
    Handle &h = w->h;
    DeviceGuard guard(h.device);
    if (x && (!h.built || x != h.x_built)) FMM_TRY(do_build(h, x));
    if (!h.built) {
        set_error("fmm_evaluate_batch: no tree (call fmm_build or pass x)");
        return FMM_ERR_STATE;
    }
    const int ev0 = 2 * kPhases + 6, ev1 = 2 * kPhases + 7;
    if (h.events_ready) cudaEventRecord(h.ev[ev0], h.stream);
    FMM_TRY(evaluate_batch(h, q, nrhs, phi, grad));
    if (h.events_ready) cudaEventRecord(h.ev[ev1], h.stream);
    h.batch_done = true;
    return FMM_OK;
}

int fmm_evaluate_host(fmm_handle *w, const double *x_host, const float *q_host, float *phi_host, float *grad_host)
{
    if (!w || !x_host || !q_host || (!phi_host && !grad_host)) {
        set_error("fmm_evaluate_host: null argument");
        return FMM_ERR_ARG;
    }
    Handle &h = w->h;
    DeviceGuard guard(h.device);
    const int64_t N = h.N;
    FMM_TRY(h.hx.reserve(N * 3 * sizeof(double)));
    FMM_TRY(h.hq.reserve(N * sizeof(float)));
    FMM_TRY(h.hphi.reserve(N * sizeof(float)));
    FMM_TRY(h.hgrad.reserve(N * 3 * sizeof(float)));
    FMM_CUDA(cudaMemcpyAsync(h.hx.p, x_host, N * 3 * sizeof(double), cudaMemcpyHostToDevice, h.stream));
    FMM_CUDA(cudaMemcpyAsync(h.hq.p, q_host, N * sizeof(float), cudaMemcpyHostToDevice, h.stream));
    FMM_TRY(do_build(h, h.hx.as<double>()));
    FMM_TRY(do_evaluate(h, h.hq.as<float>(), phi_host ? h.hphi.as<float>() : nullptr,
                        grad_host ? h.hgrad.as<float>() : nullptr));
    if (phi_host)
        FMM_CUDA(cudaMemcpyAsync(phi_host, h.hphi.p, N * sizeof(float), cudaMemcpyDeviceToHost, h.stream));
    if (grad_host)
        FMM_CUDA(cudaMemcpyAsync(grad_host, h.hgrad.p, N * 3 * sizeof(float), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    // the device copy of x is internal: a later fmm_evaluate(x = caller pointer) must rebuild
    h.x_built = nullptr;
    return check_async_errors(h);
}

int fmm_energy(fmm_handle *w, double *E)
{
    if (!w || !E) {
        set_error("fmm_energy: null argument");
        return FMM_ERR_ARG;
    }
    Handle &h = w->h;
    if (!h.evaluated) {
        set_error("fmm_energy: no evaluation yet");
        return FMM_ERR_STATE;
    }
    DeviceGuard guard(h.device);
    FMM_TRY(check_async_errors(h));
    return energy_reduce(h, E);
}

int fmm_backward(fmm_handle *w, const float *dphi, const float *dgrad, float *dq, float *dx)
{
    if (!w) {
        set_error("fmm_backward: null handle");
        return FMM_ERR_ARG;
    }
    if (!dq && !dx) {
        set_error("fmm_backward: dq and dx are both NULL");
        return FMM_ERR_ARG;
    }
    Handle &h = w->h;
    if (!h.evaluated) {
        set_error("fmm_backward: no evaluation to differentiate");
        return FMM_ERR_STATE;
    }
    DeviceGuard guard(h.device);
    const int ev0 = 2 * kPhases + 4, ev1 = 2 * kPhases + 5;
    if (h.events_ready) cudaEventRecord(h.ev[ev0], h.stream);
    // far field of the adjoint sources: dipole P2M, M2M, M2L, L2L (same lists)
    FMM_TRY(adjoint_upward(h, dphi, dgrad));
    FMM_TRY(h.La.reserve((size_t)h.ncells * h.TP * sizeof(float)));
    FMM_TRY(evaluate_m2l(h, h.Ma.as<float>(), h.La.as<float>()));
    FMM_TRY(evaluate_downward(h, h.La.as<float>()));
    // near field, far-field terms at the targets and the scatter
    FMM_TRY(adjoint_p2p(h, dq, dx));
    if (h.events_ready) cudaEventRecord(h.ev[ev1], h.stream);
    h.backward_done = true;
    return FMM_OK;
}

int fmm_set_hybrid(fmm_handle *w, int64_t min_pairs)
{
    if (!w) {
        set_error("fmm_set_hybrid: null handle");
        return FMM_ERR_ARG;
    }
    w->h.hybrid_min_pairs = min_pairs < 0 ? -1 : min_pairs;
    w->h.built = false;   // the lists change: the next evaluate needs a build
    return FMM_OK;
}

// Median device time (ms) of build + evaluate over reps runs after one warm-up.
static int time_config(int64_t N, int P, float theta, int ncrit, int64_t hybrid, const double *x, const float *q,
                       int reps, const fmm_options *opt, double *ms_out)
{
    fmm_handle *w = nullptr;
    fmm_options o = opt ? *opt : fmm_options{nullptr, -1, 0u};
    o.flags &= ~FMM_FLAG_TIMING;
    FMM_TRY(fmm_create(&w, N, P, theta, ncrit, &o));
    Handle &h = w->h;
    h.hybrid_min_pairs = hybrid;
    int rc = FMM_OK;
    DevBuf phi, grad;
    std::vector<float> times;
    {
        DeviceGuard guard(h.device);
        rc = phi.reserve((size_t)N * sizeof(float));
        if (rc == FMM_OK) rc = grad.reserve((size_t)N * 3 * sizeof(float));
        if (rc == FMM_OK && !h.events_ready) {
            set_error("autotuner: no CUDA events");
            rc = FMM_ERR_CUDA;
        }
        for (int r = 0; r <= reps && rc == FMM_OK; ++r) {   // r = 0: warm-up
            // do_build records the build's start event and synchronises at its end
            rc = do_build(h, x);
            if (rc == FMM_OK) rc = do_evaluate(h, q, phi.as<float>(), grad.as<float>());
            if (rc == FMM_OK) {
                cudaEventRecord(h.ev[2 * kPhases + 1], h.stream);
                cudaEventSynchronize(h.ev[2 * kPhases + 1]);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, h.ev[2 * kPhases], h.ev[2 * kPhases + 1]);
                if (r > 0) times.push_back(ms);
            }
        }
        phi.release();
        grad.release();
    }
    fmm_destroy(w);
    if (rc != FMM_OK) return rc;
    std::sort(times.begin(), times.end());
    *ms_out = times[times.size() / 2];
    return FMM_OK;
}

int fmm_tune_ncrit(int64_t N, int P, float theta, const double *x, const float *q, const int *candidates,
                   int ncand, int reps, const fmm_options *opt, int *best, double *ms_out)
{
    if (!x || !q || !candidates || ncand < 1 || reps < 1 || !best) {
        set_error("fmm_tune_ncrit: null argument or empty candidate list");
        return FMM_ERR_ARG;
    }
    double best_ms = 1e300;
    *best = candidates[0];
    for (int k = 0; k < ncand; ++k) {
        double ms = 0.0;
        FMM_TRY(time_config(N, P, theta, candidates[k], -1, x, q, reps, opt, &ms));
        if (ms_out) ms_out[k] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            *best = candidates[k];
        }
    }
    return FMM_OK;
}

int fmm_tune_hybrid(int64_t N, int P, float theta, int ncrit, const double *x, const float *q,
                    const int64_t *candidates, int ncand, int reps, const fmm_options *opt, int64_t *best,
                    double *ms_out)
{
    if (!x || !q || !candidates || ncand < 1 || reps < 1 || !best) {
        set_error("fmm_tune_hybrid: null argument or empty candidate list");
        return FMM_ERR_ARG;
    }
    double best_ms = 1e300;
    *best = candidates[0];
    for (int k = 0; k < ncand; ++k) {
        double ms = 0.0;
        FMM_TRY(time_config(N, P, theta, ncrit, candidates[k] < 0 ? -1 : candidates[k], x, q, reps, opt, &ms));
        if (ms_out) ms_out[k] = ms;
        if (ms < best_ms) {
            best_ms = ms;
            *best = candidates[k];
        }
    }
    return FMM_OK;
}

int fmm_stats(fmm_handle *w, struct fmm_stats *s)
{
    if (!w || !s) {
        set_error("fmm_stats: null argument");
        return FMM_ERR_ARG;
    }
    Handle &h = w->h;
    DeviceGuard guard(h.device);
    FMM_TRY(check_async_errors(h));
    std::memset(s, 0, sizeof(*s));
    s->n = h.N;
    s->ncells = h.ncells;
    s->nleaves = h.nleaves;
    s->nlevels = h.nlevels;
    s->P = h.P;
    s->n_m2l = h.n_m2l;
    s->n_p2p = h.n_p2p;
    s->p2p_pairs = h.p2p_pairs;
    s->kernel_launches = h.launches;
    if (h.events_ready) {
        FMM_CUDA(cudaStreamSynchronize(h.stream));
        s->ms_build = h.ms_build;
        float ms = 0.f;
        if (h.evaluated && cudaEventElapsedTime(&ms, h.ev[2 * kPhases + 2], h.ev[2 * kPhases + 3]) == cudaSuccess)
            s->ms_evaluate = ms;
        if (h.backward_done && cudaEventElapsedTime(&ms, h.ev[2 * kPhases + 4], h.ev[2 * kPhases + 5]) == cudaSuccess)
            s->ms_backward = ms;
        if (h.batch_done && cudaEventElapsedTime(&ms, h.ev[2 * kPhases + 6], h.ev[2 * kPhases + 7]) == cudaSuccess)
            s->ms_batch = ms;
        if (h.flags & FMM_FLAG_TIMING)
            for (int p = 0; p < kPhases; ++p) {
                ms = 0.f;
                if (cudaEventElapsedTime(&ms, h.ev[2 * p], h.ev[2 * p + 1]) == cudaSuccess) s->ms_phase[p] = ms;
            }
        cudaGetLastError();   // an unrecorded phase event is not an error of this call
    }
    return FMM_OK;
}

int fmm_get_norm(fmm_handle *w, double *centre, double *scale)
{
    if (!w || !centre || !scale) {
        set_error("fmm_get_norm: null argument");
        return FMM_ERR_ARG;
    }
    if (!w->h.built) {
        set_error("fmm_get_norm: no tree");
        return FMM_ERR_STATE;
    }
    for (int a = 0; a < 3; ++a) centre[a] = w->h.norm_host[a];
    *scale = w->h.norm_host[3];
    return FMM_OK;
}

int fmm_get_sorted(fmm_handle *w, uint64_t *keys, int32_t *perm)
{
    if (!w) {
        set_error("fmm_get_sorted: null handle");
        return FMM_ERR_ARG;
    }
    Handle &h = w->h;
    if (!h.built) {
        set_error("fmm_get_sorted: no tree");
        return FMM_ERR_STATE;
    }
    DeviceGuard guard(h.device);
    if (keys) FMM_CUDA(cudaMemcpyAsync(keys, h.keys.p, h.N * sizeof(uint64_t), cudaMemcpyDeviceToHost, h.stream));
    if (perm) FMM_CUDA(cudaMemcpyAsync(perm, h.perm.p, h.N * sizeof(int32_t), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    return FMM_OK;
}

int fmm_get_ncells(fmm_handle *w, int64_t *ncells)
{
    if (!w || !ncells) {
        set_error("fmm_get_ncells: null argument");
        return FMM_ERR_ARG;
    }
    if (!w->h.built) {
        set_error("fmm_get_ncells: no tree");
        return FMM_ERR_STATE;
    }
    *ncells = w->h.ncells;
    return FMM_OK;
}

int fmm_get_cells(fmm_handle *w, uint64_t *canon, int32_t *level, int32_t *pbeg, int32_t *pcnt, int32_t *nchild,
                  int32_t *parent, float *centre, float *radius)
{
    if (!w) {
        set_error("fmm_get_cells: null handle");
        return FMM_ERR_ARG;
    }
    Handle &h = w->h;
    if (!h.built) {
        set_error("fmm_get_cells: no tree");
        return FMM_ERR_STATE;
    }
    DeviceGuard guard(h.device);
    const int64_t nc = h.ncells;
    auto cp = [&](void *dst, const DevBuf &b, size_t bytes) -> int {
        if (!dst) return FMM_OK;
        FMM_CUDA(cudaMemcpyAsync(dst, b.p, bytes, cudaMemcpyDeviceToHost, h.stream));
        return FMM_OK;
    };
    std::vector<int32_t> lev(nc);
    std::vector<uint64_t> pre(canon ? nc : 0);
    FMM_TRY(cp(lev.data(), h.c_level, nc * sizeof(int32_t)));
    if (canon) FMM_TRY(cp(pre.data(), h.c_prefix, nc * sizeof(uint64_t)));
    FMM_TRY(cp(pbeg, h.c_pbeg, nc * sizeof(int32_t)));
    FMM_TRY(cp(pcnt, h.c_pcnt, nc * sizeof(int32_t)));
    FMM_TRY(cp(nchild, h.c_ccnt, nc * sizeof(int32_t)));
    FMM_TRY(cp(parent, h.c_parent, nc * sizeof(int32_t)));
    std::vector<float4> geom((centre || radius) ? nc : 0);
    if (centre || radius) FMM_TRY(cp(geom.data(), h.c_geom, nc * sizeof(float4)));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    for (int64_t c = 0; c < nc; ++c) {
        if (level) level[c] = lev[c];
        if (canon) canon[c] = (1ull << (3 * lev[c])) | pre[c];
        if (centre) {
            centre[3 * c + 0] = geom[c].x;
            centre[3 * c + 1] = geom[c].y;
            centre[3 * c + 2] = geom[c].z;
        }
        if (radius) radius[c] = geom[c].w;
    }
    return FMM_OK;
}

int fmm_get_lists(fmm_handle *w, int64_t *n_m2l, int64_t *n_p2p, int32_t *m2l, int32_t *p2p)
{
    if (!w) {
        set_error("fmm_get_lists: null handle");
        return FMM_ERR_ARG;
    }
    Handle &h = w->h;
    if (!h.built) {
        set_error("fmm_get_lists: no tree");
        return FMM_ERR_STATE;
    }
    DeviceGuard guard(h.device);
    if (n_m2l) *n_m2l = h.n_m2l;
    if (n_p2p) *n_p2p = h.n_p2p;
    const int64_t nc = h.ncells;
    auto expand = [&](int32_t *out, const DevBuf &src, const DevBuf &off, int64_t n) -> int {
        if (!out) return FMM_OK;
        std::vector<int32_t> s(n), o(nc + 1);
        if (n) FMM_CUDA(cudaMemcpyAsync(s.data(), src.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h.stream));
        FMM_CUDA(cudaMemcpyAsync(o.data(), off.p, (nc + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, h.stream));
        FMM_CUDA(cudaStreamSynchronize(h.stream));
        for (int64_t c = 0; c < nc; ++c)
            for (int32_t e = o[c]; e < o[c + 1]; ++e) {
                out[2 * (int64_t)e] = (int32_t)c;
                out[2 * (int64_t)e + 1] = s[e];
            }
        return FMM_OK;
    };
    FMM_TRY(expand(m2l, h.m2l_src, h.m2l_off, h.n_m2l));
    FMM_TRY(expand(p2p, h.p2p_src, h.p2p_off, h.n_p2p));
    return FMM_OK;
}

}  // extern "C"
