// api.cu -- the C ABI of include/sslic.h: parameter validation, workspace
// management and the orchestration of the kernels on the caller's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace sslic {

int set_error(sslic_ctx* c, int code, const char* fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_check(sslic_ctx* c, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return SSLIC_OK;
    return set_error(c, e == cudaErrorMemoryAllocation ? SSLIC_ENOMEM : SSLIC_ECUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

int prof_begin(sslic_ctx* c, int phase, cudaStream_t st)
{
    if (!c->prof_on) return -1;
    const size_t need = 2 * (c->prof.size() + 1);
    while (c->prof_pool.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        c->prof_pool.push_back(e);
    }
    ProfRec r;
    r.phase = phase;
    r.start = c->prof_pool[need - 2];
    r.stop = c->prof_pool[need - 1];
    if (cudaEventRecord(r.start, st) != cudaSuccess) return -1;
    c->prof.push_back(r);
    return (int)c->prof.size() - 1;
}

void prof_end(sslic_ctx* c, int rec, cudaStream_t st)
{
    if (rec < 0) return;
    cudaEventRecord(c->prof[rec].stop, st);
}

template <typename P>
static int dalloc(sslic_ctx* c, P** p, size_t count, const char* what)
{
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(P));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(c, SSLIC_ENOMEM, "cudaMalloc %s (%zu bytes): %s", what, count * sizeof(P),
                         cudaGetErrorString(e));
    }
    return SSLIC_OK;
}

template <typename P>
static void dfree(P*& p)
{
    if (p) cudaFree((void*)p);
    p = nullptr;
}

static int validate(const sslic_params* p, Geom* g)
{
    if (!p) return SSLIC_EINVAL;
    if (p->ndim < 1 || p->ndim > kMaxDims) return SSLIC_EINVAL;
    if (p->channels < 1 || p->channels > kMaxChannels) return SSLIC_EINVAL;
    if (p->dtype != SSLIC_U8 && p->dtype != SSLIC_U16 && p->dtype != SSLIC_F32) return SSLIC_EINVAL;
    if (!(p->m > 0.0f) || !std::isfinite(p->m)) return SSLIC_EINVAL;
    if (p->max_iter < 1) return SSLIC_EINVAL;
    if (p->perturb != 0 && p->perturb != 1) return SSLIC_EINVAL;
    if (p->enforce_connectivity != 0 && p->enforce_connectivity != 1) return SSLIC_EINVAL;
    if (p->precision != 0 && p->precision != 1) return SSLIC_EINVAL;
    if (p->precision == 1) {
        // the tensor-core feature term: float images with 32..128 channels, 2-D / 3-D
        if (p->channels < 32) return SSLIC_EINVAL;
        if (p->dtype != SSLIC_F32 || p->channels > 128 || (p->ndim != 2 && p->ndim != 3)) return SSLIC_EUNSUPPORTED;
    }
    Geom& G = *g;
    memset(&G, 0, sizeof(G));
    G.n = p->ndim;
    G.C = p->channels;
    G.dtype = p->dtype;
    G.CW = G.C + (G.n > 3 ? G.n : 3);
    G.AW = G.CW + 1;
    G.V = 1;
    G.K = 1;
    G.sprod = 1;
    const double m = (double)p->m;
    for (int d = 0; d < kMaxDims; ++d) {
        if (d < G.n) {
            if (p->size[d] < 1 || p->size[d] > (1 << 24)) return SSLIC_EINVAL;
            if (p->grid[d] < 1 || p->grid[d] > (1 << 24)) return SSLIC_EINVAL;
            G.N[d] = p->size[d];
            G.S[d] = p->grid[d];
            G.sprod *= G.S[d];
        } else {
            G.N[d] = 1;
            G.S[d] = 1;
        }
        G.nb[d] = (G.N[d] + G.S[d] - 1) / G.S[d];
        G.off[d] = (G.N[d] - 1 - (G.nb[d] - 1) * G.S[d]) / 2;
        G.V *= G.N[d];
        G.K *= G.nb[d];
        const double s = (double)G.S[d];
        G.w64[d] = (m * m) / (s * s);
        G.w[d] = (float)G.w64[d];
    }
    if (G.K >= (1LL << 30)) return SSLIC_EUNSUPPORTED;  // labels are int32, with room for new ones
    return SSLIC_OK;
}

int make_geom(const sslic_params* p, Geom* g)
{
    return validate(p, g);
}

int ensure_ccl_capacity(sslic_ctx* c, int64_t m)
{
    Workspace& w = c->ws;
    const Geom& g = c->g;
    int rc;
    if (!w.lid) {
        if ((rc = dalloc(c, &w.lid, (size_t)g.V, "component ids"))) return rc;
        w.lid_cap = g.V;
        w.n_ccl_tiles = ccl_num_tiles(g);
        if ((rc = dalloc(c, &w.tile_base, (size_t)w.n_ccl_tiles, "tile bases"))) return rc;
        if ((rc = dalloc(c, &w.tile_cnt, (size_t)w.n_ccl_tiles, "tile counts"))) return rc;
        if ((rc = dalloc(c, &w.counters, 4, "counters"))) return rc;
    }
    if (m <= w.m_cap) return SSLIC_OK;
    dfree(w.comp_label); dfree(w.gparent);
    dfree(w.root_size); dfree(w.root_first); dfree(w.fin); dfree(w.out_label); dfree(w.link);
    dfree(w.new_key); dfree(w.new_val);
    w.m_cap = 0;
    const size_t n = (size_t)m;
    if ((rc = dalloc(c, &w.comp_label, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.gparent, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.root_size, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.root_first, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.fin, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.out_label, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.link, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.new_key, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.new_val, n, "components"))) return rc;
    w.m_cap = m;
    return SSLIC_OK;
}

int grow_ccl_records(sslic_ctx* c, int64_t m, int64_t keep, cudaStream_t st)
{
    Workspace& w = c->ws;
    if (m <= w.m_cap) return SSLIC_OK;
    int rc;
    // the arrays the tile pass fills: copied; the later passes' arrays: fresh
    int* comp_label = nullptr;
    int* gparent = nullptr;
    unsigned long long* root_size = nullptr;
    unsigned long long* root_first = nullptr;
    uint8_t* fin = nullptr;
    const size_t n = (size_t)m;
    if ((rc = dalloc(c, &comp_label, n, "components")) || (rc = dalloc(c, &gparent, n, "components")) ||
        (rc = dalloc(c, &root_size, n, "components")) || (rc = dalloc(c, &root_first, n, "components")) ||
        (rc = dalloc(c, &fin, n, "components"))) {
        dfree(comp_label); dfree(gparent); dfree(root_size); dfree(root_first); dfree(fin);
        return rc;
    }
    const size_t k = (size_t)keep;
    if (k > 0 &&
        ((rc = cuda_check(c, cudaMemcpyAsync(comp_label, w.comp_label, k * sizeof(int), cudaMemcpyDeviceToDevice, st), "grow")) ||
         (rc = cuda_check(c, cudaMemcpyAsync(gparent, w.gparent, k * sizeof(int), cudaMemcpyDeviceToDevice, st), "grow")) ||
         (rc = cuda_check(c, cudaMemcpyAsync(root_size, w.root_size, k * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st), "grow")) ||
         (rc = cuda_check(c, cudaMemcpyAsync(root_first, w.root_first, k * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st), "grow")) ||
         (rc = cuda_check(c, cudaMemcpyAsync(fin, w.fin, k, cudaMemcpyDeviceToDevice, st), "grow")) ||
         (rc = cuda_check(c, cudaStreamSynchronize(st), "sync")))) {
        dfree(comp_label); dfree(gparent); dfree(root_size); dfree(root_first); dfree(fin);
        return rc;
    }
    dfree(w.comp_label); dfree(w.gparent); dfree(w.root_size); dfree(w.root_first); dfree(w.fin);
    w.comp_label = comp_label; w.gparent = gparent; w.root_size = root_size; w.root_first = root_first; w.fin = fin;
    dfree(w.out_label); dfree(w.link); dfree(w.new_key); dfree(w.new_val);
    w.m_cap = 0;
    if ((rc = dalloc(c, &w.out_label, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.link, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.new_key, n, "components"))) return rc;
    if ((rc = dalloc(c, &w.new_val, n, "components"))) return rc;
    w.m_cap = m;
    return SSLIC_OK;
}

int ensure_conn_slab_scratch(sslic_ctx* c)
{
    Workspace& w = c->ws;
    const Geom& g = c->g;
    int rc;
    if (!w.conn_seed && (rc = dalloc(c, &w.conn_seed, (size_t)g.K, "connectivity seeds"))) return rc;
    if (!w.conn_carry) {
        int64_t plane = 1;
        for (int d = 0; d < g.n - 1; ++d) plane *= g.N[d];
        if ((rc = dalloc(c, &w.conn_carry, (size_t)(g.S[g.n - 1] * plane), "connectivity carry"))) return rc;
    }
    return SSLIC_OK;
}

static void free_all(sslic_ctx* c)
{
    Workspace& w = c->ws;
    dfree(w.ctr); dfree(w.acc); dfree(w.facc); dfree(w.resid_k); dfree(w.nonempty_k);
    dfree(w.resid_part); dfree(w.resid_cnt_part); dfree(w.resid_out);
    dfree(w.bin_count); dfree(w.bin_start); dfree(w.bin_cursor); dfree(w.bin_items); dfree(w.bin_of);
    dfree(w.scan_tmp); dfree(w.ovf_tiles); dfree(w.ovf_count); dfree(w.tile_lists); dfree(w.hc_err); dfree(w.hc_rechecks);
    dfree(w.lid); dfree(w.tile_base); dfree(w.tile_cnt); dfree(w.counters);
    dfree(w.comp_label); dfree(w.gparent);
    dfree(w.root_size); dfree(w.root_first); dfree(w.fin); dfree(w.out_label); dfree(w.link);
    dfree(w.new_key); dfree(w.new_val); dfree(w.sort_key); dfree(w.sort_val);
    dfree(w.img_dev); dfree(w.lab_dev); dfree(w.cen_dev);
    dfree(w.conn_seed); dfree(w.conn_carry);
    for (int i = 0; i < 2; ++i) { dfree(w.slab_img[i]); dfree(w.slab_lab[i]); }
    for (int i = 0; i < 8; ++i)
        if (w.slab_ev[i]) { cudaEventDestroy(w.slab_ev[i]); w.slab_ev[i] = nullptr; }
    if (w.copy_stream) { cudaStreamDestroy(w.copy_stream); w.copy_stream = nullptr; }
    if (w.down_stream) { cudaStreamDestroy(w.down_stream); w.down_stream = nullptr; }
}

sslic_ctx* conn_ctx_create(int device, int sms)
{
    sslic_ctx* c = new (std::nothrow) sslic_ctx();
    if (!c) return nullptr;
    c->device = device;
    c->sms = sms;
    c->loop_graph = 0;
    return c;
}

int conn_ctx_run(sslic_ctx* c, const sslic_params& p, const Geom& g, const float* ctr, int32_t* labels,
                 cudaStream_t st, int64_t* num_labels)
{
    Workspace& w = c->ws;
    c->p = p;
    c->g = g;
    // the per-voxel ids and per-tile arrays follow the largest image so far
    if (w.lid && (g.V > w.lid_cap || ccl_num_tiles(g) > w.n_ccl_tiles)) {
        dfree(w.lid); dfree(w.tile_base); dfree(w.tile_cnt); dfree(w.counters);
        w.lid_cap = 0;
        w.n_ccl_tiles = 0;
    }
    int rc = ensure_ccl_capacity(c, 32 * g.K + g.V / 1024 + 4096);
    if (rc) return rc;
    w.ctr = const_cast<float*>(ctr);  // read by phase 1 only; borrowed for the call
    rc = run_connectivity(c, labels, labels, st, num_labels);
    w.ctr = nullptr;
    return rc;
}

void conn_ctx_destroy(sslic_ctx* c)
{
    if (!c) return;
    c->ws.ctr = nullptr;
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    free_all(c);
    delete c;
}

static int alloc_core(sslic_ctx* c)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    int rc;
    const size_t K = (size_t)g.K;
    if ((rc = dalloc(c, &w.ctr, K * g.CW, "centres"))) return rc;
    if ((rc = dalloc(c, &w.acc, K * g.AW, "sums"))) return rc;
    if (g.dtype == SSLIC_F32 && (rc = dalloc(c, &w.facc, K * g.C, "float sums"))) return rc;
    if ((rc = dalloc(c, &w.resid_k, K, "residual"))) return rc;
    if ((rc = dalloc(c, &w.nonempty_k, K, "residual"))) return rc;
    if ((rc = dalloc(c, &w.resid_part, 256, "residual"))) return rc;
    if ((rc = dalloc(c, &w.resid_cnt_part, 256, "residual"))) return rc;
    if ((rc = dalloc(c, &w.resid_out, 1, "residual"))) return rc;
    if ((rc = dalloc(c, &w.bin_count, K + 1, "bins"))) return rc;
    if ((rc = dalloc(c, &w.bin_start, K + 1, "bins"))) return rc;
    if ((rc = dalloc(c, &w.bin_cursor, K, "bins"))) return rc;
    if ((rc = dalloc(c, &w.bin_items, K, "bins"))) return rc;
    if ((rc = dalloc(c, &w.bin_of, K, "bins"))) return rc;
    w.scan_tmp_len = scan_tmp_needed((int64_t)K + 1);
    if ((rc = dalloc(c, &w.scan_tmp, w.scan_tmp_len, "scan"))) return rc;
    w.n_assign_tiles = assign_num_tiles(g);
    if (hc_applies(g)) w.n_assign_tiles = imax64(w.n_assign_tiles, hc_num_tiles(g));
    if ((rc = dalloc(c, &w.hc_err, 1, "status"))) return rc;
    if ((rc = dalloc(c, &w.hc_rechecks, 1, "counters"))) return rc;
    if ((rc = cuda_check(c, cudaMemset(w.hc_err, 0, sizeof(unsigned)), "memset"))) return rc;
    if ((rc = cuda_check(c, cudaMemset(w.hc_rechecks, 0, sizeof(unsigned long long)), "memset"))) return rc;
    if ((rc = dalloc(c, &w.ovf_tiles, (size_t)w.n_assign_tiles, "tiles"))) return rc;
    if ((rc = dalloc(c, &w.ovf_count, 1, "tiles"))) return rc;
    {
        // candidate records for the tile kernels (the largest tiling any shape makes)
        int64_t nrec = has_tile_kernel(g) ? assign_num_tiles(g) : 0;
        if (hc_applies(g)) nrec = imax64(nrec, hc_num_tiles(g));
        if (nrec > 0 && (rc = dalloc(c, &w.tile_lists, (size_t)nrec * tile_list_stride(), "tile lists"))) return rc;
    }
    if ((rc = cuda_check(c, cudaMemset(w.acc, 0, K * g.AW * sizeof(unsigned long long)), "memset sums"))) return rc;
    if (w.facc && (rc = cuda_check(c, cudaMemset(w.facc, 0, K * g.C * sizeof(double)), "memset sums"))) return rc;
    if ((rc = cuda_check(c, cudaMemset(w.resid_out, 0, sizeof(double)), "memset"))) return rc;
    if (c->p.enforce_connectivity) {
        // components: about a dozen local pieces per cluster; grown on demand
        if ((rc = ensure_ccl_capacity(c, 32 * (int64_t)K + g.V / 1024 + 4096))) return rc;
    }
    return SSLIC_OK;
}

// bounded device waits (tensor-core MMA completion, TMA copies): a wait
// that ran out is reported (and its flag cleared) after the stream drains
static int check_precision_status(sslic_ctx* c, cudaStream_t st)
{
    if (c->p.precision != 1 && !c->status_pending) return SSLIC_OK;
    c->status_pending = 0;
    unsigned h = 0;
    int rc = cuda_check(c, cudaMemcpyAsync(&h, c->ws.hc_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                        "read status");
    if (!rc) rc = cuda_check(c, cudaStreamSynchronize(st), "sync");
    if (rc) return rc;
    if (h) {
        cudaMemsetAsync(c->ws.hc_err, 0, sizeof(unsigned), st);
        return set_error(c, SSLIC_ETIMEOUT, "assignment: a bounded device wait ran out");
    }
    return SSLIC_OK;
}

static int read_residual(sslic_ctx* c, cudaStream_t st, double* r)
{
    int rc = cuda_check(c, cudaMemcpyAsync(r, c->ws.resid_out, sizeof(double), cudaMemcpyDeviceToHost, st),
                        "read residual");
    if (rc) return rc;
    return cuda_check(c, cudaStreamSynchronize(st), "sync");
}

// A fixed number of iterations (no convergence threshold, so no host read
// between them) launches the same dozen small kernels every iteration; on
// small images their launch latency is most of the run.  The first iteration
// runs eagerly (it sets kernel attributes and leaves nothing to allocate),
// the next is captured from a private stream into a graph, and the graph is
// replayed for the rest.  The cached executable graph is updated in place
// when the new capture has its topology (other buffers, same tile shape), else
// instantiated anew.  Phase timing records events per launch, so it runs
// eagerly.
static bool loop_graph_applies(const sslic_ctx* c)
{
    return c->loop_graph && !c->prof_on && !(c->p.conv_threshold > 0.0) && c->p.max_iter >= 2;
}

static int capture_iteration(sslic_ctx* c, const void* image, int32_t* labels, int64_t* per_iter)
{
    int rc;
    if (!c->cap_stream &&
        (rc = cuda_check(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream")))
        return rc;
    const int64_t l0 = c->launches;
    if ((rc = cuda_check(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed), "begin capture")))
        return rc;
    rc = build_bins(c, c->cap_stream);
    if (!rc) rc = launch_assign_update(c, image, labels, c->cap_stream);
    if (!rc) rc = launch_finalize(c, c->cap_stream, false);  // the residual follows the last replay
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    *per_iter = c->launches - l0;
    c->launches = l0;
    if (!rc) rc = cuda_check(c, e, "end capture");
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (c->loop_exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(c->loop_exec, graph, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(c->loop_exec);
            c->loop_exec = nullptr;
        }
    }
    if (!c->loop_exec) rc = cuda_check(c, cudaGraphInstantiate(&c->loop_exec, graph, 0), "instantiate graph");
    cudaGraphDestroy(graph);
    return rc;
}

// the loop of Sec. 3.1 from the centres already in the workspace
// (first_it iterations already ran, e.g. overlapped with the upload)
static int run_loop(sslic_ctx* c, const void* image, int32_t* labels, float* centres, cudaStream_t st,
                    sslic_result* out, int first_it = 0)
{
    int rc;
    int it = 0;
    double res = 0.0;
    const bool graph = loop_graph_applies(c);
    bool stop = false;
    if (first_it > 0 && c->p.conv_threshold > 0.0) {
        if ((rc = read_residual(c, st, &res))) return rc;
        stop = res < c->p.conv_threshold;
    }
    for (it = first_it; !stop && it < c->p.max_iter; ++it) {
        if (graph && it == 1) {
            int64_t per_iter = 0;
            if ((rc = capture_iteration(c, image, labels, &per_iter))) return rc;
            for (; it < c->p.max_iter; ++it) {
                if ((rc = cuda_check(c, cudaGraphLaunch(c->loop_exec, st), "graph launch"))) return rc;
                count_launch(c, (int)per_iter);
            }
            if ((rc = launch_residual(c, st))) return rc;
            break;
        }
        if ((rc = build_bins(c, st))) return rc;
        if ((rc = launch_assign_update(c, image, labels, st))) return rc;
        // without a threshold only the last iteration's residual is reported
        if ((rc = launch_finalize(c, st, c->p.conv_threshold > 0.0 || it == c->p.max_iter - 1))) return rc;
        if (c->p.conv_threshold > 0.0) {
            if ((rc = read_residual(c, st, &res))) return rc;
            if (res < c->p.conv_threshold) { ++it; break; }
        }
    }
    if ((rc = check_precision_status(c, st))) return rc;
    int64_t nlab = c->g.K;
    if (c->p.enforce_connectivity) {
        if ((rc = ensure_ccl_capacity(c, 32 * c->g.K + c->g.V / 1024 + 4096))) return rc;
        if ((rc = run_connectivity(c, labels, labels, st, &nlab))) return rc;
    }
    if (centres && (rc = launch_export_centres(c, centres, st))) return rc;
    if (out) {
        if ((rc = read_residual(c, st, &res))) return rc;
        out->num_clusters = c->g.K;
        out->num_labels = nlab;
        out->iterations = it;
        out->residual = res;
    }
    return SSLIC_OK;
}

}  // namespace sslic

using namespace sslic;

extern "C" {

int sslic_default_params(int32_t ndim, sslic_params* p)
{
    if (!p || ndim < 1 || ndim > kMaxDims) return SSLIC_EINVAL;
    memset(p, 0, sizeof(*p));
    p->ndim = ndim;
    for (int d = 0; d < 4; ++d) {
        p->size[d] = 1;
        p->grid[d] = d < ndim ? 16 : 1;
    }
    p->channels = 3;
    p->dtype = SSLIC_U8;
    p->m = 10.0f;
    p->max_iter = ndim >= 3 ? 5 : 10;
    p->conv_threshold = 0.0;
    p->perturb = 1;
    p->enforce_connectivity = 1;
    p->precision = 0;
    return SSLIC_OK;
}

int sslic_create(const sslic_params* p, sslic_ctx** out)
{
    if (!out) return SSLIC_EINVAL;
    *out = nullptr;
    Geom g;
    int rc = validate(p, &g);
    if (rc) return rc;
    sslic_ctx* c = new (std::nothrow) sslic_ctx();
    if (!c) return SSLIC_ENOMEM;
    c->p = *p;
    c->g = g;
    if ((rc = cuda_check(c, cudaGetDevice(&c->device), "cudaGetDevice")) ||
        (rc = cuda_check(c, cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device),
                         "SM count"))) {
        delete c;
        return rc;
    }
    if ((rc = alloc_core(c))) {
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return SSLIC_OK;
}

int sslic_num_clusters(const sslic_ctx* c, int64_t* K)
{
    if (!c || !K) return SSLIC_EINVAL;
    *K = c->g.K;
    return SSLIC_OK;
}

int sslic_run(sslic_ctx* c, const void* image_dev, int32_t* labels_dev, float* centres_dev, void* stream,
              sslic_result* out)
{
    if (!c || !image_dev || !labels_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_seed(c, image_dev, st);
    if (rc) return rc;
    return run_loop(c, image_dev, labels_dev, centres_dev, st, out);
}

int sslic_run_from(sslic_ctx* c, const void* image_dev, const float* init_centres_dev, int32_t* labels_dev,
                   float* centres_dev, void* stream, sslic_result* out)
{
    if (!c || !image_dev || !labels_dev || !init_centres_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_import_centres(c, init_centres_dev, st);
    if (rc) return rc;
    return run_loop(c, image_dev, labels_dev, centres_dev, st, out);
}

}  // extern "C"

namespace sslic {

// sslic_run_host's upload overlapped with seeding and the first iteration:
// images whose slabs along the last axis take the slab-restricted assignment
// launches, with lattice rows at least 8 planes apart and at least two slabs
static constexpr int64_t kHostSlab = 64;  // planes per slab: a multiple of every tile extent along that axis
static bool host_pipeline_applies(const sslic_ctx* c)
{
    const Geom& g = c->g;
    return (g.n == 2 || g.n == 3) && !hc_applies(g) && !c->p.precision && g.S[g.n - 1] >= 8 &&
           c->p.max_iter >= 1 && g.N[g.n - 1] >= 2 * kHostSlab;
}

// On the context's copy stream: first the planes that seeding reads (the
// lattice planes along the last axis and, with the perturbation, two on each
// side of them: its gradients' reach), then the rest slab by slab.  Seeding
// and the bins start once the first part is in; each slab's assignment of the
// first iteration starts once its planes are in.  Integer images: each slab
// adds its exact sums, so labels and centres equal the unsplit launch's.
static int host_upload_first_iteration(sslic_ctx* c, const void* image_host, cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    int rc;
    if (!w.copy_stream &&
        (rc = cuda_check(c, cudaStreamCreateWithFlags(&w.copy_stream, cudaStreamNonBlocking), "copy stream")))
        return rc;
    for (int i = 0; i < 2; ++i)
        if (!w.slab_ev[i] &&
            (rc = cuda_check(c, cudaEventCreateWithFlags(&w.slab_ev[i], cudaEventDisableTiming), "events")))
            return rc;
    cudaStream_t cs = w.copy_stream;
    const int ax = g.n - 1;
    const int64_t NL = g.N[ax];
    int64_t plane = 1;
    for (int d = 0; d < ax; ++d) plane *= g.N[d];
    const size_t esz = g.dtype == SSLIC_U8 ? 1 : (g.dtype == SSLIC_U16 ? 2 : 4);
    const size_t pbytes = (size_t)plane * g.C * esz;
    const unsigned char* src = (const unsigned char*)image_host;
    unsigned char* dst = (unsigned char*)w.img_dev;
    auto put = [&](int64_t a, int64_t b) {
        return cuda_check(c, cudaMemcpyAsync(dst + a * pbytes, src + a * pbytes, (size_t)(b - a) * pbytes,
                                             cudaMemcpyHostToDevice, cs),
                          "H2D");
    };
    // st waits for what is on cs so far
    auto ready = [&]() {
        int r = cuda_check(c, cudaEventRecord(w.slab_ev[1], cs), "event");
        return r ? r : cuda_check(c, cudaStreamWaitEvent(st, w.slab_ev[1], 0), "wait");
    };
    // the copies start after the work the caller queued on st
    if ((rc = cuda_check(c, cudaEventRecord(w.slab_ev[0], st), "event")) ||
        (rc = cuda_check(c, cudaStreamWaitEvent(cs, w.slab_ev[0], 0), "wait")))
        return rc;
    // 1. the planes seeding reads, as ascending disjoint intervals
    const int64_t reach = c->p.perturb ? 2 : 0;
    std::vector<int64_t> iv_lo, iv_hi;
    for (int64_t j = 0; j < g.nb[ax]; ++j) {
        const int64_t z = g.off[ax] + j * g.S[ax];
        const int64_t a = imax64(0, z - reach), b = imin64(NL, z + reach + 1);
        if (!iv_hi.empty() && a <= iv_hi.back()) {
            iv_hi.back() = imax64(iv_hi.back(), b);
        } else {
            iv_lo.push_back(a);
            iv_hi.push_back(b);
        }
    }
    const int niv = (int)iv_lo.size();
    for (int i = 0; i < niv; ++i)
        if ((rc = put(iv_lo[i], iv_hi[i]))) return rc;
    if ((rc = ready())) return rc;
    if ((rc = launch_seed(c, w.img_dev, st))) return rc;
    if ((rc = build_bins(c, st))) return rc;
    // 2. the first iteration slab by slab, each behind the rest of its planes
    int iv = 0;
    for (int64_t lo = 0; lo < NL; lo += kHostSlab) {
        const int64_t hi = imin64(NL, lo + kHostSlab);
        int64_t p = lo;
        for (; iv < niv && iv_lo[iv] < hi; ++iv) {
            if (iv_hi[iv] <= p) continue;
            if (iv_lo[iv] > p && (rc = put(p, iv_lo[iv]))) return rc;
            p = imax64(p, iv_hi[iv]);
            if (iv_hi[iv] > hi) break;  // the interval runs into the next slab
        }
        if (p < hi && (rc = put(p, hi))) return rc;
        if ((rc = ready())) return rc;
        const Slab sl{lo, hi};
        if ((rc = launch_assign_update(c, w.img_dev, w.lab_dev, st, &sl))) return rc;
    }
    return launch_finalize(c, st, c->p.conv_threshold > 0.0 || c->p.max_iter == 1);
}

}  // namespace sslic

extern "C" {

int sslic_run_host(sslic_ctx* c, const void* image_host, int32_t* labels_host, float* centres_host, void* stream,
                   sslic_result* out)
{
    if (!c || !image_host || !labels_host) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    const Geom& g = c->g;
    Workspace& w = c->ws;
    const size_t esz = g.dtype == SSLIC_U8 ? 1 : (g.dtype == SSLIC_U16 ? 2 : 4);
    const size_t img_bytes = (size_t)g.V * g.C * esz;
    const size_t lab_bytes = (size_t)g.V * sizeof(int32_t);
    const size_t cen_bytes = (size_t)g.K * (g.C + g.n) * sizeof(float);
    int rc;
    if (!w.img_dev) {
        if ((rc = dalloc(c, (char**)&w.img_dev, img_bytes, "image"))) return rc;
        if ((rc = dalloc(c, &w.lab_dev, (size_t)g.V, "labels"))) return rc;
        if ((rc = dalloc(c, &w.cen_dev, (size_t)g.K * (g.C + g.n), "centres"))) return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int first = 0;
    if (host_pipeline_applies(c)) {
        if ((rc = host_upload_first_iteration(c, image_host, st))) return rc;
        first = 1;
    } else {
        if ((rc = cuda_check(c, cudaMemcpyAsync(w.img_dev, image_host, img_bytes, cudaMemcpyHostToDevice, st),
                             "H2D")))
            return rc;
        if ((rc = launch_seed(c, w.img_dev, st))) return rc;
    }
    sslic_result r;
    // with connectivity the relabel pass sends the labels itself, slab by slab
    c->relabel_host = c->p.enforce_connectivity && (g.n == 2 || g.n == 3) ? labels_host : nullptr;
    c->relabel_sent = 0;
    rc = run_loop(c, w.img_dev, w.lab_dev, centres_host ? w.cen_dev : nullptr, st, &r, first);
    c->relabel_host = nullptr;
    if (c->relabel_sent) {
        const int rs = cuda_check(c, cudaStreamSynchronize(w.down_stream), "sync");
        if (!rc) rc = rs;
    }
    if (rc) return rc;
    if (!c->relabel_sent &&
        (rc = cuda_check(c, cudaMemcpyAsync(labels_host, w.lab_dev, lab_bytes, cudaMemcpyDeviceToHost, st), "D2H")))
        return rc;
    if (centres_host &&
        (rc = cuda_check(c, cudaMemcpyAsync(centres_host, w.cen_dev, cen_bytes, cudaMemcpyDeviceToHost, st), "D2H")))
        return rc;
    if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
    if (out) *out = r;
    return SSLIC_OK;
}

int sslic_run_streamed(sslic_ctx* c, const void* image_host, int32_t* labels_host, float* centres_host,
                       int64_t slab_planes, void* stream, sslic_result* out)
{
    if (!c || !image_host || !labels_host) return SSLIC_EINVAL;
    const Geom& g = c->g;
    if (g.n != 2 && g.n != 3) return set_error(c, SSLIC_EUNSUPPORTED, "streamed form: 2-D and 3-D images");
    if (c->p.precision) return set_error(c, SSLIC_EUNSUPPORTED, "streamed form: no precision form");
    if (slab_planes < 32 || slab_planes % 32 != 0)
        return set_error(c, SSLIC_EINVAL, "slab depth must be a positive multiple of 32 planes");
    if (c->p.enforce_connectivity && ((g.n == 2 && slab_planes % 64 != 0) || slab_planes < g.S[g.n - 1]))
        return set_error(c, SSLIC_EINVAL,
                         "streamed connectivity: slabs of a multiple of 64 rows (2-D) and at least S planes");
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    Workspace& w = c->ws;
    const int ax = g.n - 1;                      // the last axis: slabs are ranges of its planes
    const int64_t NL = g.N[ax];
    int64_t plane = 1;
    for (int d = 0; d < ax; ++d) plane *= g.N[d];
    const size_t esz = g.dtype == SSLIC_U8 ? 1 : (g.dtype == SSLIC_U16 ? 2 : 4);
    const size_t pbytes = (size_t)plane * g.C * esz;  // image bytes per plane
    const int64_t depth = imin64(slab_planes, NL);
    int rc;
    if (w.slab_planes < depth + 4) {
        for (int i = 0; i < 2; ++i) { dfree(w.slab_img[i]); dfree(w.slab_lab[i]); }
        w.slab_planes = 0;
        for (int i = 0; i < 2; ++i) {
            if ((rc = dalloc(c, &w.slab_img[i], (size_t)(depth + 4) * pbytes, "slab buffers"))) return rc;
            if ((rc = dalloc(c, &w.slab_lab[i], (size_t)depth * plane, "slab buffers"))) return rc;
        }
        w.slab_planes = depth + 4;
    }
    if (!w.copy_stream &&
        (rc = cuda_check(c, cudaStreamCreateWithFlags(&w.copy_stream, cudaStreamNonBlocking), "copy stream")))
        return rc;
    if (!w.down_stream &&
        (rc = cuda_check(c, cudaStreamCreateWithFlags(&w.down_stream, cudaStreamNonBlocking), "copy stream")))
        return rc;
    for (int i = 0; i < 8; ++i)
        if (!w.slab_ev[i] &&
            (rc = cuda_check(c, cudaEventCreateWithFlags(&w.slab_ev[i], cudaEventDisableTiming), "events")))
            return rc;
    cudaStream_t st = (cudaStream_t)stream, cs = w.copy_stream, ds = w.down_stream;
    cudaEvent_t* img_ready = w.slab_ev;      // [2]: recorded on cs after a buffer's upload
    cudaEvent_t* img_free = w.slab_ev + 2;   // [2]: recorded on st after the kernels that read it
    cudaEvent_t* lab_done = w.slab_ev + 4;   // [2]: recorded on st after the kernels that write it
    cudaEvent_t* lab_free = w.slab_ev + 6;   // [2]: recorded on cs after its download
    for (int i = 0; i < 2; ++i) {
        if ((rc = cuda_check(c, cudaEventRecord(img_free[i], st), "event"))) return rc;
        if ((rc = cuda_check(c, cudaEventRecord(lab_free[i], st), "event"))) return rc;
    }
    const int64_t nslab = (NL + depth - 1) / depth;
    // upload planes [a, b) of the image into buffer i, after its previous readers
    auto upload = [&](int i, int64_t a, int64_t bnd) -> int {
        int r;
        if ((r = cuda_check(c, cudaStreamWaitEvent(cs, img_free[i], 0), "wait"))) return r;
        if ((r = cuda_check(c, cudaMemcpyAsync(w.slab_img[i], (const unsigned char*)image_host + a * pbytes,
                                               (size_t)(bnd - a) * pbytes, cudaMemcpyHostToDevice, cs),
                            "slab upload")))
            return r;
        if ((r = cuda_check(c, cudaEventRecord(img_ready[i], cs), "event"))) return r;
        return cuda_check(c, cudaStreamWaitEvent(st, img_ready[i], 0), "wait");
    };
    // seeding reads the planes within two of a seed plane (the perturbation's
    // gradients): with S >= 8 along the last axis, only those five planes per
    // lattice row go up; with finer grids, whole slabs with a two-plane halo
    const int64_t S_l = g.S[ax];
    const int64_t nrow = S_l >= 8 ? g.nb[ax] : nslab;
    for (int64_t s = 0; s < nrow; ++s) {
        const int i = (int)(s & 1);
        int64_t lo, hi;
        if (S_l >= 8) {
            lo = g.off[ax] + s * S_l;  // the lattice row's plane
            hi = lo + 1;
        } else {
            lo = s * depth;
            hi = imin64(NL, lo + depth);
        }
        const int64_t a = imax64(0, lo - 2), bnd = imin64(NL, hi + 2);
        if ((rc = upload(i, a, bnd))) return rc;
        const Slab sl{lo, hi};
        if ((rc = launch_seed(c, w.slab_img[i] - a * pbytes, st, &sl))) return rc;
        if ((rc = cuda_check(c, cudaEventRecord(img_free[i], st), "event"))) return rc;
    }
    // iterations: every slab's assignment adds its exact sums to the centres' sums
    int it = 0;
    double res = 0.0;
    const bool thr = c->p.conv_threshold > 0.0;
    for (it = 0; it < c->p.max_iter; ++it) {
        const bool keep = thr || it == c->p.max_iter - 1;  // labels that may be the result go back
        if ((rc = build_bins(c, st))) return rc;
        for (int64_t s = 0; s < nslab; ++s) {
            const int i = (int)(s & 1);
            const int64_t lo = s * depth, hi = imin64(NL, lo + depth);
            if ((rc = upload(i, lo, hi))) return rc;
            if ((rc = cuda_check(c, cudaStreamWaitEvent(st, lab_free[i], 0), "wait"))) return rc;
            const Slab sl{lo, hi};
            if ((rc = launch_assign_update(c, w.slab_img[i] - lo * pbytes, w.slab_lab[i] - lo * plane, st, &sl)))
                return rc;
            if ((rc = cuda_check(c, cudaEventRecord(img_free[i], st), "event"))) return rc;
            if ((rc = cuda_check(c, cudaEventRecord(lab_done[i], st), "event"))) return rc;
            if (keep) {
                if ((rc = cuda_check(c, cudaStreamWaitEvent(ds, lab_done[i], 0), "wait"))) return rc;
                if ((rc = cuda_check(c, cudaMemcpyAsync(labels_host + lo * plane, w.slab_lab[i],
                                                        (size_t)(hi - lo) * plane * sizeof(int32_t),
                                                        cudaMemcpyDeviceToHost, ds),
                                     "slab labels")))
                    return rc;
                if ((rc = cuda_check(c, cudaEventRecord(lab_free[i], ds), "event"))) return rc;
            }
        }
        if ((rc = launch_finalize(c, st, thr || it == c->p.max_iter - 1))) return rc;
        if (thr) {
            if ((rc = read_residual(c, st, &res))) return rc;
            if (res < c->p.conv_threshold) { ++it; break; }
        }
    }
    if (centres_host) {
        if (!w.cen_dev && (rc = dalloc(c, &w.cen_dev, (size_t)g.K * (g.C + g.n), "centres"))) return rc;
        if ((rc = launch_export_centres(c, w.cen_dev, st))) return rc;
        if ((rc = cuda_check(c, cudaMemcpyAsync(centres_host, w.cen_dev, (size_t)g.K * (g.C + g.n) * sizeof(float),
                                                cudaMemcpyDeviceToHost, st),
                             "D2H")))
            return rc;
    }
    if ((rc = read_residual(c, st, &res))) return rc;
    if ((rc = cuda_check(c, cudaStreamSynchronize(ds), "sync"))) return rc;
    if ((rc = cuda_check(c, cudaStreamSynchronize(cs), "sync"))) return rc;
    if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
    int64_t num_labels = g.K;
    if (c->p.enforce_connectivity) {
        // connectivity slab by slab (Sec. 3.1 stage 3): the labels of each
        // slab go up once for the components and once more, relabelled, come
        // back; the component records and ids of the whole image stay on the
        // device
        const int pr = prof_begin(c, SSLIC_PHASE_CONNECTIVITY, st);
        if ((rc = conn_slabs_begin(c, st))) return rc;
        for (int64_t s = 0; s < nslab; ++s) {
            const int64_t lo = s * depth, hi = imin64(NL, lo + depth);
            if ((rc = cuda_check(c, cudaMemcpyAsync(w.slab_lab[0], labels_host + lo * plane,
                                                    (size_t)(hi - lo) * plane * sizeof(int32_t),
                                                    cudaMemcpyHostToDevice, st),
                                 "slab labels up")))
                return rc;
            if ((rc = conn_slabs_add(c, w.slab_lab[0], lo, hi, st))) return rc;
        }
        if ((rc = conn_slabs_finish(c, st, &num_labels))) return rc;
        for (int64_t s = 0; s < nslab; ++s) {
            const int i = (int)(s & 1);
            const int64_t lo = s * depth, hi = imin64(NL, lo + depth);
            if ((rc = cuda_check(c, cudaStreamWaitEvent(st, lab_free[i], 0), "wait"))) return rc;
            if ((rc = conn_slabs_relabel(c, w.slab_lab[i], lo, hi, st))) return rc;
            if ((rc = cuda_check(c, cudaEventRecord(lab_done[i], st), "event"))) return rc;
            if ((rc = cuda_check(c, cudaStreamWaitEvent(ds, lab_done[i], 0), "wait"))) return rc;
            if ((rc = cuda_check(c, cudaMemcpyAsync(labels_host + lo * plane, w.slab_lab[i],
                                                    (size_t)(hi - lo) * plane * sizeof(int32_t),
                                                    cudaMemcpyDeviceToHost, ds),
                                 "slab labels down")))
                return rc;
            if ((rc = cuda_check(c, cudaEventRecord(lab_free[i], ds), "event"))) return rc;
        }
        if ((rc = cuda_check(c, cudaStreamSynchronize(ds), "sync"))) return rc;
        if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
        prof_end(c, pr, st);
    }
    if (out) {
        out->num_clusters = g.K;
        out->num_labels = num_labels;
        out->iterations = it;
        out->residual = res;
    }
    return SSLIC_OK;
}

int sslic_seed(sslic_ctx* c, const void* image_dev, float* centres_dev, void* stream)
{
    if (!c || !image_dev || !centres_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = launch_seed(c, image_dev, st);
    if (rc) return rc;
    return launch_export_centres(c, centres_dev, st);
}

int sslic_iterate(sslic_ctx* c, const void* image_dev, const float* centres_in_dev, int32_t* labels_dev,
                  float* centres_out_dev, void* stream, double* residual_host)
{
    if (!c || !image_dev || !centres_in_dev || !labels_dev || !centres_out_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = launch_import_centres(c, centres_in_dev, st))) return rc;
    if ((rc = build_bins(c, st))) return rc;
    if ((rc = launch_assign_update(c, image_dev, labels_dev, st))) return rc;
    if ((rc = launch_finalize(c, st))) return rc;
    if ((rc = launch_export_centres(c, centres_out_dev, st))) return rc;
    if ((rc = check_precision_status(c, st))) return rc;
    if (residual_host) return read_residual(c, st, residual_host);
    return SSLIC_OK;
}

int sslic_connectivity(sslic_ctx* c, const float* centres_dev, const int32_t* labels_in_dev,
                       int32_t* labels_out_dev, void* stream, int64_t* num_labels_host)
{
    if (!c || !centres_dev || !labels_in_dev || !labels_out_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = ensure_ccl_capacity(c, 32 * c->g.K + c->g.V / 1024 + 4096))) return rc;
    if ((rc = launch_import_centres(c, centres_dev, st))) return rc;
    int64_t n = 0;
    if ((rc = run_connectivity(c, labels_in_dev, labels_out_dev, st, &n))) return rc;
    if (num_labels_host) *num_labels_host = n;
    return SSLIC_OK;
}

int sslic_profile_enable(sslic_ctx* c, int32_t on)
{
    if (!c) return SSLIC_EINVAL;
    c->prof_on = on ? 1 : 0;
    c->prof.clear();
    c->launches = 0;
    return cuda_check(c, cudaMemset(c->ws.hc_rechecks, 0, sizeof(unsigned long long)), "reset counters");
}

int sslic_set_loop_graph(sslic_ctx* c, int32_t enable)
{
    if (!c) return SSLIC_EINVAL;
    c->loop_graph = enable ? 1 : 0;
    return SSLIC_OK;
}

int sslic_profile_read(sslic_ctx* c, sslic_profile* out)
{
    if (!c || !out) return SSLIC_EINVAL;
    memset(out, 0, sizeof(*out));
    for (const ProfRec& r : c->prof) {
        int rc = cuda_check(c, cudaEventSynchronize(r.stop), "profile event");
        if (rc) return rc;
        float ms = 0.0f;
        if ((rc = cuda_check(c, cudaEventElapsedTime(&ms, r.start, r.stop), "profile elapsed"))) return rc;
        if (r.phase >= 0 && r.phase < 8) {
            out->ms[r.phase] += ms;
            out->calls[r.phase] += 1;
        }
    }
    out->kernel_launches = c->launches;
    unsigned long long rk = 0;
    int rc = cuda_check(c, cudaMemcpy(&rk, c->ws.hc_rechecks, sizeof(rk), cudaMemcpyDeviceToHost), "read counters");
    out->rechecks = (int64_t)rk;
    return rc;
}

void sslic_destroy(sslic_ctx* c)
{
    if (!c) return;
    cudaDeviceSynchronize();
    for (cudaEvent_t e : c->prof_pool) cudaEventDestroy(e);
    if (c->loop_exec) cudaGraphExecDestroy(c->loop_exec);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    free_all(c);
    delete c;
}

const char* sslic_strerror(int code)
{
    switch (code) {
    case SSLIC_OK: return "ok";
    case SSLIC_EINVAL: return "invalid argument";
    case SSLIC_ENOMEM: return "out of memory";
    case SSLIC_ECUDA: return "CUDA error";
    case SSLIC_ETIMEOUT: return "device wait timed out";
    case SSLIC_EBUSY: return "context busy";
    case SSLIC_EUNSUPPORTED: return "unsupported request";
    default: return "unknown error";
    }
}

const char* sslic_last_error(const sslic_ctx* c)
{
    return c ? c->err : "";
}

}  // extern "C"
