// batch.cu -- many images per launch, and the serving loop built on it.
//
// Batching.  One iteration of SSLIC for R requests of different sizes, grids
// and types runs as one launch per phase: every kernel walks a device-side
// table of requests through prefix sums (clusters, bin-count entries, scan
// chunks, tiles, voxels) and finds its request by binary search.  The
// assignment runs the tile kernel of assign_tile.cu as a persistent grid over
// the (request, tile) queue of each (image type, tile shape) group; crowded
// tiles and image types without a tile kernel use the per-voxel kernel.  The
// arithmetic is the single-image path's, so each request's labels and
// centres are the ones sslic_run gives for it alone (float images: up to
// the order of their floating-point sums).
//
// Serving.  A worker thread keeps requests on the device and runs rounds of
// continuous batching: each round advances every admitted request by one
// iteration; requests that have done max_iter leave (their labels and
// centres are copied back and the ticket completes) and queued requests join
// as soon as the HBM budget has room for them.  Device memory for requests
// comes from one arena allocated at start-up (first fit, no cudaMalloc on
// the request path).  Uploads of joining requests overlap the current round
// on a copy stream.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"
#include "device_fns.cuh"

namespace sslic {
namespace batch {

// device record of one request
struct Req {
    TileArgs a;             // geometry, image, centres, bins, labels, sums, tile grid
    unsigned* bin_count;    // K + 1
    unsigned* bin_cursor;   // K
    int* bin_of;            // K
    unsigned* bin_start;    // K + 1 (a.bin_start, writable)
    int* bin_items;         // K
    unsigned* chunk;        // scan chunk sums
    float* cen_out;         // K x (C + n)
    int perturb;
    // requests with a convergence threshold: per-cluster residual terms and
    // the parts of their reduction (null otherwise)
    double* rk;             // K
    unsigned* ne;           // K
    double* rpart;          // kResidParts
    unsigned* rcnt;         // kResidParts
};

// ---- kernels -----------------------------------------------------------------
template <typename T>
__global__ void b_seed(const Req* __restrict__ reqs, const int64_t* __restrict__ kpre, const int* __restrict__ nR)
{
    const int R = *nR;
    const int64_t tot = kpre[R];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = prefix_find(kpre, R, i);
        const Req& q = reqs[r];
        seed_one<T>(q.a.g, (const T*)q.a.img, const_cast<float*>(q.a.ctr), q.perturb, i - kpre[r]);
    }
}

// zero bin counts (K + 1 per request) and cursors (K per request)
__global__ void b_zero_bins(const Req* __restrict__ reqs, const int64_t* __restrict__ kpre1, const int* __restrict__ nR)
{
    const int R = *nR;
    const int64_t tot = kpre1[R];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = prefix_find(kpre1, R, i);
        const int64_t j = i - kpre1[r];
        reqs[r].bin_count[j] = 0u;
        if (j < reqs[r].a.g.K) reqs[r].bin_cursor[j] = 0u;
    }
}

__global__ void b_bin_count(const Req* __restrict__ reqs, const int64_t* __restrict__ kpre, const int* __restrict__ nR)
{
    const int R = *nR;
    const int64_t tot = kpre[R];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = prefix_find(kpre, R, i);
        const Req& q = reqs[r];
        const Geom& g = q.a.g;
        const int64_t k = i - kpre[r];
        const float* p = q.a.ctr + k * g.CW + g.C;
        const int64_t b = bin_of_coord(p[0], g.S[0], g.nb[0]) +
                          g.nb[0] * (bin_of_coord(p[1], g.S[1], g.nb[1]) + g.nb[1] * bin_of_coord(p[2], g.S[2], g.nb[2]));
        q.bin_of[k] = (int)b;
        atomicAdd(&q.bin_count[b], 1u);
    }
}

// segmented exclusive scan of every request's K + 1 bin counts: chunks of
// 2048 items, then each request's chunk sums, then the chunk offsets
__global__ void __launch_bounds__(kBScanThreads)
b_scan_chunks(const Req* __restrict__ reqs, const int64_t* __restrict__ cpre, const int* __restrict__ nR)
{
    const int R = *nR;
    const int64_t tot = cpre[R];
    for (int64_t i = blockIdx.x; i < tot; i += gridDim.x) {
        const int r = prefix_find(cpre, R, i);
        const Req& q = reqs[r];
        const int64_t j = i - cpre[r];
        const int64_t n = q.a.g.K + 1;
        const int m = (int)imin64(kBScanItems, n - j * kBScanItems);
        block_scan_2048(q.bin_count + j * kBScanItems, q.bin_start + j * kBScanItems, m, q.chunk + j);
    }
}

__global__ void __launch_bounds__(kBScanThreads)
b_scan_sums(const Req* __restrict__ reqs, const int64_t* __restrict__ cpre, const int* __restrict__ nR)
{
    const int R = *nR;
    for (int r = blockIdx.x; r < R; r += gridDim.x) {
        const int nch = (int)(cpre[r + 1] - cpre[r]);  // <= 2048 (K + 1 <= 2^22)
        block_scan_2048(reqs[r].chunk, reqs[r].chunk, nch, nullptr);
    }
}

__global__ void b_scan_add(const Req* __restrict__ reqs, const int64_t* __restrict__ cpre, const int* __restrict__ nR)
{
    const int R = *nR;
    const int64_t tot = cpre[R];
    for (int64_t i = blockIdx.x; i < tot; i += gridDim.x) {
        const int r = prefix_find(cpre, R, i);
        const Req& q = reqs[r];
        const int64_t j = i - cpre[r];
        if (j == 0) continue;
        const unsigned add = q.chunk[j];
        const int64_t n = q.a.g.K + 1;
        for (int64_t t = j * kBScanItems + threadIdx.x; t < imin64(n, (j + 1) * kBScanItems); t += blockDim.x)
            q.bin_start[t] += add;
    }
}

__global__ void b_bin_scatter(const Req* __restrict__ reqs, const int64_t* __restrict__ kpre, const int* __restrict__ nR)
{
    const int R = *nR;
    const int64_t tot = kpre[R];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = prefix_find(kpre, R, i);
        const Req& q = reqs[r];
        const int64_t k = i - kpre[r];
        const int b = q.bin_of[k];
        const unsigned pos = q.bin_start[b] + atomicAdd(&q.bin_cursor[b], 1u);
        q.bin_items[pos] = (int)k;
    }
}

// per-voxel assignment of every voxel of a group (image types without a tile kernel)
template <typename T>
__global__ void b_voxel_all(const TileArgs* __restrict__ reqs, const int64_t* __restrict__ vpre, const int* __restrict__ nR)
{
    const int R = *nR;
    const int64_t tot = vpre[R];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = prefix_find(vpre, R, i);
        const TileArgs& a = reqs[r];
        const Geom& g = a.g;
        const int64_t v = i - vpre[r];
        const int64_t x = v % g.N[0], y = (v / g.N[0]) % g.N[1], z = v / (g.N[0] * g.N[1]);
        voxel_assign<T>(g, (const T*)a.img, a.ctr, a.bin_start, a.bin_items, a.labels, a.acc, a.facc, x, y, z);
    }
}

// per-voxel assignment of the crowded tiles (request << 40 | tile) of a group
template <typename T>
__global__ void b_voxel_tiles(const TileArgs* __restrict__ reqs, const int64_t* __restrict__ tiles,
                              const unsigned* __restrict__ ntiles)
{
    const int64_t nt = *ntiles;
    for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
        const int64_t e = tiles[t];
        const TileArgs& a = reqs[e >> 40];
        const int64_t tile = e & ((1LL << 40) - 1);
        const Geom& g = a.g;
        const int tv = a.tx * a.ty * a.tz;
        const int64_t X0 = (tile % a.ntx) * a.tx, Y0 = ((tile / a.ntx) % a.nty) * a.ty,
                      Z0 = (tile / ((int64_t)a.ntx * a.nty)) * a.tz;
        for (int v = threadIdx.x; v < tv; v += blockDim.x) {
            const int64_t x = X0 + v % a.tx, y = Y0 + (v / a.tx) % a.ty, z = Z0 + v / (a.tx * a.ty);
            if (x >= g.N[0] || y >= g.N[1] || z >= g.N[2]) continue;
            voxel_assign<T>(g, (const T*)a.img, a.ctr, a.bin_start, a.bin_items, a.labels, a.acc, a.facc, x, y, z);
        }
    }
}

__global__ void b_finalize(const Req* __restrict__ reqs, const int64_t* __restrict__ kpre, const int* __restrict__ nR)
{
    const int R = *nR;
    const int64_t tot = kpre[R];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = prefix_find(kpre, R, i);
        const Req& q = reqs[r];
        finalize_one(q.a.g, const_cast<float*>(q.a.ctr), q.a.acc, q.a.facc, i - kpre[r], q.rk, q.ne);
    }
}

// public centre tables K x (C + n) of the requests that are done
__global__ void b_export(const Req* __restrict__ reqs, const int64_t* __restrict__ epre, const int* __restrict__ nR)
{
    const int R = *nR;
    const int64_t tot = epre[R];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = prefix_find(epre, R, i);
        const Req& q = reqs[r];
        const Geom& g = q.a.g;
        const int W = g.C + g.n;
        const int64_t e = i - epre[r];
        q.cen_out[e] = q.a.ctr[(e / W) * g.CW + (e % W)];
    }
}

// centre residual of the requests with a convergence threshold, in the same
// fixed order as the single-image path (so each stops after the same
// iteration as sslic_run would): part blockIdx.x of request blockIdx.y, ...
__global__ void __launch_bounds__(kRedThreads)
b_resid_parts(const Req* __restrict__ reqs, const int* __restrict__ nT)
{
    const int T = *nT;
    for (int r = blockIdx.y; r < T; r += gridDim.y) {
        const Req& q = reqs[r];
        resid_part(q.rk, q.ne, q.a.g.K, blockIdx.x, &q.rpart[blockIdx.x], &q.rcnt[blockIdx.x]);
    }
}

__global__ void b_resid_final(const Req* __restrict__ reqs, const int* __restrict__ nT, double* __restrict__ out)
{
    const int T = *nT;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < T; r += gridDim.x * blockDim.x)
        out[r] = resid_combine(reqs[r].rpart, reqs[r].rcnt);
}

// ---- first-fit arena over one device allocation --------------------------------
class Arena {
public:
    int init(size_t bytes)
    {
        if (cudaMalloc(&base_, bytes) != cudaSuccess) { cudaGetLastError(); base_ = nullptr; return SSLIC_ENOMEM; }
        size_ = bytes;
        free_.clear();
        free_[0] = bytes;
        return SSLIC_OK;
    }
    ~Arena() { if (base_) cudaFree(base_); }
    // returns offset or SIZE_MAX
    size_t alloc(size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = (bytes + 255) / 256 * 256;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    unsigned char* ptr(size_t off) const { return (unsigned char*)base_ + off; }
    size_t size() const { return size_; }
    size_t peak() const { return peak_; }

private:
    void* base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

// ---- requests on the host side ------------------------------------------------
// kConnecting: iterations done, connectivity enforcement pending or running on the finisher thread
enum SlotState { kQueued = 0, kUploading = 1, kActive = 2, kFinishing = 3, kDone = 4, kFailed = 5, kConnecting = 6 };

struct Slot {
    int64_t ticket = 0;
    sslic_params p;
    Geom g;
    int group = 0;      // assignment group (type + tile shape)
    int shape = 0;
    int ntx = 1, nty = 1, ntz = 1, tx = 1, ty = 1, tz = 1;
    int64_t ntiles = 0, nchunks = 0;
    const void* h_img = nullptr;
    int32_t* h_lab = nullptr;
    float* h_cen = nullptr;
    size_t off = SIZE_MAX, bytes = 0;
    Req d;              // device record (pointers into the arena)
    int iter = 0;
    bool thr = false;        // a convergence threshold is set
    bool converged = false;  // its residual fell below it: results final, no more iterations
    int state = kQueued;
    int status = SSLIC_OK;
    cudaEvent_t ev_up = nullptr, ev_done = nullptr;
    cudaEvent_t ev_iter = nullptr;  // its last iteration has run (connectivity starts after it)
    double t_submit = 0, t_done = 0;
};

static size_t a256(size_t b) { return (b + 255) / 256 * 256; }

static bool tile_type(const Geom& g) { return has_tile_kernel(g); }

static size_t footprint(const Geom& g)
{
    const size_t esz = g.dtype == SSLIC_U8 ? 1 : (g.dtype == SSLIC_U16 ? 2 : 4);
    const size_t K = (size_t)g.K, V = (size_t)g.V;
    const size_t nch = (K + 1 + kBScanItems - 1) / kBScanItems;
    return a256(V * g.C * esz) + a256(V * 4) + a256(K * g.CW * 4) + a256(K * g.AW * 8) +
           (g.dtype == SSLIC_F32 ? a256(K * g.C * 8) : 0) + 2 * a256((K + 1) * 4) + 3 * a256(K * 4) +
           a256(nch * 4) + a256(K * (g.C + g.n) * 4);
}

// the residual scratch of a request with a convergence threshold
static size_t footprint_thr(const Geom& g)
{
    const size_t K = (size_t)g.K;
    return a256(K * 8) + a256(K * 4) + a256(kResidParts * 8) + a256(kResidParts * 4);
}

// group key: dtype, channels, dims, tile shape (-1 for the per-voxel kernel)
static int group_key(const Geom& g, int shape) { return ((g.dtype * 512 + g.C) * 8 + g.n) * 32 + (shape + 1); }
static int key_dtype(int key) { return key / (512 * 8 * 32); }
static int key_channels(int key) { return (key / (8 * 32)) % 512; }
static int key_ndim(int key) { return (key / 32) % 8; }
static int key_shape(int key) { return key % 32 - 1; }

constexpr int kMaxGroups = 16;  // assignment groups (image type + tile shape) per round

// counts of one round, read by the kernels on the device (so a captured
// round replays for any number of requests)
struct RoundHdr {
    int R;                  // requests advanced by the round
    int Rf;                 // requests finishing with it
    int nseed[3];           // joining requests per dtype
    int ngrp[kMaxGroups];   // requests per assignment group
    int nthr;               // requests with a convergence threshold
};

// Fixed layout of one round's tables for at most M requests: every table
// sits at the same device address in every round of the same parity.
struct TabLayout {
    size_t hdr, kpre, kpre1, cpre, req, fpre, fin, thr, res, seed_req[3], seed_pre[3], grp_ta[kMaxGroups],
        grp_pre[kMaxGroups], end;
    void init(int M)
    {
        size_t o = 0;
        auto put = [&](size_t bytes) { o = (o + 15) / 16 * 16; const size_t r = o; o += bytes; return r; };
        const size_t P = (size_t)(M + 1) * sizeof(int64_t);
        hdr = put(sizeof(RoundHdr));
        kpre = put(P);
        kpre1 = put(P);
        cpre = put(P);
        req = put((size_t)M * sizeof(Req));
        fpre = put(P);
        fin = put((size_t)M * sizeof(Req));
        thr = put((size_t)M * sizeof(Req));   // requests with a threshold
        res = put((size_t)M * sizeof(double));  // their residuals (device -> host)
        for (int t = 0; t < 3; ++t) { seed_req[t] = put((size_t)M * sizeof(Req)); seed_pre[t] = put(P); }
        for (int g = 0; g < kMaxGroups; ++g) { grp_ta[g] = put((size_t)M * sizeof(TileArgs)); grp_pre[g] = put(P); }
        end = (o + 255) / 256 * 256;
    }
};

}  // namespace batch
}  // namespace sslic

using namespace sslic;
using namespace sslic::batch;

struct sslic_server {
    // configuration
    int device = 0;
    int sms = 148;
    int max_active = 64;
    Arena arena;
    cudaStream_t cs = nullptr, up = nullptr;  // compute, upload
    cudaStream_t ds = nullptr;                // results to the host, off the rounds' stream
    // device + pinned staging of the round tables, double buffered
    TabLayout lay;
    unsigned char* tab_dev[2] = {nullptr, nullptr};
    unsigned char* tab_host[2] = {nullptr, nullptr};
    cudaEvent_t round_ev[2] = {nullptr, nullptr};
    bool round_pending[2] = {false, false};
    // threshold requests of the last round and its parity (their residuals
    // are read before the next round is formed)
    std::vector<Slot*> thr_prev;
    int thr_prev_par = 0;
    // captured rounds, by (parity, joining dtypes, finishing, thresholds, groups)
    std::map<std::vector<int>, cudaGraphExec_t> graphs;
    // round forms met once: a form runs eagerly the first time and is
    // captured when it comes back, so one-off forms never pay a capture
    std::set<std::vector<int>> seen;
    int64_t graph_captures = 0, graph_launches = 0, eager_rounds = 0;
    // crowded-tile lists, one per group slot in a round
    int64_t* ovf[kMaxGroups] = {};
    unsigned* ovf_cnt = nullptr;  // kMaxGroups counters
    int64_t ovf_cap = 0;
    // requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Slot*> pending;
    std::vector<Slot*> live;                    // uploading / active / finishing
    std::map<int64_t, Slot*> tickets;
    int64_t next_ticket = 1;
    bool stop = false;
    int error = SSLIC_OK;
    char err[256] = {0};
    std::thread worker;
    // connectivity enforcement (Sec. 3.1 stage 3) of the requests that ask
    // for it: a finisher thread takes them off the rounds once their
    // iterations are done and runs it on its own stream with one context
    // whose workspace follows the largest request so far, while the rounds of
    // the others go on; cap_mu keeps its allocations out of a round's capture
    std::thread finisher;
    std::deque<Slot*> conn_q;
    std::condition_variable cv_conn;
    bool conn_stop = false;
    cudaStream_t fs = nullptr;
    sslic_ctx* conn = nullptr;
    std::mutex cap_mu;
    // statistics
    int64_t submitted = 0, completed = 0, rejected = 0, rounds = 0;
    int max_seen = 0;
    double voxel_iters = 0, t_first = -1, t_last = 0;
    std::vector<double> lat_ms;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

int server_fail(sslic_server* s, int code, const char* what, cudaError_t e = cudaSuccess)
{
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error == SSLIC_OK) {
        s->error = code;
        snprintf(s->err, sizeof(s->err), "%s%s%s", what, e != cudaSuccess ? ": " : "",
                 e != cudaSuccess ? cudaGetErrorString(e) : "");
    }
    s->cv_done.notify_all();
    return code;
}

// carve a request's device state out of its arena block
void place(sslic_server* s, Slot* q)
{
    const Geom& g = q->g;
    const size_t esz = g.dtype == SSLIC_U8 ? 1 : (g.dtype == SSLIC_U16 ? 2 : 4);
    const size_t K = (size_t)g.K, V = (size_t)g.V;
    unsigned char* p = s->arena.ptr(q->off);
    auto take = [&](size_t b) { unsigned char* r = p; p += a256(b); return r; };
    Req& d = q->d;
    memset(&d, 0, sizeof(d));
    TileArgs& a = d.a;
    a.g = g;
    a.img = take(V * g.C * esz);
    a.labels = (int32_t*)take(V * 4);
    a.ctr = (float*)take(K * g.CW * 4);
    a.acc = (unsigned long long*)take(K * g.AW * 8);
    a.facc = g.dtype == SSLIC_F32 ? (double*)take(K * g.C * 8) : nullptr;
    d.bin_count = (unsigned*)take((K + 1) * 4);
    d.bin_start = (unsigned*)take((K + 1) * 4);
    d.bin_cursor = (unsigned*)take(K * 4);
    d.bin_items = (int*)take(K * 4);
    d.bin_of = (int*)take(K * 4);
    d.chunk = (unsigned*)take((size_t)q->nchunks * 4);
    d.cen_out = (float*)take(K * (g.C + g.n) * 4);
    if (q->thr) {
        d.rk = (double*)take(K * 8);
        d.ne = (unsigned*)take(K * 4);
        d.rpart = (double*)take(kResidParts * 8);
        d.rcnt = (unsigned*)take(kResidParts * 4);
    }
    a.bin_start = d.bin_start;
    a.bin_items = d.bin_items;
    a.lists = q->shape >= 0 ? (int*)take((size_t)q->ntiles * tile_list_stride() * 4) : nullptr;
    a.ntx = q->ntx;
    a.nty = q->nty;
    a.tx = q->tx;
    a.ty = q->ty;
    a.tz = q->tz;
    d.perturb = q->p.perturb;
}

// the assignment of one group; with ta == nullptr only the kernels' launch
// attributes are set (before a capture)
template <typename T>
cudaError_t launch_group(sslic_server* s, int C, int n, int shape, const TileArgs* ta, const int64_t* tp,
                         const int* nR, int gi)
{
    const int grid = s->sms * 4;
    cudaError_t e;
    if (shape < 0) {
        if (!ta) return cudaSuccess;
        b_voxel_all<T><<<grid, 256, 0, s->cs>>>(ta, tp, nR);
        return cudaGetLastError();
    }
    if (ta && (e = cudaMemsetAsync(s->ovf_cnt + gi, 0, sizeof(unsigned), s->cs)) != cudaSuccess) return e;
    // step 2 ahead of the queue for every tile of the group: the queue kernel
    // then starts each tile from its record
    if (ta && (e = launch_tile_lists_queue(n, ta, tp, nR, s->ovf[gi], s->ovf_cnt + gi, s->sms * 32, s->cs)) != cudaSuccess)
        return e;
    if constexpr (sizeof(T) == 1) {
        if (C == 3) e = n == 3 ? launch_tile_queue<uint8_t, 3, 3>(shape, ta, tp, nR, s->ovf[gi], s->ovf_cnt + gi, grid, s->cs)
                               : launch_tile_queue<uint8_t, 3, 2>(shape, ta, tp, nR, s->ovf[gi], s->ovf_cnt + gi, grid, s->cs);
        else e = n == 3 ? launch_tile_queue<uint8_t, 1, 3>(shape, ta, tp, nR, s->ovf[gi], s->ovf_cnt + gi, grid, s->cs)
                        : launch_tile_queue<uint8_t, 1, 2>(shape, ta, tp, nR, s->ovf[gi], s->ovf_cnt + gi, grid, s->cs);
    } else if constexpr (sizeof(T) == 2) {
        e = n == 3 ? launch_tile_queue<uint16_t, 1, 3>(shape, ta, tp, nR, s->ovf[gi], s->ovf_cnt + gi, grid, s->cs)
                   : launch_tile_queue<uint16_t, 1, 2>(shape, ta, tp, nR, s->ovf[gi], s->ovf_cnt + gi, grid, s->cs);
    } else {
        e = n == 3 ? launch_tile_queue<float, 3, 3>(shape, ta, tp, nR, s->ovf[gi], s->ovf_cnt + gi, grid, s->cs)
                   : launch_tile_queue<float, 3, 2>(shape, ta, tp, nR, s->ovf[gi], s->ovf_cnt + gi, grid, s->cs);
    }
    if (e != cudaSuccess || !ta) return e;
    b_voxel_tiles<T><<<grid, 256, 0, s->cs>>>(ta, s->ovf[gi], s->ovf_cnt + gi);
    return cudaGetLastError();
}

cudaError_t group_launch(sslic_server* s, int key, const TileArgs* ta, const int64_t* tp, const int* nR, int gi)
{
    const int dt = key_dtype(key), C = key_channels(key), n = key_ndim(key), sh = key_shape(key);
    if (dt == SSLIC_U8) return launch_group<uint8_t>(s, C, n, sh, ta, tp, nR, gi);
    if (dt == SSLIC_U16) return launch_group<uint16_t>(s, C, n, sh, ta, tp, nR, gi);
    return launch_group<float>(s, C, n, sh, ta, tp, nR, gi);
}

// every kernel of one round, on the compute stream, reading the tables of
// parity par: seeding of the joining requests (one launch per dtype present),
// the bin grid, the assignment of each group, the reduction, the export of
// the finishing requests
cudaError_t issue_round(sslic_server* s, int par, int seed_mask, bool has_fin, bool has_thr, const std::vector<int>& keys)
{
    const TabLayout& L = s->lay;
    unsigned char* D = s->tab_dev[par];
    const RoundHdr* h = (const RoundHdr*)(D + L.hdr);
    const int grid = s->sms * 8;
    const Req* dreq = (const Req*)(D + L.req);
    const int64_t *dk = (const int64_t*)(D + L.kpre), *dk1 = (const int64_t*)(D + L.kpre1),
                  *dc = (const int64_t*)(D + L.cpre);
    for (int t = 0; t < 3; ++t) {
        if (!(seed_mask >> t & 1)) continue;
        const Req* r = (const Req*)(D + L.seed_req[t]);
        const int64_t* pr = (const int64_t*)(D + L.seed_pre[t]);
        if (t == SSLIC_U8) b_seed<uint8_t><<<grid, 128, 0, s->cs>>>(r, pr, &h->nseed[t]);
        else if (t == SSLIC_U16) b_seed<uint16_t><<<grid, 128, 0, s->cs>>>(r, pr, &h->nseed[t]);
        else b_seed<float><<<grid, 128, 0, s->cs>>>(r, pr, &h->nseed[t]);
    }
    b_zero_bins<<<grid, 256, 0, s->cs>>>(dreq, dk1, &h->R);
    b_bin_count<<<grid, 256, 0, s->cs>>>(dreq, dk, &h->R);
    b_scan_chunks<<<grid, kBScanThreads, 0, s->cs>>>(dreq, dc, &h->R);
    b_scan_sums<<<std::min(s->max_active, 1024), kBScanThreads, 0, s->cs>>>(dreq, dc, &h->R);
    b_scan_add<<<grid, 256, 0, s->cs>>>(dreq, dc, &h->R);
    b_bin_scatter<<<grid, 256, 0, s->cs>>>(dreq, dk, &h->R);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int gi = 0; gi < (int)keys.size(); ++gi) {
        e = group_launch(s, keys[gi], (const TileArgs*)(D + L.grp_ta[gi]), (const int64_t*)(D + L.grp_pre[gi]),
                         &h->ngrp[gi], gi);
        if (e != cudaSuccess) return e;
    }
    b_finalize<<<grid, 256, 0, s->cs>>>(dreq, dk, &h->R);
    if (has_thr) {
        const Req* dthr = (const Req*)(D + L.thr);
        b_resid_parts<<<dim3(kResidParts, std::min(s->max_active, 64)), kRedThreads, 0, s->cs>>>(dthr, &h->nthr);
        b_resid_final<<<1, 64, 0, s->cs>>>(dthr, &h->nthr, (double*)(D + L.res));
    }
    if (has_fin) b_export<<<grid, 256, 0, s->cs>>>((const Req*)(D + L.fin), (const int64_t*)(D + L.fpre), &h->Rf);
    return cudaGetLastError();
}

void drop_graphs(sslic_server* s)
{
    for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
    s->graphs.clear();
}

// one round: seed the joining requests, one iteration for all, export the finished
int run_round(sslic_server* s, std::vector<Slot*>& join, std::vector<Slot*>& act)
{
    const int par = (int)(s->rounds & 1);
    cudaError_t e;
    if (s->round_pending[par]) {
        if ((e = cudaEventSynchronize(s->round_ev[par])) != cudaSuccess) return server_fail(s, SSLIC_ECUDA, "round", e);
        s->round_pending[par] = false;
    }
    // residuals of the previous round's threshold requests: that round must
    // have finished (the next round's form depends on them)
    if (!s->thr_prev.empty()) {
        const int pp = s->thr_prev_par;
        if (s->round_pending[pp]) {
            if ((e = cudaEventSynchronize(s->round_ev[pp])) != cudaSuccess) return server_fail(s, SSLIC_ECUDA, "round", e);
            s->round_pending[pp] = false;
        }
        const double* res = (const double*)(s->tab_host[pp] + s->lay.res);
        for (size_t i = 0; i < s->thr_prev.size(); ++i) {
            Slot* q = s->thr_prev[i];
            if (q->state == kActive && res[i] < q->p.conv_threshold) q->converged = true;
        }
        s->thr_prev.clear();
    }
    // requests that converged leave without another iteration: their labels
    // are those of the last assignment and their centres those of the last update
    std::vector<Slot*> all, fin;
    for (Slot* q : act) (q->converged ? fin : all).push_back(q);
    all.insert(all.end(), join.begin(), join.end());
    const int R = (int)all.size();
    for (Slot* q : all)
        if (q->iter + 1 >= q->p.max_iter) fin.push_back(q);
    const int Rf = (int)fin.size();
    std::vector<Slot*> thr;
    for (Slot* q : all)
        if (q->thr && q->iter + 1 < q->p.max_iter) thr.push_back(q);
    std::map<int, std::vector<Slot*>> groups;
    for (Slot* q : all) groups[q->group].push_back(q);
    if ((int)groups.size() > kMaxGroups) return server_fail(s, SSLIC_EUNSUPPORTED, "too many image types");
    if (R > s->max_active) return server_fail(s, SSLIC_EINVAL, "round larger than the request cap");
    // tables
    const TabLayout& L = s->lay;
    unsigned char* H = s->tab_host[par];
    RoundHdr* hdr = (RoundHdr*)(H + L.hdr);
    memset(hdr, 0, sizeof(*hdr));
    hdr->R = R;
    hdr->Rf = Rf;
    Req* hreq = (Req*)(H + L.req);
    int64_t *kpre = (int64_t*)(H + L.kpre), *kpre1 = (int64_t*)(H + L.kpre1), *cpre = (int64_t*)(H + L.cpre);
    kpre[0] = kpre1[0] = cpre[0] = 0;
    for (int i = 0; i < R; ++i) {
        hreq[i] = all[i]->d;
        kpre[i + 1] = kpre[i] + all[i]->g.K;
        kpre1[i + 1] = kpre1[i] + all[i]->g.K + 1;
        cpre[i + 1] = cpre[i] + all[i]->nchunks;
    }
    Req* hfin = (Req*)(H + L.fin);
    int64_t* fpre = (int64_t*)(H + L.fpre);
    fpre[0] = 0;
    for (int i = 0; i < Rf; ++i) { hfin[i] = fin[i]->d; fpre[i + 1] = fpre[i] + fin[i]->g.K * (fin[i]->g.C + fin[i]->g.n); }
    Req* hthr = (Req*)(H + L.thr);
    for (size_t i = 0; i < thr.size(); ++i) hthr[i] = thr[i]->d;
    hdr->nthr = (int)thr.size();
    int seed_mask = 0;
    for (Slot* q : join) {
        const int t = q->g.dtype;
        Req* hr = (Req*)(H + L.seed_req[t]);
        int64_t* hp = (int64_t*)(H + L.seed_pre[t]);
        const int i = hdr->nseed[t]++;
        if (i == 0) hp[0] = 0;
        hr[i] = q->d;
        hp[i + 1] = hp[i] + q->g.K;
        seed_mask |= 1 << t;
    }
    std::vector<int> keys;
    int64_t ovf_need = 0;
    for (auto& kv : groups) {
        const int gi = (int)keys.size();
        keys.push_back(kv.first);
        TileArgs* ta = (TileArgs*)(H + L.grp_ta[gi]);
        int64_t* tp = (int64_t*)(H + L.grp_pre[gi]);
        tp[0] = 0;
        for (size_t i = 0; i < kv.second.size(); ++i) {
            Slot* q = kv.second[i];
            ta[i] = q->d.a;
            tp[i + 1] = tp[i] + (q->shape < 0 ? q->g.V : q->ntiles);
        }
        hdr->ngrp[gi] = (int)kv.second.size();
        if (kv.second[0]->shape >= 0) ovf_need = std::max(ovf_need, tp[kv.second.size()]);
    }
    if (ovf_need > s->ovf_cap) {
        // the lists move: every captured round that points at them goes
        if ((e = cudaStreamSynchronize(s->cs)) != cudaSuccess) return server_fail(s, SSLIC_ECUDA, "sync", e);
        drop_graphs(s);
        for (int i = 0; i < kMaxGroups; ++i) { cudaFree(s->ovf[i]); s->ovf[i] = nullptr; }
        s->ovf_cap = 0;
        for (int i = 0; i < kMaxGroups; ++i)
            if ((e = cudaMalloc(&s->ovf[i], ovf_need * sizeof(int64_t))) != cudaSuccess)
                return server_fail(s, SSLIC_ENOMEM, "crowded-tile lists", e);
        s->ovf_cap = ovf_need;
    }
    const size_t used = keys.empty() ? L.grp_ta[0] : L.grp_pre[keys.size() - 1] + (size_t)(s->max_active + 1) * 8;
    if ((e = cudaMemcpyAsync(s->tab_dev[par], H, used, cudaMemcpyHostToDevice, s->cs)) != cudaSuccess)
        return server_fail(s, SSLIC_ECUDA, "tables", e);
    for (Slot* q : join)
        if ((e = cudaStreamWaitEvent(s->cs, q->ev_up, 0)) != cudaSuccess) return server_fail(s, SSLIC_ECUDA, "wait", e);
    // the round's kernels: replayed from a captured graph of the same form
    std::vector<int> sig{par, seed_mask, Rf > 0 ? 1 : 0, thr.empty() ? 0 : 1};
    sig.insert(sig.end(), keys.begin(), keys.end());
    auto it = s->graphs.find(sig);
    bool eager = false;
    if (it == s->graphs.end()) {
        for (int gi = 0; gi < (int)keys.size(); ++gi)
            if ((e = group_launch(s, keys[gi], nullptr, nullptr, nullptr, gi)) != cudaSuccess)
                return server_fail(s, SSLIC_ECUDA, "kernel attributes", e);
        if (s->seen.insert(sig).second) {
            if (s->seen.size() > 4096) s->seen.clear();
            eager = true;
        }
    }
    if (eager) {
        if ((e = issue_round(s, par, seed_mask, Rf > 0, !thr.empty(), keys)) != cudaSuccess)
            return server_fail(s, SSLIC_ECUDA, "round", e);
        s->eager_rounds += 1;
    } else if (it == s->graphs.end()) {
        if (s->graphs.size() >= 256) drop_graphs(s);
        cudaGraph_t gr = nullptr;
        cudaGraphExec_t ex = nullptr;
        std::unique_lock<std::mutex> cap(s->cap_mu);
        if ((e = cudaStreamBeginCapture(s->cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return server_fail(s, SSLIC_ECUDA, "begin capture", e);
        const cudaError_t ei = issue_round(s, par, seed_mask, Rf > 0, !thr.empty(), keys);
        e = cudaStreamEndCapture(s->cs, &gr);
        cap.unlock();
        if (ei != cudaSuccess || e != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            return server_fail(s, SSLIC_ECUDA, "capture", ei != cudaSuccess ? ei : e);
        }
        e = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return server_fail(s, SSLIC_ECUDA, "instantiate", e);
        it = s->graphs.emplace(sig, ex).first;
        s->graph_captures += 1;
    }
    if (!eager) {
        if ((e = cudaGraphLaunch(it->second, s->cs)) != cudaSuccess) return server_fail(s, SSLIC_ECUDA, "round launch", e);
        s->graph_launches += 1;
    }
    if (!thr.empty()) {
        if ((e = cudaMemcpyAsync(H + L.res, s->tab_dev[par] + L.res, thr.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, s->cs)) != cudaSuccess)
            return server_fail(s, SSLIC_ECUDA, "residuals", e);
        s->thr_prev = thr;
        s->thr_prev_par = par;
    }
    std::vector<Slot*> conn;
    for (Slot* q : fin) {
        const Geom& g = q->g;
        if (q->p.enforce_connectivity) {
            // labels and centres go back after connectivity (finisher thread)
            if ((e = cudaEventRecord(q->ev_iter, s->cs)) != cudaSuccess) return server_fail(s, SSLIC_ECUDA, "event", e);
            q->state = kConnecting;
            conn.push_back(q);
            continue;
        }
        // the copies run on their own stream, so the next rounds need not wait for them
        if ((e = cudaEventRecord(q->ev_iter, s->cs)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s->ds, q->ev_iter, 0)) != cudaSuccess)
            return server_fail(s, SSLIC_ECUDA, "event", e);
        if ((e = cudaMemcpyAsync(q->h_lab, q->d.a.labels, (size_t)g.V * 4, cudaMemcpyDeviceToHost, s->ds)) != cudaSuccess)
            return server_fail(s, SSLIC_ECUDA, "labels to host", e);
        if (q->h_cen &&
            (e = cudaMemcpyAsync(q->h_cen, q->d.cen_out, (size_t)g.K * (g.C + g.n) * 4, cudaMemcpyDeviceToHost, s->ds)) != cudaSuccess)
            return server_fail(s, SSLIC_ECUDA, "centres to host", e);
        if ((e = cudaEventRecord(q->ev_done, s->ds)) != cudaSuccess) return server_fail(s, SSLIC_ECUDA, "event", e);
        q->state = kFinishing;
    }
    for (Slot* q : all) {
        q->iter += 1;
        if (q->state != kFinishing && q->state != kConnecting) q->state = kActive;
    }
    if (!conn.empty()) {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Slot* q : conn) s->conn_q.push_back(q);
        s->cv_conn.notify_all();
    }
    if ((e = cudaEventRecord(s->round_ev[par], s->cs)) != cudaSuccess) return server_fail(s, SSLIC_ECUDA, "event", e);
    s->round_pending[par] = true;
    s->rounds += 1;
    return SSLIC_OK;
}

void worker_main(sslic_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        std::vector<Slot*> join, act, done;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            // reap finished requests
            for (Slot* q : s->live) {
                if (q->state == kFinishing && cudaEventQuery(q->ev_done) == cudaSuccess) done.push_back(q);
            }
            const double t = s->now();
            for (Slot* q : done) {
                s->arena.release(q->off, q->bytes);
                q->state = kDone;
                q->t_done = t;
                s->completed += 1;
                s->lat_ms.push_back((q->t_done - q->t_submit) * 1e3);
                s->voxel_iters += (double)q->g.V * q->p.max_iter;
                s->t_last = t;
            }
            if (!done.empty()) {
                s->live.erase(std::remove_if(s->live.begin(), s->live.end(),
                                             [](Slot* q) { return q->state == kDone; }),
                              s->live.end());
                s->cv_done.notify_all();
            }
            // admit queued requests while the budget has room (first come, first served)
            while (!s->pending.empty() && (int)s->live.size() < s->max_active && s->error == SSLIC_OK) {
                Slot* q = s->pending.front();
                const size_t off = s->arena.alloc(q->bytes);
                if (off == SIZE_MAX) break;
                s->pending.pop_front();
                q->off = off;
                place(s, q);
                const size_t esz = q->g.dtype == SSLIC_U8 ? 1 : (q->g.dtype == SSLIC_U16 ? 2 : 4);
                cudaError_t e = cudaMemcpyAsync((void*)q->d.a.img, q->h_img, (size_t)q->g.V * q->g.C * esz,
                                                cudaMemcpyHostToDevice, s->up);
                if (e == cudaSuccess) e = cudaMemsetAsync(q->d.a.acc, 0, (size_t)q->g.K * q->g.AW * 8, s->up);
                if (e == cudaSuccess && q->d.a.facc)
                    e = cudaMemsetAsync(q->d.a.facc, 0, (size_t)q->g.K * q->g.C * 8, s->up);
                if (e == cudaSuccess) e = cudaEventRecord(q->ev_up, s->up);
                if (e != cudaSuccess) {
                    lk.unlock();
                    server_fail(s, SSLIC_ECUDA, "upload", e);
                    lk.lock();
                    break;
                }
                if (s->t_first < 0) s->t_first = s->now();
                q->state = kUploading;
                s->live.push_back(q);
            }
            s->max_seen = std::max(s->max_seen, (int)s->live.size());
            // a request joins the round after its upload has landed, so that
            // no round waits for another request's copy
            bool uploading = false;
            for (Slot* q : s->live) {
                if (q->state == kUploading) {
                    const cudaError_t eq = cudaEventQuery(q->ev_up);
                    if (eq == cudaSuccess) join.push_back(q);
                    else if (eq == cudaErrorNotReady) uploading = true;
                    else {
                        lk.unlock();
                        server_fail(s, SSLIC_ECUDA, "upload", eq);
                        lk.lock();
                    }
                } else if (q->state == kActive) {
                    act.push_back(q);
                }
            }
            if (s->error != SSLIC_OK) {
                for (Slot* q : s->live) { q->state = kFailed; q->status = s->error; }
                for (Slot* q : s->pending) { q->state = kFailed; q->status = s->error; }
                s->cv_done.notify_all();
                if (s->stop) return;
                s->cv_work.wait_for(lk, std::chrono::milliseconds(5));
                continue;
            }
            const bool finishing = uploading || std::any_of(s->live.begin(), s->live.end(), [](Slot* q) {
                return q->state == kFinishing || q->state == kConnecting;
            });
            if (join.empty() && act.empty()) {
                if (s->stop && s->pending.empty() && s->live.empty()) return;
                if (!finishing) s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                else {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(50));
                }
                continue;
            }
        }
        run_round(s, join, act);
    }
}

// connectivity of the requests that finished their iterations, one at a time,
// then their labels and centres to the host; the worker reaps them as usual
void finisher_main(sslic_server* s)
{
    cudaSetDevice(s->device);
    for (;;) {
        Slot* q = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_conn.wait(lk, [&] { return s->conn_stop || !s->conn_q.empty(); });
            if (s->conn_q.empty()) return;
            q = s->conn_q.front();
            s->conn_q.pop_front();
            if (s->error != SSLIC_OK) {
                q->state = kFailed;
                q->status = s->error;
                s->cv_done.notify_all();
                continue;
            }
        }
        const Geom& g = q->g;
        int rc = SSLIC_OK;
        const char* what = "connectivity";
        cudaError_t e = cudaStreamWaitEvent(s->fs, q->ev_iter, 0);
        if (e != cudaSuccess) rc = SSLIC_ECUDA;
        if (rc == SSLIC_OK) {
            std::lock_guard<std::mutex> cl(s->cap_mu);
            if (!s->conn) s->conn = conn_ctx_create(s->device, s->sms);
            if (!s->conn) rc = SSLIC_ENOMEM;
            else {
                int64_t nl = 0;
                rc = conn_ctx_run(s->conn, q->p, g, q->d.a.ctr, q->d.a.labels, s->fs, &nl);
                if (rc != SSLIC_OK) what = s->conn->err;
            }
        }
        if (rc == SSLIC_OK) {
            e = cudaMemcpyAsync(q->h_lab, q->d.a.labels, (size_t)g.V * 4, cudaMemcpyDeviceToHost, s->fs);
            if (e == cudaSuccess && q->h_cen)
                e = cudaMemcpyAsync(q->h_cen, q->d.cen_out, (size_t)g.K * (g.C + g.n) * 4, cudaMemcpyDeviceToHost, s->fs);
            if (e == cudaSuccess) e = cudaEventRecord(q->ev_done, s->fs);
            if (e != cudaSuccess) {
                rc = SSLIC_ECUDA;
                what = "connectivity results to host";
            }
        }
        if (rc != SSLIC_OK) server_fail(s, rc, what, e);
        std::lock_guard<std::mutex> lk(s->mu);
        if (rc == SSLIC_OK) {
            q->state = kFinishing;
        } else {
            q->state = kFailed;
            q->status = rc;
            s->cv_done.notify_all();
        }
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" {

int sslic_server_create(int64_t hbm_budget_bytes, int32_t max_active, sslic_server** out)
{
    if (!out || hbm_budget_bytes <= 0 || max_active < 1) return SSLIC_EINVAL;
    *out = nullptr;
    sslic_server* s = new (std::nothrow) sslic_server();
    if (!s) return SSLIC_ENOMEM;
    s->max_active = max_active;
    int rc = SSLIC_OK;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->fs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->ds, cudaStreamNonBlocking);
    s->lay.init(max_active);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaMalloc(&s->tab_dev[i], s->lay.end);
        if (e == cudaSuccess) e = cudaMallocHost(&s->tab_host[i], s->lay.end);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->round_ev[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->ovf_cnt, kMaxGroups * sizeof(unsigned));
    if (e != cudaSuccess) rc = e == cudaErrorMemoryAllocation ? SSLIC_ENOMEM : SSLIC_ECUDA;
    if (rc == SSLIC_OK) rc = s->arena.init((size_t)hbm_budget_bytes);
    if (rc != SSLIC_OK) {
        cudaGetLastError();
        sslic_server_destroy(s);
        return rc;
    }
    s->worker = std::thread(worker_main, s);
    s->finisher = std::thread(finisher_main, s);
    *out = s;
    return SSLIC_OK;
}

int sslic_server_submit(sslic_server* s, const sslic_params* p, const void* image_host, int32_t* labels_host,
                        float* centres_host, int64_t* ticket)
{
    if (!s || !p || !image_host || !labels_host || !ticket) return SSLIC_EINVAL;
    Geom g;
    int rc = make_geom(p, &g);
    if (rc) return rc;
    if (g.n > 3) return SSLIC_EUNSUPPORTED;  // the batched tables are laid out for up to three axes
    if (g.K + 1 > (int64_t)kBScanItems * kBScanItems) return SSLIC_EUNSUPPORTED;
    Slot* q = new (std::nothrow) Slot();
    if (!q) return SSLIC_ENOMEM;
    q->p = *p;
    q->g = g;
    q->shape = tile_type(g) ? tuned_tile_shape(g) : -1;
    if (tile_type(g) && q->shape < 0) q->shape = default_tile_shape(g);
    if (q->shape >= 0) {
        tile_dims(g.n, q->shape, &q->tx, &q->ty, &q->tz);
        q->ntx = (int)((g.N[0] + q->tx - 1) / q->tx);
        q->nty = (int)((g.N[1] + q->ty - 1) / q->ty);
        q->ntz = (int)((g.N[2] + q->tz - 1) / q->tz);
        q->ntiles = (int64_t)q->ntx * q->nty * q->ntz;
    }
    q->group = group_key(g, q->shape);
    q->nchunks = (g.K + 1 + kBScanItems - 1) / kBScanItems;
    q->thr = p->conv_threshold > 0.0;
    q->bytes = footprint(g) + (q->thr ? footprint_thr(g) : 0) +
               (q->shape >= 0 ? a256((size_t)q->ntiles * tile_list_stride() * 4) : 0);
    q->h_img = image_host;
    q->h_lab = labels_host;
    q->h_cen = centres_host;
    if (cudaEventCreateWithFlags(&q->ev_up, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->ev_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&q->ev_iter, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (q->ev_up) cudaEventDestroy(q->ev_up);
        if (q->ev_done) cudaEventDestroy(q->ev_done);
        delete q;
        return SSLIC_ECUDA;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error != SSLIC_OK) {
        cudaEventDestroy(q->ev_up); cudaEventDestroy(q->ev_done); cudaEventDestroy(q->ev_iter);
        delete q;
        return s->error;
    }
    if (q->bytes > s->arena.size()) {
        s->rejected += 1;
        cudaEventDestroy(q->ev_up);
        cudaEventDestroy(q->ev_done);
        cudaEventDestroy(q->ev_iter);
        delete q;
        return SSLIC_ENOMEM;  // larger than the whole budget: never admissible
    }
    q->ticket = s->next_ticket++;
    q->t_submit = s->now();
    s->tickets[q->ticket] = q;
    s->pending.push_back(q);
    s->submitted += 1;
    *ticket = q->ticket;
    s->cv_work.notify_one();
    return SSLIC_OK;
}

int sslic_server_wait(sslic_server* s, int64_t ticket, int32_t timeout_ms, double* latency_ms)
{
    if (!s) return SSLIC_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) return SSLIC_EINVAL;
    Slot* q = it->second;
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                        [&] { return q->state == kDone || q->state == kFailed; });
    if (!ok) return SSLIC_ETIMEOUT;
    const int st = q->state == kDone ? SSLIC_OK : q->status;
    if (latency_ms) *latency_ms = (q->t_done - q->t_submit) * 1e3;
    s->tickets.erase(it);
    cudaEventDestroy(q->ev_up);
    cudaEventDestroy(q->ev_done);
    cudaEventDestroy(q->ev_iter);
    delete q;
    return st;
}

int sslic_server_stats_get(sslic_server* s, sslic_server_stats* out)
{
    if (!s || !out) return SSLIC_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->rounds = s->rounds;
    out->max_active = s->max_seen;
    out->peak_bytes = (int64_t)s->arena.peak();
    out->voxel_iters = s->voxel_iters;
    out->busy_s = s->t_first >= 0 ? s->t_last - s->t_first : 0.0;
    if (!s->lat_ms.empty()) {
        std::vector<double> v(s->lat_ms);
        std::sort(v.begin(), v.end());
        auto pct = [&](double f) { return v[std::min(v.size() - 1, (size_t)(f * (double)(v.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double sum = 0;
        for (double x : v) sum += x;
        out->mean_ms = sum / (double)v.size();
    }
    out->graph_launches = s->graph_launches;
    out->eager_rounds = s->eager_rounds;
    out->graph_captures = s->graph_captures;
    out->status = s->error;
    return SSLIC_OK;
}

void sslic_server_destroy(sslic_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->conn_stop = true;
        s->cv_conn.notify_all();
    }
    if (s->finisher.joinable()) s->finisher.join();
    if (s->fs) cudaStreamSynchronize(s->fs);
    if (s->ds) cudaStreamSynchronize(s->ds);
    conn_ctx_destroy(s->conn);
    s->conn = nullptr;
    if (s->cs) cudaStreamSynchronize(s->cs);
    if (s->up) cudaStreamSynchronize(s->up);
    for (auto& kv : s->tickets) {
        cudaEventDestroy(kv.second->ev_up);
        cudaEventDestroy(kv.second->ev_done);
        cudaEventDestroy(kv.second->ev_iter);
        delete kv.second;
    }
    for (int i = 0; i < 2; ++i) {
        if (s->tab_dev[i]) cudaFree(s->tab_dev[i]);
        if (s->tab_host[i]) cudaFreeHost(s->tab_host[i]);
        if (s->round_ev[i]) cudaEventDestroy(s->round_ev[i]);
    }
    drop_graphs(s);
    for (int i = 0; i < kMaxGroups; ++i)
        if (s->ovf[i]) cudaFree(s->ovf[i]);
    if (s->ovf_cnt) cudaFree(s->ovf_cnt);
    if (s->cs) cudaStreamDestroy(s->cs);
    if (s->up) cudaStreamDestroy(s->up);
    if (s->fs) cudaStreamDestroy(s->fs);
    if (s->ds) cudaStreamDestroy(s->ds);
    delete s;
}

}  // extern "C"
