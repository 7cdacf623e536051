// bins.cu -- device-wide exclusive scan and the bin grid of the current
// centres.
//
// The bin grid has one cell per seed-lattice cell: bin_d = floor(c_d) / S_d.
// A voxel x can only be covered by centres with x_d - S_d < c_d <= x_d + S_d,
// i.e. in bins floor(x_d/S_d) - 1 .. floor(x_d/S_d) + 1 along every axis, so
// the voxel-centric search over 3^n bins meets exactly the centres whose
// 2S window (Sec. 2.2) covers the voxel.  The grid is rebuilt every
// iteration by a counting sort: count, exclusive scan, scatter.
#include "common.cuh"

namespace sslic {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;                       // per thread
constexpr int kScanBlock = kScanThreads * kScanItems;  // 2048 items per block

// exclusive scan of one block's items; writes the block total to sums
__global__ void scan_block_kernel(const unsigned* __restrict__ in, unsigned* __restrict__ out,
                                  unsigned* __restrict__ sums, int64_t n)
{
    __shared__ unsigned warp_tot[kScanThreads / 32];
    const int tid = threadIdx.x;
    const int64_t base = blockIdx.x * (int64_t)kScanBlock + tid * kScanItems;
    unsigned v[kScanItems];
    unsigned run = 0;
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        unsigned t = v[i];
        v[i] = run;
        run += t;
    }
    // inclusive warp scan of per-thread totals
    unsigned x = run;
    const int lane = tid & 31, warp = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
        unsigned s = w;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = s - w;  // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1 && sums) sums[blockIdx.x] = s;
    }
    __syncthreads();
    unsigned pre = warp_tot[warp] + (x - run);
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) out[base + i] = v[i] + pre;
}

__global__ void scan_add_kernel(unsigned* __restrict__ out, const unsigned* __restrict__ offs, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const unsigned o = offs[blockIdx.x];
    for (int j = 0; j < kScanItems; ++j) {
        int64_t q = i + j * kScanThreads;
        if (q < n) out[q] += o;
    }
}

size_t scan_tmp_needed(int64_t n)
{
    size_t tot = 0;
    while (n > kScanBlock) {
        n = (n + kScanBlock - 1) / kScanBlock;
        tot += (size_t)n;
    }
    return tot + 1;
}

// recursive: scan blocks, scan the block sums, add offsets
static int scan_rec(sslic_ctx* c, const unsigned* in, unsigned* out, int64_t n, unsigned* tmp,
                    cudaStream_t st)
{
    int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb <= 1) {
        scan_block_kernel<<<1, kScanThreads, 0, st>>>(in, out, nullptr, n);
        count_launch(c);
        return cuda_check(c, cudaGetLastError(), "scan_block_kernel");
    }
    unsigned* sums = tmp;
    scan_block_kernel<<<nb, kScanThreads, 0, st>>>(in, out, sums, n);
    count_launch(c);
    int rc = cuda_check(c, cudaGetLastError(), "scan_block_kernel");
    if (rc) return rc;
    rc = scan_rec(c, sums, sums, nb, tmp + nb, st);
    if (rc) return rc;
    scan_add_kernel<<<nb, kScanThreads, 0, st>>>(out, sums, n);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "scan_add_kernel");
}

int scan_exclusive_u32(sslic_ctx* c, const unsigned* in, unsigned* out, int64_t n, cudaStream_t st)
{
    if (n <= 0) return SSLIC_OK;
    return scan_rec(c, in, out, n, c->ws.scan_tmp, st);
}

__global__ void bin_count_kernel(Geom g, const float* __restrict__ ctr, int* __restrict__ bin_of,
                                 unsigned* __restrict__ count)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= g.K) return;
    const float* p = ctr + k * g.CW + g.C;
    int64_t b0 = bin_of_coord(p[0], g.S[0], g.nb[0]);
    int64_t b1 = bin_of_coord(p[1], g.S[1], g.nb[1]);
    int64_t b2 = bin_of_coord(p[2], g.S[2], g.nb[2]);
    int64_t b3 = g.n >= 4 ? bin_of_coord(p[3], g.S[3], g.nb[3]) : 0;
    int64_t b = b0 + g.nb[0] * (b1 + g.nb[1] * (b2 + g.nb[2] * b3));
    bin_of[k] = (int)b;
    atomicAdd(&count[b], 1u);
}

__global__ void bin_scatter_kernel(Geom g, const int* __restrict__ bin_of,
                                   const unsigned* __restrict__ start, unsigned* __restrict__ cursor,
                                   int* __restrict__ items)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= g.K) return;
    int b = bin_of[k];
    unsigned pos = start[b] + atomicAdd(&cursor[b], 1u);
    items[pos] = (int)k;
}

// Small centre sets: the whole counting sort in one CTA, the counts in shared
// memory (count, exclusive scan, scatter with the counts turned into
// cursors) -- one launch instead of two memsets and four kernels, which on
// small images is most of the bin grid's time.
constexpr int kSmallBinsThreads = 1024;
// K + 1 counts; with 9728 centres (ten per thread) the one-CTA sort measured
// slower than the device-wide passes, with 256 faster
constexpr int kSmallBins = 2048;
constexpr int kSmallPer = (kSmallBins + kSmallBinsThreads - 1) / kSmallBinsThreads;  // centres per thread

__global__ void __launch_bounds__(kSmallBinsThreads)
bins_small_kernel(Geom g, const float* __restrict__ ctr, unsigned* __restrict__ start, int* __restrict__ items)
{
    __shared__ unsigned cnt[kSmallBins];
    __shared__ unsigned warp_tot[kSmallBinsThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int K = (int)g.K, nbins = K + 1;
    for (int i = tid; i < nbins; i += kSmallBinsThreads) cnt[i] = 0u;
    // each thread's centres (k = tid + j * threads): their bins, kept in
    // registers for the scatter, with all the position loads in flight at once
    int bk[kSmallPer];
#pragma unroll
    for (int j = 0; j < kSmallPer; ++j) {
        const int k = tid + j * kSmallBinsThreads;
        bk[j] = -1;
        if (k < K) {
            const float* p = ctr + (int64_t)k * g.CW + g.C;
            const int64_t b0 = bin_of_coord(p[0], g.S[0], g.nb[0]);
            const int64_t b1 = bin_of_coord(p[1], g.S[1], g.nb[1]);
            const int64_t b2 = bin_of_coord(p[2], g.S[2], g.nb[2]);
            const int64_t b3 = g.n >= 4 ? bin_of_coord(p[3], g.S[3], g.nb[3]) : 0;
            bk[j] = (int)(b0 + g.nb[0] * (b1 + g.nb[1] * (b2 + g.nb[2] * b3)));
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSmallPer; ++j)
        if (bk[j] >= 0) atomicAdd(&cnt[bk[j]], 1u);
    __syncthreads();
    // exclusive scan: each thread a run of consecutive counts
    const int per = (nbins + kSmallBinsThreads - 1) / kSmallBinsThreads;
    const int a0 = tid * per, a1 = min(nbins, a0 + per);
    unsigned run = 0;
    for (int i = a0; i < a1; ++i) run += cnt[i];
    unsigned x = run;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const unsigned wv = warp_tot[lane];
        unsigned sc = wv;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane >= o) sc += y;
        }
        warp_tot[lane] = sc - wv;
    }
    __syncthreads();
    unsigned pre = warp_tot[warp] + (x - run);
    for (int i = a0; i < a1; ++i) {
        const unsigned v = cnt[i];
        start[i] = pre;
        cnt[i] = pre;  // the bin's cursor
        pre += v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSmallPer; ++j)
        if (bk[j] >= 0) items[atomicAdd(&cnt[bk[j]], 1u)] = tid + j * kSmallBinsThreads;
}

int build_bins(sslic_ctx* c, cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    const int pr = prof_begin(c, SSLIC_PHASE_BINS, st);
    if (g.K + 1 <= kSmallBins) {
        bins_small_kernel<<<1, kSmallBinsThreads, 0, st>>>(g, w.ctr, w.bin_start, w.bin_items);
        count_launch(c);
        prof_end(c, pr, st);
        return cuda_check(c, cudaGetLastError(), "bins_small_kernel");
    }
    int rc = cuda_check(c, cudaMemsetAsync(w.bin_count, 0, (g.K + 1) * sizeof(unsigned), st), "memset bins");
    if (rc) return rc;
    rc = cuda_check(c, cudaMemsetAsync(w.bin_cursor, 0, g.K * sizeof(unsigned), st), "memset cursor");
    if (rc) return rc;
    int threads = 256;
    int64_t blocks = (g.K + threads - 1) / threads;
    bin_count_kernel<<<blocks, threads, 0, st>>>(g, w.ctr, w.bin_of, w.bin_count);
    count_launch(c);
    if ((rc = cuda_check(c, cudaGetLastError(), "bin_count_kernel"))) return rc;
    if ((rc = scan_exclusive_u32(c, w.bin_count, w.bin_start, g.K + 1, st))) return rc;
    bin_scatter_kernel<<<blocks, threads, 0, st>>>(g, w.bin_of, w.bin_start, w.bin_cursor, w.bin_items);
    count_launch(c);
    prof_end(c, pr, st);
    return cuda_check(c, cudaGetLastError(), "bin_scatter_kernel");
}

}  // namespace sslic
