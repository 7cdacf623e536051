// device_fns.cuh -- device functions shared by the single-image kernels and
// their batched (many requests per launch) forms.
#pragma once
#include "common.cuh"

namespace sslic {

constexpr float kInfF = __builtin_huge_valf();

// Assignment + map-update of one voxel (x, y, z, w) by direct search: the 3^n
// bins around it, the exact window test, the canonical single-precision D^2
// (Sec. 2.1, one rounding per operation, no FMA) and a lexicographic (D^2, k)
// comparison, so the bin visiting order does not matter.  Sums go to the
// cluster's row of acc (uint64: features of integer images, positions,
// count last) and facc (double features of float images).
template <typename T>
__device__ __forceinline__ void voxel_assign(const Geom& g, const T* __restrict__ img,
                                             const float* __restrict__ ctr,
                                             const unsigned* __restrict__ bin_start,
                                             const int* __restrict__ bin_items, int32_t* __restrict__ labels,
                                             unsigned long long* __restrict__ acc, double* __restrict__ facc,
                                             int64_t x, int64_t y, int64_t z, int64_t w = 0)
{
    const int C = g.C;
    constexpr float kInf = kInfF;
    const int64_t q = vidx(g, x, y, z, w);
    const int64_t X[kMaxDims] = {x, y, z, w};
    int64_t blo[kMaxDims], bhi[kMaxDims];
    for (int d = 0; d < kMaxDims; ++d) {
        blo[d] = imax64(0, X[d] / g.S[d] - 1);
        bhi[d] = imin64(g.nb[d] - 1, X[d] / g.S[d] + 1);
    }
    float best = kInf;
    int bestk = -1;
    for (int64_t bw = blo[3]; bw <= bhi[3]; ++bw)
    for (int64_t bz = blo[2]; bz <= bhi[2]; ++bz)
        for (int64_t by = blo[1]; by <= bhi[1]; ++by)
            for (int64_t bx = blo[0]; bx <= bhi[0]; ++bx) {
                int64_t bin = bx + g.nb[0] * (by + g.nb[1] * (bz + g.nb[2] * bw));
                for (unsigned i = bin_start[bin]; i < bin_start[bin + 1]; ++i) {
                    const int k = bin_items[i];
                    const float* row = ctr + (int64_t)k * g.CW;
                    bool inside = true;
                    for (int d = 0; d < g.n; ++d) {
                        int64_t lo = window_lo(row[C + d], g.S[d]);
                        inside = inside && X[d] >= lo && X[d] <= lo + 2 * g.S[d] - 1;
                    }
                    if (!inside) continue;
                    float dc = 0.0f;
                    for (int c = 0; c < C; ++c) {
                        float e = __fsub_rn((float)img[q * C + c], row[c]);
                        float sq = __fmul_rn(e, e);
                        dc = c == 0 ? sq : __fadd_rn(dc, sq);
                    }
                    float ds = 0.0f;
                    for (int d = 0; d < g.n; ++d) {
                        float dl = __fsub_rn((float)X[d], row[C + d]);
                        float t = __fmul_rn(g.w[d], __fmul_rn(dl, dl));
                        ds = d == 0 ? t : __fadd_rn(ds, t);
                    }
                    float D = __fadd_rn(dc, ds);
                    if (D < best || (D == best && k < bestk)) { best = D; bestk = k; }
                }
            }
    labels[q] = bestk;
    if (bestk >= 0) {
        unsigned long long* a = acc + (int64_t)bestk * g.AW;
        for (int c = 0; c < C; ++c) {
            if (sizeof(T) == 4) atomicAdd(&facc[(int64_t)bestk * C + c], (double)img[q * C + c]);
            else atomicAdd(&a[c], (unsigned long long)img[q * C + c]);
        }
        for (int d = 0; d < g.CW - C; ++d) atomicAdd(&a[C + d], (unsigned long long)X[d]);
        atomicAdd(&a[g.AW - 1], 1ull);
    }
}

// ---- seeding (Sec. 2.2 / 3.1 step 1): lattice seed k, optionally moved to the
// lowest gradient magnitude of its 3^n neighbourhood; row k of ctr written
template <typename T>
__device__ __forceinline__ int64_t grad_int(const Geom& g, const T* img, const int64_t* x, int64_t q)
{
    int64_t acc = 0;
    for (int c = 0; c < g.C; ++c) {
        for (int d = 0; d < g.n; ++d) {
            int64_t st = d == 0 ? 1 : (d == 1 ? g.N[0] : (d == 2 ? g.N[0] * g.N[1] : g.N[0] * g.N[1] * g.N[2]));
            int64_t hi = x[d] + 1 < g.N[d] ? q + st : q;
            int64_t lo = x[d] > 0 ? q - st : q;
            int64_t diff = (int64_t)img[hi * g.C + c] - (int64_t)img[lo * g.C + c];
            acc += diff * diff;
        }
    }
    return acc;
}

__device__ __forceinline__ float grad_f32(const Geom& g, const float* img, const int64_t* x, int64_t q)
{
    float acc = 0.0f;
    bool first = true;
    for (int c = 0; c < g.C; ++c) {
        for (int d = 0; d < g.n; ++d) {
            int64_t st = d == 0 ? 1 : (d == 1 ? g.N[0] : (d == 2 ? g.N[0] * g.N[1] : g.N[0] * g.N[1] * g.N[2]));
            int64_t hi = x[d] + 1 < g.N[d] ? q + st : q;
            int64_t lo = x[d] > 0 ? q - st : q;
            float diff = __fsub_rn(img[hi * g.C + c], img[lo * g.C + c]);
            float sq = __fmul_rn(diff, diff);
            acc = first ? sq : __fadd_rn(acc, sq);
            first = false;
        }
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ void seed_one(const Geom& g, const T* __restrict__ img, float* __restrict__ ctr,
                                         int perturb, int64_t k)
{
    int64_t x[kMaxDims];
    int64_t rem = k;
    for (int d = 0; d < kMaxDims; ++d) {
        int64_t j = rem % g.nb[d];
        rem /= g.nb[d];
        x[d] = g.off[d] + j * g.S[d];
    }
    int64_t best[kMaxDims] = {x[0], x[1], x[2], x[3]};
    if (perturb) {
        int64_t q0 = vidx(g, x[0], x[1], x[2], x[3]);
        constexpr bool kFloat = sizeof(T) == 4;
        int64_t bi = 0;
        float bf = 0.0f;
        if constexpr (kFloat) bf = grad_f32(g, (const float*)img, x, q0);
        else bi = grad_int(g, img, x, q0);
        // the 3^n offsets in raster order, dimension 0 fastest
        const int lo3 = g.n >= 4 ? -1 : 0, lo2 = g.n >= 3 ? -1 : 0, lo1 = g.n >= 2 ? -1 : 0;
        for (int o3 = lo3; o3 <= -lo3; ++o3)
        for (int o2 = lo2; o2 <= -lo2; ++o2)
            for (int o1 = lo1; o1 <= -lo1; ++o1)
                for (int o0 = -1; o0 <= 1; ++o0) {
                    int64_t y[kMaxDims] = {x[0] + o0, x[1] + o1, x[2] + o2, x[3] + o3};
                    bool inside = true;
                    for (int d = 0; d < kMaxDims; ++d) inside = inside && y[d] >= 0 && y[d] < g.N[d];
                    if (!inside) continue;
                    int64_t q = vidx(g, y[0], y[1], y[2], y[3]);
                    bool better;
                    if constexpr (kFloat) {
                        float gq = grad_f32(g, (const float*)img, y, q);
                        better = gq < bf;
                        if (better) bf = gq;
                    } else {
                        int64_t gq = grad_int(g, img, y, q);
                        better = gq < bi;
                        if (better) bi = gq;
                    }
                    if (better)
                        for (int d = 0; d < kMaxDims; ++d) best[d] = y[d];
                }
    }
    int64_t qb = vidx(g, best[0], best[1], best[2], best[3]);
    float* row = ctr + k * g.CW;
    for (int c = 0; c < g.C; ++c) row[c] = (float)img[qb * g.C + c];
    for (int d = 0; d < g.CW - g.C; ++d) row[g.C + d] = (float)best[d];
}

// ---- reduce step of the update (Sec. 3.1): centre k = sum / count, divided in
// double and rounded to float; an empty cluster keeps its centre; the
// cluster's residual term sqrt(D^2(C_prev, C_new)) (rk, ne may be null); the
// sums are cleared for the next iteration
__device__ __forceinline__ void finalize_one(const Geom& g, float* __restrict__ ctr,
                                             unsigned long long* __restrict__ acc, double* __restrict__ facc,
                                             int64_t k, double* __restrict__ rk, unsigned* __restrict__ ne)
{
    unsigned long long* a = acc + k * g.AW;
    const unsigned long long cnt = a[g.AW - 1];
    float* row = ctr + k * g.CW;
    double r = 0.0;
    if (cnt) {
        const double n = (double)cnt;
        for (int j = 0; j < g.C + g.n; ++j) {
            // features, then the real position axes
            const double sum = (j < g.C && g.dtype == SSLIC_F32) ? facc[k * g.C + j] : (double)a[j];
            const float v = __double2float_rn(__ddiv_rn(sum, n));
            const double diff = (double)v - (double)row[j];
            r = __dadd_rn(r, j < g.C ? __dmul_rn(diff, diff) : __dmul_rn(g.w64[j - g.C], __dmul_rn(diff, diff)));
            row[j] = v;
        }
        r = sqrt(r);
    }
    if (rk) rk[k] = r;
    if (ne) ne[k] = cnt ? 1u : 0u;
    for (int j = 0; j < g.AW; ++j) a[j] = 0ull;
    if (g.dtype == SSLIC_F32)
        for (int c = 0; c < g.C; ++c) facc[k * g.C + c] = 0.0;
}

// ---- centre residual (Sec. 3.1: distance between successive centres) ----------
// The mean over non-empty clusters of the per-cluster terms rk, reduced in a
// fixed order so every caller gets the same double: kResidParts parts of
// ceil(K / kResidParts) consecutive clusters, each summed by a block of
// kRedThreads threads (thread-strided, then a tree), then the parts in order.
constexpr int kRedThreads = 256;
constexpr int kResidParts = 256;

// one part; must be called by all kRedThreads threads of the block
__device__ __forceinline__ void resid_part(const double* __restrict__ rk, const unsigned* __restrict__ ne, int64_t K,
                                          int part, double* __restrict__ out_d, unsigned* __restrict__ out_c)
{
    __shared__ double sd[kRedThreads];
    __shared__ unsigned sc[kRedThreads];
    const int64_t per = (K + kResidParts - 1) / kResidParts;
    const int64_t lo = part * per, hi = imin64(K, lo + per);
    double d = 0.0;
    unsigned cnt = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) { d += rk[i]; cnt += ne[i]; }
    sd[threadIdx.x] = d;
    sc[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { sd[threadIdx.x] += sd[threadIdx.x + o]; sc[threadIdx.x] += sc[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { *out_d = sd[0]; *out_c = sc[0]; }
    __syncthreads();
}

__device__ __forceinline__ double resid_combine(const double* __restrict__ part, const unsigned* __restrict__ cpart)
{
    double d = 0.0;
    unsigned long long cnt = 0;
    for (int i = 0; i < kResidParts; ++i) { d += part[i]; cnt += cpart[i]; }
    return cnt ? d / (double)cnt : 0.0;
}

// ---- block-wide exclusive scan of up to 2048 unsigned values -----------------
// 512 threads x 4 items; in and out may alias; *total (if not null) gets the
// sum of the n items.  Must be called by all 512 threads of the block.
constexpr int kBScanThreads = 512;
constexpr int kBScanItems = 2048;
__device__ __forceinline__ void block_scan_2048(const unsigned* in, unsigned* out, int n, unsigned* total)
{
    __shared__ unsigned warp_tot[kBScanThreads / 32];
    const int tid = threadIdx.x;
    const int base = tid * 4;
    unsigned v[4];
    unsigned run = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const unsigned t = (base + i < n) ? in[base + i] : 0u;
        v[i] = run;
        run += t;
    }
    unsigned x = run;
    const int lane = tid & 31, warp = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const unsigned w = lane < kBScanThreads / 32 ? warp_tot[lane] : 0u;
        unsigned sc = w;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, sc, o);
            if (lane >= o) sc += y;
        }
        if (lane < kBScanThreads / 32) warp_tot[lane] = sc - w;
        if (lane == kBScanThreads / 32 - 1 && total) *total = sc;
    }
    __syncthreads();
    const unsigned pre = warp_tot[warp] + (x - run);
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (base + i < n) out[base + i] = v[i] + pre;
    __syncthreads();
}

// last r in [0, R) with pre[r] <= i (pre ascending, pre[0] = 0)
__device__ __forceinline__ int prefix_find(const int64_t* __restrict__ pre, int R, int64_t i)
{
    int lo = 0, hi = R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace sslic
