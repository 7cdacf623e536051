// assign.cu -- one SSLIC iteration: assignment (Sec. 2.1, 2.2, 3.1 step 2)
// fused with the map step of the centre update (Sec. 3.1 map-reduce), then
// the reduce step (finalize) and the centre residual.
//
// Assignment.  Every voxel x takes the argmin over the centres whose 2S
// window covers it, c_d - S_d <= x_d < c_d + S_d, of
//     D^2 = sum_c (I_c - C_c)^2 + sum_d w_d (x_d - c_d)^2,  w_d = m^2 / S_d^2
// (Sec. 2.1 with the per-axis grid of Sec. 3.3), with ties going to the
// lowest cluster index -- the outcome of the paper's centre loop in ascending
// k with a strict "<".  D^2 is evaluated in single precision with one
// rounding per operation in a fixed order (no fused multiply-add):
//     e_c = I_c - C_c;  dc = ((e_0^2 + e_1^2) + e_2^2) ...
//     t_d = w_d * (x_d - c_d)^2 (+inf outside the window);  ds = (t_0 + t_1) + t_2
//     D^2 = dc + ds
// so that integer images give bit-identical labels to a sequential
// implementation of the same order.
//
// The hot cases (integer images with 1 or 3 channels and float images with 3,
// 2-D and 3-D) run in the tile kernel of assign_tile.cu.  This file holds the per-voxel kernel
// used for every other shape (float images, other channel counts, 1-D) and
// for tiles that too many centres reach, the reduce step and the centre
// table conversions.
#include <cstdio>

#include "common.cuh"
#include "device_fns.cuh"

namespace sslic {


// ---------------------------------------------------------------------------
// per-voxel kernel: any dtype / channel count / dimensionality, and the tiles
// the tile kernel gave up on.  Same distance, same order, lexicographic
// (D^2, k) comparison so the bin visiting order does not matter.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void assign_voxel_kernel(Geom g, const T* __restrict__ img, const float* __restrict__ ctr,
                                    const unsigned* __restrict__ bin_start,
                                    const int* __restrict__ bin_items, int32_t* __restrict__ labels,
                                    unsigned long long* __restrict__ acc, double* __restrict__ facc,
                                    const int64_t* __restrict__ tiles, const unsigned* __restrict__ ntiles,
                                    int64_t ntx, int64_t nty, int tx_, int ty_, int tz_, int64_t v0, int64_t v1)
{
    // tiles == nullptr: the voxels [v0, v1) in raster order
    const int tv = tx_ * ty_ * tz_;
    int64_t nwork;
    if (tiles) nwork = (int64_t)(*ntiles) * tv;
    else nwork = v1;
    for (int64_t w = (tiles ? 0 : v0) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwork;
         w += (int64_t)gridDim.x * blockDim.x) {
        int64_t x, y, z, u = 0;
        if (tiles) {
            const int64_t t = tiles[w / tv] & ((1LL << 40) - 1);  // low bits: tile, high bits: request
            int e = (int)(w % tv);
            x = (t % ntx) * tx_ + e % tx_;
            y = ((t / ntx) % nty) * ty_ + (e / tx_) % ty_;
            z = (t / (ntx * nty)) * tz_ + e / (tx_ * ty_);
            if (x >= g.N[0] || y >= g.N[1] || z >= g.N[2]) continue;
        } else {
            x = w % g.N[0];
            y = (w / g.N[0]) % g.N[1];
            z = (w / (g.N[0] * g.N[1])) % g.N[2];
            u = w / (g.N[0] * g.N[1] * g.N[2]);
        }
        voxel_assign<T>(g, img, ctr, bin_start, bin_items, labels, acc, facc, x, y, z, u);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
int launch_voxel_tiles(sslic_ctx* c, const T* img, int32_t* labels, int tx, int ty, int tz, int ntx, int nty,
                       cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    const int pr = prof_begin(c, SSLIC_PHASE_ASSIGN_VOXEL, st);
    assign_voxel_kernel<T><<<c->sms * 4, 256, 0, st>>>(g, img, w.ctr, w.bin_start, w.bin_items, labels, w.acc,
                                                        w.facc, w.ovf_tiles, w.ovf_count, ntx, nty, tx, ty, tz, 0, 0);
    count_launch(c);
    prof_end(c, pr, st);
    return cuda_check(c, cudaGetLastError(), "assign_voxel_kernel(crowded tiles)");
}

template int launch_voxel_tiles<uint8_t>(sslic_ctx*, const uint8_t*, int32_t*, int, int, int, int, int,
                                         cudaStream_t);
template int launch_voxel_tiles<uint16_t>(sslic_ctx*, const uint16_t*, int32_t*, int, int, int, int, int,
                                          cudaStream_t);
template int launch_voxel_tiles<float>(sslic_ctx*, const float*, int32_t*, int, int, int, int, int, cudaStream_t);

template <typename T>
static int launch_voxel(sslic_ctx* c, const T* img, int32_t* labels, cudaStream_t st, const Slab* slab)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    int64_t plane = 1;
    for (int d = 0; d < g.n - 1; ++d) plane *= g.N[d];
    const int64_t v0 = slab ? slab->lo * plane : 0, v1 = slab ? slab->hi * plane : g.V;
    int64_t blocks = imax64(1, imin64((v1 - v0 + 255) / 256, (int64_t)c->sms * 16));
    const int pr = prof_begin(c, SSLIC_PHASE_ASSIGN_VOXEL, st);
    assign_voxel_kernel<T><<<blocks, 256, 0, st>>>(g, img, w.ctr, w.bin_start, w.bin_items, labels, w.acc,
                                                    w.facc, nullptr, nullptr, 1, 1, 1, 1, 1, v0, v1);
    count_launch(c);
    prof_end(c, pr, st);
    return cuda_check(c, cudaGetLastError(), "assign_voxel_kernel");
}

int launch_assign_update(sslic_ctx* c, const void* img, int32_t* labels, cudaStream_t st, const Slab* slab)
{
    const Geom& g = c->g;
    const bool tiled = g.n == 2 || g.n == 3;
    if (tiled && g.dtype == SSLIC_U8 && g.C == 3) {
        return g.n == 3 ? launch_tile_impl<uint8_t, 3, 3>(c, (const uint8_t*)img, labels, st, slab)
                        : launch_tile_impl<uint8_t, 3, 2>(c, (const uint8_t*)img, labels, st, slab);
    }
    if (tiled && g.dtype == SSLIC_U8 && g.C == 1) {
        return g.n == 3 ? launch_tile_impl<uint8_t, 1, 3>(c, (const uint8_t*)img, labels, st, slab)
                        : launch_tile_impl<uint8_t, 1, 2>(c, (const uint8_t*)img, labels, st, slab);
    }
    if (tiled && g.dtype == SSLIC_U16 && g.C == 1) {
        return g.n == 3 ? launch_tile_impl<uint16_t, 1, 3>(c, (const uint16_t*)img, labels, st, slab)
                        : launch_tile_impl<uint16_t, 1, 2>(c, (const uint16_t*)img, labels, st, slab);
    }
    if (tiled && g.dtype == SSLIC_F32 && g.C == 3) {
        return g.n == 3 ? launch_tile_impl<float, 3, 3>(c, (const float*)img, labels, st, slab)
                        : launch_tile_impl<float, 3, 2>(c, (const float*)img, labels, st, slab);
    }
    if (hc_applies(g) && !slab) return launch_hc(c, (const float*)img, labels, st);  // slabs: per-voxel kernel
    switch (g.dtype) {
    case SSLIC_U8: return launch_voxel<uint8_t>(c, (const uint8_t*)img, labels, st, slab);
    case SSLIC_U16: return launch_voxel<uint16_t>(c, (const uint16_t*)img, labels, st, slab);
    default: return launch_voxel<float>(c, (const float*)img, labels, st, slab);
    }
}

// ---------------------------------------------------------------------------
// reduce step: centre = sum / count (divided in double, rounded to float),
// empty clusters keep their centre; per-cluster residual term; clear sums.
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(Geom g, float* __restrict__ ctr, unsigned long long* __restrict__ acc,
                                double* __restrict__ facc, double* __restrict__ rk,
                                unsigned* __restrict__ ne)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < g.K) finalize_one(g, ctr, acc, facc, k, rk, ne);
}

// deterministic residual reduction (resid_part / resid_combine)
__global__ void __launch_bounds__(kRedThreads)
resid_partial_kernel(const double* __restrict__ rk, const unsigned* __restrict__ ne, int64_t K,
                     double* __restrict__ part, unsigned* __restrict__ cpart)
{
    resid_part(rk, ne, K, blockIdx.x, &part[blockIdx.x], &cpart[blockIdx.x]);
}

__global__ void resid_final_kernel(const double* __restrict__ part, const unsigned* __restrict__ cpart,
                                   double* __restrict__ out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = resid_combine(part, cpart);
}

// the residual of the last update: the per-cluster terms reduced in a fixed order
static int residual_kernels(sslic_ctx* c, cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    resid_partial_kernel<<<kResidParts, kRedThreads, 0, st>>>(w.resid_k, w.nonempty_k, g.K, w.resid_part,
                                                              w.resid_cnt_part);
    int rc = cuda_check(c, cudaGetLastError(), "resid_partial_kernel");
    if (rc) return rc;
    resid_final_kernel<<<1, 32, 0, st>>>(w.resid_part, w.resid_cnt_part, w.resid_out);
    count_launch(c, 2);
    return cuda_check(c, cudaGetLastError(), "resid_final_kernel");
}

int launch_finalize(sslic_ctx* c, cudaStream_t st, bool residual)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    int threads = 256;
    int64_t blocks = (g.K + threads - 1) / threads;
    const int pr = prof_begin(c, SSLIC_PHASE_FINALIZE, st);
    finalize_kernel<<<blocks, threads, 0, st>>>(g, w.ctr, w.acc, w.facc, w.resid_k, w.nonempty_k);
    count_launch(c);
    int rc = cuda_check(c, cudaGetLastError(), "finalize_kernel");
    if (rc) return rc;
    if (residual && (rc = residual_kernels(c, st))) return rc;
    prof_end(c, pr, st);
    return SSLIC_OK;
}

int launch_residual(sslic_ctx* c, cudaStream_t st)
{
    const int pr = prof_begin(c, SSLIC_PHASE_FINALIZE, st);
    const int rc = residual_kernels(c, st);
    prof_end(c, pr, st);
    return rc;
}

// ---------------------------------------------------------------------------
// public centre table K x (C+n)  <->  internal K x (C+3)
// ---------------------------------------------------------------------------
__global__ void export_kernel(Geom g, const float* __restrict__ ctr, float* __restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int W = g.C + g.n;
    if (i >= g.K * W) return;
    int64_t k = i / W;
    int j = (int)(i % W);
    out[i] = ctr[k * g.CW + j];
}

__global__ void import_kernel(Geom g, const float* __restrict__ in, float* __restrict__ ctr)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.K * g.CW) return;
    int64_t k = i / g.CW;
    int j = (int)(i % g.CW);
    const int W = g.C + g.n;
    ctr[i] = j < W ? in[k * W + j] : 0.0f;
}

int launch_export_centres(sslic_ctx* c, float* out, cudaStream_t st)
{
    const Geom& g = c->g;
    int64_t n = g.K * (g.C + g.n);
    export_kernel<<<(n + 255) / 256, 256, 0, st>>>(g, c->ws.ctr, out);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "export_kernel");
}

int launch_import_centres(sslic_ctx* c, const float* in, cudaStream_t st)
{
    const Geom& g = c->g;
    int64_t n = g.K * g.CW;
    import_kernel<<<(n + 255) / 256, 256, 0, st>>>(g, in, c->ws.ctr);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "import_kernel");
}

}  // namespace sslic
