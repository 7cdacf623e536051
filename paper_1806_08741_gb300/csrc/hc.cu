// hc.cu -- assignment + map update for float images with many channels
// (16 <= C <= 128; 2-D and 3-D), e.g. hyperspectral images.
//
// The distance is the one of Sec. 2.1 (feature term + weighted spatial
// term) and the candidates are the centres whose 2S window covers the voxel
// (Sec. 2.2), ties to the lowest cluster index.  Two forms:
//
//  exact (precision 0): the canonical single-precision D^2 of the per-voxel
//     kernel, e_c = I_c - C_c, dc = (((e_0^2 + e_1^2) + e_2^2) + ...), so
//     the labels are bit-identical to it;
//  tensor core (precision 1, C >= 32): the feature term of every (voxel,
//     candidate) pair from ||x~||^2 + ||c~||^2 - 2 x~.c~, where x~ = x - mu,
//     c~ = c - mu are shifted by the mean mu of the tile's candidates and
//     rounded to BF16, and x~.c~ is one tcgen05 MMA per 16 channels (M = 128
//     voxels, N = 32 candidate slots, FP32 accumulation in tensor memory).
//     A bound E_k on |approx D^2_k - canonical D^2_k| is computed per pair
//     (BF16 operand rounding enters as delta (2 ||b|| + 3 delta) with
//     delta = (2^-8 + 2^-23)(||x~|| + ||c~||), b = x~_bf - c~_bf; FP32
//     rounding of the norms, the accumulation and the canonical sum add
//     relative terms).  The best approximate candidate k1 is taken only when
//     every other covering candidate k has approx_k - E_k > approx_k1 + E_k1;
//     otherwise the voxel is re-evaluated with the exact form.  Either way
//     the label is the exact form's label.
//
// A CTA of 128 threads owns a tile of 128 voxels (16x8 pixels or 8x4x4
// voxels), one voxel per thread.  Tiles reached by more than 32 centres go
// to the per-voxel kernel.  The map step sums the voxel features per slot in
// double precision (runs along the tile's voxel order per channel), then one
// FP64 atomic per (centre, channel) leaves the tile.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace sslic {
namespace hc {

constexpr int kThreads = 128;   // one voxel per thread = one MMA row
constexpr int kTV = 128;
constexpr int kNC = 32;         // candidate slots per tile = MMA N
constexpr int kStage = 128;     // gathered centres before filtering
constexpr int kMaxC = 128;
constexpr int kMinC = 16;
constexpr int kMinCMma = 32;
constexpr uint8_t kNone = 255;
constexpr float kInfF = __builtin_huge_valf();
constexpr long long kWaitLimit = 1LL << 24;  // mbarrier polls before giving up

template <int NDIM>
struct Tile;
template <>
struct Tile<2> { static constexpr int TX = 16, TY = 8, TZ = 1; };
template <>
struct Tile<3> { static constexpr int TX = 8, TY = 4, TZ = 4; };

// byte layout of the dynamic shared memory for C channels
struct Lay {
    int CP, CK;              // fp32 row pitch (odd), channels rounded up to 16
    size_t a, b, xf, cf, psum, end;
    __host__ __device__ void init(int C)
    {
        CP = C | 1;
        CK = (C + 15) / 16 * 16;
        size_t o = 0;
        auto put = [&](size_t bytes, size_t al) { o = (o + al - 1) / al * al; const size_t r = o; o += bytes; return r; };
        a = put((size_t)kTV * CK * 2, 1024);            // BF16 x~, canonical K-major
        b = put((size_t)kNC * CK * 2, 1024);            // BF16 c~
        const size_t ab_end = o;
        psum = a;                                       // reuses A/B after the MMA
        if (a + (size_t)kNC * C * 8 > ab_end) o = a + (size_t)kNC * C * 8;
        xf = put((size_t)kTV * CP * 4, 16);              // fp32 voxel features
        cf = put((size_t)kNC * C * 4, 16);               // fp32 candidate features
        end = (o + 15) / 16 * 16;
    }
};

struct Fixed {
    float cpos[kNC][3];
    float mu[kMaxC];
    float ncb[kNC];          // sum of squares of the BF16 c~ row
    float nrc[kNC];          // ||c~|| in FP32
    unsigned pacc[kNC][4];   // local x, y, z sums and count per slot
    int cand[kNC];
    int tmp[kNC];
    int stage[kStage];
    uint8_t slot[kTV];
    uint64_t mbar;
    uint32_t tmem;
    int nstage, ncand;
    unsigned nrecheck;
};

__host__ __device__ inline size_t smem_bytes(int C)
{
    Lay L;
    L.init(C);
    return L.end + sizeof(Fixed);
}

// byte offset of element (row, k) in a canonical K-major no-swizzle operand
__device__ __forceinline__ uint32_t kmajor_off(int row, int k, int CK)
{
    return (uint32_t)(((row >> 3) * (CK >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int NDIM, bool MMA>
__global__ void __launch_bounds__(kThreads)
hc_tile_kernel(Geom g, const float* __restrict__ img, const float* __restrict__ ctr,
               const unsigned* __restrict__ bin_start, const int* __restrict__ bin_items,
               int32_t* __restrict__ labels, unsigned long long* __restrict__ acc, double* __restrict__ facc,
               int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count, unsigned* __restrict__ err,
               unsigned long long* __restrict__ rechecks, int ntx, int nty, int64_t tile0,
               float* __restrict__ dbg_dots, int* __restrict__ dbg_cand, float* __restrict__ dbg_mu)
{
    using TL = Tile<NDIM>;
    constexpr int TX = TL::TX, TY = TL::TY, TZ = TL::TZ;
    static_assert(TX * TY * TZ == kTV, "tile size");
    extern __shared__ __align__(1024) unsigned char smem[];
    const int C = g.C;
    Lay L;
    L.init(C);
    const int CP = L.CP, CK = L.CK;
    Fixed& f = *reinterpret_cast<Fixed*>(smem + L.end);
    float* xf = reinterpret_cast<float*>(smem + L.xf);
    float* cf = reinterpret_cast<float*>(smem + L.cf);
    double* psum = reinterpret_cast<double*>(smem + L.psum);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t tile = tile0 >= 0 ? tile0 : (int64_t)blockIdx.x;
    const int X0 = (int)(tile % ntx) * TX;
    const int Y0 = (int)((tile / ntx) % nty) * TY;
    const int Z0 = (int)(tile / ((int64_t)ntx * nty)) * TZ;
    const int ex = (int)imin64(TX, g.N[0] - X0), ey = (int)imin64(TY, g.N[1] - Y0), ez = (int)imin64(TZ, g.N[2] - Z0);

    if (tid == 0) { f.nstage = 0; f.ncand = 0; f.nrecheck = 0; }
    if (MMA) {
        if (warp == 0) {
            tc::tmem_alloc(&f.tmem, 32);
            tc::tmem_relinquish();
            tc::fence_before_sync();
        }
        if (tid == 0) tc::mbar_init(&f.mbar, 1);
    }
    // ---- stage the voxel features (rows of TX voxels are contiguous) ----
    for (int i = tid; i < kTV * C; i += kThreads) {
        const int v = i / C, c = i - v * C;
        const int xl = v % TX, yl = (v / TX) % TY, zl = v / (TX * TY);
        float val = 0.0f;
        if (xl < ex && yl < ey && zl < ez) val = __ldg(img + vidx(g, X0 + xl, Y0 + yl, Z0 + zl) * C + c);
        xf[v * CP + c] = val;
    }
    // ---- candidates: centres of the 3^n bins around the tile whose window meets it ----
    const int T0[3] = {X0, Y0, Z0};
    const int E[3] = {ex, ey, ez};
    int blo[3], bhi[3];
    for (int d = 0; d < 3; ++d) {
        blo[d] = max(0, T0[d] / g.S[d] - 1);
        bhi[d] = min((int)g.nb[d] - 1, (T0[d] + E[d] - 1) / g.S[d] + 1);
    }
    const int nbx = bhi[0] - blo[0] + 1, nby = bhi[1] - blo[1] + 1, nbz = bhi[2] - blo[2] + 1;
    __syncthreads();
    for (int b = tid; b < nbx * nby * nbz; b += kThreads) {
        const int bx = blo[0] + b % nbx, by = blo[1] + (b / nbx) % nby, bz = blo[2] + b / (nbx * nby);
        const int64_t bin = bx + g.nb[0] * (by + g.nb[1] * (int64_t)bz);
        for (unsigned i = bin_start[bin]; i < bin_start[bin + 1]; ++i) {
            const int pos = atomicAdd(&f.nstage, 1);
            if (pos < kStage) f.stage[pos] = bin_items[i];
        }
    }
    __syncthreads();
    const int nst = f.nstage;
    for (int i = tid; i < min(nst, kStage); i += kThreads) {
        const int k = f.stage[i];
        const float* p = ctr + (int64_t)k * g.CW + C;
        bool hit = true;
        for (int d = 0; d < NDIM; ++d) {
            const int lo = (int)ceilf(p[d]) - g.S[d];
            hit = hit && (lo <= T0[d] + E[d] - 1) && (lo + 2 * g.S[d] - 1 >= T0[d]);
        }
        if (hit) {
            const int pos = atomicAdd(&f.ncand, 1);
            if (pos < kNC) f.tmp[pos] = k;
        }
    }
    __syncthreads();
    const int nc = f.ncand;
    if (nst > kStage || nc > kNC) {
        if (tile0 < 0 && tid == 0) ovf_tiles[atomicAdd(ovf_count, 1u)] = tile;
        if (MMA && warp == 0) tc::tmem_dealloc(f.tmem, 32);
        return;  // block-uniform: the per-voxel kernel takes this tile
    }
    for (int i = tid; i < nc; i += kThreads) {
        const int k = f.tmp[i];
        int r = 0;
        for (int j = 0; j < nc; ++j) r += (f.tmp[j] < k);
        f.cand[r] = k;
        const float* row = ctr + (int64_t)k * g.CW;
        f.cpos[r][0] = row[C];
        f.cpos[r][1] = row[C + 1];
        f.cpos[r][2] = row[C + 2];
    }
    __syncthreads();
    for (int i = tid; i < nc * C; i += kThreads) {
        const int r = i / C, c = i - r * C;
        cf[i] = ctr[(int64_t)f.cand[r] * g.CW + c];
    }
    __syncthreads();

    // ---- this thread's voxel: coordinates, covering candidates, spatial terms ----
    const int v = tid;
    const int xl = v % TX, yl = (v / TX) % TY, zl = v / (TX * TY);
    const bool valid = xl < ex && yl < ey && zl < ez;
    const int X[3] = {X0 + xl, Y0 + yl, Z0 + zl};
    uint32_t cov = 0;
    if (valid) {
        for (int r = 0; r < nc; ++r) {
            bool in = true;
            for (int d = 0; d < NDIM; ++d) {
                const int lo = (int)ceilf(f.cpos[r][d]) - g.S[d];
                in = in && X[d] >= lo && X[d] <= lo + 2 * g.S[d] - 1;
            }
            cov |= (in ? 1u : 0u) << r;
        }
    }
    auto spatial = [&](int r) -> float {
        float ds = 0.0f;
        for (int d = 0; d < NDIM; ++d) {
            const float dl = __fsub_rn((float)X[d], f.cpos[r][d]);
            const float t = __fmul_rn(g.w[d], __fmul_rn(dl, dl));
            ds = d == 0 ? t : __fadd_rn(ds, t);
        }
        return ds;
    };
    // exact canonical D^2 against slot r (the per-voxel kernel's arithmetic)
    auto exact = [&](int r) -> float {
        const float* xr = xf + v * CP;
        const float* cr = cf + r * C;
        float dc = 0.0f;
        for (int c = 0; c < C; ++c) {
            const float e = __fsub_rn(xr[c], cr[c]);
            const float sq = __fmul_rn(e, e);
            dc = c == 0 ? sq : __fadd_rn(dc, sq);
        }
        return __fadd_rn(dc, spatial(r));
    };
    auto exact_best = [&]() -> int {
        float best = kInfF;
        int bs = kNone;
        for (uint32_t m = cov; m; m &= m - 1) {
            const int r = __ffs(m) - 1;
            const float D = exact(r);
            if (D < best) { best = D; bs = r; }  // ascending slots = ascending k
        }
        return bs;
    };

    int bs = kNone;
    if constexpr (!MMA) {
        bs = exact_best();
    } else {
        // shift: the mean of the candidates' features
        for (int c = tid; c < C; c += kThreads) {
            float s = 0.0f;
            for (int r = 0; r < nc; ++r) s += cf[r * C + c];
            f.mu[c] = nc ? s / (float)nc : 0.0f;
        }
        __syncthreads();
        unsigned char* A = smem + L.a;
        unsigned char* B = smem + L.b;
        // A row v: BF16 of x~ (zero-padded to CK channels); norms
        float nxt = 0.0f, nxb = 0.0f;
        for (int c = 0; c < CK; ++c) {
            float xt = 0.0f;
            if (c < C) xt = __fsub_rn(xf[v * CP + c], f.mu[c]);
            const __nv_bfloat16 hb = __float2bfloat16_rn(xt);
            const float xb = __bfloat162float(hb);
            nxt = __fadd_rn(nxt, __fmul_rn(xt, xt));
            nxb = __fadd_rn(nxb, __fmul_rn(xb, xb));
            *reinterpret_cast<__nv_bfloat16*>(A + kmajor_off(v, c, CK)) = hb;
        }
        // B rows: one thread per slot (empty slots are zero)
        if (tid < kNC) {
            const int r = tid;
            float nct = 0.0f, ncb = 0.0f;
            for (int c = 0; c < CK; ++c) {
                float ct = 0.0f;
                if (r < nc && c < C) ct = __fsub_rn(cf[r * C + c], f.mu[c]);
                const __nv_bfloat16 hb = __float2bfloat16_rn(ct);
                const float cb = __bfloat162float(hb);
                nct = __fadd_rn(nct, __fmul_rn(ct, ct));
                ncb = __fadd_rn(ncb, __fmul_rn(cb, cb));
                *reinterpret_cast<__nv_bfloat16*>(B + kmajor_off(r, c, CK)) = hb;
            }
            f.ncb[r] = ncb;
            f.nrc[r] = sqrtf(nct);
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        tc::fence_after_sync();
        const uint32_t tmem = f.tmem;
        if (tid == 0) {
            const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(B);
            const uint32_t sbo = (uint32_t)(CK / 8) * 128u;
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kTV, kNC);
            for (int ks = 0; ks < CK / 16; ++ks)
                tc::mma_bf16(tmem, tc::smem_desc(a0 + ks * 256, 128, sbo), tc::smem_desc(b0 + ks * 256, 128, sbo),
                             idesc, ks > 0);
            tc::mma_commit(&f.mbar);
        }
        bool done = false;
        for (long long it = 0; it < kWaitLimit && !done; ++it) done = tc::mbar_try_wait(&f.mbar, 0);
        if (!done) atomicExch(err, 1u);
        tc::fence_after_sync();
        float dot[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), dot);
        if (dbg_dots) {
            for (int r = 0; r < kNC; ++r) dbg_dots[v * kNC + r] = dot[r];
            if (tid < kNC) dbg_cand[tid] = tid < nc ? f.cand[tid] : -1;
            for (int c = tid; c < C; c += kThreads) dbg_mu[c] = f.mu[c];
        }
        // approximate distances, their bounds, and the separation test
        const float u = 0x1p-8f + 0x1p-23f;
        const float xn = sqrtf(nxt);
        const float gm = (float)(C + 2) * 0x1p-22f;
        float ap[32], eb[32];
        int k1 = kNone;
        float b1 = kInfF;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            ap[r] = kInfF;
            eb[r] = 0.0f;
            if (!(cov >> r & 1u)) continue;
            const float ncr = f.ncb[r];
            const float df = __fsub_rn(__fadd_rn(nxb, ncr), __fmul_rn(2.0f, dot[r]));
            const float rho = ((float)(C + 3) * 0x1p-24f * (nxb + ncr) + 2.0f * gm * sqrtf(nxb * ncr) +
                               0x1p-23f * fabsf(df)) * 1.001f;
            const float del = u * (xn + f.nrc[r]) * 1.001f;
            const float bn = sqrtf(fmaxf(df + rho, 0.0f));
            const float ef = rho + del * (2.0f * bn + 3.0f * del);
            const float ds = spatial(r);
            const float D = __fadd_rn(df, ds);
            ap[r] = D;
            eb[r] = (ef + (float)(C + 6) * 0x1p-24f * (fabsf(df) + ef + ds)) * 1.01f + 1e-30f;
            if (D < b1) { b1 = D; k1 = r; }
        }
        bool sep = k1 != kNone;
        float hi1 = 0.0f;
#pragma unroll
        for (int r = 0; r < 32; ++r)
            if (r == k1) hi1 = ap[r] + eb[r];
#pragma unroll
        for (int r = 0; r < 32; ++r)
            if ((cov >> r & 1u) && r != k1 && !(ap[r] - eb[r] > hi1)) sep = false;
        if (sep) bs = k1;
        else if (cov) {
            bs = exact_best();
            atomicAdd(&f.nrecheck, 1u);
        }
        tc::fence_before_sync();
    }
    f.slot[v] = (uint8_t)bs;
    if (valid && !dbg_dots) labels[vidx(g, X[0], X[1], X[2])] = bs == kNone ? -1 : f.cand[bs];
    __syncthreads();
    if (MMA && warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(f.tmem, 32);
    }
    if (dbg_dots) return;

    // ---- map step: per-slot sums of the tile, then one atomic per (centre, field) ----
    for (int i = tid; i < nc * C; i += kThreads) psum[i] = 0.0;
    for (int i = tid; i < nc * 4; i += kThreads) (&f.pacc[0][0])[i] = 0u;
    __syncthreads();
    if (bs != kNone) {
        atomicAdd(&f.pacc[bs][0], (unsigned)xl);
        atomicAdd(&f.pacc[bs][1], (unsigned)yl);
        atomicAdd(&f.pacc[bs][2], (unsigned)zl);
        atomicAdd(&f.pacc[bs][3], 1u);
    }
    {
        // thread -> (channel, part of the tile): runs of equal slots summed in double
        const int parts = kThreads / C;
        if (tid < parts * C) {
            const int c = tid % C, part = tid / C;
            const int v0 = part * kTV / parts, v1 = (part + 1) * kTV / parts;
            int cur = kNone;
            double s = 0.0;
            for (int w = v0; w < v1; ++w) {
                const int sl = f.slot[w];
                if (sl != cur) {
                    if (cur != kNone) atomicAdd(&psum[cur * C + c], s);
                    cur = sl;
                    s = 0.0;
                }
                if (sl != kNone) s += (double)xf[w * CP + c];
            }
            if (cur != kNone) atomicAdd(&psum[cur * C + c], s);
        }
    }
    __syncthreads();
    for (int i = tid; i < nc * C; i += kThreads) {
        const int r = i / C;
        if (f.pacc[r][3]) atomicAdd(&facc[(int64_t)f.cand[r] * C + (i - r * C)], psum[i]);
    }
    for (int i = tid; i < nc * 4; i += kThreads) {
        const int r = i / 4, j = i % 4;
        const unsigned long long cnt = f.pacc[r][3];
        if (!cnt) continue;
        unsigned long long val = f.pacc[r][j];
        if (j == 0) val += cnt * (unsigned long long)X0;
        if (j == 1) val += cnt * (unsigned long long)Y0;
        if (j == 2) val += cnt * (unsigned long long)Z0;
        atomicAdd(&acc[(int64_t)f.cand[r] * g.AW + C + j], val);
    }
    if (MMA && tid == 0 && f.nrecheck) atomicAdd(rechecks, (unsigned long long)f.nrecheck);
}

}  // namespace hc

bool hc_applies(const Geom& g)
{
    return g.dtype == SSLIC_F32 && (g.n == 2 || g.n == 3) && g.C >= hc::kMinC && g.C <= hc::kMaxC;
}

int64_t hc_num_tiles(const Geom& g)
{
    if (g.n == 3)
        return ((g.N[0] + 7) / 8) * ((g.N[1] + 3) / 4) * ((g.N[2] + 3) / 4);
    return ((g.N[0] + 15) / 16) * ((g.N[1] + 7) / 8);
}

template <int NDIM, bool MMA>
static int launch_hc_impl(sslic_ctx* c, const float* img, int32_t* labels, cudaStream_t st, int64_t tile0,
                          float* dbg_dots, int* dbg_cand, float* dbg_mu)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    using TL = hc::Tile<NDIM>;
    const int ntx = (int)((g.N[0] + TL::TX - 1) / TL::TX), nty = (int)((g.N[1] + TL::TY - 1) / TL::TY);
    const int64_t ntiles = hc_num_tiles(g);
    const size_t smem = hc::smem_bytes(g.C);
    int rc = cuda_check(c, cudaFuncSetAttribute(hc::hc_tile_kernel<NDIM, MMA>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                        "smem attribute");
    if (rc) return rc;
    if ((rc = cuda_check(c, cudaMemsetAsync(w.ovf_count, 0, sizeof(unsigned), st), "memset ovf"))) return rc;
    const int pr = tile0 < 0 ? prof_begin(c, SSLIC_PHASE_ASSIGN, st) : -1;
    hc::hc_tile_kernel<NDIM, MMA><<<tile0 < 0 ? (unsigned)ntiles : 1u, hc::kThreads, smem, st>>>(
        g, img, w.ctr, w.bin_start, w.bin_items, labels, w.acc, w.facc, w.ovf_tiles, w.ovf_count, w.hc_err,
        w.hc_rechecks, ntx, nty, tile0, dbg_dots, dbg_cand, dbg_mu);
    count_launch(c);
    prof_end(c, pr, st);
    if ((rc = cuda_check(c, cudaGetLastError(), "hc_tile_kernel"))) return rc;
    if (tile0 >= 0) return SSLIC_OK;
    return launch_voxel_tiles<float>(c, img, labels, TL::TX, TL::TY, TL::TZ, ntx, nty, st);
}

int launch_hc(sslic_ctx* c, const float* img, int32_t* labels, cudaStream_t st)
{
    const bool mma = c->p.precision == 1 && c->g.C >= hc::kMinCMma;
    if (c->g.n == 3)
        return mma ? launch_hc_impl<3, true>(c, img, labels, st, -1, nullptr, nullptr, nullptr)
                   : launch_hc_impl<3, false>(c, img, labels, st, -1, nullptr, nullptr, nullptr);
    return mma ? launch_hc_impl<2, true>(c, img, labels, st, -1, nullptr, nullptr, nullptr)
               : launch_hc_impl<2, false>(c, img, labels, st, -1, nullptr, nullptr, nullptr);
}

int launch_hc_probe(sslic_ctx* c, const float* img, int32_t* labels, int64_t tile, float* dots, int* cand,
                    float* mu, cudaStream_t st)
{
    if (c->g.n == 3) return launch_hc_impl<3, true>(c, img, labels, st, tile, dots, cand, mu);
    return launch_hc_impl<2, true>(c, img, labels, st, tile, dots, cand, mu);
}

}  // namespace sslic

using namespace sslic;

extern "C" int sslic_precision_probe(sslic_ctx* c, const void* image_dev, const float* centres_dev, int64_t tile,
                                     float* dots_host, int32_t* cand_host, float* mu_host)
{
    if (!c || !image_dev || !centres_dev || !dots_host || !cand_host || !mu_host) return SSLIC_EINVAL;
    if (c->p.precision != 1 || !hc_applies(c->g) || tile < 0 || tile >= hc_num_tiles(c->g)) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    const Geom& g = c->g;
    float* dots = nullptr;
    int* cand = nullptr;
    float* mu = nullptr;
    int rc = SSLIC_OK;
    const size_t nd = (size_t)hc::kTV * hc::kNC;
    if ((rc = cuda_check(c, cudaMalloc((void**)&dots, nd * sizeof(float)), "probe buffers")) ||
        (rc = cuda_check(c, cudaMalloc((void**)&cand, hc::kNC * sizeof(int)), "probe buffers")) ||
        (rc = cuda_check(c, cudaMalloc((void**)&mu, g.C * sizeof(float)), "probe buffers")))
        goto done;
    if ((rc = cuda_check(c, cudaMemset(cand, 0xff, hc::kNC * sizeof(int)), "memset"))) goto done;
    if ((rc = launch_import_centres(c, centres_dev, 0)) || (rc = build_bins(c, 0)) ||
        (rc = launch_hc_probe(c, (const float*)image_dev, nullptr, tile, dots, cand, mu, 0)))
        goto done;
    if ((rc = cuda_check(c, cudaDeviceSynchronize(), "probe"))) goto done;
    {
        unsigned h = 0;
        if ((rc = cuda_check(c, cudaMemcpy(&h, c->ws.ovf_count, sizeof(unsigned), cudaMemcpyDeviceToHost), "probe")))
            goto done;
        unsigned e = 0;
        if ((rc = cuda_check(c, cudaMemcpy(&e, c->ws.hc_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "probe")))
            goto done;
        if (e) {
            cudaMemset(c->ws.hc_err, 0, sizeof(unsigned));
            rc = set_error(c, SSLIC_ETIMEOUT, "probe: a bounded wait ran out");
            goto done;
        }
    }
    if ((rc = cuda_check(c, cudaMemcpy(dots_host, dots, nd * sizeof(float), cudaMemcpyDeviceToHost), "probe")) ||
        (rc = cuda_check(c, cudaMemcpy(cand_host, cand, hc::kNC * sizeof(int), cudaMemcpyDeviceToHost), "probe")) ||
        (rc = cuda_check(c, cudaMemcpy(mu_host, mu, g.C * sizeof(float), cudaMemcpyDeviceToHost), "probe")))
        goto done;
    if (cand_host[0] == -1 && cand_host[1] == -1) {
        // the kernel left before the MMA: more candidates than slots (or none)
        int any = 0;
        for (int j = 0; j < hc::kNC; ++j) any |= cand_host[j] != -1;
        if (!any) rc = set_error(c, SSLIC_EUNSUPPORTED, "probe: tile reached by more than 32 centres or none");
    }
done:
    if (dots) cudaFree(dots);
    if (cand) cudaFree(cand);
    if (mu) cudaFree(mu);
    return rc;
}
