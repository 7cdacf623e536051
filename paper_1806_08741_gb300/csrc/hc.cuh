// hc.cuh -- assignment + map update for float images with many channels
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
//     split into two BF16 parts (x~ ~ hi + lo, 16 significant bits), and
//     x~.c~ = hi.hi + hi.lo + lo.hi comes from three tcgen05 MMAs per 16
//     channels (M = 128 voxels, N = 32 candidate slots, BF16 inputs, FP32
//     accumulation in tensor memory).  A bound E_k on |approx D^2_k -
//     canonical D^2_k| is computed per pair: the split's rounding enters as
//     delta (2 ||b|| + 3 delta) with delta = (2^-16 + 2^-23)(||x~|| + ||c~||)
//     and b = (hi + lo)_x - (hi + lo)_c; the dropped lo.lo term, the FP32
//     accumulation, the FP32 norms and the canonical sum add terms in
//     ||x~|| ||c~|| and in the magnitudes.  The best approximate candidate
//     k1 is taken only when every other covering candidate k has
//     approx_k - E_k > approx_k1 + E_k1; otherwise the voxel is re-evaluated
//     with the exact form.  Either way the label is the exact form's label.
//
// A CTA of 128 threads owns a tile of 128 voxels (16x8 pixels or 8x4x4
// voxels), one voxel per thread, its features in registers (the channel
// count is a template parameter, C zero-padded to it).  Tiles reached by
// more than 32 centres go to the per-voxel kernel.  The map step sums the
// features, staged in shared memory, per (channel, part of the tile) in FP32
// along runs of equal labels, adds the runs in double per slot and the
// slots to the double-precision sums with one FP64 atomic per (slot,
// channel); positions and counts are exact integers.
#pragma once
#include <cuda_bf16.h>

#include <atomic>

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

// channel count of the instantiation serving C channels (C is zero-padded to it)
__host__ __device__ inline int ct_of(int C) { return C <= 16 ? 16 : C <= 32 ? 32 : C <= 48 ? 48 : C <= 64 ? 64 : C <= 96 ? 96 : 128; }

// dynamic shared memory for CT channels: the two BF16 planes (high and low
// parts) of the voxel operand A and the centre operand B, then the FP32
// candidate features
// then, for the map step, the tile's features in FP32, channel-major with a
// row pitch of kTV + 1 floats (the tensor-core form reuses its operand region
// once its MMAs are done)
constexpr int kXP = kTV + 1;
template <int CT, bool MMA>
struct Lay {
    static constexpr size_t A = (size_t)kTV * CT * 2, B = (size_t)kNC * CT * 2;
    static constexpr size_t a_hi = 0, a_lo = MMA ? A : 0, b_hi = MMA ? 2 * A : 0, b_lo = MMA ? 2 * A + B : 0;
    static constexpr size_t cf = MMA ? 2 * A + 2 * B : 0;
    static constexpr size_t xs = MMA ? 0 : cf + (size_t)kNC * CT * 4;
    static constexpr size_t end = MMA ? cf + (size_t)kNC * CT * 4 : xs + (size_t)CT * kXP * 4;
    static_assert(!MMA || (size_t)CT * kXP * 4 <= 2 * A + 2 * B, "features fit the operand region");
};

struct Fixed {
    float cpos[kNC][3];
    float mu[kMaxC];
    float ncs[kNC];          // sum of squares of c~_hi + c~_lo
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

template <int CT, bool MMA>
constexpr size_t smem_bytes() { return Lay<CT, MMA>::end + sizeof(Fixed); }

// byte offset of element (row, k) in a canonical K-major no-swizzle operand
template <int CT>
__device__ __forceinline__ uint32_t kmajor_off(int row, int k)
{
    return (uint32_t)(((row >> 3) * (CT >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <int NDIM, bool MMA, int CT>
__global__ void __launch_bounds__(kThreads)
hc_tile_kernel(Geom g, const float* __restrict__ img, const float* __restrict__ ctr,
               const unsigned* __restrict__ bin_start, const int* __restrict__ bin_items,
               int32_t* __restrict__ labels, unsigned long long* __restrict__ acc, double* __restrict__ facc,
               int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count, unsigned* __restrict__ err,
               unsigned long long* __restrict__ rechecks, int ntx, int nty, int64_t tile0,
               float* __restrict__ dbg_dots, int* __restrict__ dbg_cand, float* __restrict__ dbg_mu,
               const int* __restrict__ lists)
{
    using TL = Tile<NDIM>;
    using LY = Lay<CT, MMA>;
    constexpr int TX = TL::TX, TY = TL::TY, TZ = TL::TZ;
    static_assert(TX * TY * TZ == kTV, "tile size");
    extern __shared__ __align__(1024) unsigned char smem[];
    const int C = g.C;
    Fixed& f = *reinterpret_cast<Fixed*>(smem + LY::end);
    float* cf = reinterpret_cast<float*>(smem + LY::cf);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t tile = tile0 >= 0 ? tile0 : (int64_t)blockIdx.x;
    const int X0 = (int)(tile % ntx) * TX;
    const int Y0 = (int)((tile / ntx) % nty) * TY;
    const int Z0 = (int)(tile / ((int64_t)ntx * nty)) * TZ;
    const int ex = (int)imin64(TX, g.N[0] - X0), ey = (int)imin64(TY, g.N[1] - Y0), ez = (int)imin64(TZ, g.N[2] - Z0);

    // with lists: this thread's entry of the tile's candidate record (count,
    // then the indices in ascending order), loaded before the features
    int lk = -1;
    if (lists && tid < kTileListStride) lk = __ldg(lists + tile * kTileListStride + tid);
    if (tid == 0) { f.nstage = 0; f.ncand = 0; f.nrecheck = 0; }
    if (MMA) {
        if (warp == 0) {
            tc::tmem_alloc(&f.tmem, 32);
            tc::tmem_relinquish();
            tc::fence_before_sync();
        }
        if (tid == 0) tc::mbar_init(&f.mbar, 1);
    }
    // ---- this thread's voxel: features into registers (zero-padded to CT) ----
    const int v = tid;
    const int xl = v % TX, yl = (v / TX) % TY, zl = v / (TX * TY);
    const bool valid = xl < ex && yl < ey && zl < ez;
    const int X[3] = {X0 + xl, Y0 + yl, Z0 + zl};
    const int64_t q = valid ? vidx(g, X[0], X[1], X[2]) : 0;
    auto load_x = [&](float (&xv)[CT]) {
#pragma unroll
        for (int c = 0; c < CT; ++c) xv[c] = 0.0f;
        if (valid) {
            const float* src = img + q * C;
            if (C == CT) {
#pragma unroll
                for (int j = 0; j < CT / 4; ++j) {
                    const float4 t = __ldg(reinterpret_cast<const float4*>(src) + j);
                    xv[4 * j] = t.x; xv[4 * j + 1] = t.y; xv[4 * j + 2] = t.z; xv[4 * j + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int c = 0; c < CT; ++c)
                    if (c < C) xv[c] = __ldg(src + c);
            }
        }
    };
    float x[CT];
    load_x(x);
    // ---- candidates: centres of the 3^n bins around the tile whose window meets it ----
    const int T0[3] = {X0, Y0, Z0};
    const int E[3] = {ex, ey, ez};
    int blo[3], bhi[3];
    for (int d = 0; d < 3; ++d) {
        blo[d] = max(0, T0[d] / g.S[d] - 1);
        bhi[d] = min((int)g.nb[d] - 1, (T0[d] + E[d] - 1) / g.S[d] + 1);
    }
    const int nbx = bhi[0] - blo[0] + 1, nby = bhi[1] - blo[1] + 1, nbz = bhi[2] - blo[2] + 1;
    if (lists && tid == 0) f.ncand = lk;
    __syncthreads();
    int nc;
    if (lists) {
        nc = f.ncand;
        if (nc < 0 || nc > kNC) {  // block-uniform: the per-voxel kernel takes this tile
            if (nc > kNC && tid == 0) ovf_tiles[atomicAdd(ovf_count, 1u)] = tile;
            if (MMA && warp == 0) tc::tmem_dealloc(f.tmem, 32);
            return;
        }
        if (tid >= 1 && tid <= nc) {
            const int r = tid - 1;
            f.cand[r] = lk;
            const float* row = ctr + (int64_t)lk * g.CW;
            f.cpos[r][0] = row[C];
            f.cpos[r][1] = row[C + 1];
            f.cpos[r][2] = row[C + 2];
        }
    } else {
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
        nc = f.ncand;
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
    }
    __syncthreads();
    // the listed centres' features (rows beyond nc are never read)
    for (int i = tid; i < nc * CT; i += kThreads) {
        const int r = i / CT, c = i % CT;
        cf[i] = c < C ? ctr[(int64_t)f.cand[r] * g.CW + c] : 0.0f;
    }
    __syncthreads();

    // ---- covering candidates and their spatial terms ----
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
    // exact canonical D^2 against slot r (the per-voxel kernel's arithmetic;
    // the zero padding beyond C adds exact zeros)
    auto exact = [&](const float (&xv)[CT], int r) -> float {
        const float4* cr = reinterpret_cast<const float4*>(cf + r * CT);
        float dc = 0.0f;
#pragma unroll
        for (int j = 0; j < CT / 4; ++j) {
            const float4 cc = cr[j];
            const float cv[4] = {cc.x, cc.y, cc.z, cc.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float e = __fsub_rn(xv[4 * j + t], cv[t]);
                const float sq = __fmul_rn(e, e);
                dc = (j == 0 && t == 0) ? sq : __fadd_rn(dc, sq);
            }
        }
        return __fadd_rn(dc, spatial(r));
    };
    // two covering candidates at a time: their sums are independent chains
    // (each chain keeps the canonical order)
    auto exact2 = [&](const float (&xv)[CT], int ra, int rb, float& Da, float& Db) {
        const float4* ca = reinterpret_cast<const float4*>(cf + ra * CT);
        const float4* cb = reinterpret_cast<const float4*>(cf + rb * CT);
        float da = 0.0f, db = 0.0f;
#pragma unroll
        for (int j = 0; j < CT / 4; ++j) {
            const float4 u = ca[j], w = cb[j];
            const float uv[4] = {u.x, u.y, u.z, u.w}, wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float ea = __fsub_rn(xv[4 * j + t], uv[t]), eb = __fsub_rn(xv[4 * j + t], wv[t]);
                const float sa = __fmul_rn(ea, ea), sb = __fmul_rn(eb, eb);
                da = (j == 0 && t == 0) ? sa : __fadd_rn(da, sa);
                db = (j == 0 && t == 0) ? sb : __fadd_rn(db, sb);
            }
        }
        Da = __fadd_rn(da, spatial(ra));
        Db = __fadd_rn(db, spatial(rb));
    };
    auto exact_best = [&](const float (&xv)[CT]) -> int {
        float best = kInfF;
        int bs = kNone;
        for (uint32_t m = cov; m; ) {
            const int ra = __ffs(m) - 1;
            m &= m - 1;
            if (m) {
                const int rb = __ffs(m) - 1;
                m &= m - 1;
                float Da, Db;
                exact2(xv, ra, rb, Da, Db);
                if (Da < best) { best = Da; bs = ra; }  // ascending slots = ascending k
                if (Db < best) { best = Db; bs = rb; }
            } else {
                const float D = exact(xv, ra);
                if (D < best) { best = D; bs = ra; }
            }
        }
        return bs;
    };

    int bs = kNone;
    if constexpr (!MMA) {
        bs = exact_best(x);
        // the features for the map step, channel-major (the registers are free after this)
        float* xs = reinterpret_cast<float*>(smem + LY::xs);
#pragma unroll
        for (int c = 0; c < CT; ++c) xs[c * kXP + v] = x[c];
    } else {
        // shift: the mean of the candidates' features
        for (int c = tid; c < CT; c += kThreads) {
            float s = 0.0f;
            for (int r = 0; r < nc; ++r) s += cf[r * CT + c];
            f.mu[c] = (nc && c < C) ? s / (float)nc : 0.0f;
        }
        __syncthreads();
        unsigned char* Ahi = smem + LY::a_hi;
        unsigned char* Alo = smem + LY::a_lo;
        unsigned char* Bhi = smem + LY::b_hi;
        unsigned char* Blo = smem + LY::b_lo;
        // A row v: x~ = x - mu split into two BF16 parts, two channels per
        // conversion; ||x~||^2 in FP32 (its distance to ||hi + lo||^2 enters the bound)
        float nxt = 0.0f;
#pragma unroll
        for (int c = 0; c < CT; c += 2) {
            const float x0 = __fsub_rn(x[c], f.mu[c]), x1 = __fsub_rn(x[c + 1], f.mu[c + 1]);
            const __nv_bfloat162 hi = __floats2bfloat162_rn(x0, x1);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(__fsub_rn(x0, __low2float(hi)), __fsub_rn(x1, __high2float(hi)));
            nxt = __fmaf_rn(x0, x0, nxt);
            nxt = __fmaf_rn(x1, x1, nxt);
            *reinterpret_cast<__nv_bfloat162*>(Ahi + kmajor_off<CT>(v, c)) = hi;
            *reinterpret_cast<__nv_bfloat162*>(Alo + kmajor_off<CT>(v, c)) = lo;
        }
        // B rows: one thread per slot (empty slots are zero)
        if (tid < kNC) {
            const int r = tid;
            float nct = 0.0f;
            for (int c = 0; c < CT; c += 2) {
                const float c0 = r < nc ? __fsub_rn(cf[r * CT + c], f.mu[c]) : 0.0f;
                const float c1 = r < nc ? __fsub_rn(cf[r * CT + c + 1], f.mu[c + 1]) : 0.0f;
                const __nv_bfloat162 hi = __floats2bfloat162_rn(c0, c1);
                const __nv_bfloat162 lo =
                    __floats2bfloat162_rn(__fsub_rn(c0, __low2float(hi)), __fsub_rn(c1, __high2float(hi)));
                nct = __fmaf_rn(c0, c0, nct);
                nct = __fmaf_rn(c1, c1, nct);
                *reinterpret_cast<__nv_bfloat162*>(Bhi + kmajor_off<CT>(r, c)) = hi;
                *reinterpret_cast<__nv_bfloat162*>(Blo + kmajor_off<CT>(r, c)) = lo;
            }
            f.ncs[r] = nct;
            f.nrc[r] = sqrtf(nct);
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        tc::fence_after_sync();
        const uint32_t tmem = f.tmem;
        if (tid == 0) {
            // D = Ahi Bhi^T + Ahi Blo^T + Alo Bhi^T over CT / 16 K-steps
            const uint32_t ah = tc::smem_u32(Ahi), al = tc::smem_u32(Alo);
            const uint32_t bh = tc::smem_u32(Bhi), bl = tc::smem_u32(Blo);
            constexpr uint32_t sbo = (uint32_t)(CT / 8) * 128u;
            constexpr uint32_t idesc = tc::idesc_bf16_f32(kTV, kNC);
#pragma unroll 1
            for (int ks = 0; ks < CT / 16; ++ks) {
                const uint32_t o = ks * 256;
                tc::mma_bf16(tmem, tc::smem_desc(ah + o, 128, sbo), tc::smem_desc(bh + o, 128, sbo), idesc, ks > 0);
                tc::mma_bf16(tmem, tc::smem_desc(ah + o, 128, sbo), tc::smem_desc(bl + o, 128, sbo), idesc, true);
                tc::mma_bf16(tmem, tc::smem_desc(al + o, 128, sbo), tc::smem_desc(bh + o, 128, sbo), idesc, true);
            }
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
        // Error bound of the approximate D^2 of each covering candidate r
        // (see the header): a = x - c exactly, b = x~s - c~s with x~s = hi + lo
        //   ||b - a|| <= delta = (2^-16 + 2^-23)(||x~|| + ||c~||)
        //   dot = x~s.c~s - sum lo_x lo_c, |sum lo_x lo_c| <= 1.01 2^-16 ||x~|| ||c~||
        //   FP32 accumulation of 3 CT products: (3 CT + 2) 2^-22 ||x~|| ||c~|| (generous)
        //   ||x~||^2 and ||c~||^2 stand for ||x~s||^2 and ||c~s||^2: 2^-14 of each
        //   FP32 rounding of the final sum: 2^-23 |D^|
        const float xn = sqrtf(nxt);
        const float kd = 0x1p-16f + 0x1p-23f;
        const float km = 2.0f * (1.01f * 0x1p-16f + (float)(3 * CT + 2) * 0x1p-22f);
        auto approx = [&](int r, float dt, float& D, float& Eb) {
            const float ncr = f.ncs[r], cn = f.nrc[r];
            const float df = __fsub_rn(__fadd_rn(nxt, ncr), __fmul_rn(2.0f, dt));
            const float rho = (km * 1.01f * xn * cn + 0x1p-14f * 1.01f * (nxt + ncr) + 0x1p-23f * fabsf(df)) * 1.001f;
            const float del = kd * (xn + cn) * 1.001f;
            const float bn = sqrtf(fmaxf(df + rho, 0.0f));
            const float ef = rho + del * (2.0f * bn + 3.0f * del);
            const float ds = spatial(r);
            D = __fadd_rn(df, ds);
            Eb = (ef + (float)(CT + 6) * 0x1p-24f * (fabsf(df) + ef + ds)) * 1.01f + 1e-30f;
        };
        int k1 = kNone;
        float b1 = kInfF, e1 = 0.0f;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            if (!(cov >> r & 1u)) continue;
            float D, Eb;
            approx(r, dot[r], D, Eb);
            if (D < b1) { b1 = D; e1 = Eb; k1 = r; }
        }
        bool sep = k1 != kNone;
        const float hi1 = b1 + e1;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            if (!(cov >> r & 1u) || r == k1) continue;
            float D, Eb;
            approx(r, dot[r], D, Eb);
            if (!(D - Eb > hi1)) sep = false;
        }
        if (sep) bs = k1;
        else if (cov) {
            float xr[CT];  // reloaded (cache hit), so x need not stay live through the MMA
            load_x(xr);
            bs = exact_best(xr);
            atomicAdd(&f.nrecheck, 1u);
        }
        tc::fence_before_sync();
    }
    f.slot[v] = (uint8_t)bs;
    if (valid && !dbg_dots) labels[q] = bs == kNone ? -1 : f.cand[bs];
    if constexpr (MMA) {
        // the features for the map step, into the operand region: every thread
        // has seen the MMAs complete, so nothing reads it any more
        float xr2[CT];
        load_x(xr2);
        float* xs = reinterpret_cast<float*>(smem + LY::xs);
#pragma unroll
        for (int c = 0; c < CT; ++c) xs[c * kXP + v] = xr2[c];
    }
    for (int i = tid; i < nc * 4; i += kThreads) (&f.pacc[0][0])[i] = 0u;
    __syncthreads();
    if (MMA && warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(f.tmem, 32);
    }
    if (dbg_dots) return;

    // ---- map step: positions and counts per slot in shared memory; features
    //      staged channel-major, summed in FP32 along runs of equal slots,
    //      the runs added in double per slot and leaving through one FP64
    //      atomic per (slot, channel) ----
    if (bs != kNone) {
        atomicAdd(&f.pacc[bs][0], (unsigned)xl);
        atomicAdd(&f.pacc[bs][1], (unsigned)yl);
        atomicAdd(&f.pacc[bs][2], (unsigned)zl);
        atomicAdd(&f.pacc[bs][3], 1u);
    }
    // per-slot sums in double in the candidate-feature region (no longer
    // read) when they fit it; else every run goes straight to the FP64 sums
    double* dsum = reinterpret_cast<double*>(cf);
    const bool tile_sums = 2 * nc <= kNC;
    if (tile_sums)
        for (int i = tid; i < nc * CT; i += kThreads) dsum[i] = 0.0;
    __syncthreads();
    {
        const int parts = kThreads / C;
        if (tid < parts * C) {
            const int c = tid % C, part = tid / C;
            const int v0 = part * kTV / parts, v1 = (part + 1) * kTV / parts;
            const float* xr = reinterpret_cast<const float*>(smem + LY::xs) + c * kXP;
            auto flush = [&](int r, float sum) {
                if (tile_sums) atomicAdd(&dsum[r * CT + c], (double)sum);
                else atomicAdd(&facc[(int64_t)f.cand[r] * C + c], (double)sum);
            };
            int cur = kNone;
            float sum = 0.0f;
            for (int w = v0; w < v1; ++w) {
                const int sl = f.slot[w];
                if (sl != cur) {
                    if (cur != kNone) flush(cur, sum);
                    cur = sl;
                    sum = 0.0f;
                }
                if (sl != kNone) sum = __fadd_rn(sum, xr[w]);
            }
            if (cur != kNone) flush(cur, sum);
        }
    }
    __syncthreads();
    if (tile_sums)
        for (int i = tid; i < nc * C; i += kThreads) {
            const int r = i / C, c = i % C;
            if (f.pacc[r][3]) atomicAdd(&facc[(int64_t)f.cand[r] * C + c], dsum[r * CT + c]);
        }
    __syncthreads();
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

template <int NDIM, bool MMA, int CT>
int launch_hc_ct(sslic_ctx* c, const float* img, int32_t* labels, cudaStream_t st, int64_t tile0,
                        float* dbg_dots, int* dbg_cand, float* dbg_mu)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    using TL = hc::Tile<NDIM>;
    const int ntx = (int)((g.N[0] + TL::TX - 1) / TL::TX), nty = (int)((g.N[1] + TL::TY - 1) / TL::TY);
    const int64_t ntiles = hc_num_tiles(g);
    constexpr size_t smem = hc::smem_bytes<CT, MMA>();
    // the shared-memory limit is raised once per device (a host call that
    // otherwise costs every launch of this short kernel)
    static std::atomic<unsigned> smem_set{0};
    const unsigned dbit = 1u << (c->device & 31);
    int rc;
    if (!(smem_set.load(std::memory_order_relaxed) & dbit)) {
        if ((rc = cuda_check(c, cudaFuncSetAttribute(hc::hc_tile_kernel<NDIM, MMA, CT>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "smem attribute")))
            return rc;
        smem_set.fetch_or(dbit);
    }
    if ((rc = cuda_check(c, cudaMemsetAsync(w.ovf_count, 0, sizeof(unsigned), st), "memset ovf"))) return rc;
    // the tiles' candidate records (not for the one-tile probe)
    const bool lists = w.tile_lists && tile0 < 0;
    if (lists && (rc = launch_tile_lists(c, NDIM, TL::TX, TL::TY, TL::TZ, ntx, nty, 0, ntiles, st))) return rc;
    const int pr = tile0 < 0 ? prof_begin(c, SSLIC_PHASE_ASSIGN, st) : -1;
    hc::hc_tile_kernel<NDIM, MMA, CT><<<tile0 < 0 ? (unsigned)ntiles : 1u, hc::kThreads, smem, st>>>(
        g, img, w.ctr, w.bin_start, w.bin_items, labels, w.acc, w.facc, w.ovf_tiles, w.ovf_count, w.hc_err,
        w.hc_rechecks, ntx, nty, tile0, dbg_dots, dbg_cand, dbg_mu, lists ? w.tile_lists : nullptr);
    count_launch(c);
    prof_end(c, pr, st);
    if ((rc = cuda_check(c, cudaGetLastError(), "hc_tile_kernel"))) return rc;
    if (tile0 >= 0) return SSLIC_OK;
    return launch_voxel_tiles<float>(c, img, labels, TL::TX, TL::TY, TL::TZ, ntx, nty, st);
}

}  // namespace sslic

// explicit instantiation of the launcher for one (dims, form, channel count)
#define SSLIC_HC_INSTANTIATE(NDIM, MMA, CT)                                                                  \
    template int sslic::launch_hc_ct<NDIM, MMA, CT>(sslic_ctx*, const float*, int32_t*, cudaStream_t, int64_t, \
                                                    float*, int*, float*);
