// assign_tile.cu -- the fused assignment + map-update kernel for integer
// images with 1 or 3 channels (2-D and 3-D): one SSLIC iteration's hot loop.
//
// Assignment (Sec. 2.1, 2.2, 3.1 step 2): every voxel takes the argmin of
//     D^2 = sum_c (I_c - C_c)^2 + sum_d w_d (x_d - c_d)^2,  w_d = m^2 / S_d^2
// over the centres whose window c_d - S_d <= x_d < c_d + S_d covers it, ties
// to the lowest cluster index (the paper visits centres in ascending k and
// replaces only on a strictly smaller distance).  D^2 is computed with one
// IEEE single-precision rounding per operation in a fixed order, no fused
// multiply-add:
//     e_c = I_c - C_c;  dc = ((e_0^2 + e_1^2) + e_2^2);  t_d = w_d (x_d - c_d)^2
//     ds = ((t_0 + t_1) + t_2);  D^2 = dc + ds
// The map step of the update (Sec. 3.1) is fused: [I(x), x, 1] is summed
// per label in the same pass, so the image is read once per iteration.
//
// Work decomposition.  A CTA (4 warps) owns a tile of 32x8x8 voxels (3-D) or
// 64x32 pixels (2-D):
//  1. stages the tile's channels as bank-padded planes in shared memory;
//  2. gathers the centres of the bins that can reach the tile (3 bins per
//     axis around it), keeps those whose window meets the tile, sorts them by
//     index, and builds per centre the feature pair (C_c, C_c) and per axis
//     the table t_d(x_d) for the tile's coordinates, +inf outside the window
//     (the window test is folded into the distance);
//  3. each warp sweeps 4x4x4 (3-D) / 8x8 (2-D) boxes, two voxels per lane in
//     packed .f32x2 arithmetic, visiting only the centres that reach its box;
//  4. per box, the winners' [I, x, 1] sums are reduced across the warp with
//     redux.sync on bit-packed words (one word carries several small sums)
//     into per-warp accumulators;
//  5. labels leave through coalesced int32 stores, per-tile sums through one
//     uint64 atomic per (centre, field).
// Tiles reached by more than kCap centres are handed to the per-voxel kernel.
#include "common.cuh"

namespace sslic {

namespace tile {

constexpr float kInf = __builtin_huge_valf();
constexpr int kThreads = 128;
constexpr int kWarps = kThreads / 32;
constexpr int kCap = 64;     // candidate centres per tile
constexpr int kStage = 512;  // gathered centres before filtering

template <int NDIM>
struct Cfg;
template <>
struct Cfg<3> {
    static constexpr int TX = 32, TY = 8, TZ = 8;  // 2048 voxels
    static constexpr int WX = 2, WY = 4, WZ = 4;   // lanes -> box 4x4x4 (pairs along x)
};
template <>
struct Cfg<2> {
    static constexpr int TX = 64, TY = 32, TZ = 1;  // 2048 pixels
    static constexpr int WX = 4, WY = 8, WZ = 1;    // box 8x8
};

// per-candidate record in shared memory
template <int C, int NDIM>
struct Cand {
    float2 fe[C];            // (C_c, C_c)
    float2 t1[Cfg<NDIM>::TY];  // (t_1, t_1) by local y
    float2 t2[Cfg<NDIM>::TZ];  // (t_2, t_2) by local z
    float t0[Cfg<NDIM>::TX];   // t_0 by local x
};

// ---- bit-packed per-box sums ------------------------------------------------
__host__ __device__ constexpr int bits_for(unsigned long long v)
{
    int b = 0;
    while (v) { ++b; v >>= 1; }
    return b;
}

// fields: C features, x, y, z (local), count; per warp box of 64 voxels
template <typename T, int C, int NDIM>
struct Pack {
    static constexpr int F = C + 4;
    static constexpr unsigned long long kVmax = sizeof(T) == 1 ? 255ull : 65535ull;
    __host__ __device__ static constexpr int width(int f)
    {
        return f < C ? bits_for(64ull * kVmax)
                     : f == C ? bits_for(64ull * (Cfg<NDIM>::TX - 1))
                     : f == C + 1 ? bits_for(64ull * (Cfg<NDIM>::TY - 1))
                     : f == C + 2 ? bits_for(64ull * (Cfg<NDIM>::TZ - 1))
                                  : bits_for(64ull);
    }
    // greedy first-fit into 32-bit words
    __host__ __device__ static constexpr int word(int f)
    {
        int w = 0, used = 0;
        for (int i = 0; i <= f; ++i) {
            if (used + width(i) > 32) { ++w; used = 0; }
            if (i == f) return w;
            used += width(i);
        }
        return w;
    }
    __host__ __device__ static constexpr int shift(int f)
    {
        int used = 0;
        for (int i = 0; i <= f; ++i) {
            if (used + width(i) > 32) used = 0;
            if (i == f) return used;
            used += width(i);
        }
        return 0;
    }
    static constexpr int NW = word(F - 1) + 1;
};

template <typename T, int C, int NDIM>
struct Smem {
    using G = Cfg<NDIM>;
    static constexpr int TX = G::TX, TY = G::TY, TZ = G::TZ, TV = TX * TY * TZ;
    // channel planes, padded so the lanes of a warp box hit distinct banks
    static constexpr int RPB = TX * (int)sizeof(T) + 4;   // row pitch, bytes
    static constexpr int PPB = TY * RPB + 8;              // plane (z) pitch, bytes
    static constexpr int CPB = ((TZ * PPB + 15) / 16) * 16;  // channel pitch, bytes
    Cand<C, NDIM> cd[kCap];
    alignas(16) unsigned char planes[C * CPB];
    unsigned accw[kWarps][kCap][C + 4];   // per-warp sums: features, x, y, z, count
    float cpos[kCap][3];
    int cand[kCap];
    int tmp[kCap];
    int stage[kStage];
    uint32_t bmask[kCap];
    alignas(4) uint8_t slot[TV];
    int nstage, ncand;
};

template <typename T, int C, int NDIM>
__device__ __forceinline__ unsigned plane_pair(const Smem<T, C, NDIM>& s, int c, int xl, int yl, int zl)
{
    using S = Smem<T, C, NDIM>;
    const unsigned char* p = s.planes + c * S::CPB + zl * S::PPB + yl * S::RPB + xl * (int)sizeof(T);
    if constexpr (sizeof(T) == 1) return *reinterpret_cast<const uint16_t*>(p);
    else return *reinterpret_cast<const uint32_t*>(p);
}

template <typename T>
__device__ __forceinline__ void split_pair(unsigned v, unsigned& lo, unsigned& hi)
{
    if constexpr (sizeof(T) == 1) { lo = v & 0xffu; hi = v >> 8; }
    else { lo = v & 0xffffu; hi = v >> 16; }
}

template <typename T, int C, int NDIM>
__global__ void __launch_bounds__(kThreads, 6)
assign_tile_kernel(Geom g, const T* __restrict__ img, const float* __restrict__ ctr,
                   const unsigned* __restrict__ bin_start, const int* __restrict__ bin_items,
                   int32_t* __restrict__ labels, unsigned long long* __restrict__ acc,
                   int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count, int ntx, int nty)
{
    using G = Cfg<NDIM>;
    using S = Smem<T, C, NDIM>;
    using P = Pack<T, C, NDIM>;
    constexpr int TX = G::TX, TY = G::TY, TZ = G::TZ, TV = TX * TY * TZ;
    constexpr int WX = G::WX, WY = G::WY, WZ = G::WZ;
    constexpr int BX = 2 * WX, BY = WY, BZ = WZ;
    constexpr int NBX = TX / BX, NBY = TY / BY, NBZ = TZ / BZ;
    constexpr int NBOX = NBX * NBY * NBZ;
    constexpr int PASSES = NBOX / kWarps;
    constexpr int F = C + 4;
    static_assert(NBOX % kWarps == 0, "boxes per warp");
    static_assert(NBX + NBY + NBZ <= 32, "box mask bits");
    static_assert(BX * BY * BZ == 64, "64 voxels per warp box");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    S& s = *reinterpret_cast<S*>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const int X0 = (tile % ntx) * TX;
    const int Y0 = ((tile / ntx) % nty) * TY;
    const int Z0 = (tile / (ntx * nty)) * TZ;
    const int N0 = (int)g.N[0], N1 = (int)g.N[1], N2 = (int)g.N[2];
    const int ex = min(TX, N0 - X0), ey = min(TY, N1 - Y0), ez = min(TZ, N2 - Z0);

    if (tid == 0) { s.nstage = 0; s.ncand = 0; }
    for (int i = tid; i < kWarps * kCap * F; i += kThreads) (&s.accw[0][0][0])[i] = 0u;

    // ---- 1. stage the tile as channel planes --------------------------------
    if constexpr (sizeof(T) == 1 && C == 3) {
        // full rows: 12-byte groups (4 voxels) -> 3 words per plane row segment
        const bool fast = (ex == TX) && ((N0 * 3) % 4 == 0) && (((uintptr_t)img & 3) == 0);
        if (fast) {
            constexpr int GPR = TX / 4;  // groups per row
            for (int i = tid; i < TY * TZ * GPR; i += kThreads) {
                const int r = i / GPR, gi = i % GPR, yl = r % TY, zl = r / TY;
                uint32_t a = 0, b = 0, cc = 0;
                if (yl < ey && zl < ez) {
                    const uint32_t* src = reinterpret_cast<const uint32_t*>(
                        img + (vidx(g, X0, Y0 + yl, Z0 + zl) + gi * 4) * 3);
                    a = __ldg(src);
                    b = __ldg(src + 1);
                    cc = __ldg(src + 2);
                }
                // bytes: a = R0 G0 B0 R1, b = G1 B1 R2 G2, cc = B2 R3 G3 B3
                const uint32_t R = __byte_perm(__byte_perm(a, b, 0x0630), cc, 0x5210);
                const uint32_t Gv = __byte_perm(__byte_perm(a, b, 0x0741), cc, 0x6210);
                const uint32_t B = __byte_perm(__byte_perm(a, b, 0x0052), cc, 0x7410);
                unsigned char* row = s.planes + zl * S::PPB + yl * S::RPB + gi * 4;
                *reinterpret_cast<uint32_t*>(row) = R;
                *reinterpret_cast<uint32_t*>(row + S::CPB) = Gv;
                *reinterpret_cast<uint32_t*>(row + 2 * S::CPB) = B;
            }
        } else {
            for (int i = tid; i < TV; i += kThreads) {
                const int xl = i % TX, yl = (i / TX) % TY, zl = i / (TX * TY);
                uint8_t v[3] = {0, 0, 0};
                if (xl < ex && yl < ey && zl < ez) {
                    const int64_t q = vidx(g, X0 + xl, Y0 + yl, Z0 + zl) * 3;
                    v[0] = img[q]; v[1] = img[q + 1]; v[2] = img[q + 2];
                }
                unsigned char* p = s.planes + zl * S::PPB + yl * S::RPB + xl;
                p[0] = v[0]; p[S::CPB] = v[1]; p[2 * S::CPB] = v[2];
            }
        }
    } else {
        for (int i = tid; i < TV * C; i += kThreads) {
            const int e = i / C, c = i % C;
            const int xl = e % TX, yl = (e / TX) % TY, zl = e / (TX * TY);
            T v = T(0);
            if (xl < ex && yl < ey && zl < ez) v = img[vidx(g, X0 + xl, Y0 + yl, Z0 + zl) * C + c];
            *reinterpret_cast<T*>(s.planes + c * S::CPB + zl * S::PPB + yl * S::RPB + xl * (int)sizeof(T)) = v;
        }
    }

    // ---- 2. gather, filter, sort the centres that reach the tile -----------
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
        const unsigned st = bin_start[bin], en = bin_start[bin + 1];
        for (unsigned i = st; i < en; ++i) {
            const int pos = atomicAdd(&s.nstage, 1);
            if (pos < kStage) s.stage[pos] = bin_items[i];
        }
    }
    __syncthreads();
    const int nst = s.nstage;
    for (int i = tid; i < min(nst, kStage); i += kThreads) {
        const int k = s.stage[i];
        const float* p = ctr + (int64_t)k * g.CW + C;
        bool hit = true;
#pragma unroll
        for (int d = 0; d < NDIM; ++d) {
            const int lo = (int)ceilf(p[d]) - g.S[d];
            hit = hit && (lo <= T0[d] + E[d] - 1) && (lo + 2 * g.S[d] - 1 >= T0[d]);
        }
        if (hit) {
            const int pos = atomicAdd(&s.ncand, 1);
            if (pos < kCap) s.tmp[pos] = k;
        }
    }
    __syncthreads();
    const int nc = s.ncand;
    if (nst > kStage || nc > kCap) {
        if (tid == 0) ovf_tiles[atomicAdd(ovf_count, 1u)] = tile;
        return;  // block-uniform: the per-voxel kernel takes this tile
    }
    for (int i = tid; i < nc; i += kThreads) {
        const int k = s.tmp[i];
        int r = 0;
        for (int j = 0; j < nc; ++j) r += (s.tmp[j] < k);
        s.cand[r] = k;
        const float* row = ctr + (int64_t)k * g.CW;
#pragma unroll
        for (int c = 0; c < C; ++c) s.cd[r].fe[c] = make_float2(row[c], row[c]);
        s.cpos[r][0] = row[C];
        s.cpos[r][1] = row[C + 1];
        s.cpos[r][2] = row[C + 2];
    }
    __syncthreads();

    // ---- per-centre tables and warp-box reach masks -------------------------
    constexpr int TT = TX + (NDIM >= 2 ? TY : 0) + (NDIM >= 3 ? TZ : 0);
    for (int i = tid; i < nc * TT; i += kThreads) {
        const int sl = i / TT;
        int j = i % TT;
        int d = 0;
        if (j >= TX) { j -= TX; d = 1; if (j >= TY) { j -= TY; d = 2; } }
        const float c = s.cpos[sl][d];
        const int lo = (int)ceilf(c) - g.S[d];
        const int x = T0[d] + j;
        float t = kInf;
        if (x >= lo && x <= lo + 2 * g.S[d] - 1) {
            const float dl = __fsub_rn((float)x, c);
            t = __fmul_rn(g.w[d], __fmul_rn(dl, dl));
        }
        if (d == 0) s.cd[sl].t0[j] = t;
        else if (d == 1) s.cd[sl].t1[j] = make_float2(t, t);
        else s.cd[sl].t2[j] = make_float2(t, t);
    }
    for (int i = tid; i < nc; i += kThreads) {
        uint32_t m = 0;
        const int NB[3] = {NBX, NBY, NBZ}, BB[3] = {BX, BY, BZ}, SH[3] = {0, NBX, NBX + NBY};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= NDIM) { m |= 1u << SH[d]; continue; }
            const int lo = (int)ceilf(s.cpos[i][d]) - g.S[d], hi = lo + 2 * g.S[d] - 1;
            for (int b = 0; b < NB[d]; ++b) {
                const int a0 = T0[d] + b * BB[d], a1 = a0 + BB[d] - 1;
                if (lo <= a1 && hi >= a0) m |= 1u << (SH[d] + b);
            }
        }
        s.bmask[i] = m;
    }
    __syncthreads();

    // ---- 3-4. warp boxes: assignment + packed per-box sums ---------------------
    const int lx = lane % WX, ly = (lane / WX) % WY, lz = lane / (WX * WY);
    const uint32_t bm0 = lane < nc ? s.bmask[lane] : 0u;
    const uint32_t bm1 = lane + 32 < nc ? s.bmask[lane + 32] : 0u;
    const unsigned char* cdb = reinterpret_cast<const unsigned char*>(&s.cd[0]);
    using CandT = Cand<C, NDIM>;
    constexpr int CDS = (int)sizeof(CandT);
    constexpr int kOffT1 = 8 * C;                 // layout of Cand: fe, t1, t2, t0
    constexpr int kOffT2 = kOffT1 + 8 * TY;
    constexpr int kOffT0 = kOffT2 + 8 * TZ;
    static_assert(kOffT0 + 4 * TX == CDS, "Cand layout");
#pragma unroll 1
    for (int pass = 0; pass < PASSES; ++pass) {
        const int wb = warp + pass * kWarps;
        const int bxi = wb % NBX, byi = (wb / NBX) % NBY, bzi = wb / (NBX * NBY);
        const int xl = bxi * BX + lx * 2, yl = byi * BY + ly, zl = bzi * BZ + lz;
        const uint32_t want = (1u << bxi) | (1u << (NBX + byi)) | (1u << (NBX + NBY + bzi));
        const uint32_t m0 = __ballot_sync(0xffffffffu, (bm0 & want) == want);
        const uint32_t m1 = __ballot_sync(0xffffffffu, (bm1 & want) == want);
        unsigned fl[C], fh[C];
        uint64_t Fp[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            split_pair<T>(plane_pair(s, c, xl, yl, zl), fl[c], fh[c]);
            Fp[c] = pk2((float)fl[c], (float)fh[c]);
        }
        float b0 = kInf, b1 = kInf;
        int s0 = kNoSlot, s1 = kNoSlot;
        const int o0 = kOffT0 + xl * 4;
        const int o1 = kOffT1 + yl * 8;
        const int o2 = kOffT2 + zl * 8;
#pragma unroll 1
        for (int word = 0; word < 2; ++word) {
            uint32_t m = word ? m1 : m0;
            while (m) {
                const int sl = __ffs(m) - 1 + 32 * word;
                m &= m - 1;
                const unsigned char* base = cdb + sl * CDS;
                uint64_t dc;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint64_t e = sub2(Fp[c], *reinterpret_cast<const uint64_t*>(base + c * 8));
                    const uint64_t sq = mul2(e, e);
                    dc = c == 0 ? sq : add2(dc, sq);
                }
                uint64_t ds = *reinterpret_cast<const uint64_t*>(base + o0);
                if (NDIM >= 2) ds = add2(ds, *reinterpret_cast<const uint64_t*>(base + o1));
                if (NDIM >= 3) ds = add2(ds, *reinterpret_cast<const uint64_t*>(base + o2));
                float d0, d1;
                upk2(add2(dc, ds), d0, d1);
                if (d0 < b0) { b0 = d0; s0 = sl; }
                if (d1 < b1) { b1 = d1; s1 = sl; }
            }
        }
        const int e0 = (zl * TY + yl) * TX + xl;
        const bool in_yz = (yl < ey) && (zl < ez);
        const bool v0 = in_yz && xl < ex && s0 != kNoSlot;
        const bool v1 = in_yz && xl + 1 < ex && s1 != kNoSlot;
        *reinterpret_cast<uint16_t*>(&s.slot[e0]) = (uint16_t)(s0 | (s1 << 8));

        // packed records of the lane's voxels, merged when both have one label
        unsigned w0[P::NW], w1[P::NW];
#pragma unroll
        for (int i = 0; i < P::NW; ++i) { w0[i] = 0u; w1[i] = 0u; }
#pragma unroll
        for (int f = 0; f < F; ++f) {
            unsigned a = f < C ? fl[f < C ? f : 0] : f == C ? (unsigned)xl : f == C + 1 ? (unsigned)yl
                       : f == C + 2 ? (unsigned)zl : 1u;
            unsigned b = f < C ? fh[f < C ? f : 0] : f == C ? (unsigned)(xl + 1) : f == C + 1 ? (unsigned)yl
                       : f == C + 2 ? (unsigned)zl : 1u;
            w0[P::word(f)] += a << P::shift(f);
            w1[P::word(f)] += b << P::shift(f);
        }
        bool p0 = v0, p1 = v1;
        if (v0 && v1 && s0 == s1) {
#pragma unroll
            for (int i = 0; i < P::NW; ++i) w0[i] += w1[i];
            p1 = false;
        }
        for (;;) {
            const uint32_t pend = __ballot_sync(0xffffffffu, p0 || p1);
            if (!pend) break;
            const int leader = __ffs(pend) - 1;
            const int L = __shfl_sync(0xffffffffu, p0 ? s0 : s1, leader);
            unsigned r[P::NW];
            const bool t0 = p0 && s0 == L, t1 = p1 && s1 == L;
#pragma unroll
            for (int i = 0; i < P::NW; ++i) {
                r[i] = (t0 ? w0[i] : 0u) + (t1 ? w1[i] : 0u);
                r[i] = __reduce_add_sync(0xffffffffu, r[i]);
            }
            p0 = p0 && !t0;
            p1 = p1 && !t1;
            if (lane < F) {
                unsigned v = 0;
#pragma unroll
                for (int f = 0; f < F; ++f)
                    if (lane == f) v = (r[P::word(f)] >> P::shift(f)) & ((1u << P::width(f)) - 1u);
                s.accw[warp][L][lane] += v;
            }
        }
    }
    __syncthreads();

    // ---- 5. labels (coalesced) and per-tile sums ------------------------------
    for (int e = tid; e < TV; e += kThreads) {
        const int xl = e % TX, yl = (e / TX) % TY, zl = e / (TX * TY);
        if (xl < ex && yl < ey && zl < ez) {
            const int sl = s.slot[e];
            labels[vidx(g, X0 + xl, Y0 + yl, Z0 + zl)] = sl == kNoSlot ? -1 : s.cand[sl];
        }
    }
    for (int i = tid; i < nc * F; i += kThreads) {
        const int sl = i / F, f = i % F;
        unsigned long long cnt = 0, v = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            cnt += s.accw[w][sl][C + 3];
            v += s.accw[w][sl][f];
        }
        if (!cnt) continue;
        if (f == C) v += cnt * (unsigned long long)X0;
        if (f == C + 1) v += cnt * (unsigned long long)Y0;
        if (f == C + 2) v += cnt * (unsigned long long)Z0;
        atomicAdd(&acc[(int64_t)s.cand[sl] * F + f], v);
    }
}

}  // namespace tile

template <typename T, int C, int NDIM>
int launch_tile_impl(sslic_ctx* c, const T* img, int32_t* labels, cudaStream_t st)
{
    using G = tile::Cfg<NDIM>;
    const Geom& g = c->g;
    Workspace& w = c->ws;
    const int ntx = (int)((g.N[0] + G::TX - 1) / G::TX);
    const int nty = (int)((g.N[1] + G::TY - 1) / G::TY);
    const int ntz = (int)((g.N[2] + G::TZ - 1) / G::TZ);
    const int64_t ntiles = (int64_t)ntx * nty * ntz;
    const size_t smem = sizeof(tile::Smem<T, C, NDIM>);
    int rc = cuda_check(c, cudaFuncSetAttribute(tile::assign_tile_kernel<T, C, NDIM>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                        "smem attribute");
    if (rc) return rc;
    if ((rc = cuda_check(c, cudaMemsetAsync(w.ovf_count, 0, sizeof(unsigned), st), "memset ovf"))) return rc;
    const int pr = prof_begin(c, SSLIC_PHASE_ASSIGN, st);
    tile::assign_tile_kernel<T, C, NDIM><<<(unsigned)ntiles, tile::kThreads, smem, st>>>(
        g, img, w.ctr, w.bin_start, w.bin_items, labels, w.acc, w.ovf_tiles, w.ovf_count, ntx, nty);
    count_launch(c);
    prof_end(c, pr, st);
    if ((rc = cuda_check(c, cudaGetLastError(), "assign_tile_kernel"))) return rc;
    return launch_voxel_tiles(c, img, labels, G::TX, G::TY, G::TZ, ntx, nty, st);
}

template int launch_tile_impl<uint8_t, 3, 3>(sslic_ctx*, const uint8_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint8_t, 3, 2>(sslic_ctx*, const uint8_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint8_t, 1, 3>(sslic_ctx*, const uint8_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint8_t, 1, 2>(sslic_ctx*, const uint8_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint16_t, 1, 3>(sslic_ctx*, const uint16_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint16_t, 1, 2>(sslic_ctx*, const uint16_t*, int32_t*, cudaStream_t);

int64_t assign_num_tiles(const Geom& g)
{
    if (g.n == 3) {
        using T3 = tile::Cfg<3>;
        return ((g.N[0] + T3::TX - 1) / T3::TX) * ((g.N[1] + T3::TY - 1) / T3::TY) * ((g.N[2] + T3::TZ - 1) / T3::TZ);
    }
    using T2 = tile::Cfg<2>;
    return ((g.N[0] + T2::TX - 1) / T2::TX) * ((g.N[1] + T2::TY - 1) / T2::TY) * g.N[2];
}

}  // namespace sslic
