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
// Work decomposition.  A CTA (8 warps) owns a tile of 32x16x8 voxels (3-D)
// or 64x32 pixels (2-D):
//  1. stages the tile's channels as bank-padded planes in shared memory;
//  2. gathers the centres of the bins that can reach the tile (3 bins per
//     axis around it), keeps those whose window meets the tile, sorts them by
//     index, and builds per centre the feature pair (C_c, C_c) and per axis
//     the table t_d(x_d) over the tile's coordinates, +inf outside the window
//     (the window test is folded into the distance);
//  3. each warp sweeps 4x4x4 (3-D) / 8x8 (2-D) boxes, two voxels per lane in
//     packed .f32x2 arithmetic, visiting only the centres that reach its box,
//     and leaves the winning slot of every voxel in shared memory;
//  4. one sweep over 16-voxel row segments writes the int32 labels with
//     16-byte stores and sums [I, x, y, z, 1] along runs of equal slots (a
//     run of four equal slots takes one byte-sum instruction per channel)
//     into per-tile accumulators;
//  5. per-tile sums leave through one uint64 atomic per (centre, field).
// Tiles reached by more than kCap centres are handed to the per-voxel kernel.
#include "common.cuh"

namespace sslic {

namespace tile {

constexpr float kInf = __builtin_huge_valf();
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCap = 48;     // candidate centres per tile (a 32x16x8 tile at S = 16 sees ~23, <= 40)
constexpr int kStage = 256;  // gathered centres before filtering
constexpr int kSeg = 16;     // voxels per row segment in the label / sum sweep

template <int NDIM>
struct Cfg;
template <>
struct Cfg<3> {
    static constexpr int TX = 32, TY = 16, TZ = 8;  // 4096 voxels
    static constexpr int WX = 2, WY = 4, WZ = 4;    // lanes -> box 4x4x4 (pairs along x)
};
template <>
struct Cfg<2> {
    static constexpr int TX = 64, TY = 32, TZ = 1;  // 2048 pixels
    static constexpr int WX = 4, WY = 8, WZ = 1;    // box 8x8
};

// per-candidate record in shared memory
template <int C, int NDIM>
struct Cand {
    float2 fe[C];              // (C_c, C_c)
    float2 t1[Cfg<NDIM>::TY];  // (t_1, t_1) by local y
    float2 t2[Cfg<NDIM>::TZ];  // (t_2, t_2) by local z
    float t0[Cfg<NDIM>::TX];   // t_0 by local x
};

template <typename T, int C, int NDIM>
struct Smem {
    using G = Cfg<NDIM>;
    static constexpr int TX = G::TX, TY = G::TY, TZ = G::TZ, TV = TX * TY * TZ;
    // channel planes: row pitch 4 bytes past the row, plane pitch chosen so a
    // plane advances 4 banks -- the 4x4 (y, z) lanes of a warp box then hit
    // distinct banks
    static constexpr int RPB = TX * (int)sizeof(T) + 4;
    static constexpr int PPB_RAW = TY * RPB;
    static constexpr int PPB = PPB_RAW + 4 * ((4 - (PPB_RAW / 4) % 32 + 32) % 32);
    static constexpr int CPB = ((TZ * PPB + 15) / 16) * 16;
    static constexpr int NBOX = (TX / (2 * G::WX)) * (TY / G::WY) * (TZ / G::WZ);
    Cand<C, NDIM> cd[kCap + 1];          // [kCap]: a dummy centre that reaches nothing
    uint8_t blist[NBOX][kCap + 2];       // per warp box: reaching slots, ascending, even length
    uint8_t bcnt[NBOX];
    alignas(16) unsigned char planes[C * CPB];
    unsigned acc[kCap][C + 4];   // per-tile sums: features, x, y, z (local), count
    float cpos[kCap][3];
    int cand[kCap];
    int tmp[kCap];
    int stage[kStage];
    uint32_t bmask[kCap];
    alignas(16) uint8_t slot[TV];
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

__device__ __forceinline__ uint64_t lds64(uint32_t addr)
{
    uint64_t v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

template <typename T>
__device__ __forceinline__ void split_pair(unsigned v, unsigned& lo, unsigned& hi)
{
    if constexpr (sizeof(T) == 1) { lo = v & 0xffu; hi = v >> 8; }
    else { lo = v & 0xffffu; hi = v >> 16; }
}

template <int C>
__device__ __forceinline__ void flush_run(unsigned (*acc)[C + 4], int cur, const unsigned* fs, unsigned xs,
                                          unsigned cnt, int yl, int zl)
{
    if (cur == kNoSlot || cnt == 0) return;
#pragma unroll
    for (int c = 0; c < C; ++c) atomicAdd(&acc[cur][c], fs[c]);
    atomicAdd(&acc[cur][C], xs);
    atomicAdd(&acc[cur][C + 1], cnt * (unsigned)yl);
    atomicAdd(&acc[cur][C + 2], cnt * (unsigned)zl);
    atomicAdd(&acc[cur][C + 3], cnt);
}

template <typename T, int C, int NDIM>
__global__ void __launch_bounds__(kThreads, 4)
assign_tile_kernel(Geom g, const T* __restrict__ img, const float* __restrict__ ctr,
                   const unsigned* __restrict__ bin_start, const int* __restrict__ bin_items,
                   int32_t* __restrict__ labels, unsigned long long* __restrict__ acc,
                   int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count, int ntx, int nty)
{
    using G = Cfg<NDIM>;
    using S = Smem<T, C, NDIM>;
    constexpr int TX = G::TX, TY = G::TY, TZ = G::TZ, TV = TX * TY * TZ;
    constexpr int WX = G::WX, WY = G::WY, WZ = G::WZ;
    constexpr int BX = 2 * WX, BY = WY, BZ = WZ;
    constexpr int NBX = TX / BX, NBY = TY / BY, NBZ = TZ / BZ;
    constexpr int NBOX = NBX * NBY * NBZ;
    constexpr int PASSES = NBOX / kWarps;
    constexpr int F = C + 4;
    constexpr int SPR = TX / kSeg;  // segments per row
    static_assert(NBOX % kWarps == 0, "boxes per warp");
    static_assert(NBX + NBY + NBZ <= 32, "box mask bits");
    static_assert(TX % kSeg == 0, "row segments");

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
    for (int i = tid; i < kCap * F; i += kThreads) (&s.acc[0][0])[i] = 0u;

    // ---- 1. stage the tile as channel planes --------------------------------
    if constexpr (sizeof(T) == 1 && C == 3) {
        // full rows: 12-byte groups (4 voxels) -> one word per plane
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
    // t_d entry: w_d (x - c)^2 with one rounding per operation, +inf outside
    auto entry = [&](int d, int j, float c) -> float {
        const int lo = (int)ceilf(c) - g.S[d];
        const int x = T0[d] + j;
        if (x < lo || x > lo + 2 * g.S[d] - 1) return kInf;
        const float dl = __fsub_rn((float)x, c);
        return __fmul_rn(g.w[d], __fmul_rn(dl, dl));
    };
    for (int i = tid; i < nc * TX; i += kThreads) {
        const int sl = i / TX, j = i % TX;
        s.cd[sl].t0[j] = entry(0, j, s.cpos[sl][0]);
    }
    if constexpr (NDIM >= 2) {
        for (int i = tid; i < nc * TY; i += kThreads) {
            const int sl = i / TY, j = i % TY;
            const float t = entry(1, j, s.cpos[sl][1]);
            s.cd[sl].t1[j] = make_float2(t, t);
        }
    }
    if constexpr (NDIM >= 3) {
        for (int i = tid; i < nc * TZ; i += kThreads) {
            const int sl = i / TZ, j = i % TZ;
            const float t = entry(2, j, s.cpos[sl][2]);
            s.cd[sl].t2[j] = make_float2(t, t);
        }
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
    for (int i = tid; i < TX; i += kThreads) s.cd[kCap].t0[i] = kInf;
    for (int i = tid; i < TY; i += kThreads) s.cd[kCap].t1[i] = make_float2(kInf, kInf);
    for (int i = tid; i < TZ; i += kThreads) s.cd[kCap].t2[i] = make_float2(kInf, kInf);
    if (tid < C) s.cd[kCap].fe[tid] = make_float2(0.0f, 0.0f);
    __syncthreads();
    // per warp box: the slots whose window reaches it, ascending, padded to
    // an even count with the dummy so the sweep takes two centres per step
    for (int wb = warp; wb < NBOX; wb += kWarps) {
        const int bxi = wb % NBX, byi = (wb / NBX) % NBY, bzi = wb / (NBX * NBY);
        const uint32_t want = (1u << bxi) | (1u << (NBX + byi)) | (1u << (NBX + NBY + bzi));
        const bool h0 = lane < nc && (s.bmask[lane] & want) == want;
        const bool h1 = lane + 32 < nc && (s.bmask[lane + 32] & want) == want;
        const uint32_t m0 = __ballot_sync(0xffffffffu, h0);
        const uint32_t m1 = __ballot_sync(0xffffffffu, h1);
        const uint32_t lt = (1u << lane) - 1u;
        const int n0 = __popc(m0), n = n0 + __popc(m1);
        if (h0) s.blist[wb][__popc(m0 & lt)] = (uint8_t)lane;
        if (h1) s.blist[wb][n0 + __popc(m1 & lt)] = (uint8_t)(lane + 32);
        if (lane == 0) {
            if (n & 1) s.blist[wb][n] = (uint8_t)kCap;
            s.bcnt[wb] = (uint8_t)((n + 1) & ~1);
        }
    }
    __syncthreads();

    // ---- 3. warp boxes: assignment ------------------------------------------
    const int lx = lane % WX, ly = (lane / WX) % WY, lz = lane / (WX * WY);
    const uint32_t cdb = (uint32_t)__cvta_generic_to_shared(&s.cd[0]);
    using CandT = Cand<C, NDIM>;
    constexpr int CDS = (int)sizeof(CandT);
    constexpr int kOffT1 = 8 * C;  // layout of Cand: fe, t1, t2, t0
    constexpr int kOffT2 = kOffT1 + 8 * TY;
    constexpr int kOffT0 = kOffT2 + 8 * TZ;
    static_assert(kOffT0 + 4 * TX == CDS, "Cand layout");
#pragma unroll 1
    for (int pass = 0; pass < PASSES; ++pass) {
        const int wb = warp + pass * kWarps;
        const int bxi = wb % NBX, byi = (wb / NBX) % NBY, bzi = wb / (NBX * NBY);
        const int xl = bxi * BX + lx * 2, yl = byi * BY + ly, zl = bzi * BZ + lz;
        uint64_t Fp[C];
#pragma unroll
        for (int c = 0; c < C; ++c) {
            unsigned lo, hi;
            split_pair<T>(plane_pair(s, c, xl, yl, zl), lo, hi);
            Fp[c] = pk2((float)lo, (float)hi);
        }
        float b0 = kInf, b1 = kInf;
        int s0 = kNoSlot, s1 = kNoSlot;
        const uint32_t a0 = cdb + kOffT0 + xl * 4;
        const uint32_t a1 = cdb + kOffT1 + yl * 8;
        const uint32_t a2 = cdb + kOffT2 + zl * 8;
        const int nb = s.bcnt[wb];
        const uint16_t* lst = reinterpret_cast<const uint16_t*>(&s.blist[wb][0]);
        // D^2 of both voxels of the lane against the centre in slot sl
        auto dist2 = [&](int sl) -> uint64_t {
            const uint32_t so = (uint32_t)(sl * CDS);
            uint64_t dc;
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const uint64_t e = sub2(Fp[c], lds64(cdb + so + c * 8));
                const uint64_t sq = mul2(e, e);
                dc = c == 0 ? sq : add2(dc, sq);
            }
            uint64_t ds = lds64(a0 + so);
            if (NDIM >= 2) ds = add2(ds, lds64(a1 + so));
            if (NDIM >= 3) ds = add2(ds, lds64(a2 + so));
            return add2(dc, ds);
        };
#pragma unroll 1
        for (int i = 0; i < nb; i += 2) {
            const unsigned two = lst[i >> 1];
            const int sa = (int)(two & 0xffu), sb = (int)(two >> 8);
            const uint64_t Da = dist2(sa);
            const uint64_t Db = dist2(sb);
            float d0, d1;
            upk2(Da, d0, d1);
            if (d0 < b0) { b0 = d0; s0 = sa; }
            if (d1 < b1) { b1 = d1; s1 = sa; }
            upk2(Db, d0, d1);
            if (d0 < b0) { b0 = d0; s0 = sb; }
            if (d1 < b1) { b1 = d1; s1 = sb; }
        }
        *reinterpret_cast<uint16_t*>(&s.slot[(zl * TY + yl) * TX + xl]) = (uint16_t)(s0 | (s1 << 8));
    }
    __syncthreads();

    // ---- 4. row segments: labels out, run sums in -------------------------------
    const bool vec_ok = (N0 % 4 == 0) && (((uintptr_t)labels & 15) == 0);
    for (int sg = tid; sg < TY * TZ * SPR; sg += kThreads) {
        // lanes of a warp take segments in different z planes (different
        // labels, fewer same-address flushes); 2-D: consecutive segments
        int h, yl, zl;
        if constexpr (TZ > 1) {
            zl = sg % TZ;
            h = (sg / TZ) % SPR;
            yl = sg / (TZ * SPR);
        } else {
            h = sg % SPR;
            yl = sg / SPR;
            zl = 0;
        }
        const int r = zl * TY + yl;
        if (yl >= ey || zl >= ez) continue;
        const int xs0 = h * kSeg;
        const int n = min(kSeg, ex - xs0);
        if (n <= 0) continue;
        int32_t* lrow = labels + vidx(g, X0 + xs0, Y0 + yl, Z0 + zl);
        const unsigned char* prow = s.planes + zl * S::PPB + yl * S::RPB;
        // the segment's slots, read word by word in a lane-rotated order
        // (spreads the lanes of a warp over the banks)
        uint32_t sw[kSeg / 4];
        const uint32_t* sp = reinterpret_cast<const uint32_t*>(&s.slot[r * TX + xs0]);
#pragma unroll
        for (int j = 0; j < kSeg / 4; ++j) {
            const int jj = (j + (TZ > 1 ? (lane & 7) : (lane >> 3))) & (kSeg / 4 - 1);
            sw[jj] = sp[jj];
        }
        int cur = kNoSlot, curlab = -1;
        unsigned fs[C], xs = 0, cnt = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) fs[c] = 0;
        // start a new run at slot sl (flushing the previous one)
        auto next_run = [&](int sl) {
            flush_run<C>(s.acc, cur, fs, xs, cnt, yl, zl);
            cur = sl;
            curlab = sl == kNoSlot ? -1 : s.cand[sl];
#pragma unroll
            for (int c = 0; c < C; ++c) fs[c] = 0;
            xs = 0;
            cnt = 0;
        };
        if (n == kSeg) {
#pragma unroll
            for (int j = 0; j < kSeg / 4; ++j) {
                const uint32_t w = sw[j];
                const int xq = xs0 + 4 * j;
                int lab4[4];
                if (sizeof(T) == 1 && w == (w & 0xffu) * 0x01010101u) {
                    // four voxels, one slot: byte sums of the planes' words
                    const int sl = (int)(w & 0xffu);
                    if (sl != cur) next_run(sl);
                    if (sl != kNoSlot) {
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            fs[c] += __vsadu4(*reinterpret_cast<const uint32_t*>(prow + c * S::CPB + xq), 0u);
                        xs += 4u * (unsigned)xq + 6u;
                        cnt += 4u;
                    }
                    lab4[0] = lab4[1] = lab4[2] = lab4[3] = curlab;
                } else {
                    uint32_t pw[C];
                    if constexpr (sizeof(T) == 1) {
#pragma unroll
                        for (int c = 0; c < C; ++c)
                            pw[c] = *reinterpret_cast<const uint32_t*>(prow + c * S::CPB + xq);
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int sl = (int)((w >> (8 * b)) & 0xffu);
                        if (sl != cur) next_run(sl);
                        if (sl != kNoSlot) {
#pragma unroll
                            for (int c = 0; c < C; ++c) {
                                if constexpr (sizeof(T) == 1) fs[c] += (pw[c] >> (8 * b)) & 0xffu;
                                else fs[c] += (unsigned)*reinterpret_cast<const T*>(
                                    prow + c * S::CPB + (xq + b) * (int)sizeof(T));
                            }
                            xs += (unsigned)(xq + b);
                            cnt += 1u;
                        }
                        lab4[b] = curlab;
                    }
                }
                if (vec_ok) {
                    *reinterpret_cast<int4*>(lrow + 4 * j) = make_int4(lab4[0], lab4[1], lab4[2], lab4[3]);
                } else {
#pragma unroll
                    for (int b = 0; b < 4; ++b) lrow[4 * j + b] = lab4[b];
                }
            }
        } else {
            for (int b = 0; b < n; ++b) {
                const uint32_t wb = b < 4 ? sw[0] : (b < 8 ? sw[1] : (b < 12 ? sw[2] : sw[3]));
                const int sl = (int)((wb >> (8 * (b & 3))) & 0xffu);
                if (sl != cur) next_run(sl);
                if (sl != kNoSlot) {
#pragma unroll
                    for (int c = 0; c < C; ++c)
                        fs[c] += (unsigned)*reinterpret_cast<const T*>(prow + c * S::CPB + (xs0 + b) * (int)sizeof(T));
                    xs += (unsigned)(xs0 + b);
                    cnt += 1u;
                }
                lrow[b] = curlab;
            }
        }
        flush_run<C>(s.acc, cur, fs, xs, cnt, yl, zl);
    }
    __syncthreads();

    // ---- 5. per-tile sums, shifted to global coordinates ----------------------
    for (int i = tid; i < nc * F; i += kThreads) {
        const int sl = i / F, f = i % F;
        const unsigned long long cnt = s.acc[sl][C + 3];
        if (!cnt) continue;
        unsigned long long v = s.acc[sl][f];
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
