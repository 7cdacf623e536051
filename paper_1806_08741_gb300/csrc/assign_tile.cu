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

// Tile shapes.  A tile must stay within kCap reaching centres: about
// prod_d (T_d + 2 S_d - 1) / S_d of them, so small grids take small tiles.
// Lanes: WX pairs along x times WY times WZ; a warp box is 2WX x WY x WZ.
template <int NDIM_, int TX_, int TY_, int TZ_, int WX_, int WY_, int WZ_>
struct Shape {
    static constexpr int NDIM = NDIM_, TX = TX_, TY = TY_, TZ = TZ_, WX = WX_, WY = WY_, WZ = WZ_;
};
using Shape3L = Shape<3, 32, 16, 8, 2, 4, 4>;   // 4096 voxels, grids S >= 12
using Shape3S = Shape<3, 16, 8, 8, 2, 4, 4>;    // 1024 voxels, smaller grids
using Shape2L = Shape<2, 64, 32, 1, 4, 8, 1>;   // 2048 pixels
using Shape2S = Shape<2, 32, 16, 1, 4, 8, 1>;   // 512 pixels

// per-candidate record in shared memory
template <int C, typename SH>
struct Cand {
    float2 fe[C];        // (C_c, C_c)
    float2 t1[SH::TY];   // (t_1, t_1) by local y
    float2 t2[SH::TZ];   // (t_2, t_2) by local z
    float t0[SH::TX];    // t_0 by local x
};

template <typename T, int C, typename SH>
struct Smem {
    using G = SH;
    static constexpr int TX = G::TX, TY = G::TY, TZ = G::TZ, TV = TX * TY * TZ;
    // channel planes: row pitch 4 bytes past the row, plane pitch chosen so a
    // plane advances 4 banks -- the 4x4 (y, z) lanes of a warp box then hit
    // distinct banks
    static constexpr int RPB = TX * (int)sizeof(T) + 4;
    static constexpr int PPB_RAW = TY * RPB;
    static constexpr int PPB = PPB_RAW + 4 * ((4 - (PPB_RAW / 4) % 32 + 32) % 32);
    static constexpr int CPB = ((TZ * PPB + 15) / 16) * 16;
    static constexpr int NBOX = (TX / (2 * G::WX)) * (TY / G::WY) * (TZ / G::WZ);
    Cand<C, SH> cd[kCap + 1];          // [kCap]: a dummy centre that reaches nothing
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

template <typename T, int C, typename SH>
__device__ __forceinline__ unsigned plane_pair(const Smem<T, C, SH>& s, int c, int xl, int yl, int zl)
{
    using S = Smem<T, C, SH>;
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

// One tile of one image (request req): everything of steps 1-5 above.  A
// tile reached by more than kCap centres is appended to the crowded-tile
// list as (req << 40 | tile) and left to the per-voxel kernel.
template <typename T, int C, typename SH>
__device__ __forceinline__ void tile_body(const TileArgs& a, int tile, int64_t req, Smem<T, C, SH>& s,
                                          int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count)
{
    const Geom& g = a.g;
    const T* __restrict__ img = (const T*)a.img;
    const float* __restrict__ ctr = a.ctr;
    const unsigned* __restrict__ bin_start = a.bin_start;
    const int* __restrict__ bin_items = a.bin_items;
    int32_t* __restrict__ labels = a.labels;
    unsigned long long* __restrict__ acc = a.acc;
    const int ntx = a.ntx, nty = a.nty;
    constexpr int NDIM = SH::NDIM;
    using G = SH;
    using S = Smem<T, C, SH>;
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

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
        if (tid == 0) ovf_tiles[atomicAdd(ovf_count, 1u)] = (req << 40) | (int64_t)tile;
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
        const int NB[3] = {NBX, NBY, NBZ}, BB[3] = {BX, BY, BZ}, SHF[3] = {0, NBX, NBX + NBY};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (d >= NDIM) { m |= 1u << SHF[d]; continue; }
            const int lo = (int)ceilf(s.cpos[i][d]) - g.S[d], hi = lo + 2 * g.S[d] - 1;
            for (int b = 0; b < NB[d]; ++b) {
                const int a0 = T0[d] + b * BB[d], a1 = a0 + BB[d] - 1;
                if (lo <= a1 && hi >= a0) m |= 1u << (SHF[d] + b);
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
    using CandT = Cand<C, SH>;
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

// one image: one CTA per tile
template <typename T, int C, typename SH>
__global__ void __launch_bounds__(kThreads, 4)
assign_tile_kernel(TileArgs a, int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_body<T, C, SH>(a, blockIdx.x, 0, *reinterpret_cast<Smem<T, C, SH>*>(smem_raw), ovf_tiles, ovf_count);
}

// many images: a persistent grid walks one queue of (request, tile) work
// items; request r owns global tile numbers [tpre[r], tpre[r + 1])
template <typename T, int C, typename SH>
__global__ void __launch_bounds__(kThreads, 4)
assign_tile_queue_kernel(const TileArgs* __restrict__ reqs, const int64_t* __restrict__ tpre, int R,
                         int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<T, C, SH>& s = *reinterpret_cast<Smem<T, C, SH>*>(smem_raw);
    const int64_t total = tpre[R];
    for (int64_t i = blockIdx.x; i < total; i += gridDim.x) {
        int lo = 0, hi = R - 1;  // last r with tpre[r] <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tpre[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        __syncthreads();  // the previous tile's shared state is no longer read
        tile_body<T, C, SH>(reqs[lo], (int)(i - tpre[lo]), lo, s, ovf_tiles, ovf_count);
    }
}

}  // namespace tile

template <typename SH>
static void tile_grid(const Geom& g, int& ntx, int& nty, int& ntz)
{
    ntx = (int)((g.N[0] + SH::TX - 1) / SH::TX);
    nty = (int)((g.N[1] + SH::TY - 1) / SH::TY);
    ntz = (int)((g.N[2] + SH::TZ - 1) / SH::TZ);
}

// expected number of centres reaching a tile of shape (tx, ty, tz)
static double reach(const Geom& g, int tx, int ty, int tz)
{
    const int T[3] = {tx, ty, tz};
    double r = 1.0;
    for (int d = 0; d < g.n; ++d) r *= (double)(T[d] + 2 * g.S[d] - 1) / g.S[d];
    return r;
}

int default_tile_shape(const Geom& g)
{
    // the large tile while it stays well inside the candidate capacity
    const double lim = 0.75 * tile::kCap;
    if (g.n == 3) return reach(g, tile::Shape3L::TX, tile::Shape3L::TY, tile::Shape3L::TZ) <= lim ? 0 : 1;
    return reach(g, tile::Shape2L::TX, tile::Shape2L::TY, 1) <= lim ? 0 : 1;
}

template <typename T, int C, typename SH>
static int launch_tile_shape(sslic_ctx* c, const T* img, int32_t* labels, cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    int ntx, nty, ntz;
    tile_grid<SH>(g, ntx, nty, ntz);
    const int64_t ntiles = (int64_t)ntx * nty * ntz;
    const size_t smem = sizeof(tile::Smem<T, C, SH>);
    int rc = cuda_check(c, cudaFuncSetAttribute(tile::assign_tile_kernel<T, C, SH>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                        "smem attribute");
    if (rc) return rc;
    if ((rc = cuda_check(c, cudaMemsetAsync(w.ovf_count, 0, sizeof(unsigned), st), "memset ovf"))) return rc;
    TileArgs a;
    a.g = g;
    a.img = img;
    a.ctr = w.ctr;
    a.bin_start = w.bin_start;
    a.bin_items = w.bin_items;
    a.labels = labels;
    a.acc = w.acc;
    a.facc = w.facc;
    a.ntx = ntx;
    a.nty = nty;
    a.tx = SH::TX;
    a.ty = SH::TY;
    a.tz = SH::TZ;
    const int pr = prof_begin(c, SSLIC_PHASE_ASSIGN, st);
    tile::assign_tile_kernel<T, C, SH><<<(unsigned)ntiles, tile::kThreads, smem, st>>>(a, w.ovf_tiles, w.ovf_count);
    count_launch(c);
    prof_end(c, pr, st);
    if ((rc = cuda_check(c, cudaGetLastError(), "assign_tile_kernel"))) return rc;
    return launch_voxel_tiles(c, img, labels, SH::TX, SH::TY, SH::TZ, ntx, nty, st);
}

template <typename T, int C, int NDIM>
int launch_tile_impl(sslic_ctx* c, const T* img, int32_t* labels, cudaStream_t st)
{
    const int shape = c->tile_shape >= 0 ? c->tile_shape : default_tile_shape(c->g);
    if constexpr (NDIM == 3) {
        return shape == 0 ? launch_tile_shape<T, C, tile::Shape3L>(c, img, labels, st)
                          : launch_tile_shape<T, C, tile::Shape3S>(c, img, labels, st);
    } else {
        return shape == 0 ? launch_tile_shape<T, C, tile::Shape2L>(c, img, labels, st)
                          : launch_tile_shape<T, C, tile::Shape2S>(c, img, labels, st);
    }
}

template int launch_tile_impl<uint8_t, 3, 3>(sslic_ctx*, const uint8_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint8_t, 3, 2>(sslic_ctx*, const uint8_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint8_t, 1, 3>(sslic_ctx*, const uint8_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint8_t, 1, 2>(sslic_ctx*, const uint8_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint16_t, 1, 3>(sslic_ctx*, const uint16_t*, int32_t*, cudaStream_t);
template int launch_tile_impl<uint16_t, 1, 2>(sslic_ctx*, const uint16_t*, int32_t*, cudaStream_t);

// batched form: one persistent launch over the (request, tile) queue of all
// requests of one type and shape; returns the CUDA error of the launch
template <typename T, int C, typename SH>
static cudaError_t launch_queue_shape(const TileArgs* reqs, const int64_t* tpre, int R, int64_t* ovf,
                                      unsigned* ovf_count, int grid, cudaStream_t st)
{
    const size_t smem = sizeof(tile::Smem<T, C, SH>);
    cudaError_t e = cudaFuncSetAttribute(tile::assign_tile_queue_kernel<T, C, SH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tile::assign_tile_queue_kernel<T, C, SH><<<grid, tile::kThreads, smem, st>>>(reqs, tpre, R, ovf, ovf_count);
    return cudaGetLastError();
}

template <typename T, int C, int NDIM>
cudaError_t launch_tile_queue(int shape, const TileArgs* reqs, const int64_t* tpre, int R, int64_t* ovf,
                              unsigned* ovf_count, int grid, cudaStream_t st)
{
    if constexpr (NDIM == 3)
        return shape == 0 ? launch_queue_shape<T, C, tile::Shape3L>(reqs, tpre, R, ovf, ovf_count, grid, st)
                          : launch_queue_shape<T, C, tile::Shape3S>(reqs, tpre, R, ovf, ovf_count, grid, st);
    else
        return shape == 0 ? launch_queue_shape<T, C, tile::Shape2L>(reqs, tpre, R, ovf, ovf_count, grid, st)
                          : launch_queue_shape<T, C, tile::Shape2S>(reqs, tpre, R, ovf, ovf_count, grid, st);
}

template cudaError_t launch_tile_queue<uint8_t, 3, 3>(int, const TileArgs*, const int64_t*, int, int64_t*, unsigned*, int, cudaStream_t);
template cudaError_t launch_tile_queue<uint8_t, 3, 2>(int, const TileArgs*, const int64_t*, int, int64_t*, unsigned*, int, cudaStream_t);
template cudaError_t launch_tile_queue<uint8_t, 1, 3>(int, const TileArgs*, const int64_t*, int, int64_t*, unsigned*, int, cudaStream_t);
template cudaError_t launch_tile_queue<uint8_t, 1, 2>(int, const TileArgs*, const int64_t*, int, int64_t*, unsigned*, int, cudaStream_t);
template cudaError_t launch_tile_queue<uint16_t, 1, 3>(int, const TileArgs*, const int64_t*, int, int64_t*, unsigned*, int, cudaStream_t);
template cudaError_t launch_tile_queue<uint16_t, 1, 2>(int, const TileArgs*, const int64_t*, int, int64_t*, unsigned*, int, cudaStream_t);

// tile dimensions of a shape (host side)
void tile_dims(int ndim, int shape, int* tx, int* ty, int* tz)
{
    if (ndim == 3) {
        *tx = shape == 0 ? tile::Shape3L::TX : tile::Shape3S::TX;
        *ty = shape == 0 ? tile::Shape3L::TY : tile::Shape3S::TY;
        *tz = shape == 0 ? tile::Shape3L::TZ : tile::Shape3S::TZ;
    } else {
        *tx = shape == 0 ? tile::Shape2L::TX : tile::Shape2S::TX;
        *ty = shape == 0 ? tile::Shape2L::TY : tile::Shape2S::TY;
        *tz = 1;
    }
}

// the most tiles any shape cuts the image into (sizes the crowded-tile list)
int64_t assign_num_tiles(const Geom& g)
{
    int ntx, nty, ntz;
    if (g.n == 3) tile_grid<tile::Shape3S>(g, ntx, nty, ntz);
    else tile_grid<tile::Shape2S>(g, ntx, nty, ntz);
    return (int64_t)ntx * nty * ntz;
}

}  // namespace sslic
