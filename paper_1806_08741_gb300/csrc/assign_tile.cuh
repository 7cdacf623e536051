// assign_tile.cuh -- the fused assignment + map-update kernel for integer
// images with 1 or 3 channels (2-D and 3-D): one SSLIC iteration's hot loop.
// The kernel templates live here; assign_tile_<type>.cu files instantiate
// them per image type (separate translation units compile in parallel) and
// assign_tile.cu holds the shape table.
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
// Work decomposition.  A CTA (8 warps) owns a tile (32x16x8 voxels for the
// large 3-D shape, 64x32 pixels for the large 2-D one):
//  1. stages the tile's channels as bank-padded planes in shared memory;
//  2. gathers the centres of the bins that can reach the tile (3 bins per
//     axis around it), keeps those whose window meets the tile, sorts them by
//     index, and builds per centre the feature pair (C_c, C_c) and per axis
//     the table t_d(x_d) over the tile's coordinates, +inf outside the window
//     (the window test is folded into the distance);
//  3. each warp sweeps boxes of 32 lanes x VL voxels (VL = 2 or 4 consecutive
//     voxels along x per lane, in packed .f32x2 pairs), visiting only the
//     centres that reach its box.  Integer images finish the box at once:
//     each lane writes its voxels' int32 labels (one vector store) and adds
//     every voxel's [I, x, y, z, 1] to its slot's per-tile sums with C + 2
//     shared atomics.  Float images leave the winning slot of every voxel in
//     shared memory instead, and
//  4. one sweep over 16-voxel row segments writes their labels and sums the
//     features in FP32 along runs of equal slots;
//  5. per-tile sums leave through one uint64 atomic per (centre, field).
// Tiles reached by more than kCap centres are handed to the per-voxel kernel.
#pragma once
#include <cuda.h>

#include <type_traits>

#include "common.cuh"
#include "tc.cuh"

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
// Lanes: WX along x times WY times WZ, each lane VL consecutive voxels along
// x (VL / 2 packed pairs); a warp box is VL WX x WY x WZ.  More voxels per
// lane share each centre's shared-memory reads among more voxels; a larger
// box is reached by a few more centres.
template <int NDIM_, int TX_, int TY_, int TZ_, int WX_, int WY_, int WZ_, int VL_>
struct Shape {
    static constexpr int NDIM = NDIM_, TX = TX_, TY = TY_, TZ = TZ_, WX = WX_, WY = WY_, WZ = WZ_, VL = VL_;
};
using Shape3L = Shape<3, 32, 16, 8, 2, 4, 4, 2>;   // 4096 voxels, grids S >= 12
using Shape3S = Shape<3, 16, 8, 8, 2, 4, 4, 2>;    // 1024 voxels, smaller grids
using Shape3L4 = Shape<3, 32, 16, 8, 2, 4, 4, 4>;  // as 3L, 8x4x4 warp boxes
using Shape3S4 = Shape<3, 16, 8, 8, 2, 4, 4, 4>;   // as 3S, 8x4x4 warp boxes
using Shape3M = Shape<3, 32, 8, 8, 2, 4, 4, 2>;    // 2048 voxels: half the staging of 3L (float planes)
using Shape3M4 = Shape<3, 32, 8, 8, 2, 4, 4, 4>;   // as 3M, 8x4x4 warp boxes
using Shape2L = Shape<2, 64, 32, 1, 4, 8, 1, 2>;   // 2048 pixels
using Shape2S = Shape<2, 32, 16, 1, 4, 8, 1, 2>;   // 512 pixels
using Shape2L4 = Shape<2, 64, 32, 1, 4, 8, 1, 4>;  // as 2L, 16x8 warp boxes

// Per-candidate record in shared memory, CDS bytes: t_0 by local x (float,
// 16-byte aligned for the 4-voxel lanes), (t_1, t_1) by local y, (t_2, t_2)
// by local z, (C_c, C_c) per channel.
template <int C, typename SH>
struct CandLayout {
    static constexpr int kOffT0 = 0;
    static constexpr int kOffT1 = kOffT0 + 4 * SH::TX;
    static constexpr int kOffT2 = kOffT1 + 8 * SH::TY;
    static constexpr int kOffFe = kOffT2 + 8 * SH::TZ;
    static constexpr int CDS = ((kOffFe + 8 * C) + 15) / 16 * 16;
    static_assert(SH::TX % 4 == 0, "t_0 alignment");
};

template <typename T, int C, typename SH>
struct Smem {
    using G = SH;
    static constexpr int TX = G::TX, TY = G::TY, TZ = G::TZ, TV = TX * TY * TZ;
    // channel planes: row pitch 4 bytes past the row, plane pitch chosen so a
    // plane advances 4 banks -- the 4x4 (y, z) lanes of a warp box then hit
    // distinct banks
    // (float planes: pitches kept multiples of 8 bytes for the 64-bit pair loads)
    static constexpr bool kF = std::is_same<T, float>::value;
    static constexpr int RPB = TX * (int)sizeof(T) + (kF ? 8 : 4);
    static constexpr int PPB_RAW = TY * RPB;
    static constexpr int PPB = kF ? (PPB_RAW + 8 + 15) / 16 * 16 : PPB_RAW + 4 * ((4 - (PPB_RAW / 4) % 32 + 32) % 32);
    static constexpr int CPB = ((TZ * PPB + 15) / 16) * 16;
    static constexpr int NBOX = (TX / (G::VL * G::WX)) * (TY / G::WY) * (TZ / G::WZ);
    // integer images take the map step inside the box pass (each voxel adds
    // its [I, x, y, z, 1] with C + 2 shared atomics); float images keep the
    // slot array and the row-segment sweep
    static constexpr bool kInBox = !kF;
    alignas(16) unsigned char cd[(kCap + 1) * CandLayout<C, SH>::CDS];  // [kCap]: a dummy that reaches nothing
    uint8_t blist[NBOX][kCap + 2];       // per warp box: reaching slots, ascending, even length
    uint8_t bcnt[NBOX];
    alignas(16) unsigned char planes[C * CPB];
    // per-tile sums: kCopies copies (lane & 7 picks one, so lanes of a warp
    // adding to the same slot seldom meet on one address), each kCap x (C + 2)
    // words -- features, then two packed words (see PackedSums) -- with an odd
    // copy stride so the copies of one word sit in different banks
    static constexpr int kCopies = 8, kPkStride = kCap * (C + 2) + 1;
    // integer images: kIntCopies copies of each word side by side (word w of
    // copy j at w * kIntCopies + j), the copy chosen by lane, so that the
    // lanes of one atomic instruction land in distinct banks (two lanes per
    // copy: 32 copies measured slower, their shared memory costs a CTA per SM)
    static constexpr int kIntCopies = 16;
    alignas(16) unsigned pk[kInBox ? kCap * (C + 2) * kIntCopies : kCopies * kPkStride];
    unsigned psum[kInBox ? kCap * (C + 2) : 1];  // integer images: the copies' sums
    float cpos[kCap][3];
    int cand[kCap];
    int tmp[kCap];
    int stage[kStage];
    uint32_t bmask[kCap];
    alignas(16) uint8_t slot[kInBox ? 16 : TV];
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

// two consecutive voxels of a float plane as one packed pair
template <typename T, int C, typename SH>
__device__ __forceinline__ uint64_t plane_pair_f(const Smem<T, C, SH>& s, int c, int xl, int yl, int zl)
{
    using S = Smem<T, C, SH>;
    return *reinterpret_cast<const uint64_t*>(s.planes + c * S::CPB + zl * S::PPB + yl * S::RPB + xl * 4);
}

// typed views of one candidate record
template <int C, typename SH, typename U>
__device__ __forceinline__ U* cand_at(unsigned char* cd, int slot, int off)
{
    return reinterpret_cast<U*>(cd + slot * CandLayout<C, SH>::CDS + off);
}

__device__ __forceinline__ void lds128(uint32_t addr, uint64_t& a, uint64_t& b)
{
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr));
}

__device__ __forceinline__ uint64_t lds64(uint32_t addr)
{
    uint64_t v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}

// The two integer values of a pair word (two 8-bit or two 16-bit voxels) as
// a packed FP32 pair, exactly: each value v is placed below the exponent of
// 2^23 (the float with bits 0x4B000000 | v is 2^23 + v, for v < 2^23) and
// 2^23 is subtracted from both halves at once.
template <typename T>
__device__ __forceinline__ uint64_t int_pair_to_f32x2(unsigned v)
{
    const unsigned lo = sizeof(T) == 1 ? __byte_perm(v, 0x4B000000u, 0x7540) : __byte_perm(v, 0x4B000000u, 0x7410);
    const unsigned hi = sizeof(T) == 1 ? __byte_perm(v, 0x4B000000u, 0x7541) : __byte_perm(v, 0x4B000000u, 0x7432);
    return sub2(pk2(__uint_as_float(lo), __uint_as_float(hi)), pk2(8388608.0f, 8388608.0f));
}

template <typename T>
__device__ __forceinline__ void split_pair(unsigned v, unsigned& lo, unsigned& hi)
{
    if constexpr (sizeof(T) == 1) { lo = v & 0xffu; hi = v >> 8; }
    else { lo = v & 0xffffu; hi = v >> 16; }
}

// Per-tile sums of one slot: one 32-bit word per feature, then sum x (17
// bits) with the count (13 bits) in one word and sum y (16 bits) with sum z
// (15 bits) in another, so a run of equal labels leaves through C + 2
// shared atomics.  The widths hold a whole tile: at most 4096 voxels, local
// x < 64, y < 32, z < 8.
struct PackedSums {
    static constexpr int kCnt = 17, kZ = 16;
};

// Float images keep their feature words as FP32 (run partials in FP32, added
// into the tile's FP32 words; the tile's sums then go to FP64 global sums).
template <typename T>
using FeatAcc = typename std::conditional<std::is_same<T, float>::value, float, unsigned>::type;

template <typename T, int C>
__device__ __forceinline__ void flush_run(unsigned* pk, int cur, const FeatAcc<T>* fs, unsigned xs, unsigned cnt, int yl,
                                          int zl)
{
    if (cur == kNoSlot || cnt == 0) return;
    unsigned* w = pk + cur * (C + 2);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if constexpr (std::is_same<T, float>::value) atomicAdd(reinterpret_cast<float*>(&w[c]), fs[c]);
        else atomicAdd(&w[c], fs[c]);
    }
    atomicAdd(&w[C], xs | (cnt << PackedSums::kCnt));
    atomicAdd(&w[C + 1], (cnt * (unsigned)yl) | ((cnt * (unsigned)zl) << PackedSums::kZ));
}

// ---- per-tile candidate lists ------------------------------------------------
// Step 2 done ahead of the tile kernel, one warp per tile, for a whole image:
// the warp gathers the centres of the bins that can reach the tile, keeps
// those whose window meets it and writes them sorted by index into the
// tile's record: [0] = their count, [1 .. count] = the indices, the rest -1.
// A tile with more than kStage gathered or kCap kept centres gets count -1
// and goes to the crowded-tile list here.  The tile kernel then starts from
// one coalesced load of the record instead of the chain of dependent loads,
// shared atomics and barriers of the in-kernel gather (which a tile kernel
// given no records still runs).  The batched queue has its own form below:
// one warp per (request, tile) of a group, each request's records in its
// arena block.
constexpr int kListStride = kCap + 1;
constexpr int kListWarps = 8;

// one tile's record (the warp's work; stage / kept are the warp's scratch)
template <int NDIM>
__device__ __forceinline__ void list_one_tile(const Geom& g, const float* __restrict__ ctr,
                                              const unsigned* __restrict__ bin_start,
                                              const int* __restrict__ bin_items, int* __restrict__ lists, int64_t tile,
                                              int ntx, int nty, int TX, int TY, int TZ, int64_t ovf_key,
                                              int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count,
                                              int* stage, int* kept, int lane)
{
    const int Tn[3] = {TX, TY, TZ};
    const unsigned t32 = (unsigned)tile;  // tile counts stay below 2^31: 32-bit division
    const unsigned txy = t32 / (unsigned)ntx;
    const int T0[3] = {(int)(t32 - txy * (unsigned)ntx) * TX, (int)(txy % (unsigned)nty) * TY,
                       (int)(txy / (unsigned)nty) * TZ};
    int E[3], blo[3], nbd[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        E[d] = min(Tn[d], (int)g.N[d] - T0[d]);
        blo[d] = max(0, T0[d] / g.S[d] - 1);
        nbd[d] = min((int)g.nb[d] - 1, (T0[d] + E[d] - 1) / g.S[d] + 1) - blo[d] + 1;
    }
    // gather: bins 32 at a time, items placed by a prefix sum of the counts
    const int nbins = nbd[0] * nbd[1] * nbd[2];
    int total = 0;
    for (int b0 = 0; b0 < nbins; b0 += 32) {
        const int b = b0 + lane;
        unsigned first = 0, cnt = 0;
        if (b < nbins) {
            const unsigned bq = (unsigned)b / (unsigned)nbd[0];
            const int bx = blo[0] + (int)((unsigned)b - bq * (unsigned)nbd[0]),
                      by = blo[1] + (int)(bq % (unsigned)nbd[1]), bz = blo[2] + (int)(bq / (unsigned)nbd[1]);
            const int64_t bin = bx + g.nb[0] * (by + g.nb[1] * (int64_t)bz);
            first = bin_start[bin];
            cnt = bin_start[bin + 1] - first;
        }
        unsigned inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        const unsigned base = (unsigned)total + inc - cnt;
        for (unsigned j = 0; j < cnt; ++j)
            if (base + j < (unsigned)kStage) stage[base + j] = bin_items[first + j];
        total += (int)__shfl_sync(0xffffffffu, inc, 31);
    }
    __syncwarp();
    // filter: windows that meet the tile, compacted by ballot
    int nc = 0;
    if (total <= kStage) {
        for (int i0 = 0; i0 < total; i0 += 32) {
            const int i = i0 + lane;
            bool hit = false;
            int k = 0;
            if (i < total) {
                k = stage[i];
                const float* pos = ctr + (int64_t)k * g.CW + g.C;
                hit = true;
#pragma unroll
                for (int d = 0; d < NDIM; ++d) {
                    const int lo = (int)ceilf(pos[d]) - g.S[d];
                    hit = hit && (lo <= T0[d] + E[d] - 1) && (lo + 2 * g.S[d] - 1 >= T0[d]);
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            const int at = nc + __popc(m & ((1u << lane) - 1u));
            if (hit && at < kCap) kept[at] = k;
            nc += __popc(m);
        }
    }
    __syncwarp();
    int* rec = lists + tile * kListStride;
    if (total > kStage || nc > kCap) {
        for (int i = lane; i < kListStride; i += 32) rec[i] = -1;
        if (lane == 0) ovf_tiles[atomicAdd(ovf_count, 1u)] = ovf_key;
    } else {
        // rank sort (the indices are distinct: a centre sits in one bin)
        for (int i = lane; i < kCap; i += 32) {
            int v = -1, r = i;
            if (i < nc) {
                v = kept[i];
                r = 0;
                for (int j = 0; j < nc; ++j) r += (kept[j] < v);
            }
            rec[1 + r] = v;
        }
        if (lane == 0) rec[0] = nc;
    }
}

template <int NDIM>
__global__ void __launch_bounds__(kListWarps * 32)
tile_lists_kernel(Geom g, const float* __restrict__ ctr, const unsigned* __restrict__ bin_start,
                  const int* __restrict__ bin_items, int* __restrict__ lists, int64_t tile0, int64_t ntiles, int ntx,
                  int nty, int TX, int TY, int TZ, int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count)
{
    __shared__ int stage_all[kListWarps][kStage];
    __shared__ int kept_all[kListWarps][kCap];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int64_t tile = tile0 + (int64_t)blockIdx.x * kListWarps + wp; tile < tile0 + ntiles;
         tile += (int64_t)gridDim.x * kListWarps) {
        list_one_tile<NDIM>(g, ctr, bin_start, bin_items, lists, tile, ntx, nty, TX, TY, TZ, tile, ovf_tiles, ovf_count,
                            stage_all[wp], kept_all[wp], lane);
        __syncwarp();
    }
}

// the same for the batched queue: one warp per (request, tile) work item of
// the requests of one group (request r owns items [tpre[r], tpre[r + 1]));
// crowded tiles go to the group's list as (r << 40 | tile)
template <int NDIM>
__global__ void __launch_bounds__(kListWarps * 32)
tile_lists_queue_kernel(const TileArgs* __restrict__ reqs, const int64_t* __restrict__ tpre,
                        const int* __restrict__ nR, int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count)
{
    __shared__ int stage_all[kListWarps][kStage];
    __shared__ int kept_all[kListWarps][kCap];
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int R = *nR;
    const int64_t total = tpre[R];
    for (int64_t i = (int64_t)blockIdx.x * kListWarps + wp; i < total; i += (int64_t)gridDim.x * kListWarps) {
        int lo = 0, hi = R - 1;  // last r with tpre[r] <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tpre[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const TileArgs& a = reqs[lo];
        const int64_t tile = i - tpre[lo];
        list_one_tile<NDIM>(a.g, a.ctr, a.bin_start, a.bin_items, const_cast<int*>(a.lists), tile, a.ntx, a.nty, a.tx, a.ty, a.tz,
                            ((int64_t)lo << 40) | tile, ovf_tiles, ovf_count, stage_all[wp], kept_all[wp], lane);
        __syncwarp();
    }
}

// One tile of one image (request req): everything of steps 1-5 above.  A
// tile reached by more than kCap centres is appended to the crowded-tile
// list as (req << 40 | tile) and left to the per-voxel kernel.
template <typename T, int C, typename SH, bool STAGED = false>
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
    using CL = CandLayout<C, SH>;
    constexpr int TX = G::TX, TY = G::TY, TZ = G::TZ, TV = TX * TY * TZ;
    constexpr int WX = G::WX, WY = G::WY, WZ = G::WZ, VL = G::VL, NP = VL / 2;
    constexpr int BX = VL * WX, BY = WY, BZ = WZ;
    static_assert(VL == 2 || VL == 4, "voxels per lane");
    constexpr int NBX = TX / BX, NBY = TY / BY, NBZ = TZ / BZ;
    constexpr int NBOX = NBX * NBY * NBZ;
    constexpr int PASSES = NBOX / kWarps;
    constexpr int F = C + 4;
    constexpr int SPR = TX / kSeg;  // segments per row
    static_assert(NBOX % kWarps == 0, "boxes per warp");
    static_assert(TV <= 4096 && TX <= 64 && TY <= 32 && TZ <= 8, "packed per-tile sums");
    static_assert(!S::kInBox || C == 1 || (C == 3 && sizeof(T) == 1), "packed 64-bit feature sums");
    static_assert(NBX + NBY + NBZ <= 32, "box mask bits");
    static_assert(TX % kSeg == 0, "row segments");

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int X0 = (tile % ntx) * TX;
    const int Y0 = ((tile / ntx) % nty) * TY;
    const int Z0 = (tile / (ntx * nty)) * TZ;
    const int N0 = (int)g.N[0], N1 = (int)g.N[1], N2 = (int)g.N[2];
    const int ex = min(TX, N0 - X0), ey = min(TY, N1 - Y0), ez = min(TZ, N2 - Z0);

    // lists mode: this thread's entry of the tile's candidate record, loaded
    // before the staging so its latency overlaps it
    const bool lists = a.lists != nullptr;
    int lk = -1;
    if (lists && tid < kListStride) lk = __ldg(a.lists + (int64_t)tile * kListStride + tid);

    if (tid == 0) { s.nstage = 0; s.ncand = 0; }
    if constexpr (sizeof(s.pk) % 16 == 0) {
        for (int i = tid; i < (int)(sizeof(s.pk) / 16); i += kThreads) reinterpret_cast<uint4*>(s.pk)[i] = make_uint4(0u, 0u, 0u, 0u);
    } else {
        for (int i = tid; i < (int)(sizeof(s.pk) / sizeof(unsigned)); i += kThreads) s.pk[i] = 0u;
    }

    // ---- 1. stage the tile as channel planes (done by the caller when STAGED) ----
    // 8-bit colour images with full rows: every thread issues the loads of its
    // 12-byte groups (4 voxels) here and writes them into the planes only
    // after the candidate tables are built, so that the image's latency
    // overlaps the record's rows and the tables
    constexpr int GPR = TX / 4;                                 // groups per row
    constexpr int NG = TY * TZ * GPR;                           // groups per tile
    constexpr int GPT = (NG + kThreads - 1) / kThreads;         // groups per thread
    constexpr bool kDefer = !STAGED && sizeof(T) == 1 && C == 3;
    uint32_t ga[kDefer ? GPT : 1], gb[kDefer ? GPT : 1], gc[kDefer ? GPT : 1];
    bool fast = false;
    if constexpr (STAGED) {
    } else if constexpr (sizeof(T) == 1 && C == 3) {
        fast = (ex == TX) && ((N0 * 3) % 4 == 0) && (((uintptr_t)img & 3) == 0);
        if (fast) {
#pragma unroll
            for (int k = 0; k < GPT; ++k) {
                const int i = tid + k * kThreads;
                const int r = i / GPR, gi = i % GPR, yl = r % TY, zl = r / TY;
                ga[k] = gb[k] = gc[k] = 0;
                if (i < NG && yl < ey && zl < ez) {
                    const uint32_t* src = reinterpret_cast<const uint32_t*>(
                        img + (vidx(g, X0, Y0 + yl, Z0 + zl) + gi * 4) * 3);
                    ga[k] = __ldg(src);
                    gb[k] = __ldg(src + 1);
                    gc[k] = __ldg(src + 2);
                }
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
    } else if constexpr (S::kF && C == 3) {
        // full rows of 16-byte groups (4 floats: voxel x = e / 3, channel e % 3)
        const bool fast = (ex == TX) && (N0 % 4 == 0) && (((uintptr_t)img & 15) == 0);
        if (fast) {
            constexpr int GPR = TX * 3 / 4;  // groups per row
            for (int i = tid; i < TY * TZ * GPR; i += kThreads) {
                const int r = i / GPR, gi = i % GPR, yl = r % TY, zl = r / TY;
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (yl < ey && zl < ez)
                    v = __ldg(reinterpret_cast<const float4*>(img + vidx(g, X0, Y0 + yl, Z0 + zl) * 3) + gi);
                const float f4[4] = {v.x, v.y, v.z, v.w};
                unsigned char* row = s.planes + zl * S::PPB + yl * S::RPB;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int e = 4 * gi + j;
                    *reinterpret_cast<float*>(row + (e % 3) * S::CPB + (e / 3) * 4) = f4[j];
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
    // lists mode: the rows of the record's centres, fetched before the barrier
    float rowv[C + NDIM];
    if (lists) {
        if (tid >= 1 && tid < kListStride && lk >= 0 && lk < g.K) {
            const float* row = ctr + (int64_t)lk * g.CW;
#pragma unroll
            for (int j = 0; j < C + NDIM; ++j) rowv[j] = row[j];
        }
        if (tid == 0) s.ncand = lk;
    }
    __syncthreads();
    int nc;
    if (lists) {
        nc = s.ncand;
        if (nc < 0) return;  // block-uniform: the list kernel sent the tile to the per-voxel kernel
        if (tid >= 1 && tid <= nc) {
            const int r = tid - 1;
            s.cand[r] = lk;
#pragma unroll
            for (int c = 0; c < C; ++c) cand_at<C, SH, float2>(s.cd, r, CL::kOffFe)[c] = make_float2(rowv[c], rowv[c]);
#pragma unroll
            for (int d = 0; d < 3; ++d) s.cpos[r][d] = d < NDIM ? rowv[C + d] : 0.0f;
        }
    } else {
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
        nc = s.ncand;
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
            for (int c = 0; c < C; ++c) cand_at<C, SH, float2>(s.cd, r, CL::kOffFe)[c] = make_float2(row[c], row[c]);
            s.cpos[r][0] = row[C];
            s.cpos[r][1] = row[C + 1];
            s.cpos[r][2] = row[C + 2];
        }
    }
    __syncthreads();

    // ---- per-centre tables and warp-box reach masks -------------------------
    // t_d entry: w_d (x - c)^2 with one rounding per operation, +inf outside
    // the window [ceil(c) - S_d, ceil(c) + S_d - 1].  One thread fills four
    // consecutive entries of one axis of one centre (a 16-byte store for
    // t_0, two for the paired t_1 / t_2).
    {
        constexpr int QX = TX / 4, QY = NDIM >= 2 ? TY / 4 : 0, QZ = NDIM >= 3 ? TZ / 4 : 0;
        constexpr int QA = QX + QY + QZ;
        static_assert(TX % 4 == 0 && (NDIM < 2 || TY % 4 == 0) && (NDIM < 3 || TZ % 4 == 0), "table chunks");
        for (int i = tid; i < nc * QA; i += kThreads) {
            const int sl = i / QA, q = i - sl * QA;
            const int d = q < QX ? 0 : (q < QX + QY ? 1 : 2);
            const int j0 = 4 * (d == 0 ? q : (d == 1 ? q - QX : q - QX - QY));
            const float c = s.cpos[sl][d];
            const int lo = (int)ceilf(c) - g.S[d];
            const unsigned span = 2u * (unsigned)g.S[d];
            const float wd = g.w[d];
            float t[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int x = T0[d] + j0 + e;
                const float dl = __fsub_rn((float)x, c);
                const float v = __fmul_rn(wd, __fmul_rn(dl, dl));
                t[e] = (unsigned)(x - lo) < span ? v : kInf;
            }
            if (d == 0) {
                *reinterpret_cast<float4*>(cand_at<C, SH, float>(s.cd, sl, CL::kOffT0) + j0) =
                    make_float4(t[0], t[1], t[2], t[3]);
            } else {
                float4* dst = reinterpret_cast<float4*>(
                    cand_at<C, SH, float2>(s.cd, sl, d == 1 ? CL::kOffT1 : CL::kOffT2) + j0);
                dst[0] = make_float4(t[0], t[0], t[1], t[1]);
                dst[1] = make_float4(t[2], t[2], t[3], t[3]);
            }
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
    for (int i = tid; i < TX; i += kThreads) cand_at<C, SH, float>(s.cd, kCap, CL::kOffT0)[i] = kInf;
    for (int i = tid; i < TY; i += kThreads) cand_at<C, SH, float2>(s.cd, kCap, CL::kOffT1)[i] = make_float2(kInf, kInf);
    for (int i = tid; i < TZ; i += kThreads) cand_at<C, SH, float2>(s.cd, kCap, CL::kOffT2)[i] = make_float2(kInf, kInf);
    if (tid < C) cand_at<C, SH, float2>(s.cd, kCap, CL::kOffFe)[tid] = make_float2(0.0f, 0.0f);
    if constexpr (kDefer) {
        if (fast) {
            // the staged groups into the planes
#pragma unroll
            for (int k = 0; k < GPT; ++k) {
                const int i = tid + k * kThreads;
                if (i >= NG) break;
                const int r = i / GPR, gi = i % GPR, yl = r % TY, zl = r / TY;
                const uint32_t a_ = ga[k], b_ = gb[k], c_ = gc[k];
                // bytes: a = R0 G0 B0 R1, b = G1 B1 R2 G2, c = B2 R3 G3 B3
                unsigned char* row = s.planes + zl * S::PPB + yl * S::RPB + gi * 4;
                *reinterpret_cast<uint32_t*>(row) = __byte_perm(__byte_perm(a_, b_, 0x0630), c_, 0x5210);
                *reinterpret_cast<uint32_t*>(row + S::CPB) = __byte_perm(__byte_perm(a_, b_, 0x0741), c_, 0x6210);
                *reinterpret_cast<uint32_t*>(row + 2 * S::CPB) = __byte_perm(__byte_perm(a_, b_, 0x0052), c_, 0x7410);
            }
        }
    }
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
    const bool lvec4 = (N0 % 4 == 0) && (((uintptr_t)labels & 15) == 0);
    const bool lvec2 = (N0 % 2 == 0) && (((uintptr_t)labels & 7) == 0);
    const uint32_t cdb = (uint32_t)__cvta_generic_to_shared(&s.cd[0]);
    constexpr int CDS = CL::CDS;
#pragma unroll 1
    for (int pass = 0; pass < PASSES; ++pass) {
        const int wb = warp + pass * kWarps;
        const int bxi = wb % NBX, byi = (wb / NBX) % NBY, bzi = wb / (NBX * NBY);
        const int xl = bxi * BX + lx * VL, yl = byi * BY + ly, zl = bzi * BZ + lz;
        uint64_t Fp[C][NP];  // the lane's voxels xl .. xl + VL - 1, in pairs
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                if constexpr (S::kF) Fp[c][q] = plane_pair_f(s, c, xl + 2 * q, yl, zl);
                else Fp[c][q] = int_pair_to_f32x2<T>(plane_pair(s, c, xl + 2 * q, yl, zl));
            }
        float bd[VL];
        int bs[VL];
#pragma unroll
        for (int v = 0; v < VL; ++v) { bd[v] = kInf; bs[v] = kNoSlot; }
        const uint32_t a0 = cdb + CL::kOffT0 + xl * 4;
        const uint32_t a1 = cdb + CL::kOffT1 + yl * 8;
        const uint32_t a2 = cdb + CL::kOffT2 + zl * 8;
        const uint32_t af = cdb + CL::kOffFe;
        const int nb = s.bcnt[wb];
        const uint16_t* lst = reinterpret_cast<const uint16_t*>(&s.blist[wb][0]);
        // D^2 of the lane's voxels against the centre in slot sl
        auto dist2 = [&](int sl, uint64_t (&D)[NP]) {
            const uint32_t so = (uint32_t)(sl * CDS);
            uint64_t t0[NP];
            if constexpr (NP == 1) t0[0] = lds64(a0 + so);
            else lds128(a0 + so, t0[0], t0[1]);
            uint64_t t1 = 0, t2 = 0;
            if (NDIM >= 2) t1 = lds64(a1 + so);
            if (NDIM >= 3) t2 = lds64(a2 + so);
            uint64_t fe[C];
            // feature pairs two channels per 16-byte load where the record allows
#pragma unroll
            for (int c = 0; c < C; c += 2) {
                if (c + 1 < C && CL::kOffFe % 16 == 0) {
                    lds128(af + so + c * 8, fe[c], fe[c + 1]);
                } else {
                    fe[c] = lds64(af + so + c * 8);
                    if (c + 1 < C) fe[c + 1] = lds64(af + so + (c + 1) * 8);
                }
            }
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                uint64_t dc;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const uint64_t e = sub2(Fp[c][q], fe[c]);
                    const uint64_t sq = mul2(e, e);
                    dc = c == 0 ? sq : add2(dc, sq);
                }
                uint64_t ds = t0[q];
                if (NDIM >= 2) ds = add2(ds, t1);
                if (NDIM >= 3) ds = add2(ds, t2);
                D[q] = add2(dc, ds);
            }
        };
        auto take = [&](const uint64_t (&D)[NP], int sl) {
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float d0, d1;
                upk2(D[q], d0, d1);
                if (d0 < bd[2 * q]) { bd[2 * q] = d0; bs[2 * q] = sl; }
                if (d1 < bd[2 * q + 1]) { bd[2 * q + 1] = d1; bs[2 * q + 1] = sl; }
            }
        };
#pragma unroll 1
        for (int i = 0; i < nb; i += 2) {
            const unsigned two = lst[i >> 1];
            const int sa = (int)(two & 0xffu), sb = (int)(two >> 8);
            uint64_t Da[NP], Db[NP];
            dist2(sa, Da);
            dist2(sb, Db);
            take(Da, sa);
            take(Db, sb);
        }
        if constexpr (S::kInBox) {
            // map step for the lane's own voxels: labels out (one vector
            // store when the row allows it), and [I, x, y, z, 1] of every
            // labelled voxel into its slot's packed per-tile sums
            const bool rowin = yl < ey && zl < ez;
            unsigned val[C][VL];
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int q = 0; q < NP; ++q)
                    split_pair<T>(plane_pair(s, c, xl + 2 * q, yl, zl), val[c][2 * q], val[c][2 * q + 1]);
            int lab[VL];
            // copy: the lanes that share one differ in more than one axis of
            // the box, so that they seldom add to the same slot at once
            unsigned* const mypk = s.pk + (lane & (S::kIntCopies - 1));
#pragma unroll
            for (int v = 0; v < VL; ++v) {
                const bool in = rowin && xl + v < ex && bs[v] != kNoSlot;
                lab[v] = in ? s.cand[bs[v]] : -1;
                if (in) {
                    unsigned* w = mypk + bs[v] * (C + 2) * S::kIntCopies;
#pragma unroll
                    for (int c = 0; c < C; ++c) atomicAdd(&w[c * S::kIntCopies], val[c][v]);
                    atomicAdd(&w[C * S::kIntCopies], (unsigned)(xl + v) | (1u << PackedSums::kCnt));
                    atomicAdd(&w[(C + 1) * S::kIntCopies], (unsigned)yl | ((unsigned)zl << PackedSums::kZ));
                }
            }
            if (rowin) {
                int32_t* lp = labels + vidx(g, X0 + xl, Y0 + yl, Z0 + zl);
                if (xl + VL <= ex && ((VL == 4 && lvec4) || (VL == 2 && lvec2))) {
                    if constexpr (VL == 4) *reinterpret_cast<int4*>(lp) = make_int4(lab[0], lab[1], lab[2], lab[3]);
                    else *reinterpret_cast<int2*>(lp) = make_int2(lab[0], lab[1]);
                } else {
#pragma unroll
                    for (int v = 0; v < VL; ++v)
                        if (xl + v < ex) lp[v] = lab[v];
                }
            }
        } else {
            uint8_t* so = &s.slot[(zl * TY + yl) * TX + xl];
            if constexpr (VL == 2) *reinterpret_cast<uint16_t*>(so) = (uint16_t)(bs[0] | (bs[1] << 8));
            else *reinterpret_cast<uint32_t*>(so) = (uint32_t)bs[0] | ((uint32_t)bs[1] << 8) |
                                                    ((uint32_t)bs[2] << 16) | ((uint32_t)bs[3] << 24);
        }
    }
    __syncthreads();

    if constexpr (!S::kInBox) {
        // ---- 4. row segments: labels out, run sums in -------------------------------
        unsigned* const mypk = s.pk + (lane & (S::kCopies - 1)) * S::kPkStride;
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
            FeatAcc<T> fs[C];
            unsigned xs = 0, cnt = 0;
#pragma unroll
            for (int c = 0; c < C; ++c) fs[c] = 0;
            // start a new run at slot sl (flushing the previous one)
            auto next_run = [&](int sl) {
                flush_run<T, C>(mypk, cur, fs, xs, cnt, yl, zl);
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
                                    else fs[c] += (FeatAcc<T>)*reinterpret_cast<const T*>(
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
                            fs[c] += (FeatAcc<T>)*reinterpret_cast<const T*>(prow + c * S::CPB + (xs0 + b) * (int)sizeof(T));
                        xs += (unsigned)(xs0 + b);
                        cnt += 1u;
                    }
                    lrow[b] = curlab;
                }
            }
            flush_run<T, C>(mypk, cur, fs, xs, cnt, yl, zl);
        }
        __syncthreads();
    }

    // ---- 5. per-tile sums, shifted to global coordinates ----------------------
    // the copies are summed word by word (each field's total fits its width)
    if constexpr (S::kInBox) {
        // one word per thread, its 16 copies as four 16-byte loads; quarter q
        // is read at step (q + word / 2) mod 4, so that the 8 threads of each
        // load phase cover the 32 banks once
        static_assert(S::kIntCopies == 16, "four 16-byte quarters per word");
        for (int wd = tid; wd < nc * (C + 2); wd += kThreads) {
            const uint4* w4 = reinterpret_cast<const uint4*>(s.pk + wd * S::kIntCopies);
            unsigned t = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint4 v = w4[(j + (wd >> 1)) & 3];
                t += (v.x + v.y) + (v.z + v.w);
            }
            s.psum[wd] = t;
        }
        __syncthreads();
    }
    for (int i = tid; i < nc * F; i += kThreads) {
        const int sl = i / F, f = i % F;
        unsigned wx = 0, wyz = 0;
        FeatAcc<T> wf = 0;
        if constexpr (S::kInBox) {
            const unsigned* w = s.psum + sl * (C + 2);
            wx = w[C];
            if (f == C + 1 || f == C + 2) wyz = w[C + 1];
            if (f < C) wf = w[f];
        } else {
#pragma unroll
            for (int k = 0; k < S::kCopies; ++k) {
                const unsigned* w = s.pk + k * S::kPkStride + sl * (C + 2);
                wx += w[C];
                if (f == C + 1 || f == C + 2) wyz += w[C + 1];
                if (f < C) {
                    if constexpr (S::kF) wf += __uint_as_float(w[f]);
                    else wf += w[f];
                }
            }
        }
        const unsigned long long cnt = wx >> PackedSums::kCnt;
        if (!cnt) continue;
        if constexpr (S::kF) {
            if (f < C) {
                atomicAdd(&a.facc[(int64_t)s.cand[sl] * C + f], (double)wf);
                continue;
            }
        }
        unsigned long long v;
        if (f < C) v = (unsigned long long)wf;
        else if (f == C) v = (wx & ((1u << PackedSums::kCnt) - 1)) + cnt * (unsigned long long)X0;
        else if (f == C + 1) v = (wyz & ((1u << PackedSums::kZ) - 1)) + cnt * (unsigned long long)Y0;
        else if (f == C + 2) v = (wyz >> PackedSums::kZ) + cnt * (unsigned long long)Z0;
        else v = cnt;
        atomicAdd(&acc[(int64_t)s.cand[sl] * F + f], v);
    }
}

// The tile as the TMA copy leaves it -- bytes [z][y][x * C * sizeof(T)], rows
// contiguous, out-of-image voxels zero -- rewritten as the channel planes.
template <typename T, int C, typename SH>
__device__ __forceinline__ void planes_from_raw(Smem<T, C, SH>& s, const unsigned char* raw)
{
    using S = Smem<T, C, SH>;
    constexpr int TX = SH::TX, TY = SH::TY, TZ = SH::TZ;
    constexpr int RB = TX * C * (int)sizeof(T);  // raw row bytes
    const int tid = threadIdx.x;
    if constexpr (sizeof(T) == 1 && C == 3) {
        constexpr int GPR = TX / 4;  // 12-byte groups (4 voxels) per row
        for (int i = tid; i < TY * TZ * GPR; i += kThreads) {
            const int r = i / GPR, gi = i % GPR, yl = r % TY, zl = r / TY;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(raw + r * RB + gi * 12);
            const uint32_t a = src[0], b = src[1], cc = src[2];
            // bytes: a = R0 G0 B0 R1, b = G1 B1 R2 G2, cc = B2 R3 G3 B3
            unsigned char* row = s.planes + zl * S::PPB + yl * S::RPB + gi * 4;
            *reinterpret_cast<uint32_t*>(row) = __byte_perm(__byte_perm(a, b, 0x0630), cc, 0x5210);
            *reinterpret_cast<uint32_t*>(row + S::CPB) = __byte_perm(__byte_perm(a, b, 0x0741), cc, 0x6210);
            *reinterpret_cast<uint32_t*>(row + 2 * S::CPB) = __byte_perm(__byte_perm(a, b, 0x0052), cc, 0x7410);
        }
    } else {
        static_assert(C == 1, "single-channel raw rows are plane rows");
        constexpr int WPR = RB / 4;  // words per row
        for (int i = tid; i < TY * TZ * WPR; i += kThreads) {
            const int r = i / WPR, wi = i % WPR, yl = r % TY, zl = r / TY;
            const uint32_t v = reinterpret_cast<const uint32_t*>(raw + r * RB)[wi];
            *reinterpret_cast<uint32_t*>(s.planes + zl * S::PPB + yl * S::RPB + wi * 4) = v;
        }
    }
}

template <typename T, int C, typename SH>
struct SmemTma {
    Smem<T, C, SH> s;
    alignas(128) unsigned char raw[SH::TX * C * sizeof(T) * SH::TY * SH::TZ];
    uint64_t mbar;
};

constexpr long long kTmaWaitLimit = 1LL << 26;  // polls of the copy's mbarrier before giving up

// One image, persistent: each CTA walks tiles blockIdx.x, + gridDim.x, ...
// and the TMA copy of its next tile's image runs while it computes the
// current one.  A wait that runs out sets *status and ends the CTA.
template <typename T, int C, typename SH>
__global__ void __launch_bounds__(kThreads, 4)
assign_tile_tma_kernel(TileArgs a, const __grid_constant__ CUtensorMap map, int64_t ntiles,
                       int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count, unsigned* __restrict__ status)
{
    extern __shared__ __align__(128) unsigned char smem_tma[];
    SmemTma<T, C, SH>& st = *reinterpret_cast<SmemTma<T, C, SH>*>(smem_tma);
    constexpr uint32_t kBytes = (uint32_t)sizeof(st.raw);
    constexpr int TX = SH::TX, TY = SH::TY, TZ = SH::TZ;
    const int tid = threadIdx.x;
    const int ntx = a.ntx, nty = a.nty;
    auto issue = [&](int64_t t) {
        const int X0 = (int)(t % ntx) * TX, Y0 = (int)((t / ntx) % nty) * TY, Z0 = (int)(t / ((int64_t)ntx * nty)) * TZ;
        tc::mbar_arrive_expect_tx(&st.mbar, kBytes);
        const int xb = X0 * C * (int)sizeof(T);  // a multiple of 16 bytes
        if constexpr (SH::NDIM == 3) tc::tma_load_3d(st.raw, &map, xb, Y0, Z0, &st.mbar);
        else tc::tma_load_2d(st.raw, &map, xb, Y0, &st.mbar);
    };
    int64_t t = blockIdx.x;
    if (tid == 0) {
        tc::mbar_init(&st.mbar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0 && t < ntiles) issue(t);
    uint32_t parity = 0;
    for (; t < ntiles; t += gridDim.x) {
        bool done = false;
        for (long long it = 0; it < kTmaWaitLimit && !done; ++it) done = tc::mbar_try_wait(&st.mbar, parity);
        if (!__syncthreads_and(done)) {
            if (tid == 0) {
                atomicExch(status, 1u);
                // give the copy in flight one more bounded wait before leaving
                for (long long it = 0; it < kTmaWaitLimit && !tc::mbar_try_wait(&st.mbar, parity); ++it) {}
            }
            return;
        }
        parity ^= 1u;
        planes_from_raw<T, C, SH>(st.s, st.raw);
        __syncthreads();  // the raw buffer is free again
        if (tid == 0 && t + gridDim.x < ntiles) {
            tc::fence_proxy_async_smem();
            issue(t + gridDim.x);
        }
        tile_body<T, C, SH, true>(a, (int)t, 0, st.s, ovf_tiles, ovf_count);
        __syncthreads();  // this tile's shared state is no longer read
    }
}

// one image: one CTA per tile
template <typename T, int C, typename SH>
__global__ void __launch_bounds__(kThreads, 4)
assign_tile_kernel(TileArgs a, int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_body<T, C, SH>(a, (int)(a.tile0 + blockIdx.x), 0, *reinterpret_cast<Smem<T, C, SH>*>(smem_raw), ovf_tiles,
                        ovf_count);
}

// many images: a persistent grid walks one queue of (request, tile) work
// items; request r owns global tile numbers [tpre[r], tpre[r + 1])
template <typename T, int C, typename SH>
__global__ void __launch_bounds__(kThreads, 4)
assign_tile_queue_kernel(const TileArgs* __restrict__ reqs, const int64_t* __restrict__ tpre,
                         const int* __restrict__ nR, int64_t* __restrict__ ovf_tiles,
                         unsigned* __restrict__ ovf_count)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<T, C, SH>& s = *reinterpret_cast<Smem<T, C, SH>*>(smem_raw);
    const int R = *nR;
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
inline void tile_grid(const Geom& g, int& ntx, int& nty, int& ntz)
{
    ntx = (int)((g.N[0] + SH::TX - 1) / SH::TX);
    nty = (int)((g.N[1] + SH::TY - 1) / SH::TY);
    ntz = (int)((g.N[2] + SH::TZ - 1) / SH::TZ);
}

// calls f(SH{}) with the shape type of shape index `shape` (see tile_dims)
template <int NDIM, typename F>
inline auto with_shape(int shape, F&& f)
{
    if constexpr (NDIM == 3) {
        switch (shape) {
        case 1: return f(tile::Shape3S{});
        case 2: return f(tile::Shape3L4{});
        case 3: return f(tile::Shape3S4{});
        case 4: return f(tile::Shape3M{});
        case 5: return f(tile::Shape3M4{});
        default: return f(tile::Shape3L{});
        }
    } else {
        switch (shape) {
        case 1: return f(tile::Shape2S{});
        case 2: return f(tile::Shape2L4{});
        default: return f(tile::Shape2L{});
        }
    }
}

template <typename T, int C, typename SH>
inline int launch_tile_shape(sslic_ctx* c, const T* img, int32_t* labels, cudaStream_t st, bool want_tma,
                             const Slab* slab)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    int ntx, nty, ntz;
    tile_grid<SH>(g, ntx, nty, ntz);
    // the tiles of the launch: all, or the slab's rows of tiles along the last
    // axis (tiles are numbered with that axis slowest; slab bounds are tile-aligned)
    int64_t tile0 = 0, ntiles = (int64_t)ntx * nty * ntz;
    if (slab) {
        const int64_t ext = SH::NDIM == 3 ? SH::TZ : SH::TY;
        const int64_t row = SH::NDIM == 3 ? (int64_t)ntx * nty : (int64_t)ntx;
        if (slab->lo % ext != 0 || (slab->hi % ext != 0 && slab->hi != g.N[SH::NDIM - 1]))
            return set_error(c, SSLIC_EINVAL, "slab bounds are not multiples of the tile extent");
        tile0 = slab->lo / ext * row;
        ntiles = (slab->hi + ext - 1) / ext * row - tile0;
        want_tma = false;
    }
    const size_t smem = sizeof(tile::Smem<T, C, SH>);
    int rc = cuda_check(c, cudaFuncSetAttribute(tile::assign_tile_kernel<T, C, SH>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                        "smem attribute");
    if (rc) return rc;
    if ((rc = cuda_check(c, cudaMemsetAsync(w.ovf_count, 0, sizeof(unsigned), st), "memset ovf"))) return rc;
    if (w.tile_lists) {
        // step 2 for every tile at once (timed with the bins it reads)
        const int64_t lgrid = imin64((ntiles + tile::kListWarps - 1) / tile::kListWarps, (int64_t)c->sms * 32);
        const int pr = prof_begin(c, SSLIC_PHASE_BINS, st);
        tile::tile_lists_kernel<SH::NDIM><<<(unsigned)lgrid, tile::kListWarps * 32, 0, st>>>(
            g, w.ctr, w.bin_start, w.bin_items, w.tile_lists, tile0, ntiles, ntx, nty, SH::TX, SH::TY, SH::TZ,
            w.ovf_tiles, w.ovf_count);
        count_launch(c);
        prof_end(c, pr, st);
        if ((rc = cuda_check(c, cudaGetLastError(), "tile_lists_kernel"))) return rc;
    }
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
    a.lists = w.tile_lists;
    a.tile0 = tile0;
    alignas(64) CUtensorMap map;
    const bool tma = sizeof(T) < 4 && want_tma && image_tma_ok(g, img, (int)sizeof(T)) &&
                     encode_image_map(&map, g, img, (int)sizeof(T), SH::TX, SH::TY, SH::TZ) == SSLIC_OK;
    bool launched = false;
    if constexpr (sizeof(T) < 4) {  // float planes: a TMA-staged index runs its base shape
        if (tma) {
            // persistent: as many CTAs as fit at once, each walking its share of the tiles
            const size_t smem_t = sizeof(tile::SmemTma<T, C, SH>);
            if ((rc = cuda_check(c, cudaFuncSetAttribute(tile::assign_tile_tma_kernel<T, C, SH>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t),
                                 "smem attribute")))
                return rc;
            int per_sm = 0;
            if ((rc = cuda_check(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                        &per_sm, tile::assign_tile_tma_kernel<T, C, SH>, tile::kThreads, smem_t),
                                 "occupancy")))
                return rc;
            const int64_t grid = imin64(ntiles, (int64_t)c->sms * (per_sm > 0 ? per_sm : 1));
            const int pr = prof_begin(c, SSLIC_PHASE_ASSIGN, st);
            tile::assign_tile_tma_kernel<T, C, SH><<<(unsigned)grid, tile::kThreads, smem_t, st>>>(
                a, map, ntiles, w.ovf_tiles, w.ovf_count, w.hc_err);
            count_launch(c);
            prof_end(c, pr, st);
            c->status_pending = 1;
            if ((rc = cuda_check(c, cudaGetLastError(), "assign_tile_tma_kernel"))) return rc;
            launched = true;
        }
    }
    if (!launched) {
        const int pr = prof_begin(c, SSLIC_PHASE_ASSIGN, st);
        tile::assign_tile_kernel<T, C, SH><<<(unsigned)ntiles, tile::kThreads, smem, st>>>(a, w.ovf_tiles, w.ovf_count);
        count_launch(c);
        prof_end(c, pr, st);
        if ((rc = cuda_check(c, cudaGetLastError(), "assign_tile_kernel"))) return rc;
    }
    return launch_voxel_tiles(c, img, labels, SH::TX, SH::TY, SH::TZ, ntx, nty, st);
}

template <typename T, int C, int NDIM>
int launch_tile_impl(sslic_ctx* c, const T* img, int32_t* labels, cudaStream_t st, const Slab* slab)
{
    int shape = c->tile_shape;
    if (shape < 0) shape = tuned_tile_shape(c->g);
    if (shape < 0) shape = default_tile_shape(c->g);
    const int b = num_base_shapes(NDIM);
    return with_shape<NDIM>(shape % b, [&](auto sh) {
        return launch_tile_shape<T, C, decltype(sh)>(c, img, labels, st, shape >= b, slab);
    });
}

// batched form: one persistent launch over the (request, tile) queue of all
// requests of one type and shape (*nR of them, read on the device); returns
// the CUDA error of the launch.  With reqs == nullptr it only sets the
// kernel's shared-memory limit (done before a stream capture).
template <typename T, int C, typename SH>
inline cudaError_t launch_queue_shape(const TileArgs* reqs, const int64_t* tpre, const int* nR, int64_t* ovf,
                                      unsigned* ovf_count, int grid, cudaStream_t st)
{
    const size_t smem = sizeof(tile::Smem<T, C, SH>);
    if (!reqs)
        return cudaFuncSetAttribute(tile::assign_tile_queue_kernel<T, C, SH>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tile::assign_tile_queue_kernel<T, C, SH><<<grid, tile::kThreads, smem, st>>>(reqs, tpre, nR, ovf, ovf_count);
    return cudaGetLastError();
}

template <typename T, int C, int NDIM>
cudaError_t launch_tile_queue(int shape, const TileArgs* reqs, const int64_t* tpre, const int* nR, int64_t* ovf,
                              unsigned* ovf_count, int grid, cudaStream_t st)
{
    // the batched queue stages with plain loads: a TMA-staged index runs its base shape
    return with_shape<NDIM>(shape % num_base_shapes(NDIM), [&](auto sh) {
        return launch_queue_shape<T, C, decltype(sh)>(reqs, tpre, nR, ovf, ovf_count, grid, st);
    });
}

}  // namespace sslic

// explicit instantiation of both launchers for one image type
#define SSLIC_TILE_INSTANTIATE(T, C, NDIM)                                                                  \
    template int sslic::launch_tile_impl<T, C, NDIM>(sslic_ctx*, const T*, int32_t*, cudaStream_t,         \
                                                     const sslic::Slab*);                                   \
    template cudaError_t sslic::launch_tile_queue<T, C, NDIM>(int, const sslic::TileArgs*, const int64_t*, \
                                                              const int*, int64_t*, unsigned*, int, cudaStream_t);
