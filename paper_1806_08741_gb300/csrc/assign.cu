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
// The paper splits the image into regions and loops each region over the
// centres that reach it.  Here a CTA owns a tile of voxels; it gathers the
// centres of the 3^n-neighbouring bins, keeps those whose window meets the
// tile, sorts them by index, and builds per-centre, per-axis tables of t_d
// for the tile's coordinates (the window test becomes a +inf entry).  Each
// warp then walks the centres that meet its 4x4x4 (3-D) or 8x8 (2-D) box,
// two voxels per lane in packed f32x2 arithmetic.  The winners' slots go to
// shared memory, from where the CTA writes the int32 labels with coalesced
// stores and accumulates [I(x), x, 1] per label along runs of each row,
// flushing per-tile sums to global uint64 sums (exact, order independent).
#include <cstdio>

#include "common.cuh"

namespace sslic {

constexpr float kInf = __builtin_huge_valf();

// ---------------------------------------------------------------------------
// tile kernel configuration
// ---------------------------------------------------------------------------
template <int NDIM>
struct TileCfg;
template <>
struct TileCfg<3> {
    static constexpr int TX = 32, TY = 8, TZ = 8;  // 2048 voxels
    static constexpr int WX = 2, WY = 4, WZ = 4;   // lanes: 2 pairs x 4 x 4 -> box 4x4x4
};
template <>
struct TileCfg<2> {
    static constexpr int TX = 64, TY = 32, TZ = 1;  // 2048 pixels
    static constexpr int WX = 4, WY = 8, WZ = 1;    // box 8x8
};

constexpr int kTileThreads = 128;
constexpr int kCap = 64;        // candidate centres per tile (slot fits a byte)
constexpr int kStage = 512;     // gathered centres before filtering

template <typename T, int C, int NDIM>
struct TileSmem {
    using Cfg = TileCfg<NDIM>;
    static constexpr int TX = Cfg::TX, TY = Cfg::TY, TZ = Cfg::TZ;
    static constexpr int TV = TX * TY * TZ;
    float tab0[kCap][TX];            // t_0 by local x
    float2 tab1[kCap][TY];           // (t_1, t_1) by local y
    float2 tab2[kCap][TZ];           // (t_2, t_2) by local z
    float2 fe[kCap][C];              // (C_c, C_c)
    int cand[kCap];                  // sorted cluster indices
    int tmp[kCap];
    int stage[kStage];
    uint32_t bmask[kCap];            // which warp boxes each centre reaches
    unsigned accs[kCap][C + 4];      // per-tile sums: features, x, y, z, count
    alignas(16) T img[TV * C];
    uint8_t slot[TV];
    int nstage, ncand;
};

template <typename T>
__device__ __forceinline__ float to_f(T v) { return (float)v; }

// t_d table entry: w_d * (x - c)^2 with one rounding per op, +inf outside
__device__ __forceinline__ float tab_entry(int64_t x, float c, int64_t lo, int S, float w)
{
    if (x < lo || x > lo + 2 * S - 1) return kInf;
    float dl = __fsub_rn((float)x, c);
    return __fmul_rn(w, __fmul_rn(dl, dl));
}

template <typename T, int C, int NDIM>
__global__ void __launch_bounds__(kTileThreads, 6)
assign_tile_kernel(Geom g, const T* __restrict__ img, const float* __restrict__ ctr,
                   const unsigned* __restrict__ bin_start, const int* __restrict__ bin_items,
                   int32_t* __restrict__ labels, unsigned long long* __restrict__ acc,
                   int64_t* __restrict__ ovf_tiles, unsigned* __restrict__ ovf_count,
                   int64_t ntx, int64_t nty)
{
    using Cfg = TileCfg<NDIM>;
    constexpr int TX = Cfg::TX, TY = Cfg::TY, TZ = Cfg::TZ, TV = TX * TY * TZ;
    constexpr int WX = Cfg::WX, WY = Cfg::WY, WZ = Cfg::WZ;
    constexpr int BX = 2 * WX, BY = WY, BZ = WZ;             // warp box in voxels
    constexpr int NBX = TX / BX, NBY = TY / BY, NBZ = TZ / BZ;
    constexpr int NBOX = NBX * NBY * NBZ;
    constexpr int NWARP = kTileThreads / 32;
    constexpr int PASSES = NBOX / NWARP;
    static_assert(NBOX % NWARP == 0, "boxes per warp");
    static_assert(NBX + NBY + NBZ <= 32, "box mask bits");
    constexpr int AW = C + 4;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<T, C, NDIM>& s = *reinterpret_cast<TileSmem<T, C, NDIM>*>(smem_raw);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tile = blockIdx.x;
    const int64_t X0 = (tile % ntx) * TX;
    const int64_t Y0 = ((tile / ntx) % nty) * TY;
    const int64_t Z0 = (tile / (ntx * nty)) * TZ;
    const int ex = (int)imin64(TX, g.N[0] - X0);
    const int ey = (int)imin64(TY, g.N[1] - Y0);
    const int ez = (int)imin64(TZ, g.N[2] - Z0);

    if (tid == 0) { s.nstage = 0; s.ncand = 0; }
    for (int i = tid; i < kCap * AW; i += kTileThreads) (&s.accs[0][0])[i] = 0u;

    // ---- stage the image tile in shared memory ----------------------------
    {
        constexpr int RB = TX * C * (int)sizeof(T);  // bytes per full tile row
        const bool full = (ex == TX);
        const int64_t pitch = g.N[0] * C * (int64_t)sizeof(T);
        const char* gbase = (const char*)img;
        char* sbase = (char*)s.img;
        if (full && (pitch % 16 == 0) && (RB % 16 == 0) && (((uintptr_t)img & 15) == 0)) {
            constexpr int W = RB / 16;
            for (int i = tid; i < TY * TZ * W; i += kTileThreads) {
                int r = i / W, wi = i % W;
                int yl = r % TY, zl = r / TY;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (yl < ey && zl < ez) {
                    int64_t off = vidx(g, X0, Y0 + yl, Z0 + zl) * C * (int64_t)sizeof(T) + wi * 16;
                    v = __ldg(reinterpret_cast<const uint4*>(gbase + off));
                }
                reinterpret_cast<uint4*>(sbase + r * RB)[wi] = v;
            }
        } else {
            for (int i = tid; i < TV * C; i += kTileThreads) {
                int e = i / C, c = i % C;
                int xl = e % TX, yl = (e / TX) % TY, zl = e / (TX * TY);
                T v = T(0);
                if (xl < ex && yl < ey && zl < ez) v = img[vidx(g, X0 + xl, Y0 + yl, Z0 + zl) * C + c];
                s.img[i] = v;
            }
        }
    }
    __syncthreads();

    // ---- gather the centres of the neighbouring bins ----------------------
    int64_t blo[3], bhi[3], T0[3] = {X0, Y0, Z0};
    const int64_t E[3] = {ex, ey, ez};
    for (int d = 0; d < 3; ++d) {
        blo[d] = imax64(0, T0[d] / g.S[d] - 1);
        bhi[d] = imin64(g.nb[d] - 1, (T0[d] + E[d] - 1) / g.S[d] + 1);
    }
    const int64_t nbx = bhi[0] - blo[0] + 1, nby = bhi[1] - blo[1] + 1, nbz = bhi[2] - blo[2] + 1;
    const int64_t nbins = nbx * nby * nbz;
    for (int64_t b = tid; b < nbins; b += kTileThreads) {
        int64_t bx = blo[0] + b % nbx, by = blo[1] + (b / nbx) % nby, bz = blo[2] + b / (nbx * nby);
        int64_t bin = bx + g.nb[0] * (by + g.nb[1] * bz);
        unsigned st = bin_start[bin], en = bin_start[bin + 1];
        for (unsigned i = st; i < en; ++i) {
            int pos = atomicAdd(&s.nstage, 1);
            if (pos < kStage) s.stage[pos] = bin_items[i];
        }
    }
    __syncthreads();
    const int nst = s.nstage;
    // keep the centres whose window meets the tile
    for (int i = tid; i < min(nst, kStage); i += kTileThreads) {
        int k = s.stage[i];
        const float* p = ctr + (int64_t)k * g.CW + C;
        bool hit = true;
        for (int d = 0; d < NDIM; ++d) {
            int64_t lo = window_lo(p[d], g.S[d]);
            hit = hit && (lo <= T0[d] + E[d] - 1) && (lo + 2 * g.S[d] - 1 >= T0[d]);
        }
        if (hit) {
            int pos = atomicAdd(&s.ncand, 1);
            if (pos < kCap) s.tmp[pos] = k;
        }
    }
    __syncthreads();
    const int nc = s.ncand;
    if (nst > kStage || nc > kCap) {
        // too many centres reach this tile: the per-voxel kernel handles it
        if (tid == 0) {
            unsigned pos = atomicAdd(ovf_count, 1u);
            ovf_tiles[pos] = tile;
        }
        return;
    }
    // sort by cluster index (ascending k + strict "<" = lowest-index ties)
    for (int i = tid; i < nc; i += kTileThreads) {
        int k = s.tmp[i], r = 0;
        for (int j = 0; j < nc; ++j) r += (s.tmp[j] < k);
        s.cand[r] = k;
    }
    __syncthreads();

    // ---- per-centre tables ---------------------------------------------------
    for (int i = tid; i < nc * TX; i += kTileThreads) {
        int sl = i / TX, xl = i % TX;
        const float* p = ctr + (int64_t)s.cand[sl] * g.CW + C;
        s.tab0[sl][xl] = tab_entry(X0 + xl, p[0], window_lo(p[0], g.S[0]), g.S[0], g.w[0]);
    }
    if (NDIM >= 2) {
        for (int i = tid; i < nc * TY; i += kTileThreads) {
            int sl = i / TY, yl = i % TY;
            const float* p = ctr + (int64_t)s.cand[sl] * g.CW + C;
            float t = tab_entry(Y0 + yl, p[1], window_lo(p[1], g.S[1]), g.S[1], g.w[1]);
            s.tab1[sl][yl] = make_float2(t, t);
        }
    }
    if (NDIM >= 3) {
        for (int i = tid; i < nc * TZ; i += kTileThreads) {
            int sl = i / TZ, zl = i % TZ;
            const float* p = ctr + (int64_t)s.cand[sl] * g.CW + C;
            float t = tab_entry(Z0 + zl, p[2], window_lo(p[2], g.S[2]), g.S[2], g.w[2]);
            s.tab2[sl][zl] = make_float2(t, t);
        }
    }
    for (int i = tid; i < nc; i += kTileThreads) {
        const float* row = ctr + (int64_t)s.cand[i] * g.CW;
        for (int c = 0; c < C; ++c) s.fe[i][c] = make_float2(row[c], row[c]);
        // warp-box reach masks per axis
        uint32_t m = 0;
        const int NB[3] = {NBX, NBY, NBZ}, BB[3] = {BX, BY, BZ}, SH[3] = {0, NBX, NBX + NBY};
        for (int d = 0; d < 3; ++d) {
            if (d >= NDIM) { m |= 1u << SH[d]; continue; }
            int64_t lo = window_lo(row[C + d], g.S[d]), hi = lo + 2 * g.S[d] - 1;
            for (int b = 0; b < NB[d]; ++b) {
                int64_t a0 = T0[d] + b * BB[d], a1 = a0 + BB[d] - 1;
                if (lo <= a1 && hi >= a0) m |= 1u << (SH[d] + b);
            }
        }
        s.bmask[i] = m;
    }
    __syncthreads();

    // ---- assignment: warps sweep 4x4x4 (or 8x8) boxes, two voxels per lane ----
    const int lx = lane % WX, ly = (lane / WX) % WY, lz = lane / (WX * WY);
    const uint32_t bm0 = lane < nc ? s.bmask[lane] : 0u;
    const uint32_t bm1 = lane + 32 < nc ? s.bmask[lane + 32] : 0u;
#pragma unroll 1
    for (int pass = 0; pass < PASSES; ++pass) {
        const int wb = warp + pass * NWARP;
        const int bxi = wb % NBX, byi = (wb / NBX) % NBY, bzi = wb / (NBX * NBY);
        const int xl = bxi * BX + lx * 2, yl = byi * BY + ly, zl = bzi * BZ + lz;
        const int sh = bxi, shy = NBX + byi, shz = NBX + NBY + bzi;
        const uint32_t want = (1u << sh) | (1u << shy) | (1u << shz);
        uint32_t m0 = __ballot_sync(0xffffffffu, (bm0 & want) == want);
        uint32_t m1 = __ballot_sync(0xffffffffu, (bm1 & want) == want);
        // features of voxels (xl, yl, zl) and (xl + 1, yl, zl)
        const int e0 = (zl * TY + yl) * TX + xl;
        uint64_t F[C];
#pragma unroll
        for (int c = 0; c < C; ++c) F[c] = pk2(to_f(s.img[e0 * C + c]), to_f(s.img[(e0 + 1) * C + c]));
        float b0 = kInf, b1 = kInf;
        int s0 = kNoSlot, s1 = kNoSlot;
#pragma unroll 1
        for (int word = 0; word < 2; ++word) {
            uint32_t m = word ? m1 : m0;
            while (m) {
                const int sl = __ffs(m) - 1 + 32 * word;
                m &= m - 1;
                uint64_t dc;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    uint64_t cc = *reinterpret_cast<const uint64_t*>(&s.fe[sl][c]);
                    uint64_t e = sub2(F[c], cc);
                    uint64_t sq = mul2(e, e);
                    dc = c == 0 ? sq : add2(dc, sq);
                }
                uint64_t ds = *reinterpret_cast<const uint64_t*>(&s.tab0[sl][xl]);
                if (NDIM >= 2) ds = add2(ds, *reinterpret_cast<const uint64_t*>(&s.tab1[sl][yl]));
                if (NDIM >= 3) ds = add2(ds, *reinterpret_cast<const uint64_t*>(&s.tab2[sl][zl]));
                float d0, d1;
                upk2(add2(dc, ds), d0, d1);
                if (d0 < b0) { b0 = d0; s0 = sl; }
                if (d1 < b1) { b1 = d1; s1 = sl; }
            }
        }
        s.slot[e0] = (uint8_t)s0;
        s.slot[e0 + 1] = (uint8_t)s1;
    }
    __syncthreads();

    // ---- labels: coalesced int32 stores ------------------------------------
    for (int e = tid; e < TV; e += kTileThreads) {
        int xl = e % TX, yl = (e / TX) % TY, zl = e / (TX * TY);
        if (xl < ex && yl < ey && zl < ez) {
            int sl = s.slot[e];
            labels[vidx(g, X0 + xl, Y0 + yl, Z0 + zl)] = sl == kNoSlot ? -1 : s.cand[sl];
        }
    }
    // ---- map step of the update: runs along each row --------------------------
    for (int r = tid; r < TY * TZ; r += kTileThreads) {
        const int yl = r % TY, zl = r / TY;
        if (yl >= ey || zl >= ez) continue;
        const int rb = r * TX;
        int cur = s.slot[rb];
        unsigned cnt = 0, xs = 0, fs[C];
#pragma unroll
        for (int c = 0; c < C; ++c) fs[c] = 0;
        for (int xl = 0; xl <= ex; ++xl) {
            int sl = xl < ex ? (int)s.slot[rb + xl] : -2;
            if (sl != cur) {
                if (cur != kNoSlot && cnt) {
#pragma unroll
                    for (int c = 0; c < C; ++c) atomicAdd(&s.accs[cur][c], fs[c]);
                    atomicAdd(&s.accs[cur][C], xs);
                    atomicAdd(&s.accs[cur][C + 1], cnt * (unsigned)yl);
                    atomicAdd(&s.accs[cur][C + 2], cnt * (unsigned)zl);
                    atomicAdd(&s.accs[cur][C + 3], cnt);
                }
                cur = sl;
                cnt = 0; xs = 0;
#pragma unroll
                for (int c = 0; c < C; ++c) fs[c] = 0;
            }
            if (xl < ex) {
                ++cnt;
                xs += (unsigned)xl;
#pragma unroll
                for (int c = 0; c < C; ++c) fs[c] += (unsigned)s.img[(rb + xl) * C + c];
            }
        }
    }
    __syncthreads();
    // ---- flush per-tile sums (local coordinates shifted to global) ----------
    for (int i = tid; i < nc * AW; i += kTileThreads) {
        const int sl = i / AW, j = i % AW;
        const unsigned cnt = s.accs[sl][C + 3];
        if (!cnt) continue;
        unsigned long long v = s.accs[sl][j];
        if (j == C) v += (unsigned long long)cnt * (unsigned long long)X0;
        if (j == C + 1) v += (unsigned long long)cnt * (unsigned long long)Y0;
        if (j == C + 2) v += (unsigned long long)cnt * (unsigned long long)Z0;
        atomicAdd(&acc[(int64_t)s.cand[sl] * AW + j], v);
    }
}

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
                                    int64_t ntx, int64_t nty, int tx_, int ty_, int tz_)
{
    // tiles == nullptr: block b covers voxels [b * blockDim, ...) in raster order
    const int C = g.C;
    const int tv = tx_ * ty_ * tz_;
    int64_t nwork;
    if (tiles) nwork = (int64_t)(*ntiles) * tv;
    else nwork = g.V;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwork;
         w += (int64_t)gridDim.x * blockDim.x) {
        int64_t x, y, z;
        if (tiles) {
            int64_t t = tiles[w / tv];
            int e = (int)(w % tv);
            x = (t % ntx) * tx_ + e % tx_;
            y = ((t / ntx) % nty) * ty_ + (e / tx_) % ty_;
            z = (t / (ntx * nty)) * tz_ + e / (tx_ * ty_);
            if (x >= g.N[0] || y >= g.N[1] || z >= g.N[2]) continue;
        } else {
            x = w % g.N[0];
            y = (w / g.N[0]) % g.N[1];
            z = w / (g.N[0] * g.N[1]);
        }
        const int64_t q = vidx(g, x, y, z);
        const int64_t X[3] = {x, y, z};
        int64_t blo[3], bhi[3];
        for (int d = 0; d < 3; ++d) {
            blo[d] = imax64(0, X[d] / g.S[d] - 1);
            bhi[d] = imin64(g.nb[d] - 1, X[d] / g.S[d] + 1);
        }
        float best = kInf;
        int bestk = -1;
        for (int64_t bz = blo[2]; bz <= bhi[2]; ++bz)
            for (int64_t by = blo[1]; by <= bhi[1]; ++by)
                for (int64_t bx = blo[0]; bx <= bhi[0]; ++bx) {
                    int64_t bin = bx + g.nb[0] * (by + g.nb[1] * bz);
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
            atomicAdd(&a[C], (unsigned long long)x);
            atomicAdd(&a[C + 1], (unsigned long long)y);
            atomicAdd(&a[C + 2], (unsigned long long)z);
            atomicAdd(&a[C + 3], 1ull);
        }
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T, int C, int NDIM>
static int launch_tile(sslic_ctx* c, const T* img, int32_t* labels, cudaStream_t st)
{
    using Cfg = TileCfg<NDIM>;
    const Geom& g = c->g;
    Workspace& w = c->ws;
    const int64_t ntx = (g.N[0] + Cfg::TX - 1) / Cfg::TX;
    const int64_t nty = (g.N[1] + Cfg::TY - 1) / Cfg::TY;
    const int64_t ntz = (g.N[2] + Cfg::TZ - 1) / Cfg::TZ;
    const int64_t ntiles = ntx * nty * ntz;
    const size_t smem = sizeof(TileSmem<T, C, NDIM>);
    int rc = cuda_check(c, cudaFuncSetAttribute(assign_tile_kernel<T, C, NDIM>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                        "smem attribute");
    if (rc) return rc;
    rc = cuda_check(c, cudaMemsetAsync(w.ovf_count, 0, sizeof(unsigned), st), "memset ovf");
    if (rc) return rc;
    int pr = prof_begin(c, SSLIC_PHASE_ASSIGN, st);
    assign_tile_kernel<T, C, NDIM><<<ntiles, kTileThreads, smem, st>>>(
        g, img, w.ctr, w.bin_start, w.bin_items, labels, w.acc, w.ovf_tiles, w.ovf_count, ntx, nty);
    count_launch(c);
    prof_end(c, pr, st);
    if ((rc = cuda_check(c, cudaGetLastError(), "assign_tile_kernel"))) return rc;
    // tiles with too many reaching centres: per-voxel kernel over those tiles only
    int blocks = c->sms * 4;
    pr = prof_begin(c, SSLIC_PHASE_ASSIGN_VOXEL, st);
    assign_voxel_kernel<T><<<blocks, 256, 0, st>>>(g, img, w.ctr, w.bin_start, w.bin_items, labels, w.acc,
                                                    w.facc, w.ovf_tiles, w.ovf_count, ntx, nty, Cfg::TX,
                                                    Cfg::TY, Cfg::TZ);
    count_launch(c);
    prof_end(c, pr, st);
    return cuda_check(c, cudaGetLastError(), "assign_voxel_kernel(overflow)");
}

template <typename T>
static int launch_voxel(sslic_ctx* c, const T* img, int32_t* labels, cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    int64_t blocks = imin64((g.V + 255) / 256, (int64_t)c->sms * 16);
    const int pr = prof_begin(c, SSLIC_PHASE_ASSIGN_VOXEL, st);
    assign_voxel_kernel<T><<<blocks, 256, 0, st>>>(g, img, w.ctr, w.bin_start, w.bin_items, labels, w.acc,
                                                    w.facc, nullptr, nullptr, 1, 1, 1, 1, 1);
    count_launch(c);
    prof_end(c, pr, st);
    return cuda_check(c, cudaGetLastError(), "assign_voxel_kernel");
}

int64_t assign_num_tiles(const Geom& g)
{
    if (g.n == 3) {
        using T3 = TileCfg<3>;
        return ((g.N[0] + T3::TX - 1) / T3::TX) * ((g.N[1] + T3::TY - 1) / T3::TY) * ((g.N[2] + T3::TZ - 1) / T3::TZ);
    }
    using T2 = TileCfg<2>;
    return ((g.N[0] + T2::TX - 1) / T2::TX) * ((g.N[1] + T2::TY - 1) / T2::TY) * g.N[2];
}

int launch_assign_update(sslic_ctx* c, const void* img, int32_t* labels, cudaStream_t st)
{
    const Geom& g = c->g;
    if (g.n >= 2 && g.dtype == SSLIC_U8 && g.C == 3) {
        return g.n == 3 ? launch_tile<uint8_t, 3, 3>(c, (const uint8_t*)img, labels, st)
                        : launch_tile<uint8_t, 3, 2>(c, (const uint8_t*)img, labels, st);
    }
    if (g.n >= 2 && g.dtype == SSLIC_U8 && g.C == 1) {
        return g.n == 3 ? launch_tile<uint8_t, 1, 3>(c, (const uint8_t*)img, labels, st)
                        : launch_tile<uint8_t, 1, 2>(c, (const uint8_t*)img, labels, st);
    }
    if (g.n >= 2 && g.dtype == SSLIC_U16 && g.C == 1) {
        return g.n == 3 ? launch_tile<uint16_t, 1, 3>(c, (const uint16_t*)img, labels, st)
                        : launch_tile<uint16_t, 1, 2>(c, (const uint16_t*)img, labels, st);
    }
    switch (g.dtype) {
    case SSLIC_U8: return launch_voxel<uint8_t>(c, (const uint8_t*)img, labels, st);
    case SSLIC_U16: return launch_voxel<uint16_t>(c, (const uint16_t*)img, labels, st);
    default: return launch_voxel<float>(c, (const float*)img, labels, st);
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
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= g.K) return;
    unsigned long long* a = acc + k * g.AW;
    const unsigned long long cnt = a[g.C + 3];
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
    rk[k] = r;
    ne[k] = cnt ? 1u : 0u;
    for (int j = 0; j < g.AW; ++j) a[j] = 0ull;
    if (g.dtype == SSLIC_F32)
        for (int c = 0; c < g.C; ++c) facc[k * g.C + c] = 0.0;
}

// deterministic residual reduction: fixed-order block sums, then one block
constexpr int kRedThreads = 256;
__global__ void resid_partial_kernel(const double* __restrict__ rk, const unsigned* __restrict__ ne,
                                     int64_t K, double* __restrict__ part, unsigned* __restrict__ cpart)
{
    __shared__ double sd[kRedThreads];
    __shared__ unsigned sc[kRedThreads];
    const int64_t per = (K + gridDim.x - 1) / gridDim.x;
    const int64_t lo = blockIdx.x * per, hi = imin64(K, lo + per);
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
    if (threadIdx.x == 0) { part[blockIdx.x] = sd[0]; cpart[blockIdx.x] = sc[0]; }
}

__global__ void resid_final_kernel(const double* __restrict__ part, const unsigned* __restrict__ cpart,
                                   int nparts, double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double d = 0.0;
    unsigned long long cnt = 0;
    for (int i = 0; i < nparts; ++i) { d += part[i]; cnt += cpart[i]; }
    out[0] = cnt ? d / (double)cnt : 0.0;
}

constexpr int kResidParts = 256;

int launch_finalize(sslic_ctx* c, cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    int threads = 256;
    int64_t blocks = (g.K + threads - 1) / threads;
    const int pr = prof_begin(c, SSLIC_PHASE_FINALIZE, st);
    finalize_kernel<<<blocks, threads, 0, st>>>(g, w.ctr, w.acc, w.facc, w.resid_k, w.nonempty_k);
    count_launch(c, 3);
    int rc = cuda_check(c, cudaGetLastError(), "finalize_kernel");
    if (rc) return rc;
    resid_partial_kernel<<<kResidParts, kRedThreads, 0, st>>>(w.resid_k, w.nonempty_k, g.K, w.resid_part,
                                                              w.resid_cnt_part);
    if ((rc = cuda_check(c, cudaGetLastError(), "resid_partial_kernel"))) return rc;
    resid_final_kernel<<<1, 32, 0, st>>>(w.resid_part, w.resid_cnt_part, kResidParts, w.resid_out);
    prof_end(c, pr, st);
    return cuda_check(c, cudaGetLastError(), "resid_final_kernel");
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
