// ccl.cu -- connectivity enforcement (Sec. 3.1, stage 3).
//
// The paper marks, for every centre, the connected component of its label
// that contains the centre (or the label found in the S-box around it) as
// final when it is larger than S^n/4, then walks the image in raster order:
// each component that is not final gets a new label when large, otherwise
// the label last encountered, and becomes final.  Readings used here: face
// adjacency; seed = round-half-up(C_k) clamped, else the raster-first voxel of
// label k in the box of offsets -floor(S_d/2)..ceil(S_d/2)-1; flood fills see
// the labels before any relabelling; "last encountered" = the output label
// of x - e_d for the smallest d with x_d > 0, where x is the raster-first
// voxel of the component (the origin's component gets a new label); new
// labels count up from K in raster order of the components' first voxels.
//
// Parallel form, equal to that sequential walk:
//  1. ccl_local: per tile (2048 voxels), union-find in shared memory over
//     the row runs with atomicMin linking; local roots are the
//     tile-raster-first voxels and get dense local ids (uint16 per voxel)
//     and global record ids (tile base + local id) with label, size and
//     first voxel (left where the root statistics will be collected).
//  2. ccl_faces: union of the records across tile faces (global union-find).
//  3. flatten, with the root statistics: component size = sum, first voxel = min.
//  4. phase 1 (per centre) sets the final flag of its component.
//  5. phase 2 (per component): final -> own label; large or at the origin ->
//     new, ranked by first voxel (sort); otherwise a link to the component
//     holding x - e_d, whose first voxel is strictly smaller, so the links
//     form a forest rooted at resolved components; each pending component
//     walks its links to a resolved one.
//  6. relabel every voxel through its record.
#include <climits>
#include <vector>

#include "common.cuh"

namespace sslic {

template <int NDIM>
struct CclCfg;
template <>
struct CclCfg<3> { static constexpr int TX = 32, TY = 8, TZ = 8; };
template <>
struct CclCfg<2> { static constexpr int TX = 32, TY = 64, TZ = 1; };
template <>
struct CclCfg<1> { static constexpr int TX = 2048, TY = 1, TZ = 1; };
// 4-D: a tile is a 32x8x8 block of one slice along the fourth axis; the
// tile-local pass is the 3-D one and the slice below adds a fourth face
template <>
struct CclCfg<4> { static constexpr int TX = 32, TY = 8, TZ = 8; };

constexpr int kCclThreads = 256;
constexpr int kCclTV = 2048;

// ---- union-find with atomicMin linking (parents only ever decrease) --------
// Parent indices strictly decrease along every chain, so walks end within
// the number of nodes.  The walks over the global records are still bounded
// and report a broken invariant through *err instead of spinning; the
// tile-local walks further below mask their indices into the tile instead.
constexpr int kWalkLimit = 1 << 26;

// Every global walk checks its index against the forest's size n and gives
// up (flag 2) instead of leaving it.
__device__ __forceinline__ bool uf_bad(int x, int n, unsigned* err)
{
    if (x >= 0 && x < n) return false;
    atomicExch(err, 2u);
    return true;
}

__device__ __forceinline__ int uf_find(int* par, int x, int n, unsigned* err)
{
    // path halving: every write points a node at one of its ancestors, which
    // is in the same set and has a smaller index, so concurrent finds and
    // links keep the forest acyclic
    volatile int* vp = par;
    for (int i = 0; i < kWalkLimit; ++i) {
        if (uf_bad(x, n, err)) return -1;
        const int p = vp[x];
        if (p == x) return x;
        if (uf_bad(p, n, err)) return -1;
        const int gp = vp[p];
        if (gp == p) return p;
        vp[x] = gp;
        x = gp;
    }
    atomicExch(err, 1u);
    return -1;
}

// read-only walk to the root, for the compress / flatten passes: those run
// after every union has finished, and a halving write landing after another
// thread's final "parent = root" store would leave a non-root parent behind
__device__ __forceinline__ int uf_root(const int* par, int x, int n, unsigned* err)
{
    const volatile int* vp = par;
    for (int i = 0; i < kWalkLimit; ++i) {
        if (uf_bad(x, n, err)) return -1;
        const int p = vp[x];
        if (p == x) return x;
        x = p;
    }
    atomicExch(err, 1u);
    return -1;
}

__device__ __noinline__ void uf_unite(int* par, int a, int b, int n, unsigned* err)
{
    a = uf_find(par, a, n, err);
    b = uf_find(par, b, n, err);
    for (int i = 0; i < kWalkLimit && a != b; ++i) {
        if (a < 0 || b < 0) return;  // flagged
        if (a < b) { int t = a; a = b; b = t; }
        const int old = atomicMin(&par[a], b);
        if (old == a) return;       // a was a root and now hangs under b
        a = uf_find(par, old, n, err); // a had been re-linked meanwhile: retry from its root
        b = uf_find(par, b, n, err);
    }
    if (a != b) atomicExch(err, 1u);
}

// A tile's forest in shared memory: indices are masked into the tile, so no
// walk can leave the array, and since parents strictly decrease along a
// chain a walk ends within kCclTV steps (a broken invariant shows up as a
// root that is not a root, which the kernel checks and reports).
constexpr int kTileMask = kCclTV - 1;
static_assert((kCclTV & kTileMask) == 0, "the tile size is a power of two");

__device__ __forceinline__ int uf_find_tile(int* par, int x)
{
    volatile int* vp = par;
    x &= kTileMask;
    for (int i = 0; i < kCclTV; ++i) {
        const int p = vp[x] & kTileMask;
        if (p == x) break;
        const int gp = vp[p] & kTileMask;
        if (gp == p) return p;
        vp[x] = gp;  // path halving
        x = gp;
    }
    return x;
}

__device__ __forceinline__ int uf_root_tile(const int* par, int x)
{
    const volatile int* vp = par;
    x &= kTileMask;
    for (int i = 0; i < kCclTV; ++i) {
        const int p = vp[x] & kTileMask;
        if (p == x) break;
        x = p;
    }
    return x;
}

// The same union for a tile's forest, inlined so the walks and the link use
// shared-memory instructions
__device__ __forceinline__ void uf_unite_local(int* par, int a, int b, unsigned* err)
{
    a = uf_find_tile(par, a);
    b = uf_find_tile(par, b);
    for (int i = 0; i < kCclTV && a != b; ++i) {
        if (a < b) { int t = a; a = b; b = t; }
        const int old = atomicMin(&par[a], b);
        if (old == a) return;
        a = uf_find_tile(par, old);
        b = uf_find_tile(par, b);
    }
    if (a != b) atomicExch(err, 1u);
}

// First voxels of components are kept as packed coordinates: x in the low
// bits, then y, z and the fourth axis, each in ceil(log2 N_d) bits.  Packed
// keys compare exactly as raster indices (dimension 0 fastest) do, so the
// minimum over a component and the ranking of new labels are unchanged, and
// unpacking takes shifts and masks instead of 64-bit divisions.
struct RasterKey {
    int sh[kMaxDims];
    unsigned long long mask[kMaxDims];
};

static bool make_raster_key(const Geom& g, RasterKey& k)
{
    int s = 0;
    for (int d = 0; d < kMaxDims; ++d) {
        int b = 0;
        while (((int64_t)1 << b) < g.N[d]) ++b;
        k.sh[d] = s;
        k.mask[d] = ((unsigned long long)1 << b) - 1ull;
        s += b;
    }
    return s <= 63;
}

__device__ __forceinline__ unsigned long long raster_pack(const RasterKey& k, int64_t x, int64_t y, int64_t z,
                                                          int64_t w)
{
    return (unsigned long long)x << k.sh[0] | (unsigned long long)y << k.sh[1] | (unsigned long long)z << k.sh[2] |
           (unsigned long long)w << k.sh[3];
}

template <int NDIM>
__device__ __forceinline__ int64_t ccl_tile_of(const Geom& g, int64_t x, int64_t y, int64_t z, int64_t w, int64_t ntx,
                                               int64_t nty, int64_t ntz)
{
    using Cfg = CclCfg<NDIM>;
    return x / Cfg::TX + ntx * (y / Cfg::TY + nty * (z / Cfg::TZ + ntz * w));
}

// origin of tile t (the fourth coordinate is 0 below 4-D)
template <int NDIM>
__device__ __forceinline__ void ccl_tile_origin(int64_t t, int64_t ntx, int64_t nty, int64_t ntz, int64_t& X0,
                                                int64_t& Y0, int64_t& Z0, int64_t& W0)
{
    using Cfg = CclCfg<NDIM>;
    X0 = (t % ntx) * Cfg::TX;
    Y0 = ((t / ntx) % nty) * Cfg::TY;
    Z0 = ((t / (ntx * nty)) % ntz) * Cfg::TZ;
    W0 = t / (ntx * nty * ntz);
}

// Tile-local components.  The tile is handled as 64 rows of 32 voxels (one
// row = one warp instruction, lane = x; in 1-D a row is a 32-voxel chunk and
// consecutive chunks touch):
//  A. runs of equal labels along a row come from one ballot; every voxel's
//     parent is the first voxel of its run;
//  B. each run is united with the runs it touches in the previous row along
//     y and along z -- once per pair of touching runs, at the first voxel of
//     the overlap;
//  C. every voxel resolves its root (read-only walks after the unions);
//  D. roots (the tile-raster-first voxel of each local component) are ranked
//     by ballots and a scan over the rows;
//  E. local ids go out per voxel, component sizes are summed per run.
template <int NDIM>
__global__ void __launch_bounds__(kCclThreads)
ccl_local_kernel(Geom g, const int32_t* __restrict__ labels, uint16_t* __restrict__ lid_img,
                 int* __restrict__ tile_base, int* __restrict__ tile_cnt, int* __restrict__ comp_label,
                 unsigned long long* __restrict__ root_size, unsigned long long* __restrict__ root_first,
                 uint8_t* __restrict__ fin, int* __restrict__ gparent,
                 unsigned* __restrict__ counters, int64_t m_cap, RasterKey rk, int64_t ntx, int64_t nty, int64_t ntz,
                 int64_t tile0)
{
    using Cfg = CclCfg<NDIM>;
    constexpr int TX = Cfg::TX, TY = Cfg::TY, TZ = Cfg::TZ;
    constexpr int kRows = kCclTV / 32, kWarpsL = kCclThreads / 32, RPW = kRows / kWarpsL;
    static_assert(TX * TY * TZ == kCclTV, "tile size");
    static_assert(NDIM == 1 || TX == 32, "a row is the tile's extent along x");
    __shared__ int lab[kCclTV];
    __shared__ int par[kCclTV];
    __shared__ uint16_t lidv[kCclTV];
    __shared__ unsigned sz[kCclTV];
    __shared__ unsigned rowoff[kRows];
    __shared__ unsigned rhead[kRows];  // per row: lanes that start a run (of any label)
    __shared__ unsigned vhead[kRows];  // ... and start a run of a voxel inside the image
    __shared__ unsigned rroot[kRows];  // ... and are the root of their local component
    __shared__ unsigned s_total;
    __shared__ int s_base;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tile = tile0 + blockIdx.x;
    int64_t X0, Y0, Z0, W0;
    ccl_tile_origin<NDIM>(tile, ntx, nty, ntz, X0, Y0, Z0, W0);
    const int ex = (int)imin64(TX, g.N[0] - X0);
    const int ey = (int)imin64(TY, g.N[1] - Y0);
    const int ez = (int)imin64(TZ, g.N[2] - Z0);
    const unsigned lt = (1u << lane) - 1u;
    unsigned* err = &counters[3];
    // voxel index of tile element e: the tile origin plus in-tile offsets
    const int64_t p0 = vidx(g, X0, Y0, Z0, W0), sy = g.N[0], sxy = g.N[0] * g.N[1];
    auto vox = [&](int e) -> int64_t {
        return p0 + e % TX + (int64_t)((e / TX) % TY) * sy + (int64_t)(e / (TX * TY)) * sxy;
    };

    // A. labels in (all of the warp's rows in flight at once), run heads
    int Lr[RPW];
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
        const int e = (warp * RPW + i) * 32 + lane;
        const int xl = e % TX, yl = (e / TX) % TY, zl = e / (TX * TY);
        const bool v = xl < ex && yl < ey && zl < ez;
        Lr[i] = v ? labels[vox(e)] : INT_MIN;
    }
#pragma unroll
    for (int i = 0; i < RPW; ++i) {
        const int e = (warp * RPW + i) * 32 + lane;
        const int L = Lr[i];
        const int Lp = __shfl_up_sync(0xffffffffu, L, 1);
        const unsigned m = __ballot_sync(0xffffffffu, lane == 0 || L != Lp);
        const unsigned vm = __ballot_sync(0xffffffffu, L != INT_MIN);
        lab[e] = L;
        if (lane == 0) {
            rhead[warp * RPW + i] = m;
            vhead[warp * RPW + i] = m & vm;
        }
        const int head = 31 - __clz(m & (lt | (1u << lane)));
        par[e] = L == INT_MIN ? -1 : (e - lane + head);
    }
    __syncwarp();
    // B1. unions with the previous row inside the warp's own rows (a z-plane
    //     in 3-D, 8 consecutive rows in 2-D), so that B2 may rely on them.  A
    //     pair of touching runs is united where its overlap starts: the voxel
    //     matches the one below and either the voxel before it does not, or
    //     it starts a new run.  The warp first lists the pairs of all its rows
    //     (in the sizes array, not yet in use), then unites them one per lane,
    //     so few lanes idle while the walks run.
    if constexpr (NDIM == 1) {
#pragma unroll 1
        for (int i = 1; i < RPW; ++i) {
            const int e = (warp * RPW + i) * 32 + lane;
            if (lane == 0 && lab[e] != INT_MIN && lab[e - 1] == lab[e]) uf_unite_local(par, e, e - 1, err);
        }
    } else {
        unsigned* pl = sz + warp * (RPW * 32);  // packed pairs (a << 16 | b), a, b < 2048
        int np = 0;
#pragma unroll 1
        for (int i = 1; i < RPW; ++i) {
            const int e = (warp * RPW + i) * 32 + lane;
            const int L = lab[e];
            const int yl = (e / TX) % TY;
            const unsigned starts = rhead[warp * RPW + i];
            const unsigned my = __ballot_sync(0xffffffffu, yl > 0 && L != INT_MIN && lab[e - TX] == L);
            const unsigned want = my & (starts | ~(my << 1));
            if (want >> lane & 1u) pl[np + __popc(want & lt)] = ((unsigned)e << 16) | (unsigned)(e - TX);
            np += __popc(want);
        }
        __syncwarp();
        for (int j = lane; j < np; j += 32) uf_unite_local(par, (int)(pl[j] >> 16), (int)(pl[j] & 0xffffu), err);
    }
    __syncthreads();
    // B2. unions across warps (atomic linking): along z in 3-D, along y at
    //     the first row of each warp in 2-D, along x between the warps' chunks
    //     in 1-D.  A z-pair is skipped when the row before it has the same two
    //     labels across the same faces (that path is already united).
    if (NDIM == 1) {
        const int e = warp * RPW * 32;
        if (lane == 0 && e > 0 && lab[e] != INT_MIN && lab[e - 1] == lab[e]) uf_unite_local(par, e, e - 1, err);
    } else if (NDIM == 2) {
        const int e = warp * RPW * 32 + lane;
        const int L = lab[e];
        const int yl = (e / TX) % TY;
        const unsigned starts = __ballot_sync(0xffffffffu, lane == 0 || L != lab[e - (lane > 0)]);
        const unsigned my = __ballot_sync(0xffffffffu, yl > 0 && L != INT_MIN && lab[e - TX] == L);
        if ((my & (starts | ~(my << 1))) >> lane & 1u) uf_unite_local(par, e, e - TX, err);
    } else {
        constexpr int P = TX * TY;
        unsigned* pl = sz + warp * (RPW * 32);  // listed as in B1, then united one per lane
        int np = 0;
#pragma unroll 1
        for (int i = 0; i < RPW; ++i) {
            const int e = (warp * RPW + i) * 32 + lane;
            const int L = lab[e];
            const int yl = (e / TX) % TY, zl = e / P;
            const unsigned starts = rhead[warp * RPW + i];
            const bool zm = zl > 0 && L != INT_MIN && lab[e - P] == L;
            const bool via_y = zm && yl > 0 && lab[e - TX] == L && lab[e - TX - P] == L;
            const unsigned mz = __ballot_sync(0xffffffffu, zm);
            const unsigned want = mz & (starts | ~(mz << 1)) & ~__ballot_sync(0xffffffffu, via_y);
            if (want >> lane & 1u) pl[np + __popc(want & lt)] = ((unsigned)e << 16) | (unsigned)(e - P);
            np += __popc(want);
        }
        __syncwarp();
        for (int j = lane; j < np; j += 32) uf_unite_local(par, (int)(pl[j] >> 16), (int)(pl[j] & 0xffffu), err);
    }
    __syncthreads();
    // C. roots: every run head (the first voxel of a run; path halving may
    //    have moved its parent) finds its root and compresses its path to
    //    it -- no unions run any more, so every store writes a final root.
    //    Every parent pointer names a run head, so afterwards any voxel's
    //    root is par[par[e]].
    //    The warp lists the heads of all its rows (in the local-id array,
    //    not yet in use) and walks them one per lane.
    {
        uint16_t* hl = lidv + warp * (RPW * 32);
        int nh = 0;
#pragma unroll 1
        for (int i = 0; i < RPW; ++i) {
            const int e = (warp * RPW + i) * 32 + lane;
            sz[e] = 0u;  // the pair lists are consumed
            const unsigned hm = vhead[warp * RPW + i];
            if (hm >> lane & 1u) hl[nh + __popc(hm & lt)] = (uint16_t)e;
            nh += __popc(hm);
        }
        __syncwarp();
        for (int j = lane; j < nh; j += 32) {
            const int e = hl[j];
            const int r = uf_root_tile(par, e);
            for (int x = e, n = 0; x != r && n < kCclTV; ++n) {
                const int nx = par[x] & kTileMask;
                par[x] = r;
                x = nx;
            }
        }
    }
    __syncthreads();
    // Every voxel's parent becomes its root (-1 where the invariant broke,
    // which is reported): a concurrent reader of par[h] sees the root either
    // way.  The roots of each row are counted and their lanes kept.
    unsigned cnt_row = 0;  // lane i < RPW: roots in row warp * RPW + i
#pragma unroll 1
    for (int i = 0; i < RPW; ++i) {
        const int e = (warp * RPW + i) * 32 + lane;
        const int h = par[e];
        int r = h < 0 ? -1 : par[h];
        if (r >= 0 && par[r] != r) { atomicExch(err, 1u); r = -1; }  // broken invariant: never used as an index
        if (r != h) par[e] = r;
        const unsigned rm = __ballot_sync(0xffffffffu, r == e);
        if (lane == 0) rroot[warp * RPW + i] = rm;
        if (lane == i) cnt_row = __popc(rm);
    }
    // D. rank the roots (raster order = row order, then lane order)
    if (lane < RPW) rowoff[warp * RPW + lane] = cnt_row;
    __syncthreads();
    if (warp == 0) {
        static_assert(kRows == 64, "two rows per lane");
        const unsigned a0 = rowoff[2 * lane], a1 = rowoff[2 * lane + 1];
        unsigned incl = a0 + a1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const unsigned excl = incl - a0 - a1;
        rowoff[2 * lane] = excl;
        rowoff[2 * lane + 1] = excl + a0;
        if (lane == 31) {
            s_total = incl;
            const unsigned base = atomicAdd(&counters[0], incl);
            if ((int64_t)base + incl > m_cap) atomicExch(&counters[1], 1u);
            s_base = (int)base;
        }
    }
    __syncthreads();
    const unsigned total = s_total;
    const int base = s_base;
    if ((int64_t)base + total > m_cap) return;  // host grows the records and reruns
#pragma unroll 1
    for (int i = 0; i < RPW; ++i) {
        const int e = (warp * RPW + i) * 32 + lane;
        const unsigned rm = rroot[warp * RPW + i];
        if (rm >> lane & 1u) lidv[e] = (uint16_t)(rowoff[warp * RPW + i] + __popc(rm & lt));
    }
    __syncthreads();
    // E. local ids out; sizes per run
#pragma unroll 1
    for (int i = 0; i < RPW; ++i) {
        const int e = (warp * RPW + i) * 32 + lane;
        const int r = par[e];
        const unsigned hm = rhead[warp * RPW + i];  // first voxels of runs (of any label)
        const bool head = hm >> lane & 1u;
        if (r >= 0) {
            const uint16_t l = lidv[r];
            lid_img[vox(e)] = l;
            if (head) {
                const unsigned later = hm & ~(lt | (1u << lane));
                const int len = (later ? __ffs(later) - 1 : 32) - lane;
                atomicAdd(&sz[l], (unsigned)len);
            }
        }
    }
    __syncthreads();
    for (int e = tid; e < kCclTV; e += kCclThreads) {
        if (par[e] != e) continue;
        const int r = base + lidv[e];
        const int xl = e % TX, yl = (e / TX) % TY, zl = e / (TX * TY);
        comp_label[r] = lab[e];
        root_size[r] = sz[lidv[e]];
        root_first[r] = raster_pack(rk, X0 + xl, Y0 + yl, Z0 + zl, W0);
        fin[r] = 0;
        gparent[r] = r;
    }
    if (tid == 0) {
        tile_base[tile] = base;
        tile_cnt[tile] = (int)total;
    }
}

template <int NDIM>
__device__ __forceinline__ int gid_of(const Geom& g, const uint16_t* lid_img, const int* tile_base, int64_t x,
                                      int64_t y, int64_t z, int64_t w, int64_t ntx, int64_t nty, int64_t ntz)
{
    return tile_base[ccl_tile_of<NDIM>(g, x, y, z, w, ntx, nty, ntz)] + (int)lid_img[vidx(g, x, y, z, w)];
}

// Union across the low faces of every tile.  Each face pixel whose label
// equals that of its neighbour across the face names a pair of component
// records; a pixel whose predecessor along the face's longer axis has the
// same two labels names the same pair and is skipped, and the remaining
// pairs are deduplicated in a shared hash set, so each distinct pair of
// records is united once per tile.
// The set holds every key a tile can produce: at most 576 face pixels in
// 2-D / 3-D; in 4-D another 2048 for the slice below.
template <int NDIM>
struct FaceHash {
    static constexpr int kSize = NDIM == 4 ? 4096 : 2048;
    static constexpr int kShift = NDIM == 4 ? 20 : 21;  // 32 - log2(kSize)
    static constexpr int kPairs = NDIM == 4 ? 2624 : 576;  // face pixels of a tile, at most
};

template <int NDIM>
__global__ void __launch_bounds__(kCclThreads)
ccl_faces_kernel(Geom g, const int32_t* __restrict__ labels, const uint16_t* __restrict__ lid_img,
                 const int* __restrict__ tile_base, int* gparent, unsigned* counters, int64_t ntx,
                 int64_t nty, int64_t ntz, int64_t tile0, const int32_t* __restrict__ carry, int64_t qlo,
                 int64_t cbase)
{
    // labels of voxels before qlo (the planes below a slab, see the slab form)
    // come from the carried planes, indexed from voxel cbase
    auto lab_at = [&](int64_t q) -> int { return q < qlo ? carry[q - cbase] : labels[q]; };
    using Cfg = CclCfg<NDIM>;
    constexpr int TX = Cfg::TX, TY = Cfg::TY, TZ = Cfg::TZ;
    constexpr int HS = FaceHash<NDIM>::kSize;
    __shared__ unsigned hset[HS];
    __shared__ int2 plist[FaceHash<NDIM>::kPairs];  // the distinct pairs, united after the scan
    __shared__ unsigned npairs;
    const int64_t tile = tile0 + blockIdx.x;
    int64_t X0, Y0, Z0, W0;
    ccl_tile_origin<NDIM>(tile, ntx, nty, ntz, X0, Y0, Z0, W0);
    const int EX = (int)imin64(TX, g.N[0] - X0), EY = (int)imin64(TY, g.N[1] - Y0), EZ = (int)imin64(TZ, g.N[2] - Z0);
    for (int i = threadIdx.x; i < HS; i += kCclThreads) hset[i] = 0u;
    if (threadIdx.x == 0) npairs = 0u;
    __syncthreads();
    const int base_here = tile_base[tile];
    const int64_t sy = g.N[0], sz = g.N[0] * g.N[1], sw4 = sz * g.N[2];
    // the faces that exist (the tile is not on the image's low border there)
    const bool has[4] = {X0 > 0, NDIM >= 2 && Y0 > 0, NDIM >= 3 && Z0 > 0, NDIM >= 4 && W0 > 0};
    const int nf[4] = {has[0] ? EY * EZ : 0, has[1] ? EX * EZ : 0, has[2] ? EX * EY : 0, has[3] ? EX * EY * EZ : 0};
    const int n_all = nf[0] + nf[1] + nf[2] + nf[3];
    const int64_t p0 = vidx(g, X0, Y0, Z0, W0);
    // one pixel of one face per thread and step; its loads are issued together
    for (int idx = threadIdx.x; idx < n_all; idx += kCclThreads) {
        const int d = idx < nf[0] ? 0 : (idx < nf[0] + nf[1] ? 1 : (idx < nf[0] + nf[1] + nf[2] ? 2 : 3));
        const int i = idx - (d == 0 ? 0 : (d == 1 ? nf[0] : (d == 2 ? nf[0] + nf[1] : nf[0] + nf[1] + nf[2])));
        // in-face axes: u (the longer one, x except on the x face) and the rest
        const int nu = d == 0 ? EY : EX;
        const int64_t su = d == 0 ? sy : 1;
        const int64_t st = d == 0 ? 1 : (d == 1 ? sy : (d == 2 ? sz : sw4));
        const int iu = i % nu, iw = i / nu;
        int64_t rest;
        if (d == 3) rest = (iw % EY) * sy + (iw / EY) * sz;  // the slice face: (y, z) beyond u = x
        else rest = iw * (d == 2 ? sy : sz);
        const int64_t ia = p0 + iu * su + rest, ib = ia - st;
        const int64_t ja = iu > 0 ? ia - su : ia, jb = iu > 0 ? ib - su : ib;
        const int L = labels[ia], Lb = lab_at(ib), La1 = labels[ja], Lb1 = lab_at(jb);
        const unsigned la = lid_img[ia], lb = lid_img[ib];
        if (L != Lb) continue;
        if (iu > 0 && La1 == L && Lb1 == L) continue;  // same pair as the predecessor along u
        const int64_t nb = d == 0 ? tile - 1 : (d == 1 ? tile - ntx : (d == 2 ? tile - ntx * nty : tile - ntx * nty * ntz));
        const unsigned key = 1u + ((unsigned)d << 22 | la << 11 | lb);
        unsigned h = (key * 2654435761u) >> FaceHash<NDIM>::kShift;
        bool fresh = false;
        for (int probe = 0; probe < HS; ++probe) {
            const unsigned old = atomicCAS(&hset[h], 0u, key);
            if (old == 0u) { fresh = true; break; }
            if (old == key) break;
            h = (h + 1) & (HS - 1);
        }
        if (fresh) plist[atomicAdd(&npairs, 1u)] = make_int2(base_here + (int)la, tile_base[nb] + (int)lb);
    }
    // one union per thread (the scan leaves few fresh pairs per warp and step)
    __syncthreads();
    const int np = (int)npairs;
    for (int i = threadIdx.x; i < np; i += kCclThreads)
        uf_unite(gparent, plist[i].x, plist[i].y, (int)counters[0], &counters[3]);
}

// every record's parent becomes its root (read-only walks: a concurrent
// store only ever replaces a parent by the root), and every record that is
// not a root adds its own size and first voxel -- left in its root_size /
// root_first entries by the tile pass -- into its root's.  Only roots take
// atomics and roots add nothing, so no entry is read while it changes.
constexpr int kFlattenBatch = 2;
__global__ void ccl_flatten_kernel(int* gparent, unsigned long long* root_size, unsigned long long* root_first,
                                   unsigned* counters)
{
    // kFlattenBatch records a grid stride apart per thread: their parents,
    // then the non-roots' sizes and first voxels, are loaded together before
    // the walks
    const int64_t M = counters[0];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const volatile int* vp = gparent;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < M; i0 += stride * kFlattenBatch) {
        int par[kFlattenBatch];
        bool child[kFlattenBatch];
        unsigned long long cs[kFlattenBatch], cf[kFlattenBatch];
#pragma unroll
        for (int b = 0; b < kFlattenBatch; ++b) {
            const int64_t i = i0 + b * stride;
            par[b] = i < M ? vp[i] : -1;
            child[b] = i < M && par[b] != (int)i;
        }
#pragma unroll
        for (int b = 0; b < kFlattenBatch; ++b) {
            const int64_t i = i0 + b * stride;
            cs[b] = child[b] ? root_size[i] : 0ull;
            cf[b] = child[b] ? root_first[i] : 0ull;
        }
#pragma unroll
        for (int b = 0; b < kFlattenBatch; ++b) {
            if (!child[b]) continue;
            const int64_t i = i0 + b * stride;
            const int r = uf_root(gparent, par[b], (int)M, &counters[3]);
            if (r < 0) continue;  // flagged
            if (r != par[b]) gparent[i] = r;
            atomicAdd(&root_size[r], cs[b]);
            atomicMin(&root_first[r], cf[b]);
        }
    }
}

// phase 1: one component per centre, final if 4 * size > prod S
template <int NDIM>
__global__ void conn_phase1_kernel(Geom g, const float* __restrict__ ctr, const int32_t* __restrict__ labels,
                                   const uint16_t* __restrict__ lid_img, const int* __restrict__ tile_base,
                                   const int* __restrict__ gparent, const unsigned long long* __restrict__ root_size,
                                   uint8_t* __restrict__ fin, int64_t ntx, int64_t nty, int64_t ntz)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= g.K) return;
    const float* pc = ctr + k * g.CW + g.C;
    int64_t p[kMaxDims] = {0, 0, 0, 0};
    for (int d = 0; d < g.n; ++d) {
        int64_t v = (int64_t)floor((double)pc[d] + 0.5);
        p[d] = v < 0 ? 0 : (v > g.N[d] - 1 ? g.N[d] - 1 : v);
    }
    int64_t s[kMaxDims] = {-1, -1, -1, -1};
    if (labels[vidx(g, p[0], p[1], p[2], p[3])] == (int32_t)k) {
        for (int d = 0; d < kMaxDims; ++d) s[d] = p[d];
    } else {
        // the S-box around p in raster order, dimension 0 fastest
        int64_t lo[kMaxDims], hi[kMaxDims];
        for (int d = 0; d < kMaxDims; ++d) {
            lo[d] = imax64(0, p[d] - g.S[d] / 2);
            hi[d] = imin64(g.N[d] - 1, p[d] + (g.S[d] + 1) / 2 - 1);
        }
        for (int64_t w = lo[3]; w <= hi[3] && s[0] < 0; ++w)
            for (int64_t z = lo[2]; z <= hi[2] && s[0] < 0; ++z)
                for (int64_t y = lo[1]; y <= hi[1] && s[0] < 0; ++y)
                    for (int64_t x = lo[0]; x <= hi[0]; ++x)
                        if (labels[vidx(g, x, y, z, w)] == (int32_t)k) { s[0] = x; s[1] = y; s[2] = z; s[3] = w; break; }
    }
    if (s[0] < 0) return;
    const int G = gparent[gid_of<NDIM>(g, lid_img, tile_base, s[0], s[1], s[2], s[3], ntx, nty, ntz)];
    if (4ull * root_size[G] > (unsigned long long)g.sprod) fin[G] = 1;
}

// Slab form, phase 1's seed voxel: every centre whose S-box ends in the
// planes [lo, hi) of the last axis finds it here -- the voxel at its rounded
// centre when that carries its label, else the raster-first voxel of its
// label in the box (the same rule as conn_phase1_kernel).  The box spans at
// most S planes along the last axis, so the planes below lo that it reaches
// are among the carried ones (labels of voxels before qlo come from carry,
// indexed from voxel cbase).  -1: no such voxel.
template <int NDIM>
__global__ void conn_seek_kernel(Geom g, const float* __restrict__ ctr, const int32_t* __restrict__ labels,
                                 const int32_t* __restrict__ carry, int64_t qlo, int64_t cbase, int64_t lo,
                                 int64_t hi, long long* __restrict__ seed_vox)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= g.K) return;
    const int L = g.n - 1;
    const float* pc = ctr + k * g.CW + g.C;
    int64_t p[kMaxDims] = {0, 0, 0, 0};
    for (int d = 0; d < g.n; ++d) {
        int64_t v = (int64_t)floor((double)pc[d] + 0.5);
        p[d] = v < 0 ? 0 : (v > g.N[d] - 1 ? g.N[d] - 1 : v);
    }
    int64_t blo[kMaxDims], bhi[kMaxDims];
    for (int d = 0; d < kMaxDims; ++d) {
        blo[d] = imax64(0, p[d] - g.S[d] / 2);
        bhi[d] = imin64(g.N[d] - 1, p[d] + (g.S[d] + 1) / 2 - 1);
    }
    if (bhi[L] < lo || bhi[L] >= hi) return;  // another slab holds the box's last plane
    auto lab = [&](int64_t q) -> int32_t { return q < qlo ? carry[q - cbase] : labels[q]; };
    long long s = -1;
    const int64_t q0 = vidx(g, p[0], p[1], p[2], p[3]);
    if (lab(q0) == (int32_t)k) {
        s = q0;
    } else {
        for (int64_t w = blo[3]; w <= bhi[3] && s < 0; ++w)
            for (int64_t z = blo[2]; z <= bhi[2] && s < 0; ++z)
                for (int64_t y = blo[1]; y <= bhi[1] && s < 0; ++y)
                    for (int64_t x = blo[0]; x <= bhi[0]; ++x) {
                        const int64_t q = vidx(g, x, y, z, w);
                        if (lab(q) == (int32_t)k) { s = q; break; }
                    }
    }
    seed_vox[k] = s;
}

// Slab form, phase 1 proper: the component through each centre's seed voxel
// is final if 4 * size > prod S (after every slab's records are united)
template <int NDIM>
__global__ void conn_phase1_seeded_kernel(Geom g, const long long* __restrict__ seed_vox,
                                          const uint16_t* __restrict__ lid_img, const int* __restrict__ tile_base,
                                          const int* __restrict__ gparent,
                                          const unsigned long long* __restrict__ root_size, uint8_t* __restrict__ fin,
                                          int64_t ntx, int64_t nty, int64_t ntz)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= g.K) return;
    const long long s = seed_vox[k];
    if (s < 0) return;
    const int64_t x = s % g.N[0], y = (s / g.N[0]) % g.N[1], z = (s / (g.N[0] * g.N[1])) % g.N[2],
                  w = s / (g.N[0] * g.N[1] * g.N[2]);
    const int G = gparent[gid_of<NDIM>(g, lid_img, tile_base, x, y, z, w, ntx, nty, ntz)];
    if (4ull * root_size[G] > (unsigned long long)g.sprod) fin[G] = 1;
}

constexpr int kPendingMerge = -2;
constexpr int kPendingNew = -3;
constexpr int kPhase2Batch = 2;

template <int NDIM>
__global__ void conn_phase2_kernel(Geom g, const int* __restrict__ gparent, const int* __restrict__ comp_label,
                                   const unsigned long long* __restrict__ root_size,
                                   const unsigned long long* __restrict__ root_first,
                                   const uint8_t* __restrict__ fin, const uint16_t* __restrict__ lid_img,
                                   const int* __restrict__ tile_base, int* __restrict__ out_label,
                                   int* __restrict__ link, unsigned long long* __restrict__ new_key,
                                   int* __restrict__ new_val, unsigned* __restrict__ counters, RasterKey rk,
                                   int64_t ntx, int64_t nty, int64_t ntz)
{
    // kPhase2Batch records a grid stride apart per thread, their loads issued
    // together (the merge lookup is two dependent random loads)
    const int64_t M = counters[0];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < M; i0 += stride * kPhase2Batch) {
        bool root[kPhase2Batch], merge[kPhase2Batch];
        uint8_t fn[kPhase2Batch];
        unsigned long long f[kPhase2Batch], sz[kPhase2Batch];
        int64_t tix[kPhase2Batch], vix[kPhase2Batch];
#pragma unroll
        for (int b = 0; b < kPhase2Batch; ++b) {
            const int64_t i = i0 + b * stride;
            root[b] = i < M && gparent[i] == (int)i;
        }
#pragma unroll
        for (int b = 0; b < kPhase2Batch; ++b) {
            const int64_t i = i0 + b * stride;
            fn[b] = root[b] ? fin[i] : 0;
            f[b] = root[b] ? root_first[i] : 0ull;
            sz[b] = root[b] ? root_size[i] : 0ull;
        }
#pragma unroll
        for (int b = 0; b < kPhase2Batch; ++b) {
            const int64_t i = i0 + b * stride;
            merge[b] = false;
            tix[b] = vix[b] = 0;
            if (!root[b]) continue;
            if (fn[b]) { out_label[i] = comp_label[i]; continue; }
            if (4ull * sz[b] > (unsigned long long)g.sprod || f[b] == 0ull) {
                unsigned pos = atomicAdd(&counters[2], 1u);
                new_key[pos] = f[b];
                new_val[pos] = (int)i;
                out_label[i] = kPendingNew;
                continue;
            }
            int64_t x[kMaxDims];
#pragma unroll
            for (int d = 0; d < kMaxDims; ++d) x[d] = (int64_t)((f[b] >> rk.sh[d]) & rk.mask[d]);
            bool stepped = false;  // x - e_d for the smallest d with x_d > 0 (f != 0, so there is one)
#pragma unroll
            for (int d = 0; d < kMaxDims; ++d)
                if (!stepped && x[d] > 0) { x[d] -= 1; stepped = true; }
            tix[b] = ccl_tile_of<NDIM>(g, x[0], x[1], x[2], x[3], ntx, nty, ntz);
            vix[b] = vidx(g, x[0], x[1], x[2], x[3]);
            merge[b] = true;
        }
        int at[kPhase2Batch];
#pragma unroll
        for (int b = 0; b < kPhase2Batch; ++b) at[b] = merge[b] ? tile_base[tix[b]] + (int)lid_img[vix[b]] : 0;
#pragma unroll
        for (int b = 0; b < kPhase2Batch; ++b) {
            if (!merge[b]) continue;
            const int64_t i = i0 + b * stride;
            link[i] = gparent[at[b]];
            out_label[i] = kPendingMerge;
        }
    }
}

// bitonic sort of (key, value) pairs -- one block, in shared memory
constexpr int kSmallSort = 2048;
__global__ void sort_small_kernel(unsigned long long* key, int* val, const unsigned* __restrict__ counters)
{
    __shared__ unsigned long long sk[kSmallSort];
    __shared__ int sv[kSmallSort];
    const int n = (int)counters[2];
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        sk[i] = i < n ? key[i] : ~0ull;
        sv[i] = i < n ? val[i] : -1;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    bool up = (i & k) == 0;
                    if ((sk[i] > sk[l]) == up) {
                        unsigned long long tk = sk[i]; sk[i] = sk[l]; sk[l] = tk;
                        int tv = sv[i]; sv[i] = sv[l]; sv[l] = tv;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) { key[i] = sk[i]; val[i] = sv[i]; }
}

__global__ void sort_pad_kernel(const unsigned long long* __restrict__ key, const int* __restrict__ val,
                                unsigned long long* __restrict__ k2, int* __restrict__ v2, int64_t n, int64_t P)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        k2[i] = i < n ? key[i] : ~0ull;
        v2[i] = i < n ? val[i] : -1;
    }
}

__global__ void sort_step_kernel(unsigned long long* key, int* val, int64_t P, int64_t k, int64_t j)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t l = i ^ j;
        if (l > i) {
            bool up = (i & k) == 0;
            if ((key[i] > key[l]) == up) {
                unsigned long long tk = key[i]; key[i] = key[l]; key[l] = tk;
                int tv = val[i]; val[i] = val[l]; val[l] = tv;
            }
        }
    }
}

__global__ void assign_new_kernel(const int* __restrict__ val, int* __restrict__ out_label, int64_t K,
                                  int64_t n)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        out_label[val[r]] = (int)(K + r);
}

// Each thread takes kResolveBatch records a grid stride apart and issues
// their loads together, so the dependent loads of one record (its link, then
// the label there) overlap those of the others.
constexpr int kResolveBatch = 4;
__global__ void conn_resolve_kernel(const int* __restrict__ gparent, const int* __restrict__ link,
                                    volatile int* out_label, unsigned* counters)
{
    const int64_t M = counters[0];
    const int* ol = const_cast<const int*>(out_label);  // plain loads for the filter
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < M; i0 += stride * kResolveBatch) {
        bool pend[kResolveBatch];
        int j[kResolveBatch], o[kResolveBatch];
#pragma unroll
        for (int b = 0; b < kResolveBatch; ++b) {
            const int64_t i = i0 + b * stride;
            pend[b] = i < M && gparent[i] == (int)i && ol[i] == kPendingMerge;
        }
#pragma unroll
        for (int b = 0; b < kResolveBatch; ++b) j[b] = pend[b] ? link[i0 + b * stride] : 0;
#pragma unroll
        for (int b = 0; b < kResolveBatch; ++b) o[b] = pend[b] ? out_label[j[b]] : 0;
        // a pending merge that links to another pending one follows the links
        // on (first voxels strictly decrease, so the walk is shorter than the
        // component count)
#pragma unroll
        for (int b = 0; b < kResolveBatch; ++b) {
            if (!pend[b]) continue;
            for (int64_t step = 0; o[b] < 0; ++step) {
                if (step > M) { atomicExch(&counters[3], 1u); o[b] = 0; break; }
                j[b] = link[j[b]];
                o[b] = out_label[j[b]];
            }
            out_label[i0 + b * stride] = o[b];
        }
    }
}

template <int NDIM>
__global__ void __launch_bounds__(kCclThreads, 8)
conn_relabel_kernel(Geom g, const uint16_t* __restrict__ lid_img, const int* __restrict__ tile_base,
                    const int* __restrict__ tile_cnt, const int* __restrict__ gparent,
                    const int* __restrict__ out_label, const int* __restrict__ comp_label,
                    int32_t* __restrict__ labels_out, int inplace, int64_t ntx, int64_t nty, int64_t ntz,
                    int64_t tile0)
{
    using Cfg = CclCfg<NDIM>;
    constexpr int TX = Cfg::TX, TY = Cfg::TY, TZ = Cfg::TZ;
    __shared__ int tab[kCclTV];  // local component -> output label
    const int64_t tile = tile0 + blockIdx.x;
    int64_t X0, Y0, Z0, W0;
    ccl_tile_origin<NDIM>(tile, ntx, nty, ntz, X0, Y0, Z0, W0);
    // the thread's voxels: their local ids are loaded first, in flight while
    // the table is built (0xffff marks a voxel outside the image)
    constexpr int PT = kCclTV / kCclThreads;
    static_assert(PT % 2 == 0, "local ids are kept two per register");
    const int64_t p0 = vidx(g, X0, Y0, Z0, W0), sy = g.N[0], sxy = g.N[0] * g.N[1];
    const int ex = (int)imin64(TX, g.N[0] - X0), ey = (int)imin64(TY, g.N[1] - Y0), ez = (int)imin64(TZ, g.N[2] - Z0);
    auto inside = [&](int e) { return e % TX < ex && (e / TX) % TY < ey && e / (TX * TY) < ez; };
    auto vox = [&](int e) -> int64_t {
        return p0 + e % TX + (int64_t)((e / TX) % TY) * sy + (int64_t)(e / (TX * TY)) * sxy;
    };
    unsigned lv[PT / 2];
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        const int e = threadIdx.x + i * kCclThreads;
        const unsigned l = inside(e) ? (unsigned)lid_img[vox(e)] : 0xffffu;
        if (i % 2 == 0) lv[i / 2] = l;
        else lv[i / 2] |= l << 16;
    }
    const int base = tile_base[tile];
    const int nloc = tile_cnt[tile];
    // the table: two records per thread and pass, so that both records'
    // dependent loads (parent, then its label) are in flight together
    int any = 0;
    for (int l = threadIdx.x; l < nloc; l += 2 * kCclThreads) {
        const bool two = l + kCclThreads < nloc;
        const int r0 = base + l, r1 = two ? r0 + kCclThreads : r0;
        const int G0 = gparent[r0], G1 = gparent[r1];
        const int c0 = comp_label[r0], c1 = comp_label[r1];
        const int o0 = out_label[G0], o1 = out_label[G1];
        tab[l] = o0;
        if (two) tab[l + kCclThreads] = o1;
        any |= (o0 != c0) | (o1 != c1);
    }
    // in place, a tile none of whose components changes label is left alone;
    // otherwise all of its voxels are stored, so that every 32-byte sector is
    // written whole
    if (!__syncthreads_or(any) && inplace) return;
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        const int e = threadIdx.x + i * kCclThreads;
        const unsigned l = (lv[i / 2] >> (16 * (i % 2))) & 0xffffu;
        if (l < (unsigned)nloc) labels_out[vox(e)] = tab[l];
    }
}

// ---------------------------------------------------------------------------
template <int NDIM>
struct CclGrid {
    int64_t ntx, nty, ntz, ntiles;
    explicit CclGrid(const Geom& g)
    {
        using Cfg = CclCfg<NDIM>;
        ntx = (g.N[0] + Cfg::TX - 1) / Cfg::TX;
        nty = (g.N[1] + Cfg::TY - 1) / Cfg::TY;
        ntz = (g.N[2] + Cfg::TZ - 1) / Cfg::TZ;
        ntiles = ntx * nty * ntz * g.N[3];  // one slice of tiles per index along a fourth axis
    }
};

// Steps 3-5 on the complete record forest (M records): flatten, phase 1
// (from the label image, or -- labels_in null -- from the seed voxels the
// slab form found), phase 2, the ranking of new labels, the link walks.
// *Mn receives the number of new labels.
template <int NDIM>
static int conn_resolve_records(sslic_ctx* c, const int32_t* labels_in, const RasterKey& rk, int64_t M,
                                cudaStream_t st, int64_t* Mn_out)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    const CclGrid<NDIM> t(g);
    int rc;
    unsigned hc[4];
    const int gb = c->sms * 8;
    // per-record passes: a few records per thread, all of them in flight at
    // once, so that the walks' latencies overlap
    auto rec_grid = [M](int batch) {
        return (unsigned)imax64(1, imin64((M + 256 * batch - 1) / (256 * batch), (int64_t)1 << 30));
    };
    ccl_flatten_kernel<<<rec_grid(kFlattenBatch), 256, 0, st>>>(w.gparent, w.root_size, w.root_first, w.counters);
    count_launch(c);
    if ((rc = cuda_check(c, cudaGetLastError(), "ccl_flatten_kernel"))) return rc;
    if (labels_in)
        conn_phase1_kernel<NDIM><<<(g.K + 255) / 256, 256, 0, st>>>(g, w.ctr, labels_in, w.lid, w.tile_base,
                                                                     w.gparent, w.root_size, w.fin, t.ntx, t.nty, t.ntz);
    else
        conn_phase1_seeded_kernel<NDIM><<<(g.K + 255) / 256, 256, 0, st>>>(g, w.conn_seed, w.lid, w.tile_base,
                                                                            w.gparent, w.root_size, w.fin, t.ntx,
                                                                            t.nty, t.ntz);
    count_launch(c);
    if ((rc = cuda_check(c, cudaGetLastError(), "conn_phase1_kernel"))) return rc;
    conn_phase2_kernel<NDIM><<<rec_grid(kPhase2Batch), 256, 0, st>>>(g, w.gparent, w.comp_label, w.root_size, w.root_first, w.fin,
                                                  w.lid, w.tile_base, w.out_label, w.link, w.new_key, w.new_val,
                                                  w.counters, rk, t.ntx, t.nty, t.ntz);
    count_launch(c);
    if ((rc = cuda_check(c, cudaGetLastError(), "conn_phase2_kernel"))) return rc;
    if ((rc = cuda_check(c, cudaMemcpyAsync(hc, w.counters, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                         "read new count")))
        return rc;
    if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
    const int64_t Mn = hc[2];
    if (g.K + Mn > INT_MAX) return set_error(c, SSLIC_EUNSUPPORTED, "label count exceeds int32");
    if (Mn > 0) {
        const int* sorted_val = w.new_val;
        if (Mn <= kSmallSort) {
            sort_small_kernel<<<1, 1024, 0, st>>>(w.new_key, w.new_val, w.counters);
            count_launch(c);
            if ((rc = cuda_check(c, cudaGetLastError(), "sort_small_kernel"))) return rc;
        } else {
            int64_t P = 1;
            while (P < Mn) P <<= 1;
            if (P > w.sort_cap) {
                cudaFree(w.sort_key);
                cudaFree(w.sort_val);
                w.sort_key = nullptr;
                w.sort_val = nullptr;
                w.sort_cap = 0;
                if (cudaMalloc(&w.sort_key, P * sizeof(unsigned long long)) != cudaSuccess ||
                    cudaMalloc(&w.sort_val, P * sizeof(int)) != cudaSuccess)
                    return set_error(c, SSLIC_ENOMEM, "sort scratch");
                w.sort_cap = P;
            }
            sort_pad_kernel<<<gb, 256, 0, st>>>(w.new_key, w.new_val, w.sort_key, w.sort_val, Mn, P);
            count_launch(c);
            for (int64_t k = 2; k <= P; k <<= 1)
                for (int64_t j = k >> 1; j > 0; j >>= 1) {
                    sort_step_kernel<<<gb, 256, 0, st>>>(w.sort_key, w.sort_val, P, k, j);
                    count_launch(c);
                }
            if ((rc = cuda_check(c, cudaGetLastError(), "sort_step_kernel"))) return rc;
            sorted_val = w.sort_val;
        }
        assign_new_kernel<<<gb, 256, 0, st>>>(sorted_val, w.out_label, g.K, Mn);
        count_launch(c);
        if ((rc = cuda_check(c, cudaGetLastError(), "assign_new_kernel"))) return rc;
    }
    conn_resolve_kernel<<<rec_grid(kResolveBatch), 256, 0, st>>>(w.gparent, w.link, w.out_label, w.counters);
    count_launch(c);
    if ((rc = cuda_check(c, cudaGetLastError(), "conn_resolve_kernel"))) return rc;
    *Mn_out = Mn;
    return SSLIC_OK;
}

// the error flag of the bounded walks, read after a stream sync
static int conn_status(sslic_ctx* c, cudaStream_t st)
{
    unsigned hc[4];
    int rc;
    if ((rc = cuda_check(c, cudaMemcpyAsync(hc, c->ws.counters, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                         "read status")))
        return rc;
    if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
    if (hc[3]) return set_error(c, SSLIC_ECUDA, "connectivity: a bounded walk ran out or an internal check failed (code %u)", hc[3]);
    return SSLIC_OK;
}

template <int NDIM>
static int connectivity_impl(sslic_ctx* c, const int32_t* labels_in, int32_t* labels_out, cudaStream_t st,
                             int64_t* num_labels)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    const CclGrid<NDIM> t(g);
    int rc;
    unsigned hc[4];
    RasterKey rk;
    if (!make_raster_key(g, rk)) return set_error(c, SSLIC_EUNSUPPORTED, "packed voxel coordinates exceed 63 bits");
    const int pr = prof_begin(c, SSLIC_PHASE_CONNECTIVITY, st);
    for (int attempt = 0; attempt < 2; ++attempt) {
        if ((rc = cuda_check(c, cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned), st), "memset counters"))) return rc;
        ccl_local_kernel<NDIM><<<t.ntiles, kCclThreads, 0, st>>>(g, labels_in, w.lid, w.tile_base, w.tile_cnt,
                                                                w.comp_label, w.root_size, w.root_first, w.fin,
                                                                w.gparent, w.counters, w.m_cap, rk, t.ntx, t.nty,
                                                                t.ntz, 0);
        count_launch(c);
        if ((rc = cuda_check(c, cudaGetLastError(), "ccl_local_kernel"))) return rc;
        if ((rc = cuda_check(c, cudaMemcpyAsync(hc, w.counters, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                             "read component count")))
            return rc;
        if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
        if (!hc[1]) break;
        if (attempt == 1) return set_error(c, SSLIC_ENOMEM, "component records still overflow");
        if ((rc = ensure_ccl_capacity(c, (int64_t)hc[0] + hc[0] / 4 + 4096))) return rc;
    }
    const int64_t M = hc[0];
    if (M > INT_MAX) return set_error(c, SSLIC_EUNSUPPORTED, "more than 2^31 components");
    ccl_faces_kernel<NDIM><<<t.ntiles, kCclThreads, 0, st>>>(g, labels_in, w.lid, w.tile_base, w.gparent,
                                                             w.counters, t.ntx, t.nty, t.ntz, 0, nullptr, 0, 0);
    count_launch(c);
    if ((rc = cuda_check(c, cudaGetLastError(), "ccl_faces_kernel"))) return rc;
    int64_t Mn = 0;
    if ((rc = conn_resolve_records<NDIM>(c, labels_in, rk, M, st, &Mn))) return rc;
    if (c->relabel_host && (NDIM == 2 || NDIM == 3)) {
        // slabs of tile planes along the last axis, each relabelled and then
        // copied to the host on the download stream while the next is relabelled
        if (!w.down_stream &&
            (rc = cuda_check(c, cudaStreamCreateWithFlags(&w.down_stream, cudaStreamNonBlocking), "copy stream")))
            return rc;
        if (!w.slab_ev[4] &&
            (rc = cuda_check(c, cudaEventCreateWithFlags(&w.slab_ev[4], cudaEventDisableTiming), "event")))
            return rc;
        const int64_t depth = NDIM == 3 ? CclCfg<3>::TZ : CclCfg<2>::TY;  // planes per layer of tiles
        const int64_t layer = NDIM == 3 ? t.ntx * t.nty : t.ntx;         // tiles per layer
        const int64_t nlayers = t.ntiles / layer;
        const int64_t per = imax64(1, (nlayers + 7) / 8);                  // layers per slab: about 8 slabs
        const int ax = NDIM - 1;
        int64_t plane = 1;
        for (int d = 0; d < ax; ++d) plane *= g.N[d];
        for (int64_t l0 = 0; l0 < nlayers; l0 += per) {
            const int64_t l1 = imin64(nlayers, l0 + per);
            conn_relabel_kernel<NDIM><<<(unsigned)((l1 - l0) * layer), kCclThreads, 0, st>>>(
                g, w.lid, w.tile_base, w.tile_cnt, w.gparent, w.out_label, w.comp_label, labels_out,
                labels_in == labels_out ? 1 : 0, t.ntx, t.nty, t.ntz, l0 * layer);
            count_launch(c);
            if ((rc = cuda_check(c, cudaGetLastError(), "conn_relabel_kernel"))) return rc;
            const int64_t p0 = l0 * depth, p1 = imin64(g.N[ax], l1 * depth);
            if ((rc = cuda_check(c, cudaEventRecord(w.slab_ev[4], st), "event")) ||
                (rc = cuda_check(c, cudaStreamWaitEvent(w.down_stream, w.slab_ev[4], 0), "wait")) ||
                (rc = cuda_check(c, cudaMemcpyAsync(c->relabel_host + p0 * plane, labels_out + p0 * plane,
                                                    (size_t)((p1 - p0) * plane) * sizeof(int32_t),
                                                    cudaMemcpyDeviceToHost, w.down_stream),
                                 "labels to host")))
                return rc;
        }
        c->relabel_sent = 1;
    } else {
        conn_relabel_kernel<NDIM><<<t.ntiles, kCclThreads, 0, st>>>(g, w.lid, w.tile_base, w.tile_cnt, w.gparent,
                                                                    w.out_label, w.comp_label, labels_out,
                                                                    labels_in == labels_out ? 1 : 0, t.ntx, t.nty,
                                                                    t.ntz, 0);
        count_launch(c);
        if ((rc = cuda_check(c, cudaGetLastError(), "conn_relabel_kernel"))) return rc;
    }
    if ((rc = conn_status(c, st))) return rc;
    prof_end(c, pr, st);
    if (num_labels) *num_labels = g.K + Mn;
    return SSLIC_OK;
}

// ---- slab form -----------------------------------------------------------
// Connectivity of an image handed over as consecutive ranges of planes along
// its last axis (the streamed form's slabs, or the slabs of the ranks that
// share an image), with the same result as connectivity_impl:
//  - each slab's tiles get their local components and records (the records
//    and the per-voxel local ids of the whole image stay on the device), and
//    their faces are united, the face towards the previous slab against the
//    planes carried over from it;
//  - every centre whose S-box ends in the slab finds its phase-1 seed voxel
//    there (the box reaches at most S planes back: those are carried);
//  - once every slab is in, steps 3-5 run on the complete forest;
//  - then each slab is relabelled through its records.
// Slab bounds are multiples of the tile's extent along the last axis, and
// every slab but the last holds at least S_last planes.
template <int NDIM>
static int64_t ccl_tile_depth()
{
    return NDIM == 3 ? CclCfg<3>::TZ : CclCfg<2>::TY;
}

template <int NDIM>
static int conn_slab_tiles(const Geom& g, int64_t lo, int64_t hi, int64_t* tile0, int64_t* ntiles)
{
    const CclGrid<NDIM> t(g);
    const int64_t td = ccl_tile_depth<NDIM>();
    const int64_t layer = NDIM == 3 ? t.ntx * t.nty : t.ntx;
    *tile0 = lo / td * layer;
    *ntiles = (hi + td - 1) / td * layer - *tile0;
    return SSLIC_OK;
}

static int64_t plane_voxels(const Geom& g)
{
    int64_t plane = 1;
    for (int d = 0; d < g.n - 1; ++d) plane *= g.N[d];
    return plane;
}

int conn_slabs_begin(sslic_ctx* c, cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    if (g.n != 2 && g.n != 3) return set_error(c, SSLIC_EUNSUPPORTED, "slab connectivity: 2-D and 3-D images");
    RasterKey rk;
    if (!make_raster_key(g, rk)) return set_error(c, SSLIC_EUNSUPPORTED, "packed voxel coordinates exceed 63 bits");
    int rc;
    if ((rc = ensure_ccl_capacity(c, 32 * g.K + g.V / 1024 + 4096))) return rc;
    if ((rc = ensure_conn_slab_scratch(c))) return rc;
    if ((rc = cuda_check(c, cudaMemsetAsync(w.counters, 0, 4 * sizeof(unsigned), st), "memset counters"))) return rc;
    if ((rc = cuda_check(c, cudaMemsetAsync(w.conn_seed, 0xff, g.K * sizeof(long long), st), "memset seeds")))
        return rc;
    w.conn_next = 0;
    w.conn_carried = 0;
    return SSLIC_OK;
}

template <int NDIM>
static int conn_slabs_add_impl(sslic_ctx* c, const int32_t* labels_slab, int64_t lo, int64_t hi, cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    const CclGrid<NDIM> t(g);
    const int L = g.n - 1;
    const int64_t NL = g.N[L], td = ccl_tile_depth<NDIM>(), SL = g.S[L];
    if (lo != w.conn_next || hi <= lo || hi > NL)
        return set_error(c, SSLIC_EINVAL, "slab connectivity: slabs must follow each other from plane 0");
    if (lo % td != 0 || (hi % td != 0 && hi != NL))
        return set_error(c, SSLIC_EINVAL, "slab connectivity: slab bounds must be multiples of %lld planes",
                         (long long)td);
    if (hi < NL && hi - lo < SL)
        return set_error(c, SSLIC_EINVAL, "slab connectivity: a slab before the last needs at least S = %lld planes",
                         (long long)SL);
    RasterKey rk;
    make_raster_key(g, rk);
    const int64_t plane = plane_voxels(g), qlo = lo * plane;
    const int32_t* lab = labels_slab - qlo;            // indexed by global voxel
    const int64_t cbase = (lo - w.conn_carried) * plane;  // first voxel the carry holds
    int64_t tile0, nt;
    conn_slab_tiles<NDIM>(g, lo, hi, &tile0, &nt);
    int rc;
    unsigned hc[4];
    if ((rc = cuda_check(c, cudaMemcpyAsync(hc, w.counters, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                         "read component count")))
        return rc;
    if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
    const unsigned m_before = hc[0];
    for (int attempt = 0; attempt < 2; ++attempt) {
        ccl_local_kernel<NDIM><<<nt, kCclThreads, 0, st>>>(g, lab, w.lid, w.tile_base, w.tile_cnt, w.comp_label,
                                                           w.root_size, w.root_first, w.fin, w.gparent, w.counters,
                                                           w.m_cap, rk, t.ntx, t.nty, t.ntz, tile0);
        count_launch(c);
        if ((rc = cuda_check(c, cudaGetLastError(), "ccl_local_kernel"))) return rc;
        if ((rc = cuda_check(c, cudaMemcpyAsync(hc, w.counters, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                             "read component count")))
            return rc;
        if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
        if (!hc[1]) break;
        if (attempt == 1) return set_error(c, SSLIC_ENOMEM, "component records still overflow");
        // grow (keeping the earlier slabs' records) and redo this slab
        if ((rc = grow_ccl_records(c, (int64_t)hc[0] + hc[0] / 4 + 4096, m_before, st))) return rc;
        const unsigned reset[2] = {m_before, 0u};
        if ((rc = cuda_check(c, cudaMemcpyAsync(w.counters, reset, 2 * sizeof(unsigned), cudaMemcpyHostToDevice, st),
                             "reset counters")))
            return rc;
        if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
    }
    if (hc[0] > (unsigned)INT_MAX) return set_error(c, SSLIC_EUNSUPPORTED, "more than 2^31 components");
    ccl_faces_kernel<NDIM><<<nt, kCclThreads, 0, st>>>(g, lab, w.lid, w.tile_base, w.gparent, w.counters, t.ntx,
                                                       t.nty, t.ntz, tile0, w.conn_carry, qlo, cbase);
    count_launch(c);
    if ((rc = cuda_check(c, cudaGetLastError(), "ccl_faces_kernel"))) return rc;
    conn_seek_kernel<NDIM><<<(g.K + 255) / 256, 256, 0, st>>>(g, w.ctr, lab, w.conn_carry, qlo, cbase, lo, hi,
                                                             w.conn_seed);
    count_launch(c);
    if ((rc = cuda_check(c, cudaGetLastError(), "conn_seek_kernel"))) return rc;
    // carry the last S planes (those the next slab's boxes and faces reach)
    if (hi < NL) {
        const int64_t keep = imin64(SL, hi);
        if ((rc = cuda_check(c, cudaMemcpyAsync(w.conn_carry, labels_slab + (hi - keep - lo) * plane,
                                                (size_t)(keep * plane) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st),
                             "carry planes")))
            return rc;
        w.conn_carried = keep;
    }
    w.conn_next = hi;
    return SSLIC_OK;
}

int conn_slabs_add(sslic_ctx* c, const int32_t* labels_slab, int64_t lo, int64_t hi, cudaStream_t st)
{
    if (c->g.n == 3) return conn_slabs_add_impl<3>(c, labels_slab, lo, hi, st);
    if (c->g.n == 2) return conn_slabs_add_impl<2>(c, labels_slab, lo, hi, st);
    return set_error(c, SSLIC_EUNSUPPORTED, "slab connectivity: 2-D and 3-D images");
}

int conn_slabs_finish(sslic_ctx* c, cudaStream_t st, int64_t* num_labels)
{
    const Geom& g = c->g;
    if (g.n != 2 && g.n != 3) return set_error(c, SSLIC_EUNSUPPORTED, "slab connectivity: 2-D and 3-D images");
    if (c->ws.conn_next != g.N[g.n - 1])
        return set_error(c, SSLIC_EINVAL, "slab connectivity: not every plane has been added");
    RasterKey rk;
    make_raster_key(g, rk);
    unsigned hc[4];
    int rc;
    if ((rc = cuda_check(c, cudaMemcpyAsync(hc, c->ws.counters, 4 * sizeof(unsigned), cudaMemcpyDeviceToHost, st),
                         "read component count")))
        return rc;
    if ((rc = cuda_check(c, cudaStreamSynchronize(st), "sync"))) return rc;
    int64_t Mn = 0;
    rc = g.n == 3 ? conn_resolve_records<3>(c, nullptr, rk, hc[0], st, &Mn)
                  : conn_resolve_records<2>(c, nullptr, rk, hc[0], st, &Mn);
    if (rc) return rc;
    if ((rc = conn_status(c, st))) return rc;
    if (num_labels) *num_labels = g.K + Mn;
    return SSLIC_OK;
}

template <int NDIM>
static int conn_slabs_relabel_impl(sslic_ctx* c, int32_t* labels_out_slab, int64_t lo, int64_t hi, cudaStream_t st)
{
    const Geom& g = c->g;
    Workspace& w = c->ws;
    const CclGrid<NDIM> t(g);
    const int64_t NL = g.N[g.n - 1], td = ccl_tile_depth<NDIM>();
    if (lo < 0 || hi <= lo || hi > NL || lo % td != 0 || (hi % td != 0 && hi != NL))
        return set_error(c, SSLIC_EINVAL, "slab connectivity: slab bounds must be multiples of %lld planes",
                         (long long)td);
    int64_t tile0, nt;
    conn_slab_tiles<NDIM>(g, lo, hi, &tile0, &nt);
    conn_relabel_kernel<NDIM><<<nt, kCclThreads, 0, st>>>(g, w.lid, w.tile_base, w.tile_cnt, w.gparent, w.out_label,
                                                          w.comp_label, labels_out_slab - lo * plane_voxels(g), 0,
                                                          t.ntx, t.nty, t.ntz, tile0);
    count_launch(c);
    return cuda_check(c, cudaGetLastError(), "conn_relabel_kernel");
}

int conn_slabs_relabel(sslic_ctx* c, int32_t* labels_out_slab, int64_t lo, int64_t hi, cudaStream_t st)
{
    if (c->g.n == 3) return conn_slabs_relabel_impl<3>(c, labels_out_slab, lo, hi, st);
    if (c->g.n == 2) return conn_slabs_relabel_impl<2>(c, labels_out_slab, lo, hi, st);
    return set_error(c, SSLIC_EUNSUPPORTED, "slab connectivity: 2-D and 3-D images");
}

int64_t ccl_num_tiles(const Geom& g)
{
    if (g.n == 4) {
        using C4 = CclCfg<4>;
        return ((g.N[0] + C4::TX - 1) / C4::TX) * ((g.N[1] + C4::TY - 1) / C4::TY) * ((g.N[2] + C4::TZ - 1) / C4::TZ) *
               g.N[3];
    }
    if (g.n == 3) {
        using C3 = CclCfg<3>;
        return ((g.N[0] + C3::TX - 1) / C3::TX) * ((g.N[1] + C3::TY - 1) / C3::TY) * ((g.N[2] + C3::TZ - 1) / C3::TZ);
    }
    if (g.n == 2) {
        using C2 = CclCfg<2>;
        return ((g.N[0] + C2::TX - 1) / C2::TX) * ((g.N[1] + C2::TY - 1) / C2::TY);
    }
    return (g.N[0] + CclCfg<1>::TX - 1) / CclCfg<1>::TX;
}

int run_connectivity(sslic_ctx* c, const int32_t* labels_in, int32_t* labels_out, cudaStream_t st,
                     int64_t* num_labels)
{
    switch (c->g.n) {
    case 4: return connectivity_impl<4>(c, labels_in, labels_out, st, num_labels);
    case 3: return connectivity_impl<3>(c, labels_in, labels_out, st, num_labels);
    case 2: return connectivity_impl<2>(c, labels_in, labels_out, st, num_labels);
    default: return connectivity_impl<1>(c, labels_in, labels_out, st, num_labels);
    }
}

}  // namespace sslic
