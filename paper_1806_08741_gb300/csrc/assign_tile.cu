// assign_tile.cu -- the tile shapes of the assignment kernel (host side).
//
// Shape indices: 3-D 0 = 32x16x8 / 2 voxels per lane, 1 = 16x8x8 / 2,
// 2 = 32x16x8 / 4, 3 = 16x8x8 / 4, 4 = 32x8x8 / 2, 5 = 32x8x8 / 4; 2-D
// 0 = 64x32 / 2, 1 = 32x16 / 2, 2 = 64x32 / 4.  Each base shape comes twice: index b stages the tile with
// plain loads, index b + (number of base shapes) with a TMA copy of the next
// tile in flight while the current one is computed (used where the image
// rows are 16-byte multiples; otherwise it is the plain form).  The default
// follows the expected number of centres that reach a tile; sslic_autotune
// measures the shapes instead.
#include "assign_tile.cuh"

namespace sslic {

int num_base_shapes(int ndim) { return ndim == 3 ? 6 : (ndim == 2 ? 3 : 0); }
int num_tile_shapes(int ndim) { return 2 * num_base_shapes(ndim); }

void tile_dims(int ndim, int shape, int* tx, int* ty, int* tz)
{
    auto f = [&](auto sh) {
        using SH = decltype(sh);
        *tx = SH::TX;
        *ty = SH::TY;
        *tz = SH::TZ;
        return 0;
    };
    const int b = num_base_shapes(ndim);
    if (ndim == 3) with_shape<3>(shape % b, f);
    else with_shape<2>(shape % b, f);
}

int tile_voxels_per_lane(int ndim, int shape)
{
    auto f = [](auto sh) { return decltype(sh)::VL; };
    const int b = num_base_shapes(ndim);
    return ndim == 3 ? with_shape<3>(shape % b, f) : with_shape<2>(shape % b, f);
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
    if (g.n == 3) {
        // float channel planes: the 2048-voxel tile keeps four CTAs per SM
        if (g.dtype == SSLIC_F32)
            return reach(g, tile::Shape3M::TX, tile::Shape3M::TY, tile::Shape3M::TZ) <= lim ? 4 : 1;
        return reach(g, tile::Shape3L::TX, tile::Shape3L::TY, tile::Shape3L::TZ) <= lim ? 0 : 1;
    }
    return reach(g, tile::Shape2L::TX, tile::Shape2L::TY, 1) <= lim ? 0 : 1;
}

int tile_list_stride() { return tile::kListStride; }
static_assert(tile::kListStride == kTileListStride, "record layout");

int launch_tile_lists(sslic_ctx* c, int ndim, int tx, int ty, int tz, int ntx, int nty, int64_t tile0,
                      int64_t ntiles, cudaStream_t st)
{
    const Workspace& w = c->ws;
    const int64_t lgrid = imax64(1, imin64((ntiles + tile::kListWarps - 1) / tile::kListWarps, (int64_t)c->sms * 32));
    const int pr = prof_begin(c, SSLIC_PHASE_BINS, st);  // timed with the bins it reads
    if (ndim == 3)
        tile::tile_lists_kernel<3><<<(unsigned)lgrid, tile::kListWarps * 32, 0, st>>>(
            c->g, w.ctr, w.bin_start, w.bin_items, w.tile_lists, tile0, ntiles, ntx, nty, tx, ty, tz, w.ovf_tiles,
            w.ovf_count);
    else
        tile::tile_lists_kernel<2><<<(unsigned)lgrid, tile::kListWarps * 32, 0, st>>>(
            c->g, w.ctr, w.bin_start, w.bin_items, w.tile_lists, tile0, ntiles, ntx, nty, tx, ty, tz, w.ovf_tiles,
            w.ovf_count);
    count_launch(c);
    prof_end(c, pr, st);
    return cuda_check(c, cudaGetLastError(), "tile_lists_kernel");
}

// the batched queue's records: one warp per (request, tile) of a group
cudaError_t launch_tile_lists_queue(int ndim, const TileArgs* reqs, const int64_t* tpre, const int* nR, int64_t* ovf,
                                    unsigned* ovf_count, int grid, cudaStream_t st)
{
    if (ndim == 3)
        tile::tile_lists_queue_kernel<3><<<grid, tile::kListWarps * 32, 0, st>>>(reqs, tpre, nR, ovf, ovf_count);
    else
        tile::tile_lists_queue_kernel<2><<<grid, tile::kListWarps * 32, 0, st>>>(reqs, tpre, nR, ovf, ovf_count);
    return cudaGetLastError();
}

// the most tiles any shape cuts the image into (sizes the crowded-tile list)
int64_t assign_num_tiles(const Geom& g)
{
    int64_t best = 0;
    for (int s = 0; s < num_base_shapes(g.n == 3 ? 3 : 2); ++s) {
        int tx, ty, tz;
        tile_dims(g.n == 3 ? 3 : 2, s, &tx, &ty, &tz);
        const int64_t n = ((g.N[0] + tx - 1) / tx) * ((g.N[1] + ty - 1) / ty) * ((g.N[2] + tz - 1) / tz);
        best = n > best ? n : best;
    }
    return best;
}

}  // namespace sslic
