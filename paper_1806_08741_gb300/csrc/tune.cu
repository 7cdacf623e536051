// tune.cu -- measured choice of the assignment kernel's tile shape.
//
// The tile shape (tile extent and voxels per lane) changes only how the
// assignment is scheduled, never its result.  sslic_autotune times one
// assign + update iteration per shape on the caller's image, from the same
// seeded centres, and keeps the fastest: in the context, and in a
// process-wide table keyed by (dtype, channels, dims, grid) that contexts
// created later and the serving loop consult before the built-in rule.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace sslic {

namespace {
using TuneKey = std::tuple<int, int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tuned;

TuneKey key_of(const Geom& g) { return TuneKey(g.dtype, g.C, g.n, g.S[0], g.S[1], g.S[2]); }

}  // namespace

bool has_tile_kernel(const Geom& g)
{
    return (g.n == 2 || g.n == 3) && ((g.dtype == SSLIC_U8 && (g.C == 1 || g.C == 3)) ||
                                      (g.dtype == SSLIC_U16 && g.C == 1) || (g.dtype == SSLIC_F32 && g.C == 3));
}

int tuned_tile_shape(const Geom& g)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key_of(g));
    return it == g_tuned.end() ? -1 : it->second;
}

}  // namespace sslic

using namespace sslic;

extern "C" {

int sslic_num_tile_shapes(int32_t ndim, int32_t* count)
{
    if (!count || ndim < 1 || ndim > 3) return SSLIC_EINVAL;
    *count = num_tile_shapes(ndim);
    return SSLIC_OK;
}

int sslic_tile_shape_info(int32_t ndim, int32_t shape, int32_t* dims, int32_t* voxels_per_lane,
                          int32_t* tma_staged)
{
    if (!dims || ndim < 2 || ndim > 3 || shape < 0 || shape >= num_tile_shapes(ndim)) return SSLIC_EINVAL;
    tile_dims(ndim, shape, &dims[0], &dims[1], &dims[2]);
    const int b = num_base_shapes(ndim);
    if (voxels_per_lane) *voxels_per_lane = tile_voxels_per_lane(ndim, shape);
    if (tma_staged) *tma_staged = shape >= b ? 1 : 0;
    return SSLIC_OK;
}

int sslic_set_tile_shape(sslic_ctx* c, int32_t shape)
{
    if (!c || shape < -1 || (shape >= 0 && shape >= num_tile_shapes(c->g.n))) return SSLIC_EINVAL;
    if (shape >= 0 && !has_tile_kernel(c->g)) return SSLIC_EUNSUPPORTED;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    c->tile_shape = shape;
    return SSLIC_OK;
}

int sslic_get_tile_shape(const sslic_ctx* c, int32_t* shape)
{
    if (!c || !shape) return SSLIC_EINVAL;
    if (!has_tile_kernel(c->g)) *shape = -1;
    else if (c->tile_shape >= 0) *shape = c->tile_shape;
    else {
        const int t = tuned_tile_shape(c->g);
        *shape = t >= 0 ? t : default_tile_shape(c->g);
    }
    return SSLIC_OK;
}

int sslic_autotune(sslic_ctx* c, const void* image_dev, int32_t* labels_dev, void* stream, int32_t reps,
                   int32_t* best, float* ms_out)
{
    if (!c || !image_dev || !labels_dev || reps < 1) return SSLIC_EINVAL;
    if (!has_tile_kernel(c->g)) return set_error(c, SSLIC_EUNSUPPORTED, "no tile kernel for this image type");
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    cudaStream_t st = (cudaStream_t)stream;
    const Geom& g = c->g;
    const int ns = num_tile_shapes(g.n);
    const int saved = c->tile_shape;
    const int prof = c->prof_on;
    c->prof_on = 0;
    float* start = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SSLIC_OK;
    std::vector<float> med(ns, 0.0f);
    const size_t cbytes = (size_t)g.K * (g.C + g.n) * sizeof(float);
    if ((rc = cuda_check(c, cudaMalloc((void**)&start, cbytes), "autotune centres"))) goto done;
    if ((rc = cuda_check(c, cudaEventCreate(&e0), "event")) || (rc = cuda_check(c, cudaEventCreate(&e1), "event")))
        goto done;
    if ((rc = launch_seed(c, image_dev, st)) || (rc = launch_export_centres(c, start, st))) goto done;
    for (int s = 0; s < ns; ++s) {
        c->tile_shape = s;
        std::vector<float> t;
        for (int r = 0; r <= reps; ++r) {  // the first run warms up
            if ((rc = launch_import_centres(c, start, st))) goto done;
            if ((rc = cuda_check(c, cudaEventRecord(e0, st), "event"))) goto done;
            if ((rc = build_bins(c, st)) || (rc = launch_assign_update(c, image_dev, labels_dev, st)) ||
                (rc = launch_finalize(c, st)))
                goto done;
            if ((rc = cuda_check(c, cudaEventRecord(e1, st), "event")) ||
                (rc = cuda_check(c, cudaEventSynchronize(e1), "event")))
                goto done;
            float ms = 0.0f;
            if ((rc = cuda_check(c, cudaEventElapsedTime(&ms, e0, e1), "elapsed"))) goto done;
            if (r > 0) t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        med[s] = t[t.size() / 2];
    }
    {
        const int bi = (int)(std::min_element(med.begin(), med.end()) - med.begin());
        c->tile_shape = bi;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key_of(g)] = bi;
        }
        if (best) *best = bi;
        if (ms_out)
            for (int s = 0; s < ns; ++s) ms_out[s] = med[s];
    }
done:
    if (rc) c->tile_shape = saved;
    c->prof_on = prof;
    if (start) cudaFree(start);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

int sslic_tune_record(const sslic_params* p, int32_t shape)
{
    Geom g;
    if (!p || make_geom(p, &g) != SSLIC_OK) return SSLIC_EINVAL;
    if (!has_tile_kernel(g)) return SSLIC_EUNSUPPORTED;
    if (shape < 0 || shape >= num_tile_shapes(g.n)) return SSLIC_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key_of(g)] = shape;
    return SSLIC_OK;
}

int sslic_tune_lookup(const sslic_params* p, int32_t* shape)
{
    Geom g;
    if (!p || !shape || make_geom(p, &g) != SSLIC_OK) return SSLIC_EINVAL;
    if (!has_tile_kernel(g)) return SSLIC_EUNSUPPORTED;
    *shape = tuned_tile_shape(g);
    return SSLIC_OK;
}

int sslic_tune_forget(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
    return SSLIC_OK;
}

}  // extern "C"
