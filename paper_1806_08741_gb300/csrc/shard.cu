// shard.cu -- one image shared by several GPUs, each holding a slab of
// planes along the last axis (the C ABI's sslic_shard_* and
// sslic_conn_slabs_* calls).
//
// The paper parallelises SSLIC over non-overlapping regions of the image:
// each thread assigns the pixels of its region and maps them into per-label
// sums, and a reduce merges the regions' sums before the centres are
// divided out (Sec. 3.1).  Here a region is a GPU's slab.  Assignment is
// voxel-centric and reads only the centres and their bins, which every rank
// keeps whole, so slabs need no halo for it; the map leaves exact integer
// sums, whose sum over the ranks does not depend on the order of the
// additions, so every rank that divides the same summed sums gets the
// centres of the single-GPU run bit for bit.  The library does no
// communication itself: the caller's collective (NCCL across GPUs) sums the
// buffers between sslic_shard_map and sslic_shard_finalize.
#include "common.cuh"

namespace sslic {

static int64_t slab_align(const Geom& g) { return g.n == 3 ? 8 : 64; }

static int64_t plane_count(const Geom& g)
{
    int64_t plane = 1;
    for (int d = 0; d < g.n - 1; ++d) plane *= g.N[d];
    return plane;
}

static size_t elem_size(const Geom& g) { return g.dtype == SSLIC_U8 ? 1 : (g.dtype == SSLIC_U16 ? 2 : 4); }

// the checks every shard call makes on a slab
static int check_slab(sslic_ctx* c, int64_t lo, int64_t hi)
{
    const Geom& g = c->g;
    if (g.n != 2 && g.n != 3) return set_error(c, SSLIC_EUNSUPPORTED, "shards: 2-D and 3-D images");
    if (c->p.precision) return set_error(c, SSLIC_EUNSUPPORTED, "shards: no precision form");
    const int64_t NL = g.N[g.n - 1], al = slab_align(g);
    if (lo < 0 || hi <= lo || hi > NL || lo % al != 0 || (hi % al != 0 && hi != NL))
        return set_error(c, SSLIC_EINVAL, "shard slab [%lld, %lld): bounds must be multiples of %lld planes",
                         (long long)lo, (long long)hi, (long long)al);
    return SSLIC_OK;
}

}  // namespace sslic

using namespace sslic;

extern "C" {

int sslic_shard_seed(sslic_ctx* c, const void* image_dev, int64_t lo, int64_t hi, float* centres_dev, void* stream)
{
    if (!c || !image_dev || !centres_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    int rc;
    if ((rc = check_slab(c, lo, hi))) return rc;
    const Geom& g = c->g;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t a = imax64(0, lo - 2);
    const size_t pbytes = (size_t)plane_count(g) * g.C * elem_size(g);
    if ((rc = cuda_check(c, cudaMemsetAsync(c->ws.ctr, 0, (size_t)g.K * g.CW * sizeof(float), st), "clear centres")))
        return rc;
    const Slab sl{lo, hi};
    if ((rc = launch_seed(c, (const unsigned char*)image_dev - a * pbytes, st, &sl))) return rc;
    return launch_export_centres(c, centres_dev, st);
}

int sslic_shard_sums_size(const sslic_ctx* c, int64_t* n_u64, int64_t* n_f64)
{
    if (!c || !n_u64 || !n_f64) return SSLIC_EINVAL;
    *n_u64 = c->g.K * c->g.AW;
    *n_f64 = c->g.dtype == SSLIC_F32 ? c->g.K * c->g.C : 0;
    return SSLIC_OK;
}

int sslic_shard_map(sslic_ctx* c, const void* image_dev, int32_t* labels_dev, int64_t lo, int64_t hi,
                    const float* centres_dev, void* sums_dev, void* stream)
{
    if (!c || !image_dev || !labels_dev || !centres_dev || !sums_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    int rc;
    if ((rc = check_slab(c, lo, hi))) return rc;
    const Geom& g = c->g;
    Workspace& w = c->ws;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t plane = plane_count(g);
    const size_t nu = (size_t)(g.K * g.AW), nf = g.dtype == SSLIC_F32 ? (size_t)(g.K * g.C) : 0;
    if ((rc = launch_import_centres(c, centres_dev, st))) return rc;
    if ((rc = cuda_check(c, cudaMemsetAsync(w.acc, 0, nu * sizeof(unsigned long long), st), "clear sums"))) return rc;
    if (nf && (rc = cuda_check(c, cudaMemsetAsync(w.facc, 0, nf * sizeof(double), st), "clear sums"))) return rc;
    if ((rc = build_bins(c, st))) return rc;
    const Slab sl{lo, hi};
    if ((rc = launch_assign_update(c, (const unsigned char*)image_dev - lo * plane * g.C * elem_size(g),
                                   labels_dev - lo * plane, st, &sl)))
        return rc;
    unsigned char* out = (unsigned char*)sums_dev;
    if ((rc = cuda_check(c, cudaMemcpyAsync(out, w.acc, nu * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st),
                         "export sums")))
        return rc;
    if (nf && (rc = cuda_check(c, cudaMemcpyAsync(out + nu * sizeof(unsigned long long), w.facc, nf * sizeof(double),
                                                   cudaMemcpyDeviceToDevice, st),
                                "export sums")))
        return rc;
    return SSLIC_OK;
}

int sslic_shard_finalize(sslic_ctx* c, const void* sums_dev, const float* centres_prev_dev, float* centres_out_dev,
                         double* residual_host, void* stream)
{
    if (!c || !sums_dev || !centres_prev_dev || !centres_out_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    const Geom& g = c->g;
    if (g.n != 2 && g.n != 3) return set_error(c, SSLIC_EUNSUPPORTED, "shards: 2-D and 3-D images");
    Workspace& w = c->ws;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nu = (size_t)(g.K * g.AW), nf = g.dtype == SSLIC_F32 ? (size_t)(g.K * g.C) : 0;
    const unsigned char* in = (const unsigned char*)sums_dev;
    int rc;
    if ((rc = launch_import_centres(c, centres_prev_dev, st))) return rc;
    if ((rc = cuda_check(c, cudaMemcpyAsync(w.acc, in, nu * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st),
                         "import sums")))
        return rc;
    if (nf && (rc = cuda_check(c, cudaMemcpyAsync(w.facc, in + nu * sizeof(unsigned long long), nf * sizeof(double),
                                                   cudaMemcpyDeviceToDevice, st),
                                "import sums")))
        return rc;
    if ((rc = launch_finalize(c, st))) return rc;
    if ((rc = launch_export_centres(c, centres_out_dev, st))) return rc;
    if (residual_host) {
        if ((rc = cuda_check(c, cudaMemcpyAsync(residual_host, w.resid_out, sizeof(double), cudaMemcpyDeviceToHost, st),
                             "read residual")))
            return rc;
        return cuda_check(c, cudaStreamSynchronize(st), "sync");
    }
    return SSLIC_OK;
}

int sslic_conn_slabs_begin(sslic_ctx* c, const float* centres_dev, void* stream)
{
    if (!c || !centres_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if ((rc = launch_import_centres(c, centres_dev, st))) return rc;
    return conn_slabs_begin(c, st);
}

int sslic_conn_slabs_add(sslic_ctx* c, const int32_t* labels_dev, int64_t lo, int64_t hi, void* stream)
{
    if (!c || !labels_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    return conn_slabs_add(c, labels_dev, lo, hi, (cudaStream_t)stream);
}

int sslic_conn_slabs_finish(sslic_ctx* c, void* stream, int64_t* num_labels_host)
{
    if (!c) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    int64_t n = 0;
    const int rc = conn_slabs_finish(c, (cudaStream_t)stream, &n);
    if (!rc && num_labels_host) *num_labels_host = n;
    return rc;
}

int sslic_conn_slabs_relabel(sslic_ctx* c, int32_t* labels_out_dev, int64_t lo, int64_t hi, void* stream)
{
    if (!c || !labels_out_dev) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    return conn_slabs_relabel(c, labels_out_dev, lo, hi, (cudaStream_t)stream);
}

}  // extern "C"
