// hc.cu -- dispatch of the many-channel float kernels of hc.cuh (one
// instantiation file per dims x form, compiled in parallel) and the
// diagnostic entry point of the tensor-core form.
#include "hc.cuh"

namespace sslic {

bool hc_applies(const Geom& g)
{
    return g.dtype == SSLIC_F32 && (g.n == 2 || g.n == 3) && g.C >= hc::kMinC && g.C <= hc::kMaxC;
}

int64_t hc_num_tiles(const Geom& g)
{
    if (g.n == 3)
        return ((g.N[0] + 7) / 8) * ((g.N[1] + 3) / 4) * ((g.N[2] + 3) / 4);
    return ((g.N[0] + 15) / 16) * ((g.N[1] + 7) / 8);
}


// instantiated in hc_<dims>_<form>.cu
#define SSLIC_HC_EXTERN(NDIM, MMA)                                                                          \
    extern template int launch_hc_ct<NDIM, MMA, 16>(sslic_ctx*, const float*, int32_t*, cudaStream_t, int64_t, float*, int*, float*); \
    extern template int launch_hc_ct<NDIM, MMA, 32>(sslic_ctx*, const float*, int32_t*, cudaStream_t, int64_t, float*, int*, float*); \
    extern template int launch_hc_ct<NDIM, MMA, 48>(sslic_ctx*, const float*, int32_t*, cudaStream_t, int64_t, float*, int*, float*); \
    extern template int launch_hc_ct<NDIM, MMA, 64>(sslic_ctx*, const float*, int32_t*, cudaStream_t, int64_t, float*, int*, float*); \
    extern template int launch_hc_ct<NDIM, MMA, 96>(sslic_ctx*, const float*, int32_t*, cudaStream_t, int64_t, float*, int*, float*); \
    extern template int launch_hc_ct<NDIM, MMA, 128>(sslic_ctx*, const float*, int32_t*, cudaStream_t, int64_t, float*, int*, float*);
SSLIC_HC_EXTERN(2, false)
SSLIC_HC_EXTERN(2, true)
SSLIC_HC_EXTERN(3, false)
SSLIC_HC_EXTERN(3, true)

template <int NDIM, bool MMA>
static int launch_hc_impl(sslic_ctx* c, const float* img, int32_t* labels, cudaStream_t st, int64_t tile0,
                          float* dbg_dots, int* dbg_cand, float* dbg_mu)
{
    switch (hc::ct_of(c->g.C)) {
    case 16: return launch_hc_ct<NDIM, MMA, 16>(c, img, labels, st, tile0, dbg_dots, dbg_cand, dbg_mu);
    case 32: return launch_hc_ct<NDIM, MMA, 32>(c, img, labels, st, tile0, dbg_dots, dbg_cand, dbg_mu);
    case 48: return launch_hc_ct<NDIM, MMA, 48>(c, img, labels, st, tile0, dbg_dots, dbg_cand, dbg_mu);
    case 64: return launch_hc_ct<NDIM, MMA, 64>(c, img, labels, st, tile0, dbg_dots, dbg_cand, dbg_mu);
    case 96: return launch_hc_ct<NDIM, MMA, 96>(c, img, labels, st, tile0, dbg_dots, dbg_cand, dbg_mu);
    default: return launch_hc_ct<NDIM, MMA, 128>(c, img, labels, st, tile0, dbg_dots, dbg_cand, dbg_mu);
    }
}

int launch_hc(sslic_ctx* c, const float* img, int32_t* labels, cudaStream_t st)
{
    const bool mma = c->p.precision == 1 && c->g.C >= hc::kMinCMma;
    if (c->g.n == 3)
        return mma ? launch_hc_impl<3, true>(c, img, labels, st, -1, nullptr, nullptr, nullptr)
                   : launch_hc_impl<3, false>(c, img, labels, st, -1, nullptr, nullptr, nullptr);
    return mma ? launch_hc_impl<2, true>(c, img, labels, st, -1, nullptr, nullptr, nullptr)
               : launch_hc_impl<2, false>(c, img, labels, st, -1, nullptr, nullptr, nullptr);
}

int launch_hc_probe(sslic_ctx* c, const float* img, int32_t* labels, int64_t tile, float* dots, int* cand,
                    float* mu, cudaStream_t st)
{
    if (c->g.n == 3) return launch_hc_impl<3, true>(c, img, labels, st, tile, dots, cand, mu);
    return launch_hc_impl<2, true>(c, img, labels, st, tile, dots, cand, mu);
}

}  // namespace sslic

using namespace sslic;

extern "C" int sslic_precision_probe(sslic_ctx* c, const void* image_dev, const float* centres_dev, int64_t tile,
                                     float* dots_host, int32_t* cand_host, float* mu_host)
{
    if (!c || !image_dev || !centres_dev || !dots_host || !cand_host || !mu_host) return SSLIC_EINVAL;
    if (c->p.precision != 1 || !hc_applies(c->g) || tile < 0 || tile >= hc_num_tiles(c->g)) return SSLIC_EINVAL;
    Busy b(c);
    if (!b.ok) return SSLIC_EBUSY;
    const Geom& g = c->g;
    float* dots = nullptr;
    int* cand = nullptr;
    float* mu = nullptr;
    int rc = SSLIC_OK;
    const size_t nd = (size_t)hc::kTV * hc::kNC;
    if ((rc = cuda_check(c, cudaMalloc((void**)&dots, nd * sizeof(float)), "probe buffers")) ||
        (rc = cuda_check(c, cudaMalloc((void**)&cand, hc::kNC * sizeof(int)), "probe buffers")) ||
        (rc = cuda_check(c, cudaMalloc((void**)&mu, g.C * sizeof(float)), "probe buffers")))
        goto done;
    if ((rc = cuda_check(c, cudaMemset(cand, 0xff, hc::kNC * sizeof(int)), "memset"))) goto done;
    if ((rc = launch_import_centres(c, centres_dev, 0)) || (rc = build_bins(c, 0)) ||
        (rc = launch_hc_probe(c, (const float*)image_dev, nullptr, tile, dots, cand, mu, 0)))
        goto done;
    if ((rc = cuda_check(c, cudaDeviceSynchronize(), "probe"))) goto done;
    {
        unsigned h = 0;
        if ((rc = cuda_check(c, cudaMemcpy(&h, c->ws.ovf_count, sizeof(unsigned), cudaMemcpyDeviceToHost), "probe")))
            goto done;
        unsigned e = 0;
        if ((rc = cuda_check(c, cudaMemcpy(&e, c->ws.hc_err, sizeof(unsigned), cudaMemcpyDeviceToHost), "probe")))
            goto done;
        if (e) {
            cudaMemset(c->ws.hc_err, 0, sizeof(unsigned));
            rc = set_error(c, SSLIC_ETIMEOUT, "probe: a bounded wait ran out");
            goto done;
        }
    }
    if ((rc = cuda_check(c, cudaMemcpy(dots_host, dots, nd * sizeof(float), cudaMemcpyDeviceToHost), "probe")) ||
        (rc = cuda_check(c, cudaMemcpy(cand_host, cand, hc::kNC * sizeof(int), cudaMemcpyDeviceToHost), "probe")) ||
        (rc = cuda_check(c, cudaMemcpy(mu_host, mu, g.C * sizeof(float), cudaMemcpyDeviceToHost), "probe")))
        goto done;
    if (cand_host[0] == -1 && cand_host[1] == -1) {
        // the kernel left before the MMA: more candidates than slots (or none)
        int any = 0;
        for (int j = 0; j < hc::kNC; ++j) any |= cand_host[j] != -1;
        if (!any) rc = set_error(c, SSLIC_EUNSUPPORTED, "probe: tile reached by more than 32 centres or none");
    }
done:
    if (dots) cudaFree(dots);
    if (cand) cudaFree(cand);
    if (mu) cudaFree(mu);
    return rc;
}
