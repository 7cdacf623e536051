// seed.cu -- seeding on the regular lattice and gradient perturbation.
//
// Sec. 2.2 / 3.1 step 1: centres are sampled at fixed intervals S_d and each
// is moved, in parallel, to the lowest gradient magnitude in its 3^n
// neighbourhood (multi-channel: Frobenius norm of the Jacobian).  Lattice:
// nb_d = ceil(N_d / S_d) seeds per axis at o_d + j S_d, cluster index = raster
// index of (j_0, j_1, j_2), j_0 fastest.  Gradient^2 = sum_c sum_d
// (I_c(x + e_d) - I_c(x - e_d))^2 with border clamping; exact in int64 for
// integer images, one rounding per operation (channel outer, axis inner) for
// float images.  The seed keeps ties; the other offsets are visited in raster
// order (axis 0 fastest) and win only on a strictly smaller gradient.
#include "common.cuh"

namespace sslic {

template <typename T>
__device__ __forceinline__ int64_t grad_int(const Geom& g, const T* img, const int64_t* x, int64_t q)
{
    int64_t acc = 0;
    for (int c = 0; c < g.C; ++c) {
        for (int d = 0; d < g.n; ++d) {
            int64_t st = d == 0 ? 1 : (d == 1 ? g.N[0] : g.N[0] * g.N[1]);
            int64_t hi = x[d] + 1 < g.N[d] ? q + st : q;
            int64_t lo = x[d] > 0 ? q - st : q;
            int64_t diff = (int64_t)img[hi * g.C + c] - (int64_t)img[lo * g.C + c];
            acc += diff * diff;
        }
    }
    return acc;
}

__device__ __forceinline__ float grad_f32(const Geom& g, const float* img, const int64_t* x, int64_t q)
{
    float acc = 0.0f;
    bool first = true;
    for (int c = 0; c < g.C; ++c) {
        for (int d = 0; d < g.n; ++d) {
            int64_t st = d == 0 ? 1 : (d == 1 ? g.N[0] : g.N[0] * g.N[1]);
            int64_t hi = x[d] + 1 < g.N[d] ? q + st : q;
            int64_t lo = x[d] > 0 ? q - st : q;
            float diff = __fsub_rn(img[hi * g.C + c], img[lo * g.C + c]);
            float sq = __fmul_rn(diff, diff);
            acc = first ? sq : __fadd_rn(acc, sq);
            first = false;
        }
    }
    return acc;
}

template <typename T>
__global__ void seed_kernel(Geom g, const T* __restrict__ img, float* __restrict__ ctr, int perturb)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= g.K) return;
    int64_t x[3];
    int64_t rem = k;
    for (int d = 0; d < 3; ++d) {
        int64_t j = rem % g.nb[d];
        rem /= g.nb[d];
        x[d] = g.off[d] + j * g.S[d];
    }
    int64_t best[3] = {x[0], x[1], x[2]};
    if (perturb) {
        int64_t q0 = vidx(g, x[0], x[1], x[2]);
        constexpr bool kFloat = sizeof(T) == 4;
        int64_t bi = 0;
        float bf = 0.0f;
        if constexpr (kFloat) bf = grad_f32(g, (const float*)img, x, q0);
        else bi = grad_int(g, img, x, q0);
        const int lo2 = g.n >= 3 ? -1 : 0, lo1 = g.n >= 2 ? -1 : 0;
        for (int o2 = lo2; o2 <= -lo2; ++o2)
            for (int o1 = lo1; o1 <= -lo1; ++o1)
                for (int o0 = -1; o0 <= 1; ++o0) {
                    int64_t y[3] = {x[0] + o0, x[1] + o1, x[2] + o2};
                    if (y[0] < 0 || y[0] >= g.N[0] || y[1] < 0 || y[1] >= g.N[1] || y[2] < 0 ||
                        y[2] >= g.N[2])
                        continue;
                    int64_t q = vidx(g, y[0], y[1], y[2]);
                    bool better;
                    if constexpr (kFloat) {
                        float gq = grad_f32(g, (const float*)img, y, q);
                        better = gq < bf;
                        if (better) bf = gq;
                    } else {
                        int64_t gq = grad_int(g, img, y, q);
                        better = gq < bi;
                        if (better) bi = gq;
                    }
                    if (better) { best[0] = y[0]; best[1] = y[1]; best[2] = y[2]; }
                }
    }
    int64_t qb = vidx(g, best[0], best[1], best[2]);
    float* row = ctr + k * g.CW;
    for (int c = 0; c < g.C; ++c) row[c] = (float)img[qb * g.C + c];
    for (int d = 0; d < 3; ++d) row[g.C + d] = (float)best[d];
}

int launch_seed(sslic_ctx* c, const void* img, cudaStream_t st)
{
    const Geom& g = c->g;
    int threads = 128;
    int64_t blocks = (g.K + threads - 1) / threads;
    const int pr = prof_begin(c, SSLIC_PHASE_SEED, st);
    count_launch(c);
    switch (g.dtype) {
    case SSLIC_U8:
        seed_kernel<uint8_t><<<blocks, threads, 0, st>>>(g, (const uint8_t*)img, c->ws.ctr, c->p.perturb);
        break;
    case SSLIC_U16:
        seed_kernel<uint16_t><<<blocks, threads, 0, st>>>(g, (const uint16_t*)img, c->ws.ctr, c->p.perturb);
        break;
    default:
        seed_kernel<float><<<blocks, threads, 0, st>>>(g, (const float*)img, c->ws.ctr, c->p.perturb);
    }
    prof_end(c, pr, st);
    return cuda_check(c, cudaGetLastError(), "seed_kernel");
}

}  // namespace sslic
