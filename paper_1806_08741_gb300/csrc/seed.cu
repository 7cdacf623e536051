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
#include "device_fns.cuh"

namespace sslic {

template <typename T>
__global__ void seed_kernel(Geom g, const T* __restrict__ img, float* __restrict__ ctr, int perturb, int64_t k0,
                            int64_t k1)
{
    const int64_t k = k0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < k1) seed_one<T>(g, img, ctr, perturb, k);
}

// With a slab: the seeds whose lattice coordinate along the last axis lies in
// [lo, hi); the buffer must hold the planes [lo - 2, hi + 2) (clamped to the
// image), which the perturbation's gradients reach.
int launch_seed(sslic_ctx* c, const void* img, cudaStream_t st, const Slab* slab)
{
    const Geom& g = c->g;
    int64_t k0 = 0, k1 = g.K;
    if (slab) {
        const int a = g.n - 1;  // the last axis
        int64_t per = 1;
        for (int d = 0; d < a; ++d) per *= g.nb[d];
        auto first_at_or_after = [&](int64_t v) {  // smallest j with off + j S >= v
            const int64_t t = v - g.off[a];
            return t <= 0 ? 0 : imin64(g.nb[a], (t + g.S[a] - 1) / g.S[a]);
        };
        k0 = first_at_or_after(slab->lo) * per;
        k1 = first_at_or_after(slab->hi) * per;
        if (k1 <= k0) return SSLIC_OK;
    }
    int threads = 128;
    int64_t blocks = (k1 - k0 + threads - 1) / threads;
    const int pr = prof_begin(c, SSLIC_PHASE_SEED, st);
    count_launch(c);
    switch (g.dtype) {
    case SSLIC_U8:
        seed_kernel<uint8_t><<<blocks, threads, 0, st>>>(g, (const uint8_t*)img, c->ws.ctr, c->p.perturb, k0, k1);
        break;
    case SSLIC_U16:
        seed_kernel<uint16_t><<<blocks, threads, 0, st>>>(g, (const uint16_t*)img, c->ws.ctr, c->p.perturb, k0, k1);
        break;
    default:
        seed_kernel<float><<<blocks, threads, 0, st>>>(g, (const float*)img, c->ws.ctr, c->p.perturb, k0, k1);
    }
    prof_end(c, pr, st);
    return cuda_check(c, cudaGetLastError(), "seed_kernel");
}

}  // namespace sslic
