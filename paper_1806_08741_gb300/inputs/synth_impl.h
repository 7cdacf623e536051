/*
 * synth_impl.h -- the per-voxel generator of synth.h, written once as inline
 * integer code and compiled both by the host C compiler (synth.c) and by
 * nvcc for the device (synth_gpu.cu).  Input generation only.
 */
#ifndef SSLIC_SYNTH_IMPL_H
#define SSLIC_SYNTH_IMPL_H
#include "synth.h"

#ifdef __CUDACC__
#define SYN_FN static __host__ __device__ inline
#else
#define SYN_FN static inline
#endif

SYN_FN uint64_t syn_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

SYN_FN uint64_t syn_hash(uint64_t seed, uint64_t stream, uint64_t i)
{
    return syn_splitmix64(syn_splitmix64(seed * 256ULL + stream) + i);
}

SYN_FN int64_t syn_floordiv(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

SYN_FN int64_t syn_bound(const synth_spec* s, int d, int64_t j)
{
    return j * s->size[d] / s->sites[d];
}

/* site coordinate along axis d of the site with cell index j_d and raster id sid */
SYN_FN int64_t syn_site_coord(const synth_spec* s, int d, int64_t jd, uint64_t sid)
{
    int64_t lo = syn_bound(s, d, jd);
    int64_t w = syn_bound(s, d, jd + 1) - lo;
    return lo + (int64_t)(syn_hash(s->seed, 10 + d, sid) % (uint64_t)w);
}

/* region (site id) of voxel x, and that site's position */
SYN_FN int64_t syn_region(const synth_spec* s, const int64_t* x, int64_t* site_pos)
{
    int64_t j[3];
    for (int d = 0; d < 3; ++d) j[d] = ((x[d] + 1) * s->sites[d] - 1) / s->size[d];
    int64_t best = -1, bestd = 0;
    int64_t bp[3] = {0, 0, 0};
    for (int64_t a2 = j[2] - 1; a2 <= j[2] + 1; ++a2) {
        if (a2 < 0 || a2 >= s->sites[2]) continue;
        for (int64_t a1 = j[1] - 1; a1 <= j[1] + 1; ++a1) {
            if (a1 < 0 || a1 >= s->sites[1]) continue;
            for (int64_t a0 = j[0] - 1; a0 <= j[0] + 1; ++a0) {
                if (a0 < 0 || a0 >= s->sites[0]) continue;
                int64_t sid = a0 + s->sites[0] * (a1 + s->sites[1] * a2);
                int64_t p0 = syn_site_coord(s, 0, a0, (uint64_t)sid);
                int64_t p1 = syn_site_coord(s, 1, a1, (uint64_t)sid);
                int64_t p2 = syn_site_coord(s, 2, a2, (uint64_t)sid);
                int64_t e0 = x[0] - p0, e1 = x[1] - p1, e2 = x[2] - p2;
                int64_t dd = e0 * e0 + e1 * e1 + e2 * e2;
                if (best < 0 || dd < bestd || (dd == bestd && sid < best)) {
                    best = sid; bestd = dd; bp[0] = p0; bp[1] = p1; bp[2] = p2;
                }
            }
        }
    }
    if (site_pos) { site_pos[0] = bp[0]; site_pos[1] = bp[1]; site_pos[2] = bp[2]; }
    return best;
}

SYN_FN int64_t syn_value(const synth_spec* s, const int64_t* x, int64_t region,
                         const int64_t* site, int c)
{
    const int64_t vmax = s->dtype == 0 ? 255 : 65535;
    const int64_t C = s->channels;
    int64_t v = (int64_t)(syn_hash(s->seed, 20, (uint64_t)(region * C + c)) % (uint64_t)(vmax + 1));
    if (s->ramp_amp != 0) {
        int64_t acc = 0;
        for (int d = 0; d < s->ndim; ++d) {
            int64_t a = (int64_t)(syn_hash(s->seed, 30 + d, (uint64_t)(region * C + c)) % 2049ULL) - 1024;
            acc += a * (x[d] - site[d]);
        }
        v += syn_floordiv(s->ramp_amp * acc, 1024 * s->ramp_len);
    }
    if (s->sigma != 0) {
        uint64_t q = (uint64_t)(x[0] + s->size[0] * (x[1] + s->size[1] * x[2]));
        uint64_t r = syn_hash(s->seed, 40, q * (uint64_t)C + (uint64_t)c);
        int64_t u = (int64_t)(r & 0xFFFF) + (int64_t)((r >> 16) & 0xFFFF) +
                    (int64_t)((r >> 32) & 0xFFFF) + (int64_t)((r >> 48) & 0xFFFF) - 131070;
        v += syn_floordiv(2 * u * s->sigma + 37837, 2 * 37837);
    }
    if (v < 0) v = 0;
    if (v > vmax) v = vmax;
    return v;
}

SYN_FN int syn_check(const synth_spec* s)
{
    if (s->ndim < 1 || s->ndim > 3 || s->channels < 1) return -1;
    if (s->dtype != 0 && s->dtype != 1) return -1;
    for (int d = 0; d < 3; ++d) {
        if (s->size[d] < 1 || s->sites[d] < 1 || s->sites[d] > s->size[d]) return -1;
        if (d >= s->ndim && (s->size[d] != 1 || s->sites[d] != 1)) return -1;
    }
    if (s->ramp_amp != 0 && s->ramp_len < 1) return -1;
    return 0;
}
#endif
