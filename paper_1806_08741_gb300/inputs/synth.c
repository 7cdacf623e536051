/* synth.c -- CPU side of the synthetic image generator (definition in synth.h). */
#include "synth_impl.h"

int synth_fill(const synth_spec* s, const int64_t* origin, const int64_t* extent, void* out)
{
    if (syn_check(s) != 0) return -1;
    for (int d = 0; d < 3; ++d)
        if (origin[d] < 0 || extent[d] < 0 || origin[d] + extent[d] > s->size[d]) return -1;
    const int64_t C = s->channels;
    const int64_t rows = extent[1] * extent[2];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < rows; ++r) {
        int64_t y = r % extent[1], z = r / extent[1];
        for (int64_t xx = 0; xx < extent[0]; ++xx) {
            int64_t x[3] = {origin[0] + xx, origin[1] + y, origin[2] + z};
            int64_t site[3];
            int64_t reg = syn_region(s, x, site);
            int64_t o = (r * extent[0] + xx) * C;
            for (int c = 0; c < C; ++c) {
                int64_t v = syn_value(s, x, reg, site, c);
                if (s->dtype == 0) ((uint8_t*)out)[o + c] = (uint8_t)v;
                else ((uint16_t*)out)[o + c] = (uint16_t)v;
            }
        }
    }
    return 0;
}

int synth_regions(const synth_spec* s, const int64_t* origin, const int64_t* extent, int32_t* out)
{
    if (syn_check(s) != 0) return -1;
    for (int d = 0; d < 3; ++d)
        if (origin[d] < 0 || extent[d] < 0 || origin[d] + extent[d] > s->size[d]) return -1;
    const int64_t rows = extent[1] * extent[2];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < rows; ++r) {
        int64_t y = r % extent[1], z = r / extent[1];
        for (int64_t xx = 0; xx < extent[0]; ++xx) {
            int64_t x[3] = {origin[0] + xx, origin[1] + y, origin[2] + z};
            out[r * extent[0] + xx] = (int32_t)syn_region(s, x, 0);
        }
    }
    return 0;
}
