/*
 * synth.h -- seeded, counter-based synthetic image generator shared by the
 * test-suite, the benchmark and the CPU oracle's inputs.  It holds no part of
 * the superpixel method's arithmetic: it only makes images.
 *
 * Definition (implemented identically, in integer arithmetic only, by the
 * CPU code in synth.c and the CUDA code in synth_gpu.cu, so both produce the
 * same bytes):
 *
 *  h(seed, stream, i) = splitmix64(splitmix64(seed * 256 + stream) + i)
 *      splitmix64 is Steele, Lea and Flood's SplitMix64 output function
 *      (the golden-gamma increment followed by the two xor-shift-multiply
 *      rounds); all arithmetic is modulo 2^64.
 *
 *  Regions.  A jittered lattice of g_d sites per axis.  Cell j along axis d
 *      spans [b_d(j), b_d(j+1)) with b_d(j) = floor(j * N_d / g_d); the site
 *      of cell index s (raster, axis 0 fastest) sits at
 *      b_d(j_d) + h(seed, 10 + d, s) mod (b_d(j_d+1) - b_d(j_d)).
 *      Voxel x lies in cell j_d(x) = floor(((x_d + 1) * g_d - 1) / N_d); its
 *      region is the nearest site (integer squared Euclidean distance) among
 *      the 3^n cells around its own, ties to the lowest site index.
 *  Colour.  mean_c(s) = h(seed, 20, s*C + c) mod (vmax + 1).
 *  Ramp (optional, amplitude A).  coefficient a_{c,d}(s) =
 *      h(seed, 30 + d, s*C + c) mod 2049 - 1024; ramp_c(x) =
 *      floor(A * sum_d a_{c,d} (x_d - site_d) / (1024 * L)), L = ramp_len.
 *  Noise.  Irwin-Hall sum of four 16-bit uniforms taken from
 *      h(seed, 40, q*C + c) (q = raster voxel index): u = sum - 131070, whose
 *      standard deviation is 37837.2; noise = round-half-up(u * sigma / 37837).
 *  Value = clamp(mean + ramp + noise, 0, vmax).
 */
#ifndef SSLIC_SYNTH_H
#define SSLIC_SYNTH_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t ndim;        /* 1..3 */
    int64_t size[3];     /* N_d, axis 0 fastest; unused axes = 1 */
    int32_t channels;    /* C */
    int32_t dtype;       /* 0 = uint8 (vmax 255), 1 = uint16 (vmax 65535) */
    uint64_t seed;
    int64_t sites[3];    /* g_d sites per axis (>= 1, <= N_d) */
    int64_t sigma;       /* noise standard deviation, in grey levels */
    int64_t ramp_amp;    /* A; 0 disables the ramp */
    int64_t ramp_len;    /* L (>= 1) */
} synth_spec;

/* CPU: write the crop [origin, origin + extent) of the image into out
 * (C-contiguous crop, channels interleaved).  Returns 0 or -1 on bad spec. */
int synth_fill(const synth_spec* s, const int64_t* origin, const int64_t* extent, void* out);

/* CPU: region index (site index) of every voxel of the crop. */
int synth_regions(const synth_spec* s, const int64_t* origin, const int64_t* extent, int32_t* out);

/* GPU (synth_gpu.cu): write the whole image into device memory on the given
 * stream.  Returns 0, -1 on bad spec, -2 on a CUDA error. */
int synth_fill_device(const synth_spec* s, void* out_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif
