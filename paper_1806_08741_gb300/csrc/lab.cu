// lab.cu -- 8-bit sRGB to CIE-Lab float conversion on the device.
//
// SLIC clusters colour pixels as the vector [L, a, b, x, y] (Sec. 2, 2.1) and
// the paper converts its 8-bit RGB colour volume to CIE-Lab float before
// segmenting it (Sec. 4.1); jSLIC's lookup table for that conversion (Sec. 6)
// has its counterpart here in a 256-entry table of linear values per CTA.
// The paper names neither the RGB space nor the white point.  Read as sRGB
// (IEC 61966-2-1: piecewise transfer function, 4-decimal RGB->XYZ matrix)
// under the D65 white (0.95047, 1, 1.08883) and CIE 1976 L*a*b*, the reading
// whose extremes over the 8-bit cube give the L, a and b ranges Sec. 2.1
// prints:
//     lin(v) = v/12.92 if v <= 0.04045 else ((v + 0.055)/1.055)^2.4, v = code/255
//     [X Y Z] = M [lin(R) lin(G) lin(B)],  f(t) = t^(1/3) if t > (6/29)^3
//                                                  else t/(3 (6/29)^2) + 4/29
//     L = 116 f(Y) - 16,  a = 500 (f(X/Xn) - f(Y)),  b = 200 (f(Y) - f(Z/Zn))
//
// One pass, 3 bytes in and 12 bytes out per voxel: a grid-stride loop over
// groups of 4 voxels (three 32-bit loads, three 16-byte stores) where the
// pointers are aligned for it, one voxel per step otherwise and for the
// ragged tail.  Single precision throughout except the table, whose entries
// are computed in double and rounded once.
#include <cstdint>

#include "common.cuh"

namespace sslic {
namespace {

constexpr int kLabThreads = 256;
constexpr double kDelta = 6.0 / 29.0;
constexpr float kDelta3 = (float)(kDelta * kDelta * kDelta);
constexpr float kSlope = (float)(1.0 / (3.0 * kDelta * kDelta));
constexpr float kOffset = (float)(4.0 / 29.0);

__device__ __forceinline__ float lab_f(float t)
{
    return t > kDelta3 ? cbrtf(t) : t * kSlope + kOffset;
}

__device__ __forceinline__ void to_lab(const float* lin, unsigned r, unsigned g, unsigned b, float* o)
{
    const float R = lin[r], G = lin[g], B = lin[b];
    const float fx = lab_f((0.4124f * R + 0.3576f * G + 0.1805f * B) / 0.95047f);
    const float fy = lab_f(0.2126f * R + 0.7152f * G + 0.0722f * B);
    const float fz = lab_f((0.0193f * R + 0.1192f * G + 0.9505f * B) / 1.08883f);
    o[0] = 116.0f * fy - 16.0f;
    o[1] = 500.0f * (fx - fy);
    o[2] = 200.0f * (fy - fz);
}

}  // namespace

__global__ void __launch_bounds__(kLabThreads) srgb_to_lab_kernel(const uint8_t* __restrict__ rgb,
                                                                  float* __restrict__ lab, int64_t n, int vec)
{
    __shared__ float lin[256];
    {
        const double v = threadIdx.x / 255.0;
        lin[threadIdx.x] = (float)(v <= 0.04045 ? v / 12.92 : pow((v + 0.055) / 1.055, 2.4));
    }
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t first = 0;
    if (vec) {
        const int64_t ng = n / 4;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(rgb);
        float4* dst = reinterpret_cast<float4*>(lab);
        for (int64_t gi = t0; gi < ng; gi += stride) {
            // bytes: w0 = R0 G0 B0 R1, w1 = G1 B1 R2 G2, w2 = B2 R3 G3 B3
            const uint32_t w0 = __ldg(src + 3 * gi), w1 = __ldg(src + 3 * gi + 1), w2 = __ldg(src + 3 * gi + 2);
            float o[12];
            to_lab(lin, w0 & 255u, (w0 >> 8) & 255u, (w0 >> 16) & 255u, o);
            to_lab(lin, w0 >> 24, w1 & 255u, (w1 >> 8) & 255u, o + 3);
            to_lab(lin, (w1 >> 16) & 255u, w1 >> 24, w2 & 255u, o + 6);
            to_lab(lin, (w2 >> 8) & 255u, (w2 >> 16) & 255u, w2 >> 24, o + 9);
            dst[3 * gi] = make_float4(o[0], o[1], o[2], o[3]);
            dst[3 * gi + 1] = make_float4(o[4], o[5], o[6], o[7]);
            dst[3 * gi + 2] = make_float4(o[8], o[9], o[10], o[11]);
        }
        first = ng * 4;
    }
    for (int64_t i = first + t0; i < n; i += stride) {
        float o[3];
        to_lab(lin, rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], o);
        lab[3 * i] = o[0];
        lab[3 * i + 1] = o[1];
        lab[3 * i + 2] = o[2];
    }
}

}  // namespace sslic

extern "C" int sslic_srgb_to_lab(const void* rgb_dev, void* lab_dev, int64_t n, void* stream)
{
    using namespace sslic;
    if (n < 0 || (n > 0 && (!rgb_dev || !lab_dev))) return SSLIC_EINVAL;
    if (n == 0) return SSLIC_OK;
    if (n > (INT64_MAX / 12)) return SSLIC_EINVAL;
    const uintptr_t a = (uintptr_t)rgb_dev, b = (uintptr_t)lab_dev;
    if (a < b + (uintptr_t)(12 * n) && b < a + (uintptr_t)(3 * n)) return SSLIC_EINVAL;  // overlapping buffers
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return SSLIC_ECUDA;
    const int vec = (a % 4 == 0) && (b % 16 == 0);
    const int64_t work = vec ? (n + 3) / 4 : n;
    const int64_t blocks = imin64((work + kLabThreads - 1) / kLabThreads, (int64_t)sms * 8);
    srgb_to_lab_kernel<<<(unsigned)blocks, kLabThreads, 0, (cudaStream_t)stream>>>(
        (const uint8_t*)rgb_dev, (float*)lab_dev, n, vec);
    return cudaGetLastError() == cudaSuccess ? SSLIC_OK : SSLIC_ECUDA;
}
