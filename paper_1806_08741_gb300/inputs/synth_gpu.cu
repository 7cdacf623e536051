// synth_gpu.cu -- device side of the synthetic image generator (definition in
// synth.h).  One thread per voxel of a row segment; used to make the large
// volumes directly in device memory.
#include <cuda_runtime.h>
#include "synth_impl.h"

template <typename T>
__global__ void synth_kernel(synth_spec s, T* out, int64_t V)
{
    const int64_t C = s.channels;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < V;
         q += (int64_t)gridDim.x * blockDim.x) {
        int64_t x[3] = {q % s.size[0], (q / s.size[0]) % s.size[1], q / (s.size[0] * s.size[1])};
        int64_t site[3];
        int64_t reg = syn_region(&s, x, site);
        for (int c = 0; c < C; ++c) out[q * C + c] = (T)syn_value(&s, x, reg, site, c);
    }
}

extern "C" int synth_fill_device(const synth_spec* s, void* out_dev, void* stream)
{
    if (!s || !out_dev || syn_check(s) != 0) return -1;
    int64_t V = s->size[0] * s->size[1] * s->size[2];
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int blocks = sms * 8;
    cudaStream_t st = (cudaStream_t)stream;
    if (s->dtype == 0) synth_kernel<uint8_t><<<blocks, 256, 0, st>>>(*s, (uint8_t*)out_dev, V);
    else synth_kernel<uint16_t><<<blocks, 256, 0, st>>>(*s, (uint16_t*)out_dev, V);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
