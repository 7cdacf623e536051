// hc_2d_mma.cu -- instantiations of the many-channel float kernel: 2-D, tensor-core form.
#include "hc.cuh"

SSLIC_HC_INSTANTIATE(2, true, 16)
SSLIC_HC_INSTANTIATE(2, true, 32)
SSLIC_HC_INSTANTIATE(2, true, 48)
SSLIC_HC_INSTANTIATE(2, true, 64)
SSLIC_HC_INSTANTIATE(2, true, 96)
SSLIC_HC_INSTANTIATE(2, true, 128)
