// hc_3d_mma.cu -- instantiations of the many-channel float kernel: 3-D, tensor-core form.
#include "hc.cuh"

SSLIC_HC_INSTANTIATE(3, true, 16)
SSLIC_HC_INSTANTIATE(3, true, 32)
SSLIC_HC_INSTANTIATE(3, true, 48)
SSLIC_HC_INSTANTIATE(3, true, 64)
SSLIC_HC_INSTANTIATE(3, true, 96)
SSLIC_HC_INSTANTIATE(3, true, 128)
