// hc_3d_exact.cu -- instantiations of the many-channel float kernel: 3-D, exact FP32 form.
#include "hc.cuh"

SSLIC_HC_INSTANTIATE(3, false, 16)
SSLIC_HC_INSTANTIATE(3, false, 32)
SSLIC_HC_INSTANTIATE(3, false, 48)
SSLIC_HC_INSTANTIATE(3, false, 64)
SSLIC_HC_INSTANTIATE(3, false, 96)
SSLIC_HC_INSTANTIATE(3, false, 128)
