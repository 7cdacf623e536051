// hc_2d_exact.cu -- instantiations of the many-channel float kernel: 2-D, exact FP32 form.
#include "hc.cuh"

SSLIC_HC_INSTANTIATE(2, false, 16)
SSLIC_HC_INSTANTIATE(2, false, 32)
SSLIC_HC_INSTANTIATE(2, false, 48)
SSLIC_HC_INSTANTIATE(2, false, 64)
SSLIC_HC_INSTANTIATE(2, false, 96)
SSLIC_HC_INSTANTIATE(2, false, 128)
