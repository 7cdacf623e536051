// assign_tile_f32c3_2d.cu -- tile-kernel instantiations for float images, C = 3, 2-D
// (e.g. CIE-Lab colour converted by sslic_srgb_to_lab).
#include "assign_tile.cuh"

SSLIC_TILE_INSTANTIATE(float, 3, 2)
