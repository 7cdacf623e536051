// assign_tile_u8c3_3d.cu -- tile-kernel instantiations for uint8_t images, C = 3, 3-D.
#include "assign_tile.cuh"

SSLIC_TILE_INSTANTIATE(uint8_t, 3, 3)
