// assign_tile_u8c3_2d.cu -- tile-kernel instantiations for uint8_t images, C = 3, 2-D.
#include "assign_tile.cuh"

SSLIC_TILE_INSTANTIATE(uint8_t, 3, 2)
