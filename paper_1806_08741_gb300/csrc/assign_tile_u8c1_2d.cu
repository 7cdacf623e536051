// assign_tile_u8c1_2d.cu -- tile-kernel instantiations for uint8_t images, C = 1, 2-D.
#include "assign_tile.cuh"

SSLIC_TILE_INSTANTIATE(uint8_t, 1, 2)
