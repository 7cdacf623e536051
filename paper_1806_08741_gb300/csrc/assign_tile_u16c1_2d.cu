// assign_tile_u16c1_2d.cu -- tile-kernel instantiations for uint16_t images, C = 1, 2-D.
#include "assign_tile.cuh"

SSLIC_TILE_INSTANTIATE(uint16_t, 1, 2)
