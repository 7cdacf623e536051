// assign_tile_u16c1_3d.cu -- tile-kernel instantiations for uint16_t images, C = 1, 3-D.
#include "assign_tile.cuh"

SSLIC_TILE_INSTANTIATE(uint16_t, 1, 3)
