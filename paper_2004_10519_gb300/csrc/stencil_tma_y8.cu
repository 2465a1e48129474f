// The TMA-fed stencil passes (elastic, centred TTI) at a tile height of 8
// rows: the same source as stencil_tma.cu, compiled with WP_TILE_Y = 8.  Its
// entry points carry the suffix _y8; the autotuner picks the height per grid.
#define WP_TILE_Y 8
#include "stencil_tma.cu"
