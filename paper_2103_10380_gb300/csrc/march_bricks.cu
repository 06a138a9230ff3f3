// march_bricks.cu -- the ray-march kernels for FNR_LAYOUT_BRICKS caches
// (densities and records in brick pools behind a page table; empty bricks
// skipped): march.cu's template instantiated with SKIP = BRICKS = true in a
// translation unit of its own, so the kernel sets compile in parallel.
#define FNR_MARCH_BRICKS_UNIT
#include "march.cu"
