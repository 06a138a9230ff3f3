// march_skip.cu -- the ray-march kernels with empty-space skipping
// (FNR_RENDER_SKIP_EMPTY): march.cu's template instantiated with SKIP = true
// in a translation unit of its own, so both kernel sets compile in parallel.
#define FNR_MARCH_SKIP_UNIT
#include "march.cu"
