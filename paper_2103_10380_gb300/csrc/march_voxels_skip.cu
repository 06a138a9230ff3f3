// march_voxels_skip.cu -- the voxel walk's instantiations that skip the
// density loads of empty bricks (march_voxels.cuh), compiled apart from the others.
#include "march_voxels.cuh"

namespace fnr {

cudaError_t launch_march_voxels_skip(const MarchArgs &a, cudaStream_t s) { return launch_voxels_prec<kVoxSkip>(a, s); }

}  // namespace fnr
