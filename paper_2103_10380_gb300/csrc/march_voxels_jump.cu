// march_voxels_jump.cu -- the voxel walk's instantiations with the one-step
// passes over empty cubes (march_voxels.cuh), compiled apart from the others.
#include "march_voxels.cuh"

namespace fnr {

cudaError_t launch_march_voxels_jump(const MarchArgs &a, cudaStream_t s) { return launch_voxels_prec<kVoxJump>(a, s); }

}  // namespace fnr
