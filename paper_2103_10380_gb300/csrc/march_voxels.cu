// march_voxels.cu -- launcher of the voxel walk (FNR_RENDER_VOXELS; the
// kernel is in march_voxels.cuh) and its instantiations without the one-step
// passes over empty cubes.
#include "march_voxels.cuh"

namespace fnr {

cudaError_t launch_march_voxels(const MarchArgs &a, cudaStream_t s) {
    if (a.total_tiles <= 0) return cudaSuccess;
    // the passes over empty cubes need the distance field and a walk that records no cells
    bool jump = (a.r.flags & FNR_RENDER_SKIP_EMPTY) != 0u && a.c.dist != nullptr;
    for (int f = 0; f < a.n_frames; ++f)
        if (a.f[f].cells) jump = false;
    return jump ? launch_march_voxels_jump(a, s) : launch_voxels_prec<false>(a, s);
}

}  // namespace fnr
