// march_voxels.cu -- launcher of the voxel walk (FNR_RENDER_VOXELS; the
// kernel is in march_voxels.cuh) and the instantiations of its plain form.
#include "march_voxels.cuh"

namespace fnr {

cudaError_t launch_march_voxels(const MarchArgs &a, cudaStream_t s) {
    if (a.total_tiles <= 0) return cudaSuccess;
    if ((a.r.flags & FNR_RENDER_SKIP_EMPTY) == 0u) return launch_voxels_prec<kVoxPlain>(a, s);
    // the passes over empty cubes need the distance field and a walk that records no cells
    bool jump = a.c.dist != nullptr;
    for (int f = 0; f < a.n_frames; ++f)
        if (a.f[f].cells) jump = false;
    return jump ? launch_march_voxels_jump(a, s) : launch_march_voxels_skip(a, s);
}

}  // namespace fnr
