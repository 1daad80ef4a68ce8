// Host entry points of the mesh voxelizer (voxelize.cu).
#pragma once

#include "vct_internal.cuh"

namespace vct {

size_t voxelize_workspace_bytes(int n, int n_triangles);
cudaError_t launch_voxelize(const vct_mesh &m, int n, const float origin[3], float size,
                            const vct_voxel_light &light, float *out, void *ws, int sms,
                            cudaStream_t s);

}  // namespace vct
