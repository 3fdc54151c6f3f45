// dg_row3d_f32_tiles.cu -- tile variants 1 and 2 of the 3D FP32 row kernels (the default
// tiles are in dg_row3d_f32.cu); the autotuner of dg_graph_create picks
// among them per degree.
#include "dg_launch.cuh"

namespace dg {

template int launch_row_tile<3, 2, float, 1>(const DevMesh&, int, float*, float*, int, const LaunchOpts&,
                                                       Tracer*, int);
template int launch_row_tile<3, 3, float, 1>(const DevMesh&, int, float*, float*, int, const LaunchOpts&,
                                                       Tracer*, int);
template int launch_row_tile<3, 3, float, 2>(const DevMesh&, int, float*, float*, int, const LaunchOpts&,
                                                       Tracer*, int);
}  // namespace dg
