// dg_row2d_f32_tiles1.cu -- tile variants 1 of the 2D FP32 row kernels (the default
// tiles are in dg_row2d_f32.cu); the autotuner of dg_graph_create picks
// among them per degree.
#include "dg_launch.cuh"

namespace dg {

template int launch_row_tile<2, 3, float, 1>(const DevMesh&, int, float*, float*, int, const LaunchOpts&,
                                                       Tracer*, int);
template int launch_row_tile<2, 4, float, 1>(const DevMesh&, int, float*, float*, int, const LaunchOpts&,
                                                       Tracer*, int);
template int launch_row_tile<2, 5, float, 1>(const DevMesh&, int, float*, float*, int, const LaunchOpts&,
                                                       Tracer*, int);
template int launch_row_tile<2, 6, float, 1>(const DevMesh&, int, float*, float*, int, const LaunchOpts&,
                                                       Tracer*, int);
}  // namespace dg
