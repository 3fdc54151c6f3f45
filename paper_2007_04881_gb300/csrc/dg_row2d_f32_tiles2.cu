// dg_row2d_f32_tiles2.cu -- tile variants 2 of the 2D FP32 row kernels (the default
// tiles are in dg_row2d_f32.cu); the autotuner of dg_graph_create picks
// among them per degree.
#include "dg_launch.cuh"

namespace dg {

template int launch_row_tile<2, 4, float, 2>(const DevMesh&, int, float*, float*, int, const LaunchOpts&,
                                                       Tracer*, int);
template int launch_row_tile<2, 5, float, 2>(const DevMesh&, int, float*, float*, int, const LaunchOpts&,
                                                       Tracer*, int);
}  // namespace dg
