// 3D instantiations of the launch layer: the dispatch here, the
// precision-specific launches (and their kernels) in launch_d3_f64.cu and
// launch_d3_f32.cu, so that the three compile in parallel.
#include "launch_impl.cuh"
namespace afg {
extern template struct PrecOps<3, double>;
extern template struct PrecOps<3, float>;
template struct DimOps<3>;
}
