// 2D instantiations of the launch layer: the dispatch here, the
// precision-specific launches (and their kernels) in launch_d2_f64.cu and
// launch_d2_f32.cu, so that the three compile in parallel.
#include "launch_impl.cuh"
namespace afg {
extern template struct PrecOps<2, double>;
extern template struct PrecOps<2, float>;
template struct DimOps<2>;
}
