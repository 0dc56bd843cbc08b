// 2D instantiations of the launch layer.
#include "launch_impl.cuh"
namespace afg {
template struct DimOps<2>;
}
