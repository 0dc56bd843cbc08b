// 3D double launches of the launch layer (and the kernels they instantiate).
#include "launch_impl.cuh"
namespace afg {
template struct PrecOps<3, double>;
}
