// Variable-coefficient launches, 3D.
#include "launch_var.cuh"

namespace afg {
AFG_VAR_LAUNCHES(3)
}  // namespace afg
