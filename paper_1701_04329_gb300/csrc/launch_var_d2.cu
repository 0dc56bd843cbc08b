// Variable-coefficient launches, 2D.
#include "launch_var.cuh"

namespace afg {
AFG_VAR_LAUNCHES(2)
}  // namespace afg
