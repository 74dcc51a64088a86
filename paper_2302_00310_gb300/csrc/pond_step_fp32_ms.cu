// pond_step_fp32_ms.cu -- the mixed-precision instantiations of the member
// step kernel with the multiscale f-lattice.
#include "pond_step_impl.cuh"

pond::Shape pond_ms_shape_fp32(int D) { return pond::ms_shape<float>(D); }
