// pond_step_fp64_ms.cu -- the FP64 instantiations of the member step kernel
// with the multiscale f-lattice.
#include "pond_step_impl.cuh"

pond::Shape pond_ms_shape_fp64(int D) { return pond::ms_shape<double>(D); }
