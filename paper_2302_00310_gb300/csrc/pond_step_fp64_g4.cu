// pond_step_fp64_g4.cu -- the FP64 instantiations of the member step kernel
// with the g-populations on the f-lattice (D1Q4 / D2Q16).
#include "pond_step_impl.cuh"

pond::Shape pond_g4_shape_fp64(int D) { return pond::g4_shape<double>(D); }
