// pond_step_fp64_q5.cu -- the FP64 instantiations of the member step kernel on
// the D2Q25 f-lattice.
#include "pond_step_impl.cuh"

std::vector<pond::Shape> pond_shapes_fp64_q5() { return pond::all_shapes_q5<double>(); }
pond::Shape pond_iter_shape_fp64_q5() { return pond::iter_shape_q5<double>(); }
