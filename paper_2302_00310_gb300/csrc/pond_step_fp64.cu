// pond_step_fp64.cu -- the FP64 instantiations of the member step kernel.
#include "pond_step_impl.cuh"

std::vector<pond::Shape> pond_shapes_fp64(int D) { return pond::all_shapes<double>(D); }
pond::Shape pond_iter_shape_fp64(int D) { return pond::iter_shape<double>(D); }
