// pond_step_fp32.cu -- the mixed-precision (FP32 + FP64 moments)
// instantiations of the member step kernel.
#include "pond_step_impl.cuh"

std::vector<pond::Shape> pond_shapes_fp32(int D) { return pond::all_shapes<float>(D); }
pond::Shape pond_iter_shape_fp32(int D) { return pond::iter_shape<float>(D); }
