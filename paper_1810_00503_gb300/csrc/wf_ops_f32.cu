// Operator kernels and launchers instantiated for the float working type.
#include "wf_ops_impl.cuh"

WF_INSTANTIATE_OPS(float)

WF_DBG_READER(ops_f32)
