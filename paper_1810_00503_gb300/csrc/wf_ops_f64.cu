// Operator kernels and launchers instantiated for the double working type.
#include "wf_ops_impl.cuh"

WF_INSTANTIATE_OPS(double)

WF_DBG_READER(ops_f64)
