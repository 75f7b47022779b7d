// L-BFGS row-stage and streaming kernels for the float working type.
#include "wf_ops_impl.cuh"

WF_INSTANTIATE_LBROW(float)

WF_DBG_READER(lbrow_f32)
