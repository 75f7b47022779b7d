// L-BFGS column-stage kernels (every variant and radix plan) for the float working type.
#include "wf_ops_impl.cuh"

WF_INSTANTIATE_LBCOL(float)

WF_DBG_READER(lbcol_f32)
