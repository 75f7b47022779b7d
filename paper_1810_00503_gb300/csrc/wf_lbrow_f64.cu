// L-BFGS row-stage and streaming kernels for the double working type.
#include "wf_ops_impl.cuh"

WF_INSTANTIATE_LBROW(double)

WF_DBG_READER(lbrow_f64)
