// L-BFGS column-stage kernels (every variant and radix plan) for the double working type.
#include "wf_ops_impl.cuh"

WF_INSTANTIATE_LBCOL(double)

WF_DBG_READER(lbcol_f64)
