// FP32-pair instantiation of the iteration kernels: complex vectors stored as
// (hi, lo) FP32 pairs and computed with error-free FP32 transformations (48-bit
// significand on the FP32 pipes); FP64 scalars.
#include "kw_kernels.cuh"

namespace kw {
template cudaError_t launch_init<PREC_DF>(Work&);
template cudaError_t launch_iteration<PREC_DF>(Work&, int, int, cudaEvent_t*, int64_t*);
template cudaError_t launch_finish_x<PREC_DF>(Work&);
template cudaError_t launch_unfinish_x<PREC_DF>(Work&);
template cudaError_t launch_k1<PREC_DF>(Work&, void*, void*);
template cudaError_t launch_update_xp<PREC_DF>(Work&, const void*, State*, int, cudaStream_t);
template cudaError_t launch_project_x<PREC_DF>(Work&, double2*);
template cudaError_t launch_spmv_dot<PREC_DF>(Work&, const void*, void*, double2, float4, double2*);

}  // namespace kw
