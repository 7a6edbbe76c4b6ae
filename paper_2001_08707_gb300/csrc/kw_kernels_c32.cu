// Complex-FP32-vector instantiation of the iteration kernels (FP32 vectors and
// matrix values; FP64 scalars, FP64 accumulation across FP32 chunk partials).
#include "kw_kernels.cuh"

namespace kw {
template cudaError_t launch_init<PREC_C32>(Work&);
template cudaError_t launch_iteration<PREC_C32>(Work&, int, int, cudaEvent_t*, int64_t*);
template cudaError_t launch_finish_x<PREC_C32>(Work&);
template cudaError_t launch_unfinish_x<PREC_C32>(Work&);
template cudaError_t launch_k1<PREC_C32>(Work&, void*, void*);
template cudaError_t launch_update_xp<PREC_C32>(Work&, const void*, State*, int, cudaStream_t);
template cudaError_t launch_project_x<PREC_C32>(Work&, double2*);
template cudaError_t launch_spmv_dot<PREC_C32>(Work&, const void*, void*, double2, float4, double2*);

}  // namespace kw
