// FP64 instantiation of the iteration kernels (complex FP64 vectors and values).
#include "kw_kernels.cuh"

namespace kw {
template cudaError_t launch_init<PREC_F64>(Work&);
template cudaError_t launch_iteration<PREC_F64>(Work&, int, cudaEvent_t*, int64_t*);
template cudaError_t launch_finish_x<PREC_F64>(Work&);
template cudaError_t launch_project_x<PREC_F64>(Work&, double2*);
template cudaError_t launch_spmv_dot<PREC_F64>(Work&, const void*, void*, double2, float4, double2*);

cudaError_t launch_convert_f64_to_f32(const double* in, float* out, int64_t n, unsigned long long* inexact,
                                      cudaStream_t s) {
  k_f64_to_f32<<<1024, 256, 0, s>>>(in, out, n, inexact);
  return cudaGetLastError();
}

cudaError_t launch_convert_f64_to_pair(const double* in, void* out, int64_t n, cudaStream_t s) {
  k_f64_to_pair<<<1024, 256, 0, s>>>(in, (df*)out, n);
  return cudaGetLastError();
}
}  // namespace kw
