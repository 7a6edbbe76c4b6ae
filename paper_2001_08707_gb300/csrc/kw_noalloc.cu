// kw_spmv_dot_noalloc: the seed SpMV + r^T q step without any device allocation.
//
// Some callers cannot call cudaMalloc: code whose device memory is entirely
// owned by another allocator (a framework's caching pool that has reserved the
// GPU, or a fixed memory budget), and latency-critical loops that cannot pay
// for cudaMalloc's implicit device synchronisation.  This entry point needs no
// context and allocates nothing: its scratch (one FP64 partial per thread
// block, the arrival counter of the last-block reduction and the result) lives
// in the file-scope array below, which every GPU that loads this library keeps
// until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "komega_gb300.h"
#include "kw_kernels.cuh"

namespace {

// Layout of the scratch: [State | result double2 | partials 2 doubles per block].
constexpr size_t kStateBytes = (sizeof(kw::State) + 255) / 256 * 256;
constexpr size_t kResultBytes = 256;
constexpr size_t kPartBytes = (size_t)KW_NOALLOC_MAX_BLOCKS * 2 * sizeof(double);
constexpr size_t kScratchBytes = kStateBytes + kResultBytes + kPartBytes;

static __device__ __align__(256) unsigned char kw_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};
int g_resident[kMaxDevices] = {};

// Once per device, with that device current: the device address of the scratch
// array (in host code its name is only a host-side stand-in), the SM count and
// how many K1 blocks fit at once.
kw_status setup(int dev, void** addr, int* grid_cap) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, kw_noalloc_scratch) != cudaSuccess || !p) return KW_ERR_CUDA;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return KW_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kw::k_spmv_dot<kw::PREC_F64, double, 1>, 256, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    g_sms[dev] = sms;
    g_resident[dev] = per_sm * sms;
    g_addr[dev] = p;
  }
  *addr = g_addr[dev];
  *grid_cap = std::min(g_resident[dev], KW_NOALLOC_MAX_BLOCKS);
  return KW_OK;
}

}  // namespace

extern "C" kw_status kw_spmv_dot_noalloc(int64_t m, int64_t nnz, const int64_t* rowptr_dev, const int32_t* col_dev,
                                         const double* val_dev, kw_c128 zs, const kw_c128* r_dev, kw_c128* q_dev,
                                         kw_c128* t_host, void* cuda_stream) {
  if (m < 1 || m > KW_MAX_ROWS || nnz < 0 || nnz > KW_MAX_NNZ) return KW_ERR_ARG;
  if (!rowptr_dev || (nnz > 0 && (!col_dev || !val_dev)) || !r_dev || !q_dev || !t_host) return KW_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KW_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return KW_ERR_ARG;
  void* base = nullptr;
  int cap = 0;
  kw_status s = setup(dev, &base, &cap);
  if (s != KW_OK) return s;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  unsigned char* b = (unsigned char*)base;
  kw::State* st = (kw::State*)b;
  double2* result = (double2*)(b + kStateBytes);
  double* part = (double*)(b + kStateBytes + kResultBytes);
  // The arrival counter must start at zero; partials are written before they are read.
  if (cudaMemsetAsync(&st->cnt_spmv, 0, sizeof(unsigned int), stream) != cudaSuccess) return KW_ERR_CUDA;
  const int need = (int)((m + 255) / 256);
  const int grid = std::max(1, std::min(cap, need));
  kw::SpmvMode mode;
  mode.solver = 0;
  mode.zs = make_double2(zs.re, zs.im);
  mode.zs_pair = make_float4(0.f, 0.f, 0.f, 0.f);   // unused in the FP64 form
  mode.t_out = result;
  kw::k_spmv_dot<kw::PREC_F64, double, 1><<<grid, 256, 0, stream>>>(
      (int)m, rowptr_dev, col_dev, val_dev, (const double2*)r_dev, (double2*)q_dev, st, part, mode);
  if (cudaGetLastError() != cudaSuccess) return KW_ERR_CUDA;
  if (cudaMemcpyAsync(t_host, result, sizeof(kw_c128), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
    return KW_ERR_CUDA;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return KW_ERR_CUDA;
  return KW_OK;
}
