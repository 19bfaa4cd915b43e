// lbm_mass_noalloc: the FP64 mass reduction without any device allocation
// and without a workspace.
//
// Who needs it: callers whose device memory is entirely owned by someone
// else (a framework's caching allocator, a serving runtime's memory pool) and
// who are not allowed to create device allocations of their own, and loops
// that cannot afford cudaMalloc's implicit device-wide synchronisation. They
// hold a population buffer and can provide one double of device memory for
// the result, but cannot hand the library a scratch workspace.
//
// The reduction needs scratch for its per-block partial sums. Here that
// scratch is a file-scope __device__ array of fixed size, which every GPU
// that loads the library keeps until the process exits. Host code cannot use
// the array's name as a device address (on the host it is only a stand-in),
// so the first call on each device, with that device current, looks up the
// device address with cudaGetSymbolAddress and caches it; later calls reuse
// it. Make that first call on a device before any stream capture begins.
//
// Every call uses the same array. Each call writes every partial slot it
// later reads, so nothing has to be cleared between calls, but two calls
// whose work overlaps on the GPU (different streams, no ordering) race on the
// array and may both return wrong sums. Order such calls on one stream.
#include <math.h>
#include <mutex>
#include <stdio.h>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kNaThreads = 256;
constexpr long long kNaCellsPerPartial = 65536;        // cells summed by one block
constexpr int kNaMaxPartials = 4096;                   // scratch slots
constexpr long long kNaMaxCells = kNaCellsPerPartial * kNaMaxPartials;  // 2^28 cells
constexpr int kNaMaxDevices = 64;

// The scratch: one partial per block. 32 KiB per device.
static __device__ __align__(256) double g_mass_scratch[kNaMaxPartials];

void* g_scratch_ptr[kNaMaxDevices] = {};
std::mutex g_scratch_mutex;

template <int S>
__global__ void __launch_bounds__(kNaThreads)
    k_mass_partial_static(const void* pops, long long N, float w0, float w1, float w2, float w3, float w4,
                          float w5, float w6, float w7, float w8, double* scratch) {
  using T = typename Store<S>::T;
  const T* p = static_cast<const T*>(pops);
  const float base[Q] = {w0, w1, w2, w3, w4, w5, w6, w7, w8};
  const long long c0 = (long long)blockIdx.x * kNaCellsPerPartial;
  const long long c1 = c0 + kNaCellsPerPartial < N ? c0 + kNaCellsPerPartial : N;
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    for (long long c = c0 + threadIdx.x; c < c1; c += kNaThreads)
      acc += (double)Store<S>::load(p, (size_t)i * N + c, base[i]);
  __shared__ double sh[kNaThreads];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kNaThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) scratch[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kNaThreads) k_mass_final_static(const double* scratch, int nparts, double* out) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < nparts; k += kNaThreads) acc += scratch[k];
  __shared__ double sh[kNaThreads];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kNaThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

void set_msg(char* err, size_t n, const char* msg) {
  if (err && n) snprintf(err, n, "%s", msg);
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lbm_mass_noalloc(const void* d_pops, int32_t nx, int32_t ny, int32_t storage, double rho_ref,
                                void* cuda_stream, double* d_out, char* err, size_t err_len) {
  set_msg(err, err_len, "");
  if (!d_pops || !d_out) return set_msg(err, err_len, "d_pops and d_out must be device pointers"), LBM_EINVAL;
  if (nx < 1 || ny < 1) return set_msg(err, err_len, "nx and ny must be >= 1"), LBM_EINVAL;
  if (storage < LBM_F32 || storage > LBM_BF16_DEV) return set_msg(err, err_len, "bad storage"), LBM_EINVAL;
  if (!isfinite(rho_ref)) return set_msg(err, err_len, "rho_ref must be finite"), LBM_EINVAL;
  const long long N = (long long)nx * ny;
  if (N > kNaMaxCells) {
    char m[160];
    snprintf(m, sizeof(m), "box of %lld cells exceeds the static scratch limit of %lld cells", N, kNaMaxCells);
    return set_msg(err, err_len, m), LBM_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
    return set_msg(err, err_len, "no usable current CUDA device"), LBM_ECUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_mass_scratch);
      if (e != cudaSuccess || !ptr) {
        set_msg(err, err_len, cudaGetErrorString(e));
        return LBM_ECUDA;
      }
      g_scratch_ptr[dev] = ptr;
    }
    scratch = g_scratch_ptr[dev];
  }
  float wref[Q];
  for (int i = 0; i < Q; ++i) wref[i] = storage == LBM_F32 ? 0.0f : (float)(wq(i) * rho_ref);
  const int nparts = (int)((N + kNaCellsPerPartial - 1) / kNaCellsPerPartial);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  double* sp = static_cast<double*>(scratch);
  switch (storage) {
    case LBM_F32:
      k_mass_partial_static<LBM_F32><<<nparts, kNaThreads, 0, s>>>(d_pops, N, wref[0], wref[1], wref[2], wref[3],
                                                                   wref[4], wref[5], wref[6], wref[7], wref[8], sp);
      break;
    case LBM_F16_DEV:
      k_mass_partial_static<LBM_F16_DEV><<<nparts, kNaThreads, 0, s>>>(d_pops, N, wref[0], wref[1], wref[2],
                                                                       wref[3], wref[4], wref[5], wref[6], wref[7],
                                                                       wref[8], sp);
      break;
    default:
      k_mass_partial_static<LBM_BF16_DEV><<<nparts, kNaThreads, 0, s>>>(d_pops, N, wref[0], wref[1], wref[2],
                                                                        wref[3], wref[4], wref[5], wref[6], wref[7],
                                                                        wref[8], sp);
      break;
  }
  k_mass_final_static<<<1, kNaThreads, 0, s>>>(sp, nparts, d_out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_msg(err, err_len, cudaGetErrorString(e)), LBM_ECUDA;
  return LBM_OK;
}
