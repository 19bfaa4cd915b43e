// Nucleation and bubble growth (Sec. 2.1.3; main flowchart boxes "Random
// Nucleation" and "Bubble growth").
//
// Growth: the paper adds the released hydrogen to every gas point as a
// pressure increment, dp/dt = A (dn/dt) / N (Eq. 34). The increment is taken
// on the ideal-gas part of the equation of state (dp = c_s^2 drho), so a
// release is a density source split equally over the N gas points of the
// latest census and added at rest to their post-collision populations:
// f_i^out(x) += w_i drho. Buffer convention: the buffer a step writes holds
// f_i^out(x) at x (the next step pulls it from x + e_i).
//
// Nucleation: cells within a nucleus radius become gas at rest, incoming
// f_i(x) = w_i rho_g, i.e. B_i(x - e_i) in the buffer the next step reads.
#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kThreadsG = 256;

struct FieldWref {
  float w[Q];  // w_i rho_ref of 16-bit deviations (0 for FP32)
};

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__global__ void k_gas_census(const float* __restrict__ rho, long long N, float th, int32_t* __restrict__ list,
                             int* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  // every lane of a warp runs the same number of iterations (bounds tested inside)
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long c0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); c0 < N; c0 += stride) {
    const long long c = c0 + lane;
    const bool gas = c < N && rho[c] < th;
    const unsigned b = __ballot_sync(0xffffffffu, gas);
    if (!b) continue;
    int base = 0;
    if (lane == 0) base = atomicAdd(count, __popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (gas) list[base + __popc(b & ((1u << lane) - 1u))] = (int32_t)c;
  }
}

template <int S>
__global__ void k_growth(typename Store<S>::T* __restrict__ pops, const int32_t* __restrict__ list,
                         const int* __restrict__ count, long long N, double rate, double budget,
                         double* __restrict__ released, int parity) {
  const int n = *count;
  const double before = released[parity];
  double release = 0.0;
  if (n > 0) {
    const double left = budget - before;
    release = rate < left ? rate : left;
    if (!(release > 0.0)) release = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) released[parity ^ 1] = before + release;
  if (release == 0.0) return;
  const double drho = release / (double)n;
  float add[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) add[i] = (float)(wq(i) * drho);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const size_t c = (size_t)list[k];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const size_t idx = (size_t)i * N + c;
      Store<S>::store_raw(pops, idx, __fadd_rn(Store<S>::raw(pops, idx), add[i]));
    }
  }
}

// Inside test of one cell against the nuclei, in FP64 without contraction
// (the same decision as the oracle's plain expression).
__device__ __forceinline__ bool in_nucleus(const lbm_bubble* __restrict__ nu, int n, int x, int y, int nx,
                                           int ny) {
  for (int k = 0; k < n; ++k) {
    double dx = fabs((double)x - nu[k].cx), dy = fabs((double)y - nu[k].cy);
    dx = fmin(dx, __dsub_rn((double)nx, dx));
    dy = fmin(dy, __dsub_rn((double)ny, dy));
    if (__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= __dmul_rn(nu[k].r, nu[k].r)) return true;
  }
  return false;
}

template <int S>
__global__ void k_nucleate(typename Store<S>::T* __restrict__ pops, const lbm_bubble* __restrict__ nu, int n,
                           double rho_g, int nx, int ny, FieldWref wr) {
  const long long N = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)(c / nx);
    if (!in_nucleus(nu, n, x, y, nx, ny)) continue;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      // incoming f_i(x) lives at B_i(x - e_i)
      const long long src = (long long)wrap1(y - cy(i), ny) * nx + wrap1(x - cx(i), nx);
      Store<S>::store(pops, (size_t)i * N + src, (float)(wq(i) * rho_g), wr.w[i]);
    }
  }
}

unsigned grid_for(long long n) {
  long long b = (n + kThreadsG - 1) / kThreadsG;
  if (b > device_sm_count() * 8LL) b = device_sm_count() * 8LL;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_gas_census(const float* rho, long long N, float threshold, int32_t* list, int* count,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_gas_census<<<grid_for(N), kThreadsG, 0, s>>>(rho, N, threshold, list, count);
  return cudaGetLastError();
}

cudaError_t launch_growth(int storage, void* pops, const int32_t* list, const int* count, long long N,
                          double rate, double budget, double* released, int parity, cudaStream_t s) {
  const unsigned g = (unsigned)device_sm_count() * 4;
  switch (storage) {
    case LBM_F32:
      k_growth<LBM_F32><<<g, kThreadsG, 0, s>>>(static_cast<float*>(pops), list, count, N, rate, budget, released,
                                                parity);
      break;
    case LBM_F16_DEV:
      k_growth<LBM_F16_DEV><<<g, kThreadsG, 0, s>>>(static_cast<__half*>(pops), list, count, N, rate, budget,
                                                    released, parity);
      break;
    case LBM_BF16_DEV:
      k_growth<LBM_BF16_DEV><<<g, kThreadsG, 0, s>>>(static_cast<__nv_bfloat16*>(pops), list, count, N, rate,
                                                     budget, released, parity);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_nucleate(int storage, void* pops, const lbm_bubble* nuclei, int n, double rho_g, int nx,
                            int ny, const float* wref, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  FieldWref wr;
  for (int i = 0; i < Q; ++i) wr.w[i] = wref[i];
  const unsigned g = grid_for((long long)nx * ny);
  switch (storage) {
    case LBM_F32:
      k_nucleate<LBM_F32><<<g, kThreadsG, 0, s>>>(static_cast<float*>(pops), nuclei, n, rho_g, nx, ny, wr);
      break;
    case LBM_F16_DEV:
      k_nucleate<LBM_F16_DEV><<<g, kThreadsG, 0, s>>>(static_cast<__half*>(pops), nuclei, n, rho_g, nx, ny, wr);
      break;
    case LBM_BF16_DEV:
      k_nucleate<LBM_BF16_DEV><<<g, kThreadsG, 0, s>>>(static_cast<__nv_bfloat16*>(pops), nuclei, n, rho_g, nx,
                                                       ny, wr);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
