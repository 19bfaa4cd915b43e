// Fused time step of the extended Shan-Chen lattice Boltzmann method
// (arXiv 1708.01613): pull streaming (Sec. 2.1.1, Eq. 19), moments (Eq. 11),
// pseudopotential (Sec. 2.1.2, Eq. 30), masked neighbour-sum force (Eq. 22;
// barrier of Sec. 2.1.5), velocity-shift equilibrium (Eqs. 39-40 with
// Eq. 14) and BGK collision (Eq. 18), in one pass over the populations.
//
// Layout: structure of arrays, plane i at offset i*N, row-major, x fastest.
// The buffer read by a step holds the post-collision populations of the
// previous step at their source cell; the step pulls f_i(x) from x - e_i.
//
// Geometry: a CTA owns a strip of BX consecutive columns and marches down
// rows_per_chunk rows. For every row it pulls the populations of its cells
// (plus one halo column each side), forms rho and psi once per cell, and
// writes psi into a four-row ring in shared memory. One barrier later the
// ring holds psi for rows r-2..r, so the force and collision of row r-1 can
// run on the populations kept in registers from the previous iteration. The
// only re-read of populations is the halo (two columns per strip, two rows
// per chunk), which hits L2.
#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kBX = 256;

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

template <int S>
__device__ __forceinline__ void pull_cell(const typename Store<S>::T* __restrict__ src,
                                          const StepParams& p, long long rowm, long long row0,
                                          long long rowp, int xm, int x, int xp, float f[Q]) {
  // f_i(x, r) = f_i^out(x - c_i, r - c_iy): rows r-1 (c_y = +1), r, r+1 (c_y = -1)
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const long long row = cy(i) > 0 ? rowm : (cy(i) < 0 ? rowp : row0);
    const int xs = cx(i) > 0 ? xm : (cx(i) < 0 ? xp : x);
    f[i] = Store<S>::load(src, (size_t)i * p.N + row + xs, p.wref[i]);
  }
}

__device__ __forceinline__ float psi_of(float rho, const StepParams& p) {
  return p.rho0 * (1.0f - expf(-rho * p.inv_rho0));
}

template <int S, bool MASKED>
__global__ void __launch_bounds__(kBX) k_step_strip(const StepParams p) {
  using T = typename Store<S>::T;
  const T* __restrict__ src = static_cast<const T*>(p.src);
  T* __restrict__ dst = static_cast<T*>(p.dst);
  __shared__ float ring[4][kBX + 2];

  const int nx = p.nx, ny = p.ny;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kBX;
  const int x = x0 + tid;
  const bool active = x < nx;
  const int last = min(x0 + kBX, nx) - 1;
  const int y0 = blockIdx.y * p.rows_per_chunk;
  const int y1 = min(y0 + p.rows_per_chunk, ny);
  if (y0 >= y1) return;  // uniform over the block

  const int xc = active ? x : last;
  const int xm = wrapi(xc - 1, nx), xp = wrapi(xc + 1, nx);
  const bool do_left = tid == 0;
  const bool do_right = x == last;
  const int xl = wrapi(x0 - 1, nx), xlm = wrapi(x0 - 2, nx);
  const int xr = wrapi(last + 1, nx), xrp = wrapi(last + 2, nx);
  const int jc = tid + 1;

  float fprev[Q];
  float rho_prev = 1.f, jx_prev = 0.f, jy_prev = 0.f;
  int bad = 0;

  for (int r = y0 - 1, k = 0; r <= y1; ++r, ++k) {
    const int rr = wrapi(r, ny);
    const long long row0 = (long long)rr * nx;
    const long long rowm = (long long)wrapi(rr - 1, ny) * nx;
    const long long rowp = (long long)wrapi(rr + 1, ny) * nx;
    const int slot = k & 3;
    float f[Q];
    float rho = 1.f, jx = 0.f, jy = 0.f;
    if (active) {
      pull_cell<S>(src, p, rowm, row0, rowp, xm, x, xp, f);
      rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
      jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
      jy = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
      ring[slot][jc] = psi_of(rho, p);
    }
    if (do_left) {
      float h[Q];
      pull_cell<S>(src, p, rowm, row0, rowp, xlm, xl, x0 == 0 ? wrapi(x0, nx) : x0, h);
      const float rh = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
      ring[slot][0] = psi_of(rh, p);
    }
    if (do_right) {
      float h[Q];
      pull_cell<S>(src, p, rowm, row0, rowp, last, xr, xrp, h);
      const float rh = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
      ring[slot][last - x0 + 2] = psi_of(rh, p);
    }
    __syncthreads();
    if (k >= 2 && active) {
      // force, equilibrium and collision of row rc = r - 1
      const int rc = r - 1;
      const int sm = (k - 2) & 3, s0 = (k - 1) & 3, sp = k & 3;
      const float psi_c = ring[s0][jc];
      float sx = 0.f, sy = 0.f;
      unsigned m = 0;
      if (MASKED) m = p.mask[(size_t)rc * nx + x];
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int sl = cy(i) > 0 ? sp : (cy(i) < 0 ? sm : s0);
        float s = ring[sl][jc + cx(i)];
        if (MASKED && ((m >> (i - 1)) & 1u)) s = psi_c;
        const float ws = static_cast<float>(wq(i)) * s;
        if (cx(i) != 0) sx += cx(i) > 0 ? ws : -ws;
        if (cy(i) != 0) sy += cy(i) > 0 ? ws : -ws;
      }
      const float Fx = -p.G * psi_c * sx;
      const float Fy = -p.G * psi_c * sy;
      const float inv_rho = 1.0f / rho_prev;
      const float ux = (jx_prev + p.tau * Fx) * inv_rho;
      const float uy = (jy_prev + p.tau * Fy) * inv_rho;
      const float uu = 1.5f * (ux * ux + uy * uy);
      bad |= !(rho_prev > 0.f) | !(fabsf(ux) + fabsf(uy) < 1e30f);
      const long long base = (long long)rc * nx + x;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const float eu = cx(i) * ux + cy(i) * uy;
        const float feq = static_cast<float>(wq(i)) * rho_prev * (1.0f + 3.0f * eu + 4.5f * eu * eu - uu);
        const float fo = fprev[i] + (feq - fprev[i]) * p.inv_tau;
        Store<S>::store(dst, (size_t)i * p.N + base, fo, p.wref[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) fprev[i] = f[i];
    rho_prev = rho;
    jx_prev = jx;
    jy_prev = jy;
  }
  if (bad) atomicOr(p.flags + FLAG_NUMERIC, 1);
}

template <int S>
cudaError_t launch_typed(const StepParams& p, cudaStream_t s) {
  int gx, gy, rows, block;
  step_geometry(p.nx, p.ny, &gx, &gy, &rows, &block);
  StepParams q = p;
  q.rows_per_chunk = rows;
  dim3 grid(gx, gy);
  if (p.mask)
    k_step_strip<S, true><<<grid, block, 0, s>>>(q);
  else
    k_step_strip<S, false><<<grid, block, 0, s>>>(q);
  return cudaGetLastError();
}

}  // namespace

void step_geometry(int nx, int ny, int* grid_x, int* grid_y, int* rows_per_chunk, int* block) {
  const int gx = (nx + kBX - 1) / kBX;
  const int target = 152 * 6;  // CTAs: a few per SM
  int gy = (target + gx - 1) / gx;
  if (gy > ny) gy = ny;
  if (gy < 1) gy = 1;
  int rows = (ny + gy - 1) / gy;
  gy = (ny + rows - 1) / rows;
  *grid_x = gx;
  *grid_y = gy;
  *rows_per_chunk = rows;
  *block = kBX;
}

cudaError_t launch_step(int storage, const StepParams& p, cudaStream_t s) {
  switch (storage) {
    case LBM_F32: return launch_typed<LBM_F32>(p, s);
    case LBM_F16_DEV: return launch_typed<LBM_F16_DEV>(p, s);
    case LBM_BF16_DEV: return launch_typed<LBM_BF16_DEV>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
