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

// ---------------------------------------------------------------------------
// TMA-staged variant. The same strip/row march, but the populations of each
// output row (for plane i: source row r - c_iy, columns x0 - PAD .. x0 + W +
// PAD, wrapped) are brought into a ring of NSTAGE shared-memory stages by
// cp.async.bulk copies that one thread issues NSTAGE - 2 rows ahead; an
// mbarrier per stage counts the bytes in. Every thread then reads its pulls
// from shared memory, so the number of bytes in flight no longer depends on
// occupancy. Halo columns arrive inside the same copies. Needs nx % 16 == 0
// and nx >= W + 2 PAD (16-byte aligned, at most two pieces per row copy).

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: false if the phase did not complete within `limit_ns`.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = 2000000000ull) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (global_ns() - t0 < limit_ns)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

template <int S>
struct TmaGeom {
  using T = typename Store<S>::T;
  static constexpr int E = sizeof(T);
  static constexpr int PAD = 16 / E;             // halo pad in elements: 16 bytes
  static constexpr int WIN = kBX + 2 * PAD;      // elements per staged plane row
  static constexpr int ROW_BYTES = WIN * E;      // multiple of 16
};

// Copy `len` elements of a periodic row starting at column `start` (may be
// negative) into dst: one or two pieces.
template <typename T>
__device__ __forceinline__ void copy_row_wrapped(T* dst, const T* row, int start, int len, int nx,
                                                 uint64_t* bar) {
  int s0 = start < 0 ? start + nx : start;
  const int first = min(len, nx - s0);
  bulk_g2s(dst, row + s0, (uint32_t)(first * sizeof(T)), bar);
  if (first < len) bulk_g2s(dst + first, row, (uint32_t)((len - first) * sizeof(T)), bar);
}

template <int S, bool MASKED, int NSTAGE>
__device__ __forceinline__ void issue_stage(const StepParams& p, const typename Store<S>::T* src,
                                            unsigned char* stages, uint64_t* bars, int k, int y0, int x0) {
  using G = TmaGeom<S>;
  using T = typename G::T;
  constexpr uint32_t STAGE_BYTES = Q * G::ROW_BYTES + (MASKED ? kBX : 0);
  const int slot = k % NSTAGE;
  unsigned char* st = stages + (size_t)slot * STAGE_BYTES;
  uint64_t* bar = bars + slot;
  const int r = y0 - 1 + k;
  const int ny = p.ny, nx = p.nx;
  mbar_expect_tx(bar, STAGE_BYTES);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    int g = r - cy(i);
    g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
    g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
    const T* row = src + (size_t)i * p.N + (size_t)g * nx;
    copy_row_wrapped<T>(reinterpret_cast<T*>(st + i * G::ROW_BYTES), row, x0 - G::PAD, G::WIN, nx, bar);
  }
  if (MASKED) {  // columns x0 .. x0 + W (a ragged last strip wraps; those bytes are unused)
    int g = r < 0 ? r + ny : (r >= ny ? r - ny : r);
    copy_row_wrapped<uint8_t>(st + Q * G::ROW_BYTES, p.mask + (size_t)g * nx, x0, kBX, nx, bar);
  }
}

template <int S, bool MASKED, int NSTAGE, int MINB>
__global__ void __launch_bounds__(kBX, MINB) k_step_tma(const StepParams p) {
  using G = TmaGeom<S>;
  using T = typename G::T;
  constexpr int STAGE_BYTES = Q * G::ROW_BYTES + (MASKED ? kBX : 0);
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* stages = smem;
  float(*ring)[kBX + 2] = reinterpret_cast<float(*)[kBX + 2]>(smem + (size_t)NSTAGE * STAGE_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)NSTAGE * STAGE_BYTES + 4 * (kBX + 2) * 4);
  int* abort_flag = reinterpret_cast<int*>(bars + NSTAGE);

  const T* __restrict__ src = static_cast<const T*>(p.src);
  T* __restrict__ dst = static_cast<T*>(p.dst);
  const int nx = p.nx, ny = p.ny;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kBX;
  const int width = min(kBX, nx - x0);  // active columns of this strip
  const bool active = tid < width;
  const int y0 = blockIdx.y * p.rows_per_chunk;
  const int y1 = min(y0 + p.rows_per_chunk, ny);
  if (y0 >= y1) return;
  const int nst = (y1 - y0) + 2;  // stages: rows y0-1 .. y1

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(bars + s, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < NSTAGE - 2 && k < nst; ++k) issue_stage<S, MASKED, NSTAGE>(p, src, stages, bars, k, y0, x0);

  const int jc = tid + 1;
  const int pos = G::PAD + tid;  // window position of this thread's cell
  float rho_prev = 1.f, jx_prev = 0.f, jy_prev = 0.f;
  int bad = 0;
  int k_abort = 0;
  for (int k = 0; k < nst; ++k) {
    const int slot = k % NSTAGE;
    const unsigned char* st = stages + (size_t)slot * STAGE_BYTES;
    if (!mbar_wait(bars + slot, (uint32_t)((k / NSTAGE) & 1))) *abort_flag = 1;
    float rho = 1.f, jx = 0.f, jy = 0.f;
    {
      float f[Q];
      if (active) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
          f[i] = Store<S>::load_smem(reinterpret_cast<const T*>(st + i * G::ROW_BYTES), pos - cx(i), p.wref[i]);
        rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
        jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
        jy = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
        ring[k & 3][jc] = psi_of(rho, p);
      }
      // halo cells: column x0 - 1 (window PAD - 1) and x0 + width (window PAD + width)
      if (tid == 0 || tid == width - 1) {
        const int hp = tid == 0 ? G::PAD - 1 : G::PAD + width;
        float h[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i)
          h[i] = Store<S>::load_smem(reinterpret_cast<const T*>(st + i * G::ROW_BYTES), hp - cx(i), p.wref[i]);
        const float rh = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
        ring[k & 3][tid == 0 ? 0 : width + 1] = psi_of(rh, p);
      }
      if (tid == 0 && width == 1) {  // a one-column strip needs both halos from this thread
        float h[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i)
          h[i] = Store<S>::load_smem(reinterpret_cast<const T*>(st + i * G::ROW_BYTES), G::PAD + 1 - cx(i), p.wref[i]);
        const float rh = ((h[0] + h[1]) + (h[2] + h[3])) + ((h[4] + h[5]) + (h[6] + h[7])) + h[8];
        ring[k & 3][2] = psi_of(rh, p);
      }
    }
    __syncthreads();
    if (*abort_flag) {
      k_abort = k;
      break;
    }
    if (tid == 0 && k + NSTAGE - 2 < nst) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_stage<S, MASKED, NSTAGE>(p, src, stages, bars, k + NSTAGE - 2, y0, x0);
    }
    if (k >= 2 && active) {
      const int rc = y0 - 1 + k - 1;  // row collided now
      const unsigned char* sp = stages + (size_t)((k - 1) % NSTAGE) * STAGE_BYTES;
      const int sm = (k - 2) & 3, s0 = (k - 1) & 3, s1 = k & 3;
      const float psi_c = ring[s0][jc];
      unsigned m = 0;
      if (MASKED) m = sp[Q * G::ROW_BYTES + tid];
      float sx = 0.f, sy = 0.f;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int sl = cy(i) > 0 ? s1 : (cy(i) < 0 ? sm : s0);
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
      const size_t base = (size_t)rc * nx + x0 + tid;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const float fi = Store<S>::load_smem(reinterpret_cast<const T*>(sp + i * G::ROW_BYTES), pos - cx(i), p.wref[i]);
        const float eu = cx(i) * ux + cy(i) * uy;
        const float feq = static_cast<float>(wq(i)) * rho_prev * (1.0f + 3.0f * eu + 4.5f * eu * eu - uu);
        Store<S>::store(dst, (size_t)i * p.N + base, fi + (feq - fi) * p.inv_tau, p.wref[i]);
      }
    }
    rho_prev = rho;
    jx_prev = jx;
    jy_prev = jy;
  }
  if (*abort_flag) {
    // a stage never completed: record it, then wait (bounded) for the copies
    // of every stage issued and not consumed before the CTA leaves
    if (tid == 0) {
      atomicOr(p.flags + FLAG_TIMEOUT, 1);
      const int issued = min(nst, k_abort + NSTAGE - 2);
      for (int q = k_abort; q < issued; ++q)
        mbar_wait(bars + q % NSTAGE, (uint32_t)((q / NSTAGE) & 1), 500000000ull);
    }
    __syncthreads();
    return;
  }
  if (bad) atomicOr(p.flags + FLAG_NUMERIC, 1);
}

template <int S>
constexpr int tma_stages() { return S == LBM_F32 ? 6 : 10; }
template <int S>
constexpr int tma_minblocks() { return S == LBM_F32 ? 3 : 4; }

template <int S, bool MASKED>
size_t tma_smem_bytes() {
  using G = TmaGeom<S>;
  return (size_t)tma_stages<S>() * (Q * G::ROW_BYTES + (MASKED ? kBX : 0)) + 4 * (kBX + 2) * 4 +
         tma_stages<S>() * 8 + 16;
}

template <int S>
bool tma_ok(int nx) {
  return nx % 16 == 0 && nx >= TmaGeom<S>::WIN;
}

template <int S, bool MASKED>
cudaError_t launch_tma(const StepParams& q, dim3 grid, cudaStream_t s) {
  auto kern = k_step_tma<S, MASKED, tma_stages<S>(), tma_minblocks<S>()>;
  const size_t smem = tma_smem_bytes<S, MASKED>();
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kBX, smem, s>>>(q);
  return cudaGetLastError();
}

template <int S>
cudaError_t launch_typed(const StepParams& p, cudaStream_t s) {
  int gx, gy, rows, block;
  step_geometry(p.nx, p.ny, &gx, &gy, &rows, &block);
  StepParams q = p;
  q.rows_per_chunk = rows;
  dim3 grid(gx, gy);
  if (p.force_generic != 1 && tma_ok<S>(p.nx))
    return p.mask ? launch_tma<S, true>(q, grid, s) : launch_tma<S, false>(q, grid, s);
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

bool step_tma_allowed(int storage, int nx) {
  return storage == LBM_F32 ? tma_ok<LBM_F32>(nx) : (storage == LBM_F16_DEV ? tma_ok<LBM_F16_DEV>(nx) : tma_ok<LBM_BF16_DEV>(nx));
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
