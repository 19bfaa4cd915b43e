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
// Every kernel marches a strip of columns down a chunk of rows. For every
// row it pulls the populations of the strip's cells and of one halo column
// on each side, forms rho and psi once per cell, and puts psi into a
// four-row ring in shared memory; one barrier later the ring holds psi for
// rows r-2..r and the force and collision of row r-1 run on the moments kept
// in registers. All per-cell arithmetic lives in the shared device functions
// below (one cell or two), so every kernel gives bitwise the same
// populations.
//
//  - k_step_strip: plain global loads, one cell per thread; any box size.
//  - k_step_tma: the nine source rows of every output row (with halo) are
//    copied into a ring of shared-memory stages by cp.async.bulk, issued
//    NSTAGE-1 rows ahead by a ninth warp that also computes the two halo
//    cells, so the eight compute warps are balanced and the bytes in flight
//    do not depend on occupancy. Needs nx % 16 == 0 and nx >= kBX + 16.
//  - k_step_tma2: the same staging over 512-column strips with two cells per
//    thread (march2); one static row chunk per CTA.
//  - k_step_dyn: march2 over row chunks that the resident CTAs draw from a
//    device counter (the automatic choice where nx % 16 == 0).
//  - k_step_batch: march2 over work items (box, strip, row chunk) of many
//    boxes in one launch (batch.cu).
#include "lbm_internal.cuh"
#include "tma.cuh"

namespace lbm {
namespace {

constexpr int kBX = 256;           // columns per strip (= compute threads)
constexpr int kTmaThreads = kBX + 32;
constexpr float kW1 = 1.0f / 9.0f, kW5 = 1.0f / 36.0f, kW0 = 4.0f / 9.0f;

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// ---------------------------------------------------------------- cell math
// The per-cell arithmetic is written once for V = float (one cell) and
// V = float2 (two neighbouring cells, packed FP32 instructions), with every
// operation an explicitly rounded add, multiply or fused multiply-add, so all
// kernels produce bitwise the same populations.
template <typename V>
struct VOps;

template <>
struct VOps<float> {
  static __device__ __forceinline__ float set(float a) { return a; }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
  static __device__ __forceinline__ float ex(float a) { return __expf(a); }
  static __device__ __forceinline__ int bad(float rho) { return !(rho > 0.f && rho < 1e30f); }
};

// The pair type uses the packed two-wide FP32 instructions of sm_100 and
// later, whose rounding per component is that of the scalar intrinsics; a
// difference is the fused b * (-1) + a, which rounds once, exactly as a - b.
template <>
struct VOps<float2> {
  static __device__ __forceinline__ float2 set(float a) { return make_float2(a, a); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
  static __device__ __forceinline__ float2 rcp(float2 a) { return make_float2(__frcp_rn(a.x), __frcp_rn(a.y)); }
  static __device__ __forceinline__ float2 ex(float2 a) { return make_float2(__expf(a.x), __expf(a.y)); }
  static __device__ __forceinline__ int bad(float2 rho) { return VOps<float>::bad(rho.x) | VOps<float>::bad(rho.y); }
};

// Eq. 11: rho and j from the nine incoming populations.
template <typename V>
__device__ __forceinline__ void moments9(const V f[Q], V& rho, V& jx, V& jy) {
  using O = VOps<V>;
  rho = O::add(O::add(O::add(f[0], f[1]), O::add(f[2], f[3])), O::add(O::add(f[4], f[5]), O::add(f[6], f[7])));
  rho = O::add(rho, f[8]);
  jx = O::add(O::sub(f[1], f[3]), O::add(O::sub(f[5], f[7]), O::sub(f[8], f[6])));
  jy = O::add(O::sub(f[2], f[4]), O::add(O::sub(f[5], f[7]), O::sub(f[6], f[8])));
}

// Full density from the summed stored values: for 16-bit storage (DEV) the
// stored values are deviations g_i = f_i - w_i rho_ref, whose sum is
// rho - rho_ref (the weights sum to one).
template <bool DEV, typename V>
__device__ __forceinline__ V full_rho(V rho_raw, const StepParams& p) {
  return DEV ? VOps<V>::add(VOps<V>::set(p.rho_ref), rho_raw) : rho_raw;
}

// Eq. 30.
template <typename V>
__device__ __forceinline__ V psi_of(V rho, const StepParams& p) {
  using O = VOps<V>;
  return O::mul(O::set(p.rho0), O::sub(O::set(1.0f), O::ex(O::mul(rho, O::set(-p.inv_rho0)))));
}

// Eq. 22 with the barrier substitution: s[i] holds psi(x + e_i), or psi(x)
// where the edge is blocked.
template <typename V>
__device__ __forceinline__ void force_of(const V s[Q], V psi_c, float G, V& Fx, V& Fy) {
  using O = VOps<V>;
  const V w1 = O::set(kW1), w5 = O::set(kW5);
  const V d57 = O::sub(s[5], s[7]);
  const V sx = O::fma(w1, O::sub(s[1], s[3]), O::mul(w5, O::add(d57, O::sub(s[8], s[6]))));
  const V sy = O::fma(w1, O::sub(s[2], s[4]), O::mul(w5, O::add(d57, O::sub(s[6], s[8]))));
  const V gp = O::mul(O::set(-G), psi_c);
  Fx = O::mul(gp, sx);
  Fy = O::mul(gp, sy);
}

// Eqs. 39-40 (u_eq = (j + tau F)/rho), Eq. 14 evaluated by opposite pairs,
// Eq. 18 (BGK). f holds the incoming stored values and receives the outgoing
// ones. With DEV the values are deviations from w_i rho_ref: j is unchanged
// (sum e_i w_i = 0) and the equilibrium deviation is
// w_i (rho - rho_ref - 1.5 rho u^2 + rho (3 e.u + 4.5 (e.u)^2)).
template <bool TAU_ONE, bool DEV, typename V>
__device__ __forceinline__ void collide(V f[Q], V rho_raw, V jx, V jy, V Fx, V Fy, const StepParams& p, int& bad) {
  using O = VOps<V>;
  const V rho = full_rho<DEV>(rho_raw, p);
  const V ir = O::rcp(rho);
  const V tau = O::set(p.tau);
  const V ux = O::mul(O::fma(tau, Fx, jx), ir);
  const V uy = O::mul(O::fma(tau, Fy, jy), ir);
  bad |= O::bad(rho);
  const V uu = O::fma(ux, ux, O::mul(uy, uy));
  const V a = DEV ? O::fma(O::mul(O::set(-1.5f), rho), uu, rho_raw) : O::mul(rho, O::fma(O::set(-1.5f), uu, O::set(1.0f)));
  const V r3 = O::mul(O::set(3.0f), rho), r45 = O::mul(O::set(4.5f), rho);
  const V w1 = O::set(kW1), w5 = O::set(kW5);
  V feq[Q];
  feq[0] = O::mul(O::set(kW0), a);
  {
    const V s = O::fma(O::mul(r45, ux), ux, a), t = O::mul(r3, ux);
    feq[1] = O::mul(w1, O::add(s, t));
    feq[3] = O::mul(w1, O::sub(s, t));
  }
  {
    const V s = O::fma(O::mul(r45, uy), uy, a), t = O::mul(r3, uy);
    feq[2] = O::mul(w1, O::add(s, t));
    feq[4] = O::mul(w1, O::sub(s, t));
  }
  {
    const V e = O::add(ux, uy);
    const V s = O::fma(O::mul(r45, e), e, a), t = O::mul(r3, e);
    feq[5] = O::mul(w5, O::add(s, t));
    feq[7] = O::mul(w5, O::sub(s, t));
  }
  {
    const V e = O::sub(uy, ux);
    const V s = O::fma(O::mul(r45, e), e, a), t = O::mul(r3, e);
    feq[6] = O::mul(w5, O::add(s, t));
    feq[8] = O::mul(w5, O::sub(s, t));
  }
  const V om = O::set(p.inv_tau);
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = TAU_ONE ? feq[i] : O::fma(O::sub(feq[i], f[i]), om, f[i]);
}

// Force + collision + store of one cell from the psi ring.
template <int S, bool MASKED, bool TAU_ONE>
__device__ __forceinline__ void finish_cell(float f[Q], float rho, float jx, float jy, unsigned m,
                                            const float (*ring)[kBX + 2], int sm, int s0, int sp, int jc,
                                            const StepParams& p, typename Store<S>::T* __restrict__ dst,
                                            size_t base, int& bad) {
  const float psi_c = ring[s0][jc];
  float s[Q];
#pragma unroll
  for (int i = 1; i < Q; ++i) s[i] = ring[cy(i) > 0 ? sp : (cy(i) < 0 ? sm : s0)][jc + cx(i)];
  if (MASKED && m) {
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if ((m >> (i - 1)) & 1u) s[i] = psi_c;
  }
  float Fx, Fy;
  force_of(s, psi_c, p.G, Fx, Fy);
  collide<TAU_ONE, S != LBM_F32>(f, rho, jx, jy, Fx, Fy, p, bad);
#pragma unroll
  for (int i = 0; i < Q; ++i) Store<S>::store_raw(dst, (size_t)i * p.N + base, f[i]);
}

// ---------------------------------------------------------------- plain-load kernel
template <int S>
__device__ __forceinline__ void pull_cell(const typename Store<S>::T* __restrict__ src, const StepParams& p,
                                          long long rowm, long long row0, long long rowp, int xm, int x, int xp,
                                          float f[Q]) {
  // f_i(x, r) = f_i^out(x - c_ix, r - c_iy): rows r-1 (c_iy = +1), r, r+1 (c_iy = -1)
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const long long row = cy(i) > 0 ? rowm : (cy(i) < 0 ? rowp : row0);
    const int xs = cx(i) > 0 ? xm : (cx(i) < 0 ? xp : x);
    f[i] = Store<S>::raw(src, (size_t)i * p.N + row + xs);
  }
}

template <int S, bool MASKED, bool TAU_ONE>
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
    float f[Q];
    float rho = 1.f, jx = 0.f, jy = 0.f;
    if (active) {
      pull_cell<S>(src, p, rowm, row0, rowp, xm, x, xp, f);
      moments9(f, rho, jx, jy);
      ring[k & 3][jc] = psi_of(full_rho<S != LBM_F32>(rho, p), p);
    }
    if (tid == 0) {
      float h[Q], rh, hx, hy;
      pull_cell<S>(src, p, rowm, row0, rowp, xlm, xl, x0, h);
      moments9(h, rh, hx, hy);
      ring[k & 3][0] = psi_of(full_rho<S != LBM_F32>(rh, p), p);
    }
    if (x == last) {
      float h[Q], rh, hx, hy;
      pull_cell<S>(src, p, rowm, row0, rowp, last, xr, xrp, h);
      moments9(h, rh, hx, hy);
      ring[k & 3][last - x0 + 2] = psi_of(full_rho<S != LBM_F32>(rh, p), p);
    }
    __syncthreads();
    if (k >= 2 && active) {
      const int rc = r - 1;
      const unsigned m = MASKED ? p.mask[(size_t)rc * nx + x] : 0u;
      finish_cell<S, MASKED, TAU_ONE>(fprev, rho_prev, jx_prev, jy_prev, m, ring, (k - 2) & 3, (k - 1) & 3,
                                      k & 3, jc, p, dst, (size_t)rc * nx + x, bad);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) fprev[i] = f[i];
    rho_prev = rho;
    jx_prev = jx;
    jy_prev = jy;
  }
  if (bad) atomicOr(p.flags + FLAG_NUMERIC, 1);
}

// ---------------------------------------------------------------- TMA-staged kernel
template <int S>
struct TmaGeom {
  using T = typename Store<S>::T;
  static constexpr int E = sizeof(T);
  static constexpr int PAD = 16 / E;         // halo pad in elements: 16 bytes
  static constexpr int WIN = kBX + 2 * PAD;  // elements per staged plane row
  static constexpr int ROW_BYTES = WIN * E;  // multiple of 16
};

// Issued by the lanes of the ninth warp: lane 0 arms the stage's mbarrier,
// lanes 0..8 copy plane `lane`, lane 9 copies the mask row.
template <int S, bool MASKED, int NSTAGE>
__device__ __forceinline__ void issue_stage(const StepParams& p, const typename Store<S>::T* src,
                                            unsigned char* stages, uint64_t* bars, int k, int y0, int x0,
                                            int lane) {
  using G = TmaGeom<S>;
  using T = typename G::T;
  constexpr uint32_t STAGE_BYTES = Q * G::ROW_BYTES + (MASKED ? kBX : 0);
  const int slot = k % NSTAGE;
  unsigned char* st = stages + (size_t)slot * STAGE_BYTES;
  uint64_t* bar = bars + slot;
  const int r = y0 - 1 + k;
  const int ny = p.ny, nx = p.nx;
  if (lane < Q + (MASKED ? 1 : 0)) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (lane == 0) mbar_expect_tx(bar, STAGE_BYTES);
  __syncwarp();
  if (lane < Q) {
    const int i = lane;
    const int ciy = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    int g = r - ciy;
    g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
    g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
    const T* row = src + (size_t)i * p.N + (size_t)g * nx;
    copy_row_wrapped<T>(reinterpret_cast<T*>(st + i * G::ROW_BYTES), row, x0 - G::PAD, G::WIN, nx, bar);
  } else if (MASKED && lane == Q) {  // columns x0 .. x0+kBX (a ragged strip wraps; unused)
    const int g = r < 0 ? r + ny : (r >= ny ? r - ny : r);
    copy_row_wrapped<uint8_t>(st + Q * G::ROW_BYTES, p.mask + (size_t)g * nx, x0, kBX, nx, bar);
  }
}

template <int S, bool MASKED, int NSTAGE>
constexpr size_t tma_smem_bytes_c() {
  return (size_t)NSTAGE * (Q * TmaGeom<S>::ROW_BYTES + (MASKED ? kBX : 0)) + 4 * (kBX + 2) * 4 + NSTAGE * 8 + 16;
}

template <int S, bool MASKED, bool TAU_ONE, int NSTAGE, int MINB>
__global__ void __launch_bounds__(kTmaThreads, MINB) k_step_tma(const StepParams p) {
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
  const bool helper = tid >= kBX;  // the ninth warp
  const int lane = tid & 31;
  const int x0 = blockIdx.x * kBX;
  const int width = min(kBX, nx - x0);
  const bool active = !helper && tid < width;
  const int y0 = blockIdx.y * p.rows_per_chunk;
  const int y1 = min(y0 + p.rows_per_chunk, ny);
  if (y0 >= y1) return;
  const int nst = (y1 - y0) + 2;  // stages = rows y0-1 .. y1

  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(bars + s, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (helper)
    for (int k = 0; k < NSTAGE - 1 && k < nst; ++k) issue_stage<S, MASKED, NSTAGE>(p, src, stages, bars, k, y0, x0, lane);

  // halo lanes of the helper warp: lanes 0..8 pull plane `lane` of the left
  // halo cell (column x0-1), lanes 16..24 of the right one (column x0+width)
  const int hplane = lane & 15;
  const bool hlane = helper && hplane < Q;
  const int hcx = (hplane == 1 || hplane == 5 || hplane == 8) ? 1 : ((hplane == 3 || hplane == 6 || hplane == 7) ? -1 : 0);
  const int hpos = (lane < 16 ? G::PAD - 1 : G::PAD + width) - hcx;

  const int jc = tid + 1;
  const int pos = G::PAD + tid;
  float fprev[Q];
  float rho_prev = 1.f, jx_prev = 0.f, jy_prev = 0.f;
  unsigned m_prev = 0;
  int bad = 0;
  int k_abort = 0;
  for (int k = 0; k < nst; ++k) {
    const int slot = k % NSTAGE;
    const unsigned char* st = stages + (size_t)slot * STAGE_BYTES;
    if (!mbar_wait(bars + slot, (uint32_t)((k / NSTAGE) & 1))) *abort_flag = 1;
    float f[Q];
    float rho = 1.f, jx = 0.f, jy = 0.f;
    unsigned m = 0;
    if (active) {
#pragma unroll
      for (int i = 0; i < Q; ++i)
        f[i] = Store<S>::raw_smem(reinterpret_cast<const T*>(st + i * G::ROW_BYTES), pos - cx(i));
      moments9(f, rho, jx, jy);
      ring[k & 3][jc] = psi_of(full_rho<S != LBM_F32>(rho, p), p);
      if (MASKED) m = st[Q * G::ROW_BYTES + tid];
    } else if (helper) {
      // same summation order as moments9: ((f0+f1)+(f2+f3)) + ((f4+f5)+(f6+f7)) + f8
      const float v = hlane ? Store<S>::raw_smem(reinterpret_cast<const T*>(st + hplane * G::ROW_BYTES), hpos) : 0.f;
      const float t1 = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, 1));
      const float t2 = __fadd_rn(t1, __shfl_xor_sync(0xffffffffu, t1, 2));
      const float t3 = __fadd_rn(t2, __shfl_xor_sync(0xffffffffu, t2, 4));
      const float rh = full_rho<S != LBM_F32>(__fadd_rn(t3, __shfl_xor_sync(0xffffffffu, t2, 8)), p);
      if (lane == 0) ring[k & 3][0] = psi_of(rh, p);
      if (lane == 16) ring[k & 3][width + 1] = psi_of(rh, p);
    }
    __syncthreads();
    if (*abort_flag) {
      k_abort = k;
      break;
    }
    if (helper) {
      if (k + NSTAGE - 1 < nst) issue_stage<S, MASKED, NSTAGE>(p, src, stages, bars, k + NSTAGE - 1, y0, x0, lane);
    } else if (k >= 2 && active) {
      const int rc = y0 + k - 2;  // row collided now
      finish_cell<S, MASKED, TAU_ONE>(fprev, rho_prev, jx_prev, jy_prev, m_prev, ring, (k - 2) & 3, (k - 1) & 3,
                                      k & 3, jc, p, dst, (size_t)rc * nx + x0 + tid, bad);
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) fprev[i] = f[i];
    rho_prev = rho;
    jx_prev = jx;
    jy_prev = jy;
    m_prev = m;
  }
  if (*abort_flag) {
    // a stage never completed: record it, then wait (bounded) for the copies
    // of every stage issued and not consumed before the CTA leaves
    if (tid == 0) {
      atomicOr(p.flags + FLAG_TIMEOUT, 1);
      const int issued = min(nst, k_abort + NSTAGE - 1);
      for (int q = k_abort; q < issued; ++q) mbar_wait(bars + q % NSTAGE, (uint32_t)((q / NSTAGE) & 1), 500000000ull);
    }
    __syncthreads();
    return;
  }
  if (bad) atomicOr(p.flags + FLAG_NUMERIC, 1);
}

// ---------------------------------------------------------------- two-cell staged kernel
// The staged march with two neighbouring cells per thread: a CTA owns a
// strip of kBX2 = 512 columns, 256 compute threads (cells 2t and 2t+1) plus
// the helper warp. Pairs are read from the stage with one 32-bit (16-bit
// storage) or 64-bit (FP32) shared load where aligned, and with two loads and
// a byte permute where the pull shifts them by one column; the arithmetic
// runs on float2 (packed FP32); outputs leave as half2/bfloat162/float2.
constexpr int kBX2 = 512;

template <int S>
struct TmaGeom2 {
  using T = typename Store<S>::T;
  static constexpr int E = sizeof(T);
  static constexpr int PAD = 16 / E;
  static constexpr int WIN = kBX2 + 2 * PAD;
  static constexpr int ROW_BYTES = WIN * E;
};

// Two consecutive staged raw values (window positions pos, pos+1) as floats.
template <int S>
__device__ __forceinline__ float2 load_pair(const unsigned char* row, int pos, int shift);

template <>
__device__ __forceinline__ float2 load_pair<LBM_F32>(const unsigned char* row, int pos, int shift) {
  const float* r = reinterpret_cast<const float*>(row);
  if (shift == 0) return *reinterpret_cast<const float2*>(r + pos);  // pos even: 8-byte aligned
  return make_float2(r[pos], r[pos + 1]);
}

__device__ __forceinline__ uint32_t pair_bits_16(const unsigned char* row, int pos, int shift) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(row);
  if (shift == 0) return w[pos >> 1];  // pos even
  // pos odd: high half of the word at pos-1 and low half of the word at pos+1
  return __byte_perm(w[(pos - 1) >> 1], w[(pos + 1) >> 1], 0x5432);
}

// 16-bit pairs are converted element by element with the same conversion as
// the one-cell kernels (the packed conversions gave different results for
// small deviations), so all kernels agree bitwise.
template <>
__device__ __forceinline__ float2 load_pair<LBM_F16_DEV>(const unsigned char* row, int pos, int shift) {
  const uint32_t b = pair_bits_16(row, pos, shift);
  const __half2 h = *reinterpret_cast<const __half2*>(&b);
  return make_float2(__low2float(h), __high2float(h));
}

template <>
__device__ __forceinline__ float2 load_pair<LBM_BF16_DEV>(const unsigned char* row, int pos, int shift) {
  const uint32_t b = pair_bits_16(row, pos, shift);
  const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&b);
  return make_float2(__low2float(h), __high2float(h));
}

template <int S>
__device__ __forceinline__ void store_pair(typename Store<S>::T* dst, size_t idx, float2 v);

template <>
__device__ __forceinline__ void store_pair<LBM_F32>(float* dst, size_t idx, float2 v) {
  *reinterpret_cast<float2*>(dst + idx) = v;  // idx even
}

template <>
__device__ __forceinline__ void store_pair<LBM_F16_DEV>(__half* dst, size_t idx, float2 v) {
  *reinterpret_cast<__half2*>(dst + idx) = __halves2half2(__float2half_rn(v.x), __float2half_rn(v.y));
}

template <>
__device__ __forceinline__ void store_pair<LBM_BF16_DEV>(__nv_bfloat16* dst, size_t idx, float2 v) {
  *reinterpret_cast<__nv_bfloat162*>(dst + idx) = __halves2bfloat162(__float2bfloat16_rn(v.x), __float2bfloat16_rn(v.y));
}

// Copy len elements of a periodic row starting at column start (-nx <= start
// < nx) into dst, wrapping as often as needed (len <= nx + 32: at most three
// pieces). Every piece starts and ends on a 16-byte boundary when nx, start
// and len are multiples of 16 bytes' worth of elements.
template <typename T>
__device__ __forceinline__ void copy_row_wrapped3(T* dst, const T* row, int start, int len, int nx, uint64_t* bar) {
  const int s0 = start < 0 ? start + nx : start;
  const int first = min(len, nx - s0);
  bulk_g2s(dst, row + s0, (uint32_t)(first * sizeof(T)), bar);
  if (first < len) {  // wrapped past the end of the row: restart at column 0
    const int second = min(len - first, nx);
    bulk_g2s(dst + first, row, (uint32_t)(second * sizeof(T)), bar);
    if (first + second < len)  // a strip as wide as the box: its right halo wraps again
      bulk_g2s(dst + first + second, row, (uint32_t)((len - first - second) * sizeof(T)), bar);
  }
}

// Rows that do not start on 16-byte boundaries (nx % 16 != 0, variant UNAL
// of the two-cell march): a staged row keeps window element e at slot
// position e + off, where off = (index of window element 0 in the buffer,
// plane offset i N included) mod M (M = elements per 16 bytes). A window
// arrives in one bulk copy of the 16-byte-aligned span that covers its part
// inside the periodic row (up to M - 1 elements on either side land in the
// slot's slack and are never read); the mask row likewise. Where the window
// wraps (the box's first strip, and the strips that reach its last column),
// the two elements on a wrapped side that the march reads come by plain
// loads into a side area of the slot. A row slot holds 2 M more elements.
// Layout of one stage slot of the two-cell march: nine plane rows of RB bytes,
// the mask row, and (UNAL) a side area of four elements per plane for the
// window elements of a wrapped window that the staged rows cannot hold.
template <int S, bool MASKED, bool UNAL>
struct Slot2 {
  static constexpr int RB = TmaGeom2<S>::ROW_BYTES + (UNAL ? 32 : 0);  // plane row stride
  static constexpr int SIDE_OFF = Q * RB + (MASKED ? kBX2 + (UNAL ? 32 : 0) : 0);
  static constexpr int BYTES = SIDE_OFF + (UNAL ? (Q * 4 * TmaGeom2<S>::E + 15) / 16 * 16 : 0);
};

// One stage of the two-cell march: for output row r = y0 - 1 + k, plane i's
// source row r - c_iy, columns x0 - PAD .. x0 + width + PAD (wrapped), and the
// mask row r, columns x0 .. x0 + width. Slots have a fixed stride.
template <int S, bool MASKED, int NSTAGE, bool UNAL = false>
__device__ __forceinline__ void issue_stage2(const StepParams& p, const typename Store<S>::T* src,
                                             unsigned char* stages, uint64_t* bars, unsigned gk, int k, int y0,
                                             int x0, int width, int lane) {
  using G = TmaGeom2<S>;
  using T = typename G::T;
  constexpr int RB = Slot2<S, MASKED, UNAL>::RB;  // plane row stride in a slot
  constexpr uint32_t SLOT_BYTES = Slot2<S, MASKED, UNAL>::BYTES;
  const int len = width + 2 * G::PAD;
  const int slot = (int)(gk % NSTAGE);
  unsigned char* st = stages + (size_t)slot * SLOT_BYTES;
  uint64_t* bar = bars + slot;
  const int r = y0 - 1 + k;
  const int ny = p.ny, nx = p.nx;
  if (UNAL || lane < Q + (MASKED ? 1 : 0)) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (!UNAL) {
    const uint32_t bytes = (uint32_t)(Q * len * G::E + (MASKED ? width : 0));
    if (lane == 0) mbar_expect_tx(bar, bytes);
    __syncwarp();
    if (lane < Q) {
      const int i = lane;
      const int ciy = (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
      int g = r - ciy;
      g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
      g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
      const T* row = src + (size_t)i * p.N + (size_t)g * nx;
      copy_row_wrapped3<T>(reinterpret_cast<T*>(st + i * RB), row, x0 - G::PAD, len, nx, bar);
    } else if (MASKED && lane == Q) {
      const int g = r < 0 ? r + ny : (r >= ny ? r - ny : r);
      copy_row_wrapped3<uint8_t>(st + Q * RB, p.mask + (size_t)g * nx, x0, width, nx, bar);
    }
    return;
  }
  // UNAL: row q (planes 0..8, then the mask) is served by lanes 3q .. 3q + 2
  const int q = lane / 3, j = lane - 3 * q;
  uint32_t bytes = 0;
  const void* bsrc = nullptr;
  void* bdst = nullptr;
  if (q < Q) {
    constexpr int M = 16 / G::E;
    const int ciy = (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0);
    int g = r - ciy;
    g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
    g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
    const T* row = src + (size_t)q * p.N + (size_t)g * nx;
    T* dst = reinterpret_cast<T*>(st + q * RB);
    const int c0 = x0 - G::PAD;
    const long long gbase = (long long)q * p.N + (long long)g * nx;
    if (c0 >= 0 && c0 + len <= nx) {  // no wrap: one covering bulk copy to slot position 0
      const int off = (int)((gbase + c0) & (M - 1));
      if (j == 0) {
        bytes = (uint32_t)(((off + len + M - 1) / M) * 16);
        bsrc = row + c0 - off;
        bdst = dst;
      }
    } else {
      // the window wraps around the periodic row: its part inside the row
      // by one covering copy, whose slot start a + off - ra is a multiple of
      // M (0, or M after a left wrap); the wrapped elements the march reads
      // (two on a wrapped side) by plain loads into the side area, since
      // the copy's slack may cover their slot positions
      const int off = (int)((gbase + c0 + M) & (M - 1));  // gbase + c0 >= -M
      const int a = c0 < 0 ? -c0 : 0, b = c0 + len > nx ? nx - c0 : len;
      const long long ga = gbase + c0 + a;  // buffer index of the first element inside the row
      const int ra = (int)(ga & (M - 1));
      T* side = reinterpret_cast<T*>(st + Slot2<S, MASKED, UNAL>::SIDE_OFF) + 4 * q;
      if (j == 0) {
        const long long gend = gbase + c0 + b;  // one past the last element inside the row
        bytes = (uint32_t)(((gend + M - 1) / M * M - (ga - ra)) * G::E);
        bsrc = row + (c0 + a - ra);
        bdst = dst + (a + off - ra);
      } else if (j == 1 && a > 0) {  // window elements PAD - 2, PAD - 1: columns nx - 2, nx - 1
        side[0] = row[nx - 2];
        side[1] = row[nx - 1];
      } else if (j == 2 && b < len) {  // window elements b, b + 1: columns 0, 1
        side[2] = row[0];
        side[3] = row[1];
      }
    }
  } else if (MASKED && q == Q && j == 0) {
    // the mask window never wraps: one covering bulk copy to slot position 0
    const int g = r < 0 ? r + ny : (r >= ny ? r - ny : r);
    const long long gm = (long long)g * nx + x0;
    const int off = (int)(gm & 15);
    bytes = (uint32_t)(((off + width + 15) / 16) * 16);
    bsrc = p.mask + (gm - off);
    bdst = st + Q * RB;
  }
  const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
  __syncwarp();  // the plain stores above are ordered before the arrive (release)
  if (lane == 0) mbar_expect_tx(bar, total);
  __syncwarp();
  if (bytes) bulk_g2s(bdst, bsrc, bytes, bar);
}

template <int S, bool MASKED, int NSTAGE, bool UNAL = false>
constexpr size_t tma2_smem_bytes_c() {
  return (size_t)NSTAGE * Slot2<S, MASKED, UNAL>::BYTES + 4 * (kBX2 + 4) * 4 + NSTAGE * 8 + 16;
}

template <int S, bool MASKED, int NSTAGE, bool UNAL = false>
struct Tma2Smem {
  static constexpr int RB = Slot2<S, MASKED, UNAL>::RB;  // plane row stride
  static constexpr int SLOT_BYTES = Slot2<S, MASKED, UNAL>::BYTES;
  static constexpr int RW = kBX2 + 4;  // ring row: cell column c at index c + 2, halos at 1 and width + 2
  unsigned char* stages;
  float (*ring)[RW];
  uint64_t* bars;
  int* abort_flag;
  __device__ __forceinline__ explicit Tma2Smem(unsigned char* smem) {
    stages = smem;
    ring = reinterpret_cast<float(*)[RW]>(smem + (size_t)NSTAGE * SLOT_BYTES);
    bars = reinterpret_cast<uint64_t*>(smem + (size_t)NSTAGE * SLOT_BYTES + 4 * RW * 4);
    abort_flag = reinterpret_cast<int*>(bars + NSTAGE);
  }
};

// The two-cell march of one work item: columns x0 .. x0 + width (a multiple of
// 16, at most kBX2; with UNAL any width, and rows that need not start on
// 16-byte boundaries) and rows y0 .. y1 of one box. `gstage` counts the
// stages this CTA consumed before (mbarrier phases continue across items).
// Returns false if a stage wait timed out (the CTA must then leave).
template <int S, bool MASKED, bool TAU_ONE, int NSTAGE, bool FULL = false, bool UNAL = false>
__device__ __forceinline__ bool march2(const StepParams& p, const Tma2Smem<S, MASKED, NSTAGE, UNAL>& sm, int x0,
                                       int width_, int y0, int y1, unsigned& gstage, int& bad) {
  const int width = FULL ? kBX2 : width_;  // FULL: a whole strip (known at compile time)
  using G = TmaGeom2<S>;
  using T = typename G::T;
  constexpr int SLOT_BYTES = Tma2Smem<S, MASKED, NSTAGE, UNAL>::SLOT_BYTES;
  constexpr int RB = Tma2Smem<S, MASKED, NSTAGE, UNAL>::RB;
  constexpr int M = 16 / G::E;  // elements per 16 bytes
  const T* __restrict__ src = static_cast<const T*>(p.src);
  T* __restrict__ dst = static_cast<T*>(p.dst);
  const int nx = p.nx;
  const int tid = threadIdx.x;
  const bool helper = tid >= kBX;
  const int lane = tid & 31;
  const bool active = !helper && 2 * tid < width;
  const int nst = (y1 - y0) + 2;  // stages = rows y0-1 .. y1
  const unsigned g0 = gstage;

  if (helper)
    for (int k = 0; k < NSTAGE - 1 && k < nst; ++k)
      issue_stage2<S, MASKED, NSTAGE, UNAL>(p, src, sm.stages, sm.bars, g0 + k, k, y0, x0, width, lane);

  const int hplane = lane & 15;
  const bool hlane = helper && hplane < Q;
  const int hcx = (hplane == 1 || hplane == 5 || hplane == 8) ? 1 : ((hplane == 3 || hplane == 6 || hplane == 7) ? -1 : 0);
  const int hcy = (hplane == 2 || hplane == 5 || hplane == 6) ? 1 : ((hplane == 4 || hplane == 7 || hplane == 8) ? -1 : 0);
  const int hpos = (lane < 16 ? G::PAD - 1 : G::PAD + width) - hcx;

  const int jc = 2 * tid + 2;        // ring index of the first cell of the pair
  const int pos = G::PAD + 2 * tid;  // window position of the first cell
  // UNAL: window elements [PAD - 2, ea) and [eb, eb + 2) of a wrapped window
  // are read from the stage's side area (thread 0 after a left wrap, the
  // last pair before a right wrap, and the halo lanes)
  const int ea = UNAL && x0 < G::PAD ? G::PAD - x0 : 0;
  const int eb = UNAL && x0 + width + G::PAD > nx ? nx - x0 + G::PAD : (1 << 30);
  const bool fixw = UNAL && active && ((tid == 0 && ea > 0) || pos + 2 >= eb);
  float2 fprev[Q];
  float2 rho_prev = make_float2(1.f, 1.f), jx_prev = make_float2(0.f, 0.f), jy_prev = make_float2(0.f, 0.f);
  unsigned m_prev = 0;
  int k_abort = -1;
  for (int k = 0; k < nst; ++k) {
    const unsigned gk = g0 + k;
    const unsigned char* st = sm.stages + (size_t)(gk % NSTAGE) * SLOT_BYTES;
    if (!mbar_wait(sm.bars + gk % NSTAGE, (gk / NSTAGE) & 1u)) *sm.abort_flag = 1;
    float2 f[Q];
    float2 rho = make_float2(1.f, 1.f), jx = make_float2(0.f, 0.f), jy = make_float2(0.f, 0.f);
    unsigned m = 0;
    // UNAL: slot offset of plane i's source row is (i N + its row's start
    // + x0 - PAD) mod M: the rows r - 1, r, r + 1 give three bases, each
    // plane adds i N; the mask row's offset is taken mod 16
    int bm = 0, b0 = 0, bp = 0, offk = 0;
    if (UNAL) {
      const int r = y0 - 1 + k, ny = p.ny;
      const int g0r = r < 0 ? r + ny : (r >= ny ? r - ny : r);
      const int gm = g0r == 0 ? ny - 1 : g0r - 1, gp = g0r == ny - 1 ? 0 : g0r + 1;
      bm = (int)(((long long)gm * nx + x0 - G::PAD + M) & (M - 1));
      b0 = (int)(((long long)g0r * nx + x0 - G::PAD + M) & (M - 1));
      bp = (int)(((long long)gp * nx + x0 - G::PAD + M) & (M - 1));
      offk = (int)(((long long)g0r * nx + x0) & 15);
    }
    if (active) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        if (UNAL) {
          const int off = ((cy(i) > 0 ? bm : (cy(i) < 0 ? bp : b0)) + (int)((i * p.N) & (M - 1))) & (M - 1);
          const int q = pos - cx(i) + off;
          f[i] = load_pair<S>(st + i * RB, q, q & 1);
          if (fixw) {
            const T* sd = reinterpret_cast<const T*>(st + Slot2<S, MASKED, UNAL>::SIDE_OFF) + 4 * i;
            const int e0 = pos - cx(i);
            if (e0 < ea) f[i].x = Store<S>::raw_smem(sd, e0 - (G::PAD - 2));
            if (e0 >= eb) f[i].x = Store<S>::raw_smem(sd, 2 + e0 - eb);
            if (e0 + 1 >= eb) f[i].y = Store<S>::raw_smem(sd, 3 + e0 - eb);
          }
        } else {
          f[i] = load_pair<S>(st + i * RB, pos - cx(i), cx(i));
        }
      }
      moments9(f, rho, jx, jy);
      *reinterpret_cast<float2*>(&sm.ring[k & 3][jc]) = psi_of(full_rho<S != LBM_F32>(rho, p), p);
      if (MASKED) {
        if (UNAL) {
          const unsigned char* mr = st + Q * RB + offk + 2 * tid;
          m = (unsigned)mr[0] | ((unsigned)mr[1] << 8);
        } else {
          m = *reinterpret_cast<const uint16_t*>(st + Q * RB + 2 * tid);
        }
      }
    } else if (helper) {
      const int ho =
          UNAL ? ((hcy > 0 ? bm : (hcy < 0 ? bp : b0)) + (int)((hplane * p.N) & (M - 1))) & (M - 1) : 0;
      float v = hlane ? Store<S>::raw_smem(reinterpret_cast<const T*>(st + hplane * RB), hpos + ho) : 0.f;
      if (UNAL && hlane && (hpos < ea || hpos >= eb)) {
        const T* sd = reinterpret_cast<const T*>(st + Slot2<S, MASKED, UNAL>::SIDE_OFF) + 4 * hplane;
        v = Store<S>::raw_smem(sd, hpos < ea ? hpos - (G::PAD - 2) : 2 + hpos - eb);
      }
      const float t1 = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, 1));
      const float t2 = __fadd_rn(t1, __shfl_xor_sync(0xffffffffu, t1, 2));
      const float t3 = __fadd_rn(t2, __shfl_xor_sync(0xffffffffu, t2, 4));
      const float rh = full_rho<S != LBM_F32>(__fadd_rn(t3, __shfl_xor_sync(0xffffffffu, t2, 8)), p);
      if (lane == 0) sm.ring[k & 3][1] = psi_of(rh, p);
      if (lane == 16) sm.ring[k & 3][width + 2] = psi_of(rh, p);
    }
    __syncthreads();
    if (*sm.abort_flag) {
      k_abort = k;
      break;
    }
    if (helper) {
      if (k + NSTAGE - 1 < nst)
        issue_stage2<S, MASKED, NSTAGE, UNAL>(p, src, sm.stages, sm.bars, gk + NSTAGE - 1, k + NSTAGE - 1, y0, x0,
                                              width, lane);
    } else if (k >= 2 && active) {
      const int rc = y0 + k - 2;
      const int srow[3] = {(k - 2) & 3, (k - 1) & 3, k & 3};  // rows rc-1, rc, rc+1
      float2 nb[3][3];  // [row][left, centre, right] for the pair
#pragma unroll
      for (int r3 = 0; r3 < 3; ++r3) {
        const float* rr = sm.ring[srow[r3]];
        const float2 c2 = *reinterpret_cast<const float2*>(rr + jc);
        nb[r3][0] = make_float2(rr[jc - 1], c2.x);
        nb[r3][1] = c2;
        nb[r3][2] = make_float2(c2.y, rr[jc + 2]);
      }
      const float2 psi_c = nb[1][1];
      float2 sv[Q];
#pragma unroll
      for (int i = 1; i < Q; ++i) sv[i] = nb[cy(i) + 1][cx(i) + 1];
      if (MASKED && m_prev) {
        const unsigned ma = m_prev & 0xffu, mb = m_prev >> 8;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
          if ((ma >> (i - 1)) & 1u) sv[i].x = psi_c.x;
          if ((mb >> (i - 1)) & 1u) sv[i].y = psi_c.y;
        }
      }
      float2 Fx, Fy;
      force_of(sv, psi_c, p.G, Fx, Fy);
      collide<TAU_ONE, S != LBM_F32>(fprev, rho_prev, jx_prev, jy_prev, Fx, Fy, p, bad);
      const size_t base = (size_t)rc * nx + x0 + 2 * tid;
      if (UNAL) {
        // a pair at an odd buffer index (odd row start, or odd i N) cannot
        // take one vector store; with an odd width the last pair's second
        // cell is the right halo cell (computed for its psi only) and is not
        // stored
        const bool second = 2 * tid + 1 < width;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
          const size_t idx = (size_t)i * p.N + base;
          if ((idx & 1) || !second) {
            Store<S>::store_raw(dst, idx, fprev[i].x);
            if (second) Store<S>::store_raw(dst, idx + 1, fprev[i].y);
          } else {
            store_pair<S>(dst, idx, fprev[i]);
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) store_pair<S>(dst, (size_t)i * p.N + base, fprev[i]);
      }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) fprev[i] = f[i];
    rho_prev = rho;
    jx_prev = jx;
    jy_prev = jy;
    m_prev = m;
  }
  if (k_abort >= 0) {
    // a stage never completed: record it, then wait (bounded) for the copies
    // of every stage issued and not consumed before the CTA leaves
    if (tid == 0) {
      atomicOr(p.flags + FLAG_TIMEOUT, 1);
      const int issued = min(nst, k_abort + NSTAGE - 1);
      for (int q = k_abort; q < issued; ++q)
        mbar_wait(sm.bars + (g0 + q) % NSTAGE, ((g0 + q) / NSTAGE) & 1u, 500000000ull);
    }
    __syncthreads();
    return false;
  }
  gstage = g0 + nst;
  return true;
}

template <int S, bool MASKED, int NSTAGE, bool UNAL>
__device__ __forceinline__ void march2_init(const Tma2Smem<S, MASKED, NSTAGE, UNAL>& sm) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(sm.bars + s, 1);
    *sm.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// One box, one work item per CTA: strip blockIdx.x (kBX2 columns), row chunk blockIdx.y.
template <int S, bool MASKED, bool TAU_ONE, int NSTAGE, int MINB, bool UNAL>
__global__ void __launch_bounds__(kTmaThreads, MINB) k_step_tma2(const StepParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Tma2Smem<S, MASKED, NSTAGE, UNAL> sm(smem);
  const int x0 = blockIdx.x * kBX2;
  const int y0 = blockIdx.y * p.rows_per_chunk;
  const int y1 = min(y0 + p.rows_per_chunk, p.ny);
  if (y0 >= y1) return;
  march2_init(sm);
  unsigned gstage = 0;
  int bad = 0;
  const int width = min(kBX2, p.nx - x0);
  const bool ok = width == kBX2
                      ? march2<S, MASKED, TAU_ONE, NSTAGE, true, UNAL>(p, sm, x0, width, y0, y1, gstage, bad)
                      : march2<S, MASKED, TAU_ONE, NSTAGE, false, UNAL>(p, sm, x0, width, y0, y1, gstage, bad);
  if (!ok) return;
  if (bad) atomicOr(p.flags + FLAG_NUMERIC, 1);
}

// One box, dynamically scheduled: as many CTAs as fit take row chunks (of
// `rows` rows, gx strips) from a device counter until all are done. With
// chunks a few times shorter than a static split, CTAs that march fast take
// more chunks and the launch does not wait for the slowest of
// one-chunk-per-CTA (8192^2: FP32 0.817 -> 0.757 ms, FP16 0.509 -> 0.481
// ms). The counters are zero between launches: the last CTA to finish
// resets them.
template <int S, bool MASKED, bool TAU_ONE, int NSTAGE, int MINB, bool UNAL>
__global__ void __launch_bounds__(kTmaThreads, MINB) k_step_dyn(const StepParams p, int rows, int gx, int nitems) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int item_sh;
  const Tma2Smem<S, MASKED, NSTAGE, UNAL> sm(smem);
  march2_init(sm);
  int* counter = p.flags + FLAG_ITEM;
  unsigned gstage = 0;
  int bad = 0;
  for (int guard = 0; guard < nitems + 1; ++guard) {
    __syncthreads();  // the previous chunk's ring and item index are no longer read
    if (threadIdx.x == 0) item_sh = atomicAdd(counter, 1);
    __syncthreads();
    const int w = item_sh;
    if (w >= nitems) break;
    // row-major chunk order: the strips of a chunk row run together, so
    // the halo columns a strip shares with its neighbours are read while
    // still in L2 (measured for 16-bit storage at 8192^2 after the packed
    // arithmetic: 0.459 ms strip by strip, 0.450 row-major)
    const int sx = w % gx, cyk = w / gx;
    const int x0 = sx * kBX2, y0 = cyk * rows;
    const int y1 = min(y0 + rows, p.ny), width = min(kBX2, p.nx - x0);
    // full strips take the compile-time-width march (with tau != 1 the two
    // inlined copies would spill at this kernel's register budget)
    const bool ok = TAU_ONE && width == kBX2
                        ? march2<S, MASKED, TAU_ONE, NSTAGE, TAU_ONE, UNAL>(p, sm, x0, width, y0, y1, gstage, bad)
                        : march2<S, MASKED, TAU_ONE, NSTAGE, false, UNAL>(p, sm, x0, width, y0, y1, gstage, bad);
    if (!ok) break;  // a stage wait timed out (recorded); no further chunks
  }
  if (bad) atomicOr(p.flags + FLAG_NUMERIC, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    // every CTA arrives here after its last draw from the counter
    if (atomicAdd(p.flags + FLAG_DONE, 1) == (int)gridDim.x - 1) {
      *counter = 0;
      p.flags[FLAG_DONE] = 0;
    }
  }
}

// Many boxes in one launch: persistent CTAs take work items (box, strip,
// row chunk) from a device counter until the list is exhausted. Each box
// reads buffer `cur ^ parity` and writes the other. Launches alternate
// parity, so two counters take turns: this launch draws from
// counters[parity] and zeroes counters[parity ^ 1] for the next one (which
// starts only after this one has finished), so no reset is launched.
template <int S, bool MASKED, bool TAU_ONE, int NSTAGE, int MINB, bool UNAL>
__global__ void __launch_bounds__(kTmaThreads, MINB)
    k_step_batch(const BatchInst* __restrict__ insts, const BatchItem* __restrict__ items, int nitems,
                 int* __restrict__ counters, int parity) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int item_sh;
  const Tma2Smem<S, MASKED, NSTAGE, UNAL> sm(smem);
  march2_init(sm);
  int* counter = counters + parity;
  if (blockIdx.x == 0 && threadIdx.x == 0) counters[parity ^ 1] = 0;
  unsigned gstage = 0;
  for (int guard = 0; guard < nitems + 1; ++guard) {
    __syncthreads();  // the previous item's ring and item index are no longer read
    if (threadIdx.x == 0) item_sh = atomicAdd(counter, 1);
    __syncthreads();
    const int w = item_sh;
    if (w >= nitems) break;
    const BatchItem it = items[w];
    const BatchInst& in = insts[it.inst];
    StepParams p{};
    const int c = in.cur ^ parity;
    p.src = c ? in.pops1 : in.pops0;
    p.dst = c ? in.pops0 : in.pops1;
    p.mask = in.mask;
    p.flags = in.flags;
    p.nx = in.nx;
    p.ny = in.ny;
    p.N = (long long)in.nx * in.ny;
    p.tau = in.tau;
    p.inv_tau = in.inv_tau;
    p.G = in.G;
    p.rho0 = in.rho0;
    p.inv_rho0 = in.inv_rho0;
    p.rho_ref = in.rho_ref;
    int bad = 0;
    // full strips take the compile-time-width march (with tau != 1 the two
    // inlined copies would spill at this kernel's register budget)
    const bool ok = TAU_ONE && it.width == kBX2
                        ? march2<S, MASKED, TAU_ONE, NSTAGE, TAU_ONE, UNAL>(p, sm, it.x0, it.width, it.y0, it.y1,
                                                                             gstage, bad)
                        : march2<S, MASKED, TAU_ONE, NSTAGE, false, UNAL>(p, sm, it.x0, it.width, it.y0, it.y1,
                                                                         gstage, bad);
    if (!ok) return;
    if (bad) atomicOr(p.flags + FLAG_NUMERIC, 1);
  }
}

// Stage ring depth and CTAs per SM, from measured sweeps at 8192^2: with
// four CTAs per SM, prefetching two rows ahead (FP32) gave more DRAM
// throughput than deeper rings (more reads in flight lowered it).
template <int S>
constexpr int tma_stages() { return S == LBM_F32 ? 3 : 6; }
constexpr int kTmaMinBlocks = 4;

template <int S>
bool tma_ok(int nx) {
  return nx % 16 == 0 && nx >= TmaGeom<S>::WIN;
}

int sm_count() { return device_sm_count(); }

// Rows per chunk so that all CTAs are resident at once (one wave).
void tma_geometry(int nx, int ny, int resident_per_sm, int* gx, int* gy, int* rows) {
  *gx = (nx + kBX - 1) / kBX;
  const int resident = resident_per_sm * sm_count();
  int g = resident / *gx;
  if (g < 1) g = 1;
  if (g > ny) g = ny;
  *rows = (ny + g - 1) / g;
  *gy = (ny + *rows - 1) / *rows;
}

template <int S, bool MASKED, bool TAU_ONE>
cudaError_t launch_tma(const StepParams& p, cudaStream_t s) {
  constexpr int NS = tma_stages<S>();
  auto kern = k_step_tma<S, MASKED, TAU_ONE, NS, kTmaMinBlocks>;
  constexpr size_t smem = tma_smem_bytes_c<S, MASKED, NS>();
  static int resident = 0;  // per instantiation
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTmaThreads, smem);
    if (e != cudaSuccess) return e;
    resident = occ > 0 ? occ : 1;
  }
  int gx, gy, rows;
  tma_geometry(p.nx, p.ny, resident, &gx, &gy, &rows);
  StepParams q = p;
  q.rows_per_chunk = rows;
  kern<<<dim3(gx, gy), kTmaThreads, smem, s>>>(q);
  return cudaGetLastError();
}

// Measured at 8192^2 (FP16): 4 stages at 4 CTAs per SM (56 registers, no
// spills) beat deeper rings and 3 or 5 CTAs per SM.
template <int S>
constexpr int tma2_stages() { return S == LBM_F32 ? 3 : 4; }
constexpr int kTma2MinBlocks = 4;
constexpr int kDynRows = 48;  // row chunk of the dynamically scheduled step

// Rows whose starts are 16-byte aligned for every storage (and mask rows):
// whole rows are bulk-copied. Other boxes of at least 16 columns take the
// UNAL variant (each window's part inside the row by a covering bulk copy,
// the elements of a wrapped side from the slot's side area).
template <int S>
bool tma2_ok(int nx) {
  return nx % 16 == 0;
}
inline bool tma2_unal_ok(int nx) { return nx >= 16 && nx % 16 != 0; }

template <int S, bool MASKED, bool TAU_ONE, bool UNAL = false>
cudaError_t launch_tma2(const StepParams& p, cudaStream_t s) {
  constexpr int NS = tma2_stages<S>();
  // the relaxation blend (tau != 1) keeps both population sets live: fewer CTAs
  auto kern = k_step_tma2<S, MASKED, TAU_ONE, NS, TAU_ONE ? kTma2MinBlocks : 2, UNAL>;
  constexpr size_t smem = tma2_smem_bytes_c<S, MASKED, NS, UNAL>();
  static int resident = 0;  // per instantiation
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTmaThreads, smem);
    if (e != cudaSuccess) return e;
    resident = occ > 0 ? occ : 1;
  }
  const int gx = (p.nx + kBX2 - 1) / kBX2;
  int g = resident * sm_count() / gx;
  if (g < 1) g = 1;
  if (g > p.ny) g = p.ny;
  StepParams q = p;
  q.rows_per_chunk = (p.ny + g - 1) / g;
  const int gy = (p.ny + q.rows_per_chunk - 1) / q.rows_per_chunk;
  kern<<<dim3(gx, gy), kTmaThreads, smem, s>>>(q);
  return cudaGetLastError();
}

template <int S, bool MASKED, bool TAU_ONE, bool UNAL = false>
cudaError_t launch_dyn(const StepParams& p, cudaStream_t s) {
  constexpr int NS = tma2_stages<S>();
  auto kern = k_step_dyn<S, MASKED, TAU_ONE, NS, TAU_ONE ? kTma2MinBlocks : 2, UNAL>;
  constexpr size_t smem = tma2_smem_bytes_c<S, MASKED, NS, UNAL>();
  static int resident = 0;  // per instantiation: CTAs that fit the GPU at once
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTmaThreads, smem);
    if (e != cudaSuccess) return e;
    resident = (occ > 0 ? occ : 1) * sm_count();
  }
  const int gx = (p.nx + kBX2 - 1) / kBX2;
  // 48-row chunks (best at 8192^2: 4.5 waves of 608 CTAs for 16-bit
  // storage, 6 of 456 for FP32) unless they make fewer than four waves;
  // then whole waves: the fewest for 16-bit storage, at least four for FP32
  // (4096^2: FP16 0.170 -> 0.135 ms, FP32 0.214 -> 0.205 ms;
  // 5120^2: 0.224 -> 0.207, 0.320 -> 0.309; 6144^2: 0.305 -> 0.287,
  // 0.442 -> 0.437). A box of at most one wave gets one chunk per CTA.
  const int rows = dyn_chunk_rows(gx, p.ny, resident, kDynRows, 4, S == LBM_F32 ? 4 : 1);
  const long long items = (long long)gx * ((p.ny + rows - 1) / rows);
  if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int nitems = (int)items;
  // automatic choice: with no more chunks than resident CTAs there is nothing
  // to balance, and the static split saves the counter's round trips (a
  // few microseconds, a large part of a small box's step)
  if (p.force_generic == 0 && nitems <= resident) return launch_tma2<S, MASKED, TAU_ONE, UNAL>(p, s);
  const int grid = nitems < resident ? nitems : resident;
  kern<<<grid, kTmaThreads, smem, s>>>(p, rows, gx, nitems);
  return cudaGetLastError();
}

template <int S, bool MASKED, bool TAU_ONE>
cudaError_t launch_strip(const StepParams& p, cudaStream_t s) {
  int gx, gy, rows, block;
  step_geometry(p.nx, p.ny, &gx, &gy, &rows, &block);
  StepParams q = p;
  q.rows_per_chunk = rows;
  k_step_strip<S, MASKED, TAU_ONE><<<dim3(gx, gy), block, 0, s>>>(q);
  return cudaGetLastError();
}

// Variant 0 (automatic): the two-cell staged march over dynamically
// scheduled row chunks wherever rows are 16-byte multiples (measured fastest
// for every storage: 8192^2 FP32 0.757 ms against 0.815 for the one-cell
// static kernel; boxes with no more chunks than resident CTAs take the
// static split of variant 3), else plain loads; 1: plain loads; 2: one-cell staged;
// 3: two-cell staged, one chunk per CTA; 4: two-cell staged, dynamic chunks.
template <int S, bool MASKED, bool TAU_ONE>
cudaError_t launch_variant(const StepParams& p, cudaStream_t s) {
  const int v = p.force_generic;
  if ((v == 4 || v == 0) && tma2_ok<S>(p.nx)) return launch_dyn<S, MASKED, TAU_ONE>(p, s);
  // automatic choice for other widths: the unaligned staging where the box
  // has more than two strips (FP16 2047^2: 0.077 ms against 0.100 plain;
  // 2040^2: 0.074 against 0.099), plain loads for boxes of at most two
  // strips, every one of which wraps (1001^2: 0.035 plain against 0.038;
  // 511^2: 0.020 against 0.026)
  if ((v == 4 || (v == 0 && p.nx > 2 * kBX2)) && tma2_unal_ok(p.nx)) return launch_dyn<S, MASKED, TAU_ONE, true>(p, s);
  if (v == 3) {
    if (tma2_ok<S>(p.nx)) return launch_tma2<S, MASKED, TAU_ONE>(p, s);
    if (tma2_unal_ok(p.nx)) return launch_tma2<S, MASKED, TAU_ONE, true>(p, s);
  }
  if (v != 1 && tma_ok<S>(p.nx)) return launch_tma<S, MASKED, TAU_ONE>(p, s);
  return launch_strip<S, MASKED, TAU_ONE>(p, s);
}

template <int S>
cudaError_t launch_typed(const StepParams& p, cudaStream_t s) {
  const bool tau_one = p.tau == 1.0f;
  if (p.mask) return tau_one ? launch_variant<S, true, true>(p, s) : launch_variant<S, true, false>(p, s);
  return tau_one ? launch_variant<S, false, true>(p, s) : launch_variant<S, false, false>(p, s);
}

}  // namespace

int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
    cached[dev] = n;
  }
  return cached[dev];
}

void step_geometry(int nx, int ny, int* grid_x, int* grid_y, int* rows_per_chunk, int* block) {
  const int gx = (nx + kBX - 1) / kBX;
  const int target = device_sm_count() * 6;  // CTAs: a few per SM
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

// ---------------------------------------------------------------- batched launch
namespace {

template <int S, bool MASKED, bool TAU_ONE, bool UNAL>
struct BatchKernel {
  static constexpr int NS = tma2_stages<S>();
  static constexpr int MINB = TAU_ONE ? kTma2MinBlocks : 2;
  static constexpr size_t SMEM = tma2_smem_bytes_c<S, MASKED, NS, UNAL>();
  static int resident() {  // CTAs that fit the GPU at once
    static int r = 0;
    if (r == 0) {
      auto kern = k_step_batch<S, MASKED, TAU_ONE, NS, MINB, UNAL>;
      if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM) != cudaSuccess) return 0;
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTmaThreads, SMEM) != cudaSuccess) return 0;
      r = (occ > 0 ? occ : 1) * sm_count();
    }
    return r;
  }
  static cudaError_t launch(const BatchInst* insts, const BatchItem* items, int nitems, int* counters, int parity,
                            cudaStream_t s) {
    const int res = resident();
    if (res == 0) return cudaErrorInvalidConfiguration;
    const int grid = nitems < res ? nitems : res;
    if (grid <= 0) return cudaMemsetAsync(counters, 0, 2 * sizeof(int), s);  // no launch resets them
    k_step_batch<S, MASKED, TAU_ONE, NS, MINB, UNAL>
        <<<grid, kTmaThreads, SMEM, s>>>(insts, items, nitems, counters, parity);
    return cudaGetLastError();
  }
};

template <int S, bool UNAL>
cudaError_t launch_batch_su(bool masked, bool tau_one, const BatchInst* insts, const BatchItem* items, int nitems,
                            int* counter, int parity, cudaStream_t s) {
  if (masked)
    return tau_one ? BatchKernel<S, true, true, UNAL>::launch(insts, items, nitems, counter, parity, s)
                   : BatchKernel<S, true, false, UNAL>::launch(insts, items, nitems, counter, parity, s);
  return tau_one ? BatchKernel<S, false, true, UNAL>::launch(insts, items, nitems, counter, parity, s)
                 : BatchKernel<S, false, false, UNAL>::launch(insts, items, nitems, counter, parity, s);
}

template <int S>
cudaError_t launch_batch_s(bool masked, bool tau_one, bool unal, const BatchInst* insts, const BatchItem* items,
                           int nitems, int* counter, int parity, cudaStream_t s) {
  return unal ? launch_batch_su<S, true>(masked, tau_one, insts, items, nitems, counter, parity, s)
              : launch_batch_su<S, false>(masked, tau_one, insts, items, nitems, counter, parity, s);
}

template <int S>
int batch_resident_s(bool masked, bool tau_one) {
  if (masked)
    return tau_one ? BatchKernel<S, true, true, false>::resident() : BatchKernel<S, true, false, false>::resident();
  return tau_one ? BatchKernel<S, false, true, false>::resident() : BatchKernel<S, false, false, false>::resident();
}

}  // namespace

cudaError_t launch_step_batch(int storage, bool masked, bool tau_one, bool unal, const BatchInst* insts,
                              const BatchItem* items, int nitems, int* counter, int parity, cudaStream_t s) {
  switch (storage) {
    case LBM_F32: return launch_batch_s<LBM_F32>(masked, tau_one, unal, insts, items, nitems, counter, parity, s);
    case LBM_F16_DEV:
      return launch_batch_s<LBM_F16_DEV>(masked, tau_one, unal, insts, items, nitems, counter, parity, s);
    case LBM_BF16_DEV:
      return launch_batch_s<LBM_BF16_DEV>(masked, tau_one, unal, insts, items, nitems, counter, parity, s);
    default: return cudaErrorInvalidValue;
  }
}

int batch_resident_ctas(int storage, bool masked, bool tau_one) {
  switch (storage) {
    case LBM_F32: return batch_resident_s<LBM_F32>(masked, tau_one);
    case LBM_F16_DEV: return batch_resident_s<LBM_F16_DEV>(masked, tau_one);
    case LBM_BF16_DEV: return batch_resident_s<LBM_BF16_DEV>(masked, tau_one);
    default: return 0;
  }
}

bool step_tma_allowed(int storage, int nx) {
  return storage == LBM_F32 ? tma_ok<LBM_F32>(nx)
                            : (storage == LBM_F16_DEV ? tma_ok<LBM_F16_DEV>(nx) : tma_ok<LBM_BF16_DEV>(nx));
}

bool step_tma2_allowed(int storage, int nx) {
  return storage == LBM_F32 ? tma2_ok<LBM_F32>(nx)
                            : (storage == LBM_F16_DEV ? tma2_ok<LBM_F16_DEV>(nx) : tma2_ok<LBM_BF16_DEV>(nx));
}

bool step_tma2_unaligned_allowed(int nx) { return tma2_unal_ok(nx); }

cudaError_t launch_step(int storage, const StepParams& p, cudaStream_t s) {
  switch (storage) {
    case LBM_F32: return launch_typed<LBM_F32>(p, s);
    case LBM_F16_DEV: return launch_typed<LBM_F16_DEV>(p, s);
    case LBM_BF16_DEV: return launch_typed<LBM_BF16_DEV>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lbm
