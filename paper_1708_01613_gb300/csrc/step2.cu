// Two-component step: melt (m) and gas (g) lattices coupled every step
// (Sec. 2.1.5, the two-lattice description with the common velocity and the
// per-component velocities of Eqs. 36-40), read as the Shan-Chen mixture:
//
//   F_s(x) = -psi_s(x) sum_s' G_ss' S_s'(x),  S_s'(x) = sum_i w_i psi~_s'(x+e_i) e_i
//   u'     = (j_m/tau_m + j_g/tau_g) / (rho_m/tau_m + rho_g/tau_g)
//   u_s    = u' + tau_s F_s / rho_s     (u' where rho_s = 0)
//   f_s,i  <- f_s,i - (f_s,i - f^eq_i(rho_s, u_s)) / tau_s
//
// with psi_s = rho0 (1 - exp(-rho_s/rho0)) (Eq. 30), G_mg = G_gm, and the
// barrier substitution psi~ = psi_s'(x) across a blocked edge (where both
// components' populations bounce back: launch_bounce after the step). FP32 storage;
// buffer layout: 18 planes, the nine melt planes then the nine gas planes,
// each holding f^out at its source cell (the next step pulls f_i(x) from
// x - e_i).
//
// k_step2_strip marches a 256-column strip down a row chunk with plain
// loads: for each row it pulls both components of the strip's cells (and of
// one halo column per side), puts psi_m and psi_g into two four-row rings in
// shared memory, and one barrier later runs force, collision and store of
// the previous row from registers. k_step2_tma (below) is the same march
// with the rows staged by cp.async.bulk over row chunks drawn from a device
// counter; both use the per-cell functions here.
#include "lbm_internal.cuh"
#include "tma.cuh"

namespace lbm {
namespace {

constexpr int kBX2C = 256;

__device__ __forceinline__ int wrap_1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// The nine pulled populations of one component at (x, row r), rows given
// as offsets of r - 1, r, r + 1 and columns x - 1, x, x + 1 (wrapped).
__device__ __forceinline__ void pull9(const float* __restrict__ src, long long N, long long rowm, long long row0,
                                      long long rowp, int xm, int x, int xp, float f[Q]) {
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    // f_i(x) = B_i(x - e_i)
    const long long row = cy(i) > 0 ? rowm : (cy(i) < 0 ? rowp : row0);
    const int xs = cx(i) > 0 ? xm : (cx(i) < 0 ? xp : x);
    f[i] = __ldg(src + (size_t)i * N + row + xs);
  }
}

__device__ __forceinline__ void mom(const float f[Q], float& rho, float& jx, float& jy) {
  rho = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  jx = (f[1] - f[3]) + ((f[5] - f[7]) + (f[8] - f[6]));
  jy = (f[2] - f[4]) + ((f[5] - f[7]) + (f[6] - f[8]));
}

__device__ __forceinline__ float psi2(float rho, const Step2Params& p) {
  return p.rho0 * (1.0f - __expf(-rho * p.inv_rho0));
}

// S = sum_i w_i psi~(x + e_i) e_i from a ring (rows sm, s0, sp; column jc),
// psi~ = psi(x) on blocked edges.
__device__ __forceinline__ void nsum(const float (*ring)[kBX2C + 2], int sm, int s0, int sp, int jc, unsigned m,
                                     float& Sx, float& Sy) {
  const float c = ring[s0][jc];
  float s[Q];
#pragma unroll
  for (int i = 1; i < Q; ++i) s[i] = ring[cy(i) > 0 ? sp : (cy(i) < 0 ? sm : s0)][jc + cx(i)];
  if (m) {  // most cells have no blocked edge
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if ((m >> (i - 1)) & 1u) s[i] = c;
  }
  const float w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
  Sx = w1 * (s[1] - s[3]) + w5 * ((s[5] - s[7]) + (s[8] - s[6]));
  Sy = w1 * (s[2] - s[4]) + w5 * ((s[5] - s[7]) + (s[6] - s[8]));
}

// Eq. 14 by opposite pairs: with s = a + 4.5 rho (e.u)^2 and t = 3 rho e.u,
// f^eq_i = w_i (s + t) and f^eq of the opposite direction = w_i (s - t).
__device__ __forceinline__ void collide9(float f[Q], float rho, float ux, float uy, float inv_tau, bool tau_one) {
  const float uu = ux * ux + uy * uy;
  const float a = rho * (1.0f - 1.5f * uu);
  const float r3 = 3.0f * rho, r45 = 4.5f * rho;
  const float w1 = 1.0f / 9.0f, w5 = 1.0f / 36.0f;
  float feq[Q];
  feq[0] = (4.0f / 9.0f) * a;
  const float eu[4] = {ux, uy, ux + uy, uy - ux};  // directions 1, 2, 5, 6 (opposites 3, 4, 7, 8)
  const int ip[4] = {1, 2, 5, 6}, im[4] = {3, 4, 7, 8};
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    const float w = d < 2 ? w1 : w5;
    const float sv = a + r45 * eu[d] * eu[d], t = r3 * eu[d];
    feq[ip[d]] = w * (sv + t);
    feq[im[d]] = w * (sv - t);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = tau_one ? feq[i] : f[i] + (feq[i] - f[i]) * inv_tau;
}

// Force (both components, barrier substitution), common velocity, both
// collisions and the 18 stores of one cell whose psi rows sit in the rings.
template <bool TAU_ONE>
__device__ __forceinline__ void finish2(const Step2Params& p, const float (*ring_m)[kBX2C + 2],
                                        const float (*ring_g)[kBX2C + 2], int sm, int s0, int sp, int jc, unsigned m,
                                        float pm[Q], float pg[Q], float rm, float jxm, float jym, float rg, float jxg,
                                        float jyg, float* __restrict__ dst, float* __restrict__ dstg, size_t base,
                                        int& bad) {
  float Smx, Smy, Sgx, Sgy;
  nsum(ring_m, sm, s0, sp, jc, m, Smx, Smy);
  nsum(ring_g, sm, s0, sp, jc, m, Sgx, Sgy);
  const float psim = ring_m[s0][jc], psig = ring_g[s0][jc];
  const float Fmx = -psim * (p.G_mm * Smx + p.G_mg * Sgx), Fmy = -psim * (p.G_mm * Smy + p.G_mg * Sgy);
  const float Fgx = -psig * (p.G_mg * Smx + p.G_gg * Sgx), Fgy = -psig * (p.G_mg * Smy + p.G_gg * Sgy);
  const float den = rm * p.inv_tau_m + rg * p.inv_tau_g;
  bad |= !(rm >= 0.f && rg >= 0.f && den > 0.f && den < 1e30f);
  // one reciprocal per denominator (an empty component's 1/0 is never selected)
  const float iden = __frcp_rn(den), irm = __frcp_rn(rm), irg = __frcp_rn(rg);
  const float ux = (jxm * p.inv_tau_m + jxg * p.inv_tau_g) * iden;
  const float uy = (jym * p.inv_tau_m + jyg * p.inv_tau_g) * iden;
  const float tm = p.tau_m * irm, tg = p.tau_g * irg;
  const float umx = rm > 0.f ? ux + tm * Fmx : ux;
  const float umy = rm > 0.f ? uy + tm * Fmy : uy;
  const float ugx = rg > 0.f ? ux + tg * Fgx : ux;
  const float ugy = rg > 0.f ? uy + tg * Fgy : uy;
  collide9(pm, rm, umx, umy, p.inv_tau_m, TAU_ONE);
  collide9(pg, rg, ugx, ugy, p.inv_tau_g, TAU_ONE);
  const size_t N = (size_t)p.N;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    dst[(size_t)i * N + base] = pm[i];
    dstg[(size_t)i * N + base] = pg[i];
  }
}

// TAU_ONE (both relaxation times 1): the collision output is the
// equilibrium alone, so only the moments of the previous row are kept.
template <bool MASKED, bool TAU_ONE>
__global__ void __launch_bounds__(kBX2C, TAU_ONE ? 4 : 2) k_step2_strip(const Step2Params p) {
  __shared__ float ring_m[4][kBX2C + 2];
  __shared__ float ring_g[4][kBX2C + 2];
  const float* __restrict__ src = static_cast<const float*>(p.src);
  float* __restrict__ dst = static_cast<float*>(p.dst);
  const long long N = p.N;
  const float* __restrict__ srcg = src + 9 * N;
  float* __restrict__ dstg = dst + 9 * N;
  const int nx = p.nx, ny = p.ny;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * kBX2C;
  const int x = x0 + tid;
  const bool active = x < nx;
  const int last = min(x0 + kBX2C, nx) - 1;
  const int y0 = blockIdx.y * p.rows_per_chunk;
  const int y1 = min(y0 + p.rows_per_chunk, ny);
  if (y0 >= y1) return;  // uniform over the block
  const int xc = active ? x : last;
  const int xm = wrap_1(xc - 1, nx), xp = wrap_1(xc + 1, nx);
  const int xl = wrap_1(x0 - 1, nx), xlm = wrap_1(x0 - 2, nx);
  const int xr = wrap_1(last + 1, nx), xrp = wrap_1(last + 2, nx);
  const int jc = tid + 1;

  float pm[Q], pg[Q];
  float rm_p = 1.f, jxm_p = 0.f, jym_p = 0.f, rg_p = 0.f, jxg_p = 0.f, jyg_p = 0.f;
  int bad = 0;
  for (int r = y0 - 1, k = 0; r <= y1; ++r, ++k) {
    const int rr = wrap_1(r, ny);  // r in [-1, ny]
    const long long row0 = (long long)rr * nx;
    const long long rowm = (long long)wrap_1(rr - 1, ny) * nx;
    const long long rowp = (long long)wrap_1(rr + 1, ny) * nx;
    float fm[Q], fg[Q];
    float rm = 1.f, jxm = 0.f, jym = 0.f, rg = 0.f, jxg = 0.f, jyg = 0.f;
    if (active) {
      pull9(src, N, rowm, row0, rowp, xm, x, xp, fm);
      pull9(srcg, N, rowm, row0, rowp, xm, x, xp, fg);
      mom(fm, rm, jxm, jym);
      mom(fg, rg, jxg, jyg);
      ring_m[k & 3][jc] = psi2(rm, p);
      ring_g[k & 3][jc] = psi2(rg, p);
    }
    // halo cells x0 - 1 (warp 0) and last + 1 (warp 1): one population per
    // lane (melt in lanes 0-8, gas in lanes 16-24), summed per half-warp
    if (tid < 64) {
      const int lane = tid & 31, i = lane & 15;
      const bool right = tid >= 32;
      float v = 0.f;
      if (i < Q) {
        const float* base = lane < 16 ? src : srcg;
        const long long row = cy(i) > 0 ? rowm : (cy(i) < 0 ? rowp : row0);
        const int xs = cx(i) > 0 ? (right ? last : xlm) : (cx(i) < 0 ? (right ? xrp : x0) : (right ? xr : xl));
        v = __ldg(base + (size_t)i * N + row + xs);
      }
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 8);
      const int col = right ? last - x0 + 2 : 0;
      if (lane == 0) ring_m[k & 3][col] = psi2(v, p);
      if (lane == 16) ring_g[k & 3][col] = psi2(v, p);
    }
    __syncthreads();
    if (k >= 2 && active) {
      const int rc = r - 1;
      const unsigned m = MASKED ? p.mask[(size_t)rc * nx + x] : 0u;
      finish2<TAU_ONE>(p, ring_m, ring_g, (k - 2) & 3, (k - 1) & 3, k & 3, jc, m, pm, pg, rm_p, jxm_p, jym_p,
                       rg_p, jxg_p, jyg_p, dst, dstg, (size_t)rc * nx + x, bad);
    }
    if (!TAU_ONE) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        pm[i] = fm[i];
        pg[i] = fg[i];
      }
    }
    rm_p = rm;
    jxm_p = jxm;
    jym_p = jym;
    rg_p = rg;
    jxg_p = jxg;
    jyg_p = jyg;
  }
  if (bad) atomicOr(p.flags + FLAG_NUMERIC, 1);
}

// ------------------------------------------------------------------ staged
// The same march with the 18 source rows of every output row (with a
// 16-byte halo) copied into shared-memory stages by cp.async.bulk, issued
// NSTAGE - 1 rows ahead by a ninth warp that also sums the four halo cells
// (melt and gas, left and right) lane-parallel. Needs nx % 16 == 0 (16-byte
// rows and mask pieces) and nx >= kBX2C + 16 (a staged row wraps at most
// once).
constexpr int kPad2C = 4;                        // halo pad: 16 bytes of FP32
constexpr int kWin2C = kBX2C + 2 * kPad2C;       // floats per staged row
constexpr int kRow2C = kWin2C * 4;               // bytes, a multiple of 16
constexpr int kThreads2C = kBX2C + 32;

template <bool MASKED>
constexpr int stage2c_bytes() { return 2 * Q * kRow2C + (MASKED ? kBX2C : 0); }

template <bool MASKED, int NSTAGE>
constexpr size_t smem2c_bytes() {
  return (size_t)NSTAGE * stage2c_bytes<MASKED>() + 2 * 4 * (kBX2C + 2) * 4 + NSTAGE * 8 + 16;
}

// Lane l < 18 of the ninth warp copies plane l (melt 0-8, gas 9-17) of
// stage k (output row y0 - 1 + k) into the slot of the CTA's stage count gk;
// lane 18 copies the mask row.
template <bool MASKED, int NSTAGE>
__device__ __forceinline__ void issue2c(const Step2Params& p, unsigned char* stages, uint64_t* bars, unsigned gk, int k,
                                        int y0, int x0, int lane) {
  constexpr uint32_t STAGE = stage2c_bytes<MASKED>();
  const int slot = (int)(gk % NSTAGE);
  unsigned char* st = stages + (size_t)slot * STAGE;
  uint64_t* bar = bars + slot;
  const int r = y0 - 1 + k;
  const int ny = p.ny, nx = p.nx;
  if (lane < 2 * Q + (MASKED ? 1 : 0)) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (lane == 0) mbar_expect_tx(bar, STAGE);
  __syncwarp();
  if (lane < 2 * Q) {
    const int i = lane % Q;
    int g = r - cy(i);
    g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
    g = g < 0 ? g + ny : (g >= ny ? g - ny : g);
    const float* row = static_cast<const float*>(p.src) + (size_t)lane * p.N + (size_t)g * nx;
    copy_row_wrapped<float>(reinterpret_cast<float*>(st + lane * kRow2C), row, x0 - kPad2C, kWin2C, nx, bar);
  } else if (MASKED && lane == 2 * Q) {
    const int g = r < 0 ? r + ny : (r >= ny ? r - ny : r);
    copy_row_wrapped<uint8_t>(st + 2 * Q * kRow2C, p.mask + (size_t)g * nx, x0, kBX2C, nx, bar);
  }
}

// Shared-memory layout of the staged kernel.
template <bool MASKED, int NSTAGE>
struct Smem2C {
  unsigned char* stages;
  float (*ring_m)[kBX2C + 2];
  float (*ring_g)[kBX2C + 2];
  uint64_t* bars;
  int* abort_flag;
  __device__ __forceinline__ explicit Smem2C(unsigned char* smem) {
    constexpr int STAGE = stage2c_bytes<MASKED>();
    stages = smem;
    ring_m = reinterpret_cast<float(*)[kBX2C + 2]>(smem + (size_t)NSTAGE * STAGE);
    ring_g = ring_m + 4;
    bars = reinterpret_cast<uint64_t*>(smem + (size_t)NSTAGE * STAGE + 2 * 4 * (kBX2C + 2) * 4);
    abort_flag = reinterpret_cast<int*>(bars + NSTAGE);
  }
};

// The staged march of one chunk: columns x0 .. x0 + width, rows y0 .. y1.
// `gstage` counts the stages this CTA consumed before (mbarrier phases carry
// over between chunks). Returns false if a stage wait timed out (recorded;
// the CTA must leave).
template <bool MASKED, bool TAU_ONE, int NSTAGE>
__device__ __forceinline__ bool march2c(const Step2Params& p, const Smem2C<MASKED, NSTAGE>& sm, int x0, int y0, int y1,
                                        unsigned& gstage, int& bad) {
  constexpr int STAGE = stage2c_bytes<MASKED>();
  float* __restrict__ dst = static_cast<float*>(p.dst);
  float* __restrict__ dstg = dst + (size_t)Q * p.N;
  const int nx = p.nx;
  const int tid = threadIdx.x;
  const bool helper = tid >= kBX2C;
  const int lane = tid & 31;
  const int width = min(kBX2C, nx - x0);
  const bool active = !helper && tid < width;
  const int nst = (y1 - y0) + 2;  // stages = rows y0-1 .. y1
  const unsigned g0 = gstage;

  if (helper)
    for (int k = 0; k < NSTAGE - 1 && k < nst; ++k) issue2c<MASKED, NSTAGE>(p, sm.stages, sm.bars, g0 + k, k, y0, x0, lane);

  // halo lanes: lanes 0..8 the left cell (column x0 - 1), lanes 16..24 the
  // right one (column x0 + width), plane lane & 15 of the component summed
  const int hplane = lane & 15;
  const bool hlane = helper && hplane < Q;
  const int hpos = (lane < 16 ? kPad2C - 1 : kPad2C + width) - cx(hplane < Q ? hplane : 0);

  const int jc = tid + 1;
  const int pos = kPad2C + tid;
  float pm[Q], pg[Q];
  float rm_p = 1.f, jxm_p = 0.f, jym_p = 0.f, rg_p = 0.f, jxg_p = 0.f, jyg_p = 0.f;
  unsigned m_prev = 0;
  int k_abort = -1;
  for (int k = 0; k < nst; ++k) {
    const unsigned gk = g0 + k;
    const unsigned char* st = sm.stages + (size_t)(gk % NSTAGE) * STAGE;
    if (!mbar_wait(sm.bars + gk % NSTAGE, (gk / NSTAGE) & 1u)) *sm.abort_flag = 1;
    float fm[Q], fg[Q];
    float rm = 1.f, jxm = 0.f, jym = 0.f, rg = 0.f, jxg = 0.f, jyg = 0.f;
    unsigned m = 0;
    if (active) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        fm[i] = reinterpret_cast<const float*>(st + i * kRow2C)[pos - cx(i)];
        fg[i] = reinterpret_cast<const float*>(st + (Q + i) * kRow2C)[pos - cx(i)];
      }
      mom(fm, rm, jxm, jym);
      mom(fg, rg, jxg, jyg);
      sm.ring_m[k & 3][jc] = psi2(rm, p);
      sm.ring_g[k & 3][jc] = psi2(rg, p);
      if (MASKED) m = st[2 * Q * kRow2C + tid];
    } else if (helper) {
#pragma unroll
      for (int comp = 0; comp < 2; ++comp) {
        float v = hlane ? reinterpret_cast<const float*>(st + (comp * Q + hplane) * kRow2C)[hpos] : 0.f;
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        float(*ring)[kBX2C + 2] = comp ? sm.ring_g : sm.ring_m;
        if (lane == 0) ring[k & 3][0] = psi2(v, p);
        if (lane == 16) ring[k & 3][width + 1] = psi2(v, p);
      }
    }
    __syncthreads();
    if (*sm.abort_flag) {
      k_abort = k;
      break;
    }
    if (helper) {
      if (k + NSTAGE - 1 < nst)
        issue2c<MASKED, NSTAGE>(p, sm.stages, sm.bars, gk + NSTAGE - 1, k + NSTAGE - 1, y0, x0, lane);
    } else if (k >= 2 && active) {
      const int rc = y0 + k - 2;
      finish2<TAU_ONE>(p, sm.ring_m, sm.ring_g, (k - 2) & 3, (k - 1) & 3, k & 3, jc, m_prev, pm, pg, rm_p, jxm_p,
                       jym_p, rg_p, jxg_p, jyg_p, dst, dstg, (size_t)rc * nx + x0 + tid, bad);
    }
    if (!TAU_ONE) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        pm[i] = fm[i];
        pg[i] = fg[i];
      }
    }
    rm_p = rm;
    jxm_p = jxm;
    jym_p = jym;
    rg_p = rg;
    jxg_p = jxg;
    jyg_p = jyg;
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

// As many CTAs as fit draw row chunks (strip w % gx, chunk w / gx of
// `rows` rows) from a device counter until all are done, so fast CTAs take
// more chunks; the last CTA to finish resets the counters for the next
// launch.
template <bool MASKED, bool TAU_ONE, int NSTAGE, int MINB>
__global__ void __launch_bounds__(kThreads2C, MINB) k_step2_tma(const Step2Params p, int rows, int gx, int nitems) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int item_sh;
  const Smem2C<MASKED, NSTAGE> sm(smem);
  if (threadIdx.x == 0) {
    for (int q = 0; q < NSTAGE; ++q) mbar_init(sm.bars + q, 1);
    *sm.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  unsigned gstage = 0;
  int bad = 0;
  for (int guard = 0; guard < nitems + 1; ++guard) {
    __syncthreads();  // the previous chunk's ring and item index are no longer read
    if (threadIdx.x == 0) item_sh = atomicAdd(p.flags + FLAG_ITEM, 1);
    __syncthreads();
    const int w = item_sh;
    if (w >= nitems) break;
    const int y0 = (w / gx) * rows;
    if (!march2c<MASKED, TAU_ONE, NSTAGE>(p, sm, (w % gx) * kBX2C, y0, min(y0 + rows, p.ny), gstage, bad)) break;
  }
  if (bad) atomicOr(p.flags + FLAG_NUMERIC, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    // every CTA arrives here after its last draw from the counter
    if (atomicAdd(p.flags + FLAG_DONE, 1) == (int)gridDim.x - 1) {
      p.flags[FLAG_ITEM] = 0;
      p.flags[FLAG_DONE] = 0;
    }
  }
}

template <bool MASKED, bool TAU_ONE>
cudaError_t launch_step2_tma(const Step2Params& p, cudaStream_t s) {
  // measured at 8192^2 with tau = 1: since the per-cell arithmetic was cut
  // the kernel waits on its staged rows, and 3 stages at 3 CTAs per SM (72
  // registers) beat 2 stages at 4 (1.621 -> 1.498 ms; 4096^2 0.433 ->
  // 0.405, 3072^2 0.261 -> 0.237); before the cut 2 at 4 edged out 3 at 3.
  // tau != 1 keeps both components' populations across the barrier: 3 at 2.
  constexpr int NS = 3, MINB = TAU_ONE ? 3 : 2;
  auto kern = k_step2_tma<MASKED, TAU_ONE, NS, MINB>;
  constexpr size_t smem = smem2c_bytes<MASKED, NS>();
  static int resident = 0;  // per instantiation
  if (resident == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int occ = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads2C, smem);
    if (e != cudaSuccess) return e;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return cudaErrorInvalidDevice;
    resident = (occ > 0 ? occ : 1) * sms;
  }
  const int gx = (p.nx + kBX2C - 1) / kBX2C;
  // 48-row chunks when they make at least eight waves (8192^2: twelve),
  // else whole waves, at least four once one is exceeded (measured with 2
  // stages at 4 CTAs per SM: 4096^2 0.493 -> 0.432 ms, 3072^2 0.325 ->
  // 0.262, 6144^2 0.982 -> 0.935)
  const int rows = dyn_chunk_rows(gx, p.ny, resident, 48, 8, 4);
  const long long items = (long long)gx * ((p.ny + rows - 1) / rows);
  if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
  const int nitems = (int)items;
  kern<<<nitems < resident ? nitems : resident, kThreads2C, smem, s>>>(p, rows, gx, nitems);
  return cudaGetLastError();
}

// Diagnostics: melt and gas densities, the physical mixture velocity
// u = sum_s (j_s + F_s / 2) / (rho_m + rho_g) and the mixture pressure.
__global__ void k_fields2(const Step2Params p, float* __restrict__ rho_m, float* __restrict__ rho_g,
                          float* __restrict__ ux, float* __restrict__ uy, float* __restrict__ pr) {
  const float* src = static_cast<const float*>(p.src);
  const long long N = p.N;
  const int nx = p.nx, ny = p.ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)(c / nx);
    const unsigned m = p.mask ? p.mask[c] : 0u;
    float Sm[2] = {0.f, 0.f}, Sg[2] = {0.f, 0.f}, own[2] = {0.f, 0.f};
    float rm = 0.f, rg = 0.f, jx = 0.f, jy = 0.f;
    // densities of the cell and the neighbour sums from the neighbours' densities
    for (int i = 0; i < Q; ++i) {
      const int xx = wrap_1(x + cx(i), nx), yy = wrap_1(y + cy(i), ny);
      float a = 0.f, b = 0.f, ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
      for (int j = 0; j < Q; ++j) {
        const size_t idx = (size_t)wrap_1(yy - cy(j), ny) * nx + wrap_1(xx - cx(j), nx);
        const float fa = src[(size_t)j * N + idx], fb = src[(size_t)(9 + j) * N + idx];
        a += fa;
        b += fb;
        ax += cx(j) * fa;
        ay += cy(j) * fa;
        bx += cx(j) * fb;
        by += cy(j) * fb;
      }
      if (i == 0) {
        rm = a;
        rg = b;
        jx = ax + bx;
        jy = ay + by;
        own[0] = psi2(a, p);
        own[1] = psi2(b, p);
      } else {  // i = 0 comes first, so own[] is known; blocked edges take it
        const bool blocked = (m >> (i - 1)) & 1u;
        const float wa = (float)wq(i);
        const float pa = blocked ? own[0] : psi2(a, p), pb = blocked ? own[1] : psi2(b, p);
        Sm[0] += wa * cx(i) * pa;
        Sm[1] += wa * cy(i) * pa;
        Sg[0] += wa * cx(i) * pb;
        Sg[1] += wa * cy(i) * pb;
      }
    }
    const float Fx = -own[0] * (p.G_mm * Sm[0] + p.G_mg * Sg[0]) - own[1] * (p.G_mg * Sm[0] + p.G_gg * Sg[0]);
    const float Fy = -own[0] * (p.G_mm * Sm[1] + p.G_mg * Sg[1]) - own[1] * (p.G_mg * Sm[1] + p.G_gg * Sg[1]);
    const float r = rm + rg;
    if (rho_m) rho_m[c] = rm;
    if (rho_g) rho_g[c] = rg;
    if (ux) ux[c] = (jx + 0.5f * Fx) / r;
    if (uy) uy[c] = (jy + 0.5f * Fy) / r;
    if (pr)
      pr[c] = r * (1.0f / 3.0f) +
              (p.G_mm * own[0] * own[0] + 2.0f * p.G_mg * own[0] * own[1] + p.G_gg * own[1] * own[1]) *
                  (1.0f / 6.0f);
  }
}

}  // namespace

cudaError_t launch_step2(const Step2Params& p, cudaStream_t s) {
  const bool one = p.tau_m == 1.0f && p.tau_g == 1.0f;
  if (p.nx % 16 == 0 && p.nx >= kBX2C + 16) {  // staged rows
    if (p.mask) return one ? launch_step2_tma<true, true>(p, s) : launch_step2_tma<true, false>(p, s);
    return one ? launch_step2_tma<false, true>(p, s) : launch_step2_tma<false, false>(p, s);
  }
  const int gx = (p.nx + kBX2C - 1) / kBX2C;
  int g = (device_sm_count() * 4 + gx - 1) / gx;  // a few CTAs per SM
  if (g > p.ny) g = p.ny;
  if (g < 1) g = 1;
  Step2Params q = p;
  q.rows_per_chunk = (p.ny + g - 1) / g;
  const int gy = (p.ny + q.rows_per_chunk - 1) / q.rows_per_chunk;
  if (p.mask) {
    if (one) k_step2_strip<true, true><<<dim3(gx, gy), kBX2C, 0, s>>>(q);
    else k_step2_strip<true, false><<<dim3(gx, gy), kBX2C, 0, s>>>(q);
  } else {
    if (one) k_step2_strip<false, true><<<dim3(gx, gy), kBX2C, 0, s>>>(q);
    else k_step2_strip<false, false><<<dim3(gx, gy), kBX2C, 0, s>>>(q);
  }
  return cudaGetLastError();
}

cudaError_t launch_fields2(const Step2Params& p, float* rho_m, float* rho_g, float* ux, float* uy, float* pr,
                           cudaStream_t s) {
  long long b = (p.N + 255) / 256;
  if (b > device_sm_count() * 8LL) b = device_sm_count() * 8LL;
  k_fields2<<<(unsigned)b, 256, 0, s>>>(p, rho_m, rho_g, ux, uy, pr);
  return cudaGetLastError();
}

}  // namespace lbm
