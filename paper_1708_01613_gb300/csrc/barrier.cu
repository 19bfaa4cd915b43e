// Film-barrier pipeline of the extended Shan-Chen model (arXiv 1708.01613,
// Sec. 2.1.5) and the auxiliary kernels: density, gas labelling, interaction
// zones, rupture test (Eq. 41), blocked-edge mask, the bounce-back across
// blocked edges after each step, diagnostics fields, initialisation, FP64
// mass and bubble statistics.
//
// Readings used (the paper is silent on them):
//  - gas cell: rho < threshold (default ln 2, the critical density of
//    Sec. 2.1.2); bubbles are 4-connected gas components on the torus,
//    labelled by the smallest row-major index in the component;
//  - owner of a liquid cell: the bubble of the nearest gas cell within R_z
//    (the nearest-bubble rule of Sec. 2.1.5, which is where the largest
//    |xi_k| of Eq. 38 sits); -1 if there is none; -2 (a wall cell) if gas
//    cells of two or more bubbles are nearest at the same distance (the
//    flowchart places the barrier wall where the bubbles' domains are equal);
//  - rupture: at a cell with a differing-owner neighbour, n = the first such
//    lattice direction, D2 = p(x+n) - 2 p(x) + p(x-n) with p of Eq. 29; the
//    cell opens for good when |D2| <= eps or sign(D2) differs from the sign
//    stored at the previous relabel;
//  - blocked edge: owners differ, both defined (not -1; the wall's -2 is
//    defined), neither end open.
#include <math.h>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kThreads = 256;
constexpr int kUnionIters = 1 << 20;  // bound of the union/find retry loops

__device__ __forceinline__ int wrapi(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

inline unsigned blocks_for(long long n, int threads = kThreads) {
  long long b = (n + threads - 1) / threads;
  const long long cap = device_sm_count() * 64LL;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <int S>
__device__ __forceinline__ float pulled(const void* pops, const FieldParams& fp, int i, int x, int y) {
  using T = typename Store<S>::T;
  const T* p = static_cast<const T*>(pops);
  const int xs = wrapi(x - cx(i), fp.nx), ys = wrapi(y - cy(i), fp.ny);
  return Store<S>::load(p, (size_t)i * fp.N + (size_t)ys * fp.nx + xs, fp.wref[i]);
}

template <int S>
__global__ void k_density(const FieldParams fp, float* __restrict__ rho) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < fp.N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % fp.nx), y = (int)(c / fp.nx);
    float f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = pulled<S>(fp.pops, fp, i, x, y);
    rho[c] = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  }
}

// --- union-find labelling (min-root hooking: the root is the min index) ---
__global__ void k_label_init(const float* __restrict__ rho, long long N, float th, int32_t* L) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x)
    L[c] = rho[c] < th ? (int32_t)c : -1;
}

// Relabel variant of k_label_init: each new gas cell first parks its label of
// the previous relabel in keep[c] (INT_MAX where it was liquid) for the
// coalescence count; keep is the owner array, which the owner phase
// rewrites afterwards.
__global__ void k_label_init_keep(const float* __restrict__ rho, long long N, float th, int32_t* L,
                                  int32_t* __restrict__ keep) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const bool gas = rho[c] < th;
    if (gas) {
      const int32_t o = L[c];
      keep[c] = o >= 0 ? o : 0x7fffffff;
    }
    L[c] = gas ? (int32_t)c : -1;
  }
}

// Coalescence events (components of the new labelling holding gas of two or
// more components of the previous one). keep[r] of a new root r collects the
// first earlier label seen in its component (the root starts with its own);
// a member with another earlier label marks the component (-3), and the one
// that marks it first counts it, so every merged component counts once.
__device__ __forceinline__ int merge_vote(int32_t* keep, int r, int o) {
  if (o == 0x7fffffff) return 0;
  const int prev = atomicCAS(keep + r, 0x7fffffff, o);
  if (prev == 0x7fffffff || prev == o || prev == -3) return 0;
  return atomicExch(keep + r, -3) != -3;
}

__global__ void k_merge_count(long long N, const int32_t* __restrict__ L, int32_t* keep, int* flags) {
  int n = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int r = L[c];
    if (r >= 0 && r != c) n += merge_vote(keep, r, keep[c]);
  }
  if (n) atomicAdd(flags + FLAG_MERGES, n);
}

__device__ int find_root(const int32_t* L, int a, int* fail) {
  for (int it = 0; it < kUnionIters; ++it) {
    const int p = L[a];
    if (p == a) return a;
    a = p;
  }
  *fail = 1;
  return a;
}

__device__ void unite(int32_t* L, int a, int b, int* fail) {
  for (int it = 0; it < kUnionIters; ++it) {
    a = find_root(L, a, fail);
    b = find_root(L, b, fail);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    // hook the larger root a under b; if a stopped being a root meanwhile,
    // continue with the value it points to (links only ever decrease)
    const int old = atomicMin(&L[a], b);
    if (old == a) return;
    a = old;
  }
  *fail = 1;
}

__global__ void k_label_union(int nx, int ny, int32_t* L, int* flags) {
  const long long N = (long long)nx * ny;
  int fail = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    if (L[c] < 0) continue;
    const int x = (int)(c % nx), y = (int)(c / nx);
    const int right = y * nx + (x + 1 == nx ? 0 : x + 1);
    const int down = (y + 1 == ny ? 0 : y + 1) * nx + x;
    if (L[right] >= 0) unite(L, (int)c, right, &fail);
    if (L[down] >= 0) unite(L, (int)c, down, &fail);
  }
  if (fail) atomicOr(flags + FLAG_TIMEOUT, 1);
}

__global__ void k_label_flatten(long long N, int32_t* L, int* flags) {
  int fail = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    if (L[c] >= 0) L[c] = find_root(L, (int)c, &fail);
  }
  if (fail) atomicOr(flags + FLAG_TIMEOUT, 1);
}

// --- interaction zones: nearest gas cell within R; equidistant bubbles: wall (-2) ---
__global__ void k_owner(int nx, int ny, int R, const int32_t* __restrict__ L, int32_t* __restrict__ own) {
  const long long N = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int lc = L[c];
    if (lc >= 0) {
      own[c] = lc;
      continue;
    }
    const int x = (int)(c % nx), y = (int)(c / nx);
    int best = -1, bd = 0x7fffffff;
    bool tie = false;
    for (int dy = -R; dy <= R; ++dy) {
      const long long row = (long long)wrapi(y + dy, ny) * nx;
      for (int dx = -R; dx <= R; ++dx) {
        const int d2 = dx * dx + dy * dy;
        if (d2 > R * R || d2 > bd) continue;
        const int l = __ldg(L + row + wrapi(x + dx, nx));
        if (l < 0) continue;
        if (d2 < bd) {
          bd = d2;
          best = l;
          tie = false;
        } else if (l != best) {
          tie = true;
        }
      }
    }
    own[c] = tie ? -2 : best;
  }
}

// Owner of a liquid cell from a window of labels in shared memory (row0 at
// the cell, row stride W): the label of the nearest labelled cell within R,
// -1 if none, -2 if two different labels are nearest at the same distance.
__device__ __forceinline__ int window_owner(const int* row0, int W, int R) {
  int best = -1, bd = 0x7fffffff;
  bool tie = false;
  for (int dy = -R; dy <= R; ++dy) {
    const int* rowp = row0 + dy * W;
    for (int dx = -R; dx <= R; ++dx) {
      const int d2 = dx * dx + dy * dy;
      if (d2 > R * R || d2 > bd) continue;
      const int l = rowp[dx];
      if (l < 0) continue;
      if (d2 < bd) {
        bd = d2;
        best = l;
        tie = false;
      } else if (l != best) {
        tie = true;
      }
    }
  }
  return tie ? -2 : best;
}

// Tiled owner search: a 32 x 8 tile stages the labels of its window (tile
// plus R on every side, wrapped) in shared memory. A tile with no gas cell
// in that window writes -1 everywhere; otherwise each liquid cell scans the
// window from shared memory. Same result as k_owner (same scan order).
constexpr int kOTX = 32, kOTY = 8, kOMaxR = 16;

__global__ void __launch_bounds__(kOTX * kOTY) k_owner_tiled(int nx, int ny, int R, const int32_t* __restrict__ L,
                                                           int32_t* __restrict__ own) {
  __shared__ int32_t sl[(kOTY + 2 * kOMaxR) * (kOTX + 2 * kOMaxR)];
  const int W = kOTX + 2 * R, H = kOTY + 2 * R;
  const int bx0 = blockIdx.x * kOTX, by0 = blockIdx.y * kOTY;
  const int tid = threadIdx.y * kOTX + threadIdx.x;
  int any = 0;
  for (int k = tid; k < W * H; k += kOTX * kOTY) {
    const int yy = k / W, xx = k - yy * W;
    const int gy = wrapi(by0 - R + yy, ny), gx = wrapi(bx0 - R + xx, nx);
    const int l = L[(long long)gy * nx + gx];
    sl[k] = l;
    any |= l >= 0;
  }
  any = __syncthreads_or(any);
  const int x = bx0 + threadIdx.x, y = by0 + threadIdx.y;
  if (x >= nx || y >= ny) return;
  int result = -1;
  if (any) {
    const int* row0 = sl + (threadIdx.y + R) * W + threadIdx.x + R;
    const int lc = row0[0];
    if (lc >= 0) {
      result = lc;
    } else {
      result = window_owner(row0, W, R);
    }
  }
  own[(long long)y * nx + x] = result;
}

__device__ __forceinline__ float pressure_of(float rho, float G, float rho0) {
  const float s = rho0 * (1.0f - expf(-rho / rho0));
  return rho * (1.0f / 3.0f) + G * s * s * (1.0f / 6.0f);
}

__global__ void k_rupture(int nx, int ny, float G, float rho0, float eps,
                          const float* __restrict__ rho, const int32_t* __restrict__ own,
                          int8_t* __restrict__ sgn, uint8_t* __restrict__ open, int* flags) {
  const long long N = (long long)nx * ny;
  int opened = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int o = own[c];
    const int x = (int)(c % nx), y = (int)(c / nx);
    int dir = 0;
    if (o != -1) {
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int on = own[(long long)wrapi(y + cy(i), ny) * nx + wrapi(x + cx(i), nx)];
        if (dir == 0 && on != -1 && on != o) dir = i;
      }
    }
    if (dir == 0) {
      sgn[c] = 0;
      continue;
    }
    int ex = 0, ey = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i)
      if (i == dir) {
        ex = cx(i);
        ey = cy(i);
      }
    const float pp = pressure_of(rho[(long long)wrapi(y + ey, ny) * nx + wrapi(x + ex, nx)], G, rho0);
    const float p0 = pressure_of(rho[c], G, rho0);
    const float pm = pressure_of(rho[(long long)wrapi(y - ey, ny) * nx + wrapi(x - ex, nx)], G, rho0);
    const float d2 = pp - 2.0f * p0 + pm;
    const int s = (d2 > 0.f) - (d2 < 0.f);
    const int prev = sgn[c];
    if (eps >= 0.f && !open[c] && (fabsf(d2) <= eps || (prev != 0 && s != prev))) {
      open[c] = 1;
      opened += 1;
    }
    sgn[c] = (int8_t)s;
  }
  if (opened) atomicAdd(flags + FLAG_OPENED, opened);
}

__global__ void k_mask(int nx, int ny, const int32_t* __restrict__ own, const uint8_t* __restrict__ open,
                       uint8_t* __restrict__ mask) {
  const long long N = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int o = own[c];
    const int x = (int)(c % nx), y = (int)(c / nx);
    unsigned m = 0;
    if (o != -1 && !open[c]) {
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const long long nb = (long long)wrapi(y + cy(i), ny) * nx + wrapi(x + cx(i), nx);
        const int on = own[nb];
        if (on != -1 && on != o && !open[nb]) m |= 1u << (i - 1);
      }
    }
    mask[c] = (uint8_t)m;
  }
}

// --- diagnostics: rho, u = (j + F/2)/rho, p (Eq. 29) ---
template <int S>
__global__ void k_fields(const FieldParams fp, const float* __restrict__ rho,
                         const uint8_t* __restrict__ mask, uint32_t which, float* __restrict__ out) {
  const int nx = fp.nx, ny = fp.ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < fp.N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)(c / nx);
    const float r = rho[c];
    const float psi_c = fp.rho0 * (1.0f - expf(-r * fp.inv_rho0));
    float v = 0.f;
    if (which == LBM_FIELD_RHO) {
      v = r;
    } else if (which == LBM_FIELD_P) {
      v = r * (1.0f / 3.0f) + fp.G * psi_c * psi_c * (1.0f / 6.0f);
    } else {
      float f[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = pulled<S>(fp.pops, fp, i, x, y);
      const float jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
      const float jy = (f[2] - f[4]) + (f[5] - f[8]) + (f[6] - f[7]);
      const unsigned m = mask ? mask[c] : 0u;
      float sx = 0.f, sy = 0.f;
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        float s = fp.rho0 * (1.0f - expf(-rho[(long long)wrapi(y + cy(i), ny) * nx + wrapi(x + cx(i), nx)] * fp.inv_rho0));
        if ((m >> (i - 1)) & 1u) s = psi_c;
        sx += static_cast<float>(wq(i)) * s * cx(i);
        sy += static_cast<float>(wq(i)) * s * cy(i);
      }
      const float F = -fp.G * psi_c * (which == LBM_FIELD_UX ? sx : sy);
      v = ((which == LBM_FIELD_UX ? jx : jy) + 0.5f * F) / r;
    }
    out[c] = v;
  }
}

template <int S>
__global__ void k_pops_out(const FieldParams fp, int plane, float* __restrict__ out) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < fp.N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % fp.nx), y = (int)(c / fp.nx);
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i)
      if (i == plane) v = pulled<S>(fp.pops, fp, i, x, y);
    out[c] = v;
  }
}

// The stored buffer holds f_i at the source cell of the next pull: B_i(y) = f_i(y + e_i).
template <int S>
__global__ void k_init_from_rho(typename Store<S>::T* __restrict__ pops, const double* __restrict__ rho,
                                int nx, int ny, FieldParams fp) {
  const long long N = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)(c / nx);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const long long src = (long long)wrapi(y + cy(i), ny) * nx + wrapi(x + cx(i), nx);
      const float f = (float)(wq(i) * rho[src]);
      Store<S>::store(pops, (size_t)i * N + c, f, fp.wref[i]);
    }
  }
}

template <int S>
__global__ void k_load_plane(typename Store<S>::T* __restrict__ pops, const float* __restrict__ fpl,
                             int plane, int nx, int ny, float base) {
  const long long N = (long long)nx * ny;
  int ex = 0, ey = 0;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    if (i == plane) {
      ex = cx(i);
      ey = cy(i);
    }
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % nx), y = (int)(c / nx);
    const long long src = (long long)wrapi(y + ey, ny) * nx + wrapi(x + ex, nx);
    Store<S>::store(pops, (size_t)plane * N + c, fpl[src], base);
  }
}

// Initial density of a bubble set (tanh profile of the signed distance to the
// nearest interface). One CTA per 32 x 32 tile: the bubbles are filtered
// against the tile first, so each cell takes the minimum only over bubbles
// that can come within kSatQ half-widths of it. Beyond that distance the
// correctly rounded tanh is exactly 1 in FP64 (1 - tanh(20) < 1e-17 < 2^-54),
// so the result equals the minimum over all bubbles: the filter drops nothing
// that could change a single bit.
constexpr int kInitTile = 32;
constexpr int kInitChunk = 512;
constexpr double kSatQ = 20.0;

__global__ void __launch_bounds__(kThreads) k_bubbles_rho(const lbm_bubble* __restrict__ b, int n,
                                                         double rho_l, double rho_g, double width,
                                                         int nx, int ny, double* __restrict__ rho) {
  __shared__ double scx[kInitChunk], scy[kInitChunk], sr[kInitChunk];
  __shared__ int cnt;
  const int ntx = (nx + kInitTile - 1) / kInitTile;
  const int x0 = (int)(blockIdx.x % ntx) * kInitTile, y0 = (int)(blockIdx.x / ntx) * kInitTile;
  const double half = 0.5 * width;
  const double reach = kSatQ * half + 2.0;  // margin over the saturation distance
  const double tcx = x0 + 0.5 * (kInitTile - 1), tcy = y0 + 0.5 * (kInitTile - 1);
  const int tx = threadIdx.x % kInitTile, ty = threadIdx.x / kInitTile;
  constexpr int kRows = kInitTile * kInitTile / kThreads;
  double best[kRows];
#pragma unroll
  for (int j = 0; j < kRows; ++j) best[j] = INFINITY;
  for (int k0 = 0; k0 < n; k0 += kInitChunk) {
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int k = k0 + threadIdx.x; k < min(n, k0 + kInitChunk); k += kThreads) {
      // periodic distance from the tile's centre, less the tile's half extent
      double dx = fabs(tcx - b[k].cx), dy = fabs(tcy - b[k].cy);
      dx = fmax(0.0, fmin(dx, nx - dx) - 0.5 * kInitTile);
      dy = fmax(0.0, fmin(dy, ny - dy) - 0.5 * kInitTile);
      if (sqrt(dx * dx + dy * dy) - b[k].r <= reach) {
        const int slot = atomicAdd(&cnt, 1);
        scx[slot] = b[k].cx;
        scy[slot] = b[k].cy;
        sr[slot] = b[k].r;
      }
    }
    __syncthreads();
    const int m = cnt;
#pragma unroll
    for (int j = 0; j < kRows; ++j) {
      const double x = (double)(x0 + tx), y = (double)(y0 + ty + j * (kThreads / kInitTile));
      for (int k = 0; k < m; ++k) {
        double dx = fabs(x - scx[k]), dy = fabs(y - scy[k]);
        dx = fmin(dx, nx - dx);
        dy = fmin(dy, ny - dy);
        const double s = sqrt(dx * dx + dy * dy) - sr[k];
        if (s < best[j]) best[j] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < kRows; ++j) {
    const int x = x0 + tx, y = y0 + ty + j * (kThreads / kInitTile);
    if (x >= nx || y >= ny) continue;
    const double q = best[j] / half;
    const double v = q >= kSatQ ? 1.0 : tanh(q);
    rho[(size_t)y * nx + x] = 0.5 * (rho_l + rho_g) + 0.5 * (rho_l - rho_g) * v;
  }
}

// --- fixed-order FP64 reductions ---
// A fixed number of block partials (not tied to the device's SM count), so the
// summation order, and with it every reduced value, is the same on any GPU.
constexpr int kRedBlocks = 608;

template <int NV>
__device__ void block_reduce_store(double (&v)[NV], double* __restrict__ out) {
  __shared__ double sh[NV][kThreads];
#pragma unroll
  for (int j = 0; j < NV; ++j) sh[j][threadIdx.x] = v[j];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s)
#pragma unroll
      for (int j = 0; j < NV; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j * gridDim.x + blockIdx.x] = sh[j][0];
}

template <int S>
__global__ void __launch_bounds__(kThreads) k_mass_partial(const FieldParams fp, double* partials) {
  using T = typename Store<S>::T;
  const T* p = static_cast<const T*>(fp.pops);
  double acc[1] = {0.0};
  for (int i = 0; i < Q; ++i) {
    const float base = fp.wref[i];
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < fp.N;
         c += (long long)gridDim.x * blockDim.x)
      acc[0] += (double)Store<S>::load(p, (size_t)i * fp.N + c, base);
  }
  block_reduce_store<1>(acc, partials);
}

template <int NV>
__global__ void __launch_bounds__(kThreads) k_sum_partials(const double* partials, int nparts, double* out) {
  double acc[NV];
#pragma unroll
  for (int j = 0; j < NV; ++j) acc[j] = 0.0;
  for (int k = threadIdx.x; k < nparts; k += blockDim.x)
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] += partials[j * nparts + k];
  block_reduce_store<NV>(acc, out);
}

__global__ void k_area(long long N, const int32_t* __restrict__ L, int32_t* __restrict__ area) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int l = L[c];
    if (l >= 0) atomicAdd(area + l, 1);
  }
}

// Roots with their areas appended to list (warp-aggregated slots).
__global__ void k_bubble_list(long long N, const int32_t* __restrict__ L, const int32_t* __restrict__ area,
                              int32_t* __restrict__ list, int* count) {
  for (long long c0 = blockIdx.x * (long long)blockDim.x; c0 < N; c0 += (long long)gridDim.x * blockDim.x) {
    const long long c = c0 + threadIdx.x;
    const bool root = c < N && L[c] == c;
    const unsigned b = __ballot_sync(0xffffffffu, root);
    if (!b) continue;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == __ffs(b) - 1) base = atomicAdd(count, __popc(b));
    base = __shfl_sync(0xffffffffu, base, __ffs(b) - 1);
    if (root) {
      const int k = base + __popc(b & ((1u << lane) - 1u));
      list[2 * k] = (int32_t)c;
      list[2 * k + 1] = area[c];
    }
  }
}

// partial sums: [0] bubbles, [1] gas cells, [2] sum of equivalent diameters;
// histogram counts are integers, accumulated exactly with atomics
constexpr int kMaxBins = 64;
constexpr int kStatVals = 3;

__global__ void __launch_bounds__(kThreads) k_stats_partial(long long N, const int32_t* __restrict__ L,
                                                            const int32_t* __restrict__ area, int nbins,
                                                            double ldmin, double ldspan, double* partials,
                                                            int* hist) {
  double v[kStatVals] = {0.0, 0.0, 0.0};
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int l = L[c];
    if (l < 0) continue;
    v[1] += 1.0;
    if (l == c) {
      const double d = 2.0 * sqrt((double)area[c] / M_PI);
      v[0] += 1.0;
      v[2] += d;
      if (nbins > 0) {
        int b = (int)floor((log(d) - ldmin) / ldspan * nbins);
        b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
        atomicAdd(hist + b, 1);
      }
    }
  }
  block_reduce_store<kStatVals>(v, partials);
}

// ---------------------------------------------------------------------------
// Tiled barrier pipeline. The box is cut into 32 x 8 tiles; where nx or ny is
// not a multiple of the tile, the last tile column or row is ragged and its
// threads outside the box take part in the barriers only. The density pass also joins the gas cells inside
// each tile (a union-find in shared memory: a gas cell's initial label is
// the smallest index of its piece of the tile) and writes one gas flag per
// tile; the union phase then joins the pieces across tile borders. A tile is
// active when a gas cell lies within the tile span that R_z can reach. Owners, rupture signs and masks can only be
// non-trivial in active tiles (a defined owner needs gas within R_z), so the
// later kernels skip every tile that is inactive now and was inactive at the
// previous relabel: its owner/sign/mask are already -1/0/0. A tile that just
// became inactive is reset to those values. Results equal the untiled kernels.
//
// Every phase is one launch over any number of boxes (a lone box is a list
// of one): each box's CTAs follow those of the boxes before it in the entry
// list (RelabelEntry prefix sums), and a CTA finds its box by binary search.
constexpr int kTX = kRelabelTileX, kTY = kRelabelTileY;
// Mask bits of the directions 1, 2, 5, 6: each blocked edge is seen from the
// one end where its direction is among these.
constexpr unsigned kCanonBits = 0x33u;
// CTAs per box for the tile-list phases, at most: eight per SM
inline int list_ctas() { return device_sm_count() * 8; }

__device__ __forceinline__ int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

enum { kOffTiles = 0, kOffScan = 1, kOffList = 2 };

template <int F>
__device__ __forceinline__ int entry_off(const RelabelEntry& e) {
  return F == kOffTiles ? e.off_tiles : (F == kOffScan ? e.off_scan : e.off_list);
}

// Entry k owning CTA `b`: the last k < m with off(k) <= b.
template <int F>
__device__ __forceinline__ int find_entry(const RelabelEntry* __restrict__ e, int m, int b) {
  int lo = 0, hi = m - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (entry_off<F>(e[mid]) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One cell per thread. Used for two-component boxes (TWO, FP32), which also
// get the mixture pressure; one-component boxes take the four-cell kernels
// below, whose per-cell arithmetic is this kernel's.
// Union-find inside one 32 x 8 tile in shared memory (local indices
// ly * kTX + lx, -1 for liquid), hooking the larger root under the smaller,
// so a root is the smallest local index of its piece. Bounded like the
// global version.
__device__ __forceinline__ int tile_find(const int* sp, int a, int* fail) {
  for (int it = 0; it < kTX * kTY; ++it) {
    const int p = sp[a];
    if (p == a) return a;
    a = p;
  }
  *fail = 1;
  return a;
}

__device__ __forceinline__ void tile_unite(int* sp, int a, int b, int* fail) {
  for (int it = 0; it < kTX * kTY; ++it) {
    a = tile_find(sp, a, fail);
    b = tile_find(sp, b, fail);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(&sp[a], b);
    if (old == a) return;
    a = old;
  }
  *fail = 1;
}

// Global index of the tile-local root of local cell li (a gas cell).
__device__ __forceinline__ int32_t tile_root_index(const int* sp, int li, int x0, int y0, int nx, int* fail) {
  const int r = tile_find(sp, li, fail);
  return (int32_t)((y0 + r / kTX) * nx + x0 + r % kTX);
}

template <int S, bool TWO>
__global__ void __launch_bounds__(kTX * kTY) kb_density_label(const RelabelBox* __restrict__ boxes,
                                                              const RelabelEntry* __restrict__ e, int m, int parity) {
  using T = typename Store<S>::T;
  const int k = find_entry<kOffTiles>(e, m, blockIdx.x);
  const RelabelBox& B = boxes[e[k].box];
  const int t = blockIdx.x - e[k].off_tiles;
  const T* p = static_cast<const T*>(B.pops[B.cur ^ parity]);
  const int nx = B.nx, ny = B.ny;
  const size_t N = (size_t)nx * ny;
  const int x = (t % B.ntx) * kTX + threadIdx.x, y = (t / B.ntx) * kTY + threadIdx.y;
  const bool in = x < nx && y < ny;  // a ragged tile's threads outside the box only join the barriers
  const int xi = in ? x : 0, yi = in ? y : 0;
  const int xm = wrap1(xi - 1, nx), xp = wrap1(xi + 1, nx);
  const size_t r0 = (size_t)yi * nx, rm = (size_t)wrap1(yi - 1, ny) * nx, rp = (size_t)wrap1(yi + 1, ny) * nx;
  float f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const size_t row = cy(i) > 0 ? rm : (cy(i) < 0 ? rp : r0);
    const int xs = cx(i) > 0 ? xm : (cx(i) < 0 ? xp : xi);
    f[i] = Store<S>::load(p, (size_t)i * N + row + xs, B.wref[i]);
  }
  const float r = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const size_t c = r0 + xi;
  if (in) B.rho[c] = r;
  if (TWO && in) {  // two components (FP32): the gas lattice follows the melt's nine planes
    const float* pg = reinterpret_cast<const float*>(p) + (size_t)Q * N;
    float g = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const size_t row = cy(i) > 0 ? rm : (cy(i) < 0 ? rp : r0);
      const int xs = cx(i) > 0 ? xm : (cx(i) < 0 ? xp : x);
      g += __ldg(pg + (size_t)i * N + row + xs);
    }
    const float a = B.rho0 * (1.0f - expf(-r / B.rho0)), b = B.rho0 * (1.0f - expf(-g / B.rho0));
    B.pr[c] = (r + g) * (1.0f / 3.0f) + (B.G * a * a + 2.0f * B.G_mg * a * b + B.G_gg * b * b) * (1.0f / 6.0f);
  }
  const bool gas = in && r < B.threshold;
  // gas cells joined inside the tile here (shared-memory union-find); each
  // starts the global union-find pointing at the smallest index of its piece
  // of the tile, and the union phase joins the pieces across tile borders
  __shared__ int sp[kTX * kTY];
  const int li = threadIdx.y * kTX + threadIdx.x;
  sp[li] = gas ? li : -1;
  const int any = __syncthreads_or(gas);
  int32_t lab = -1;
  if (any) {
    int fail = 0;
    if (gas) {
      if (threadIdx.x + 1 < kTX && sp[li + 1] >= 0) tile_unite(sp, li, li + 1, &fail);
      if (threadIdx.y + 1 < kTY && sp[li + kTX] >= 0) tile_unite(sp, li, li + kTX, &fail);
    }
    __syncthreads();
    if (gas) lab = tile_root_index(sp, li, x - threadIdx.x, y - threadIdx.y, nx, &fail);
    if (fail) atomicOr(B.flags + FLAG_TIMEOUT, 1);
  }
  if (gas) {  // the label of the previous relabel, for the coalescence count
    const int32_t o = B.label[c];
    B.owner[c] = o >= 0 ? o : 0x7fffffff;
  }
  if (in) B.label[c] = lab;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    B.tile_gas[t] = (uint8_t)(any != 0);
    if (t == 0) {  // the tile lists are rebuilt by the next phase and the mask phase
      B.flags[FLAG_TILES] = 0;
      B.flags[FLAG_FILM] = 0;
    }
  }
}

template <int S>
__device__ __forceinline__ float dec16(unsigned short v) {
  if constexpr (S == LBM_F16_DEV) return __half2float(__ushort_as_half(v));
  else return __bfloat162float(__ushort_as_bfloat16(v));
}

// Four cells (x .. x + 3) of one tile row per thread, 8 x 8 threads per
// 32 x 8 tile: the part after the densities r, shared by the vector density
// kernels. Densities out, gas decision (rho < threshold), tile-local
// union-find, the previous labels of gas cells kept for the coalescence
// count, labels out, tile flags; the same results as kb_density_label's
// one-cell threads. vec: the four cells lie inside the row and the row's
// start is 16-byte aligned (one vector store each for densities and labels).
__device__ __forceinline__ void density_label_tail4(const RelabelBox& B, int t, int x, int y, size_t c,
                                                    const float (&r)[4], bool rowin, bool vec) {
  float* const rho = B.rho;
  int32_t* const label = B.label;
  bool in[4], gas[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    in[j] = rowin && x + j < B.nx;
    gas[j] = in[j] && r[j] < B.threshold;
  }
  if (vec) {
    *reinterpret_cast<float4*>(rho + c) = make_float4(r[0], r[1], r[2], r[3]);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (in[j]) rho[c + j] = r[j];
  }
  __shared__ int sp[kTX * kTY];  // tile-local union-find, as in kb_density_label
  const int la = threadIdx.y * kTX + 4 * threadIdx.x;
#pragma unroll
  for (int j = 0; j < 4; ++j) sp[la + j] = gas[j] ? la + j : -1;
  const int any = __syncthreads_or(gas[0] || gas[1] || gas[2] || gas[3]);
  int32_t lab[4] = {-1, -1, -1, -1};
  if (any) {
    int fail = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!gas[j]) continue;
      if (j < 3 ? gas[j + 1] : (4 * threadIdx.x + 4 < kTX && sp[la + 4] >= 0)) tile_unite(sp, la + j, la + j + 1, &fail);
      if (threadIdx.y + 1 < kTY && sp[la + j + kTX] >= 0) tile_unite(sp, la + j, la + j + kTX, &fail);
    }
    __syncthreads();
    const int x0 = x - 4 * threadIdx.x, y0 = y - threadIdx.y;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (gas[j]) lab[j] = tile_root_index(sp, la + j, x0, y0, B.nx, &fail);
    if (fail) atomicOr(B.flags + FLAG_TIMEOUT, 1);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (gas[j]) {  // the label of the previous relabel, for the coalescence count
      const int32_t o = label[c + j];
      B.owner[c + j] = o >= 0 ? o : 0x7fffffff;
    }
  if (vec) {
    *reinterpret_cast<int4*>(label + c) = make_int4(lab[0], lab[1], lab[2], lab[3]);
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (in[j]) label[c + j] = lab[j];
  }
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    B.tile_gas[t] = (uint8_t)(any != 0);
    if (t == 0) {  // the tile lists are rebuilt by the next phase and the mask phase
      B.flags[FLAG_TILES] = 0;
      B.flags[FLAG_FILM] = 0;
    }
  }
}

// Sum of the nine pulled values in kb_density_label's order, for two cells
// at once (the packed adds round per component like the scalar ones).
__device__ __forceinline__ float2 rho_pair(const float2 (&f)[Q]) {
  return __fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(f[0], f[1]), __fadd2_rn(f[2], f[3])),
                               __fadd2_rn(__fadd2_rn(f[4], f[5]), __fadd2_rn(f[6], f[7]))),
                    f[8]);
}

// One-component FP32 storage, four cells per thread. Where the box's rows
// start on 16-byte boundaries (nx % 4 == 0) and the cells and the columns
// they pull from lie inside the row, a plane arrives in one 16-byte load, a
// plane the pull shifts by one column adds the value beside it; other cells
// (the box's first and last columns, ragged tiles, other widths) load one by
// one with the periodic wrap.
__global__ void __launch_bounds__(kTX / 4 * kTY, 16) kb_density_label32(const RelabelBox* __restrict__ boxes,
                                                                        const RelabelEntry* __restrict__ e, int m,
                                                                        int parity) {
  const int k = find_entry<kOffTiles>(e, m, blockIdx.x);
  const RelabelBox& B = boxes[e[k].box];
  const int t = blockIdx.x - e[k].off_tiles;
  const float* p = static_cast<const float*>(B.pops[B.cur ^ parity]);
  const int nx = B.nx, ny = B.ny;
  const size_t N = (size_t)nx * ny;
  const int x = (t % B.ntx) * kTX + 4 * threadIdx.x, y = (t / B.ntx) * kTY + threadIdx.y;
  const bool rowin = y < ny;
  const int yi = rowin ? y : 0;
  const size_t r0 = (size_t)yi * nx, rm = (size_t)wrap1(yi - 1, ny) * nx, rp = (size_t)wrap1(yi + 1, ny) * nx;
  const bool aligned = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(B.rho) |
                         reinterpret_cast<uintptr_t>(B.label)) & 15u) == 0;
  const bool vec = rowin && aligned && (nx & 3) == 0 && x >= 1 && x + 5 <= nx;  // columns x - 1 .. x + 4
  float2 fa[Q], fb[Q];  // cells (x, x + 1) and (x + 2, x + 3)
  if (vec) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const size_t row = cy(i) > 0 ? rm : (cy(i) < 0 ? rp : r0);
      const float* q = p + (size_t)i * N + row + x;
      const float4 w = __ldg(reinterpret_cast<const float4*>(q));  // columns x .. x + 3
      if (cx(i) > 0) {  // columns x - 1 .. x + 2
        fa[i] = make_float2(__ldg(q - 1), w.x);
        fb[i] = make_float2(w.y, w.z);
      } else if (cx(i) < 0) {  // columns x + 1 .. x + 4
        fa[i] = make_float2(w.y, w.z);
        fb[i] = make_float2(w.w, __ldg(q + 4));
      } else {
        fa[i] = make_float2(w.x, w.y);
        fb[i] = make_float2(w.z, w.w);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const size_t row = cy(i) > 0 ? rm : (cy(i) < 0 ? rp : r0);
      const float* q = p + (size_t)i * N + row;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = rowin && x + j < nx ? __ldg(q + wrap1(x + j - cx(i), nx)) : 0.f;
      fa[i] = make_float2(v[0], v[1]);
      fb[i] = make_float2(v[2], v[3]);
    }
  }
  const float2 ra = rho_pair(fa), rb = rho_pair(fb);
  const float r[4] = {ra.x, ra.y, rb.x, rb.y};
  density_label_tail4(B, t, x, y, r0 + x, r, rowin, vec);
}

// 16-bit storage, four cells per thread. Where the box's rows start on
// 8-byte boundaries (nx % 4 == 0) and the four cells and the columns they
// pull from lie inside the row, a plane arrives in one 8-byte load; a plane
// the pull shifts by one column adds the 4-byte word beside it, and its
// pairs (source columns s, s + 1 with s odd) are the high half of one word
// and the low half of the next. Other cells load element by element with
// the periodic wrap. Each cell's arithmetic is kb_density_label's, so
// densities, labels and tile flags are bitwise the same.
template <int S>
__device__ __forceinline__ float2 dec16x2(uint32_t bits) {
  return make_float2(dec16<S>((unsigned short)(bits & 0xffffu)), dec16<S>((unsigned short)(bits >> 16)));
}

template <int S>
__global__ void __launch_bounds__(kTX / 4 * kTY, 16) kb_density_label16(const RelabelBox* __restrict__ boxes,
                                                                        const RelabelEntry* __restrict__ e, int m,
                                                                        int parity) {
  const int k = find_entry<kOffTiles>(e, m, blockIdx.x);
  const RelabelBox& B = boxes[e[k].box];
  const int t = blockIdx.x - e[k].off_tiles;
  const unsigned short* p = static_cast<const unsigned short*>(B.pops[B.cur ^ parity]);
  const int nx = B.nx, ny = B.ny;
  const size_t N = (size_t)nx * ny;
  const int x = (t % B.ntx) * kTX + 4 * threadIdx.x, y = (t / B.ntx) * kTY + threadIdx.y;
  const bool rowin = y < ny;
  const int yi = rowin ? y : 0;
  const size_t r0 = (size_t)yi * nx, rm = (size_t)wrap1(yi - 1, ny) * nx, rp = (size_t)wrap1(yi + 1, ny) * nx;
  const bool aligned = ((reinterpret_cast<uintptr_t>(p) | reinterpret_cast<uintptr_t>(B.rho) |
                         reinterpret_cast<uintptr_t>(B.label)) & 15u) == 0;
  const bool vec = rowin && aligned && (nx & 3) == 0 && x >= 2 && x + 6 <= nx;  // columns x - 2 .. x + 5
  float2 fa[Q], fb[Q];  // cells (x, x + 1) and (x + 2, x + 3)
  if (vec) {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const size_t row = cy(i) > 0 ? rm : (cy(i) < 0 ? rp : r0);
      const unsigned short* q = p + (size_t)i * N + row + x;
      const uint2 w = __ldg(reinterpret_cast<const uint2*>(q));  // columns x .. x + 3
      uint32_t lo = w.x, hi = w.y;
      if (cx(i) > 0) {  // columns x - 1 .. x + 2
        const uint32_t wm = __ldg(reinterpret_cast<const uint32_t*>(q - 2));
        lo = __byte_perm(wm, w.x, 0x5432);
        hi = __byte_perm(w.x, w.y, 0x5432);
      } else if (cx(i) < 0) {  // columns x + 1 .. x + 4
        const uint32_t wp = __ldg(reinterpret_cast<const uint32_t*>(q + 4));
        lo = __byte_perm(w.x, w.y, 0x5432);
        hi = __byte_perm(w.y, wp, 0x5432);
      }
      const float2 wr = make_float2(B.wref[i], B.wref[i]);
      fa[i] = __fadd2_rn(wr, dec16x2<S>(lo));
      fb[i] = __fadd2_rn(wr, dec16x2<S>(hi));
    }
  } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const size_t row = cy(i) > 0 ? rm : (cy(i) < 0 ? rp : r0);
      const unsigned short* q = p + (size_t)i * N + row;
      unsigned v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = rowin && x + j < nx ? __ldg(q + wrap1(x + j - cx(i), nx)) : 0u;
      const float2 wr = make_float2(B.wref[i], B.wref[i]);
      fa[i] = __fadd2_rn(wr, dec16x2<S>(v[0] | (v[1] << 16)));
      fb[i] = __fadd2_rn(wr, dec16x2<S>(v[2] | (v[3] << 16)));
    }
  }
  const float2 ra = rho_pair(fa), rb = rho_pair(fb);
  const float r[4] = {ra.x, ra.y, rb.x, rb.y};
  density_label_tail4(B, t, x, y, r0 + x, r, rowin, vec);
}

// Also appends every tile that needs a visit (active now or at the previous
// relabel) to the box's list; the order of the list does not affect any
// result.
__global__ void kb_active(const RelabelBox* __restrict__ boxes, const RelabelEntry* __restrict__ e, int m) {
  const int k = find_entry<kOffScan>(e, m, blockIdx.x);
  const RelabelBox& B = boxes[e[k].box];
  const int t = (blockIdx.x - e[k].off_scan) * blockDim.x + threadIdx.x;
  const int ntx = B.ntx, nty = B.nty;
  if (t >= ntx * nty) return;
  // tiles within reach of R cells; across the periodic seam of a box with a
  // ragged last tile one tile more
  const int spx = (B.R + kTX - 1) / kTX + (B.nx % kTX ? 1 : 0);
  const int spy = (B.R + kTY - 1) / kTY + (B.ny % kTY ? 1 : 0);
  const int ty = t / ntx, tx = t - ty * ntx;
  int a = 0;
  for (int dy = -spy; dy <= spy && !a; ++dy) {
    const int yy = wrapi(ty + dy, nty);
    for (int dx = -spx; dx <= spx; ++dx) a |= B.tile_gas[yy * ntx + wrapi(tx + dx, ntx)];
  }
  B.tile_active[t] = (uint8_t)(a != 0);
  if (a || B.tile_prev[t]) B.tile_list[atomicAdd(B.flags + FLAG_TILES, 1)] = t;
}

// CTA `first` of `stride` CTAs that walk box k's tile list.
struct ListWalk {
  const RelabelBox* B;
  int first, stride, n;
};

__device__ __forceinline__ ListWalk list_walk(const RelabelBox* __restrict__ boxes, const RelabelEntry* __restrict__ e,
                                              int m) {
  const int k = find_entry<kOffList>(e, m, blockIdx.x);
  ListWalk w;
  w.B = &boxes[e[k].box];
  w.first = blockIdx.x - e[k].off_list;
  w.stride = e[k + 1].off_list - e[k].off_list;
  w.n = w.B->flags[FLAG_TILES];
  return w;
}

__global__ void __launch_bounds__(kTX * kTY) kb_union(const RelabelBox* __restrict__ boxes,
                                                      const RelabelEntry* __restrict__ e, int m) {
  const ListWalk lw = list_walk(boxes, e, m);
  const RelabelBox& B = *lw.B;
  const int nx = B.nx, ny = B.ny;
  int32_t* L = B.label;
  int fail = 0;
  for (int w = lw.first; w < lw.n; w += lw.stride) {
    const int t = B.tile_list[w];
    if (!B.tile_gas[t]) continue;
    // edges inside the tile were joined by the density phase: only the
    // right and bottom borders (periodic wrap included) are left
    const int x = (t % B.ntx) * kTX + threadIdx.x, y = (t / B.ntx) * kTY + threadIdx.y;
    if (x >= nx || y >= ny) continue;
    const bool re = threadIdx.x == kTX - 1 || x == nx - 1, be = threadIdx.y == kTY - 1 || y == ny - 1;
    if (!re && !be) continue;
    const int c = y * nx + x;
    if (L[c] < 0) continue;
    if (re) {
      const int right = y * nx + (x + 1 == nx ? 0 : x + 1);
      if (L[right] >= 0) unite(L, c, right, &fail);
    }
    if (be) {
      const int down = (y + 1 == ny ? 0 : y + 1) * nx + x;
      if (L[down] >= 0) unite(L, c, down, &fail);
    }
  }
  if (fail) atomicOr(B.flags + FLAG_TIMEOUT, 1);
}

__global__ void __launch_bounds__(kTX * kTY) kb_flatten(const RelabelBox* __restrict__ boxes,
                                                        const RelabelEntry* __restrict__ e, int m) {
  const ListWalk lw = list_walk(boxes, e, m);
  const RelabelBox& B = *lw.B;
  int32_t* L = B.label;
  int fail = 0;
  for (int w = lw.first; w < lw.n; w += lw.stride) {
    const int t = B.tile_list[w];
    if (!B.tile_gas[t]) continue;
    const int x = (t % B.ntx) * kTX + threadIdx.x, y = (t / B.ntx) * kTY + threadIdx.y;
    if (x >= B.nx || y >= B.ny) continue;
    const int c = y * B.nx + x;
    if (L[c] >= 0) L[c] = find_root(L, c, &fail);
  }
  if (fail) atomicOr(B.flags + FLAG_TIMEOUT, 1);
}

// Coalescence events of the relabel (merge_vote), over the listed tiles
// with gas; runs between the flatten and the owner phase, whose owner array
// holds the earlier labels the density phase parked there.
__global__ void __launch_bounds__(kTX * kTY) kb_merge(const RelabelBox* __restrict__ boxes,
                                                      const RelabelEntry* __restrict__ e, int m) {
  const ListWalk lw = list_walk(boxes, e, m);
  const RelabelBox& B = *lw.B;
  int n = 0;
  for (int w = lw.first; w < lw.n; w += lw.stride) {
    const int t = B.tile_list[w];
    if (!B.tile_gas[t]) continue;
    const int x = (t % B.ntx) * kTX + threadIdx.x, y = (t / B.ntx) * kTY + threadIdx.y;
    if (x >= B.nx || y >= B.ny) continue;
    const int c = y * B.nx + x;
    const int r = B.label[c];
    if (r >= 0 && r != c) n += merge_vote(B.owner, r, B.owner[c]);
  }
  n = __syncthreads_count(n);
  if (n && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(B.flags + FLAG_MERGES, n);
}

// Owner from the labels within radius R of the window position row0 (window
// width W): the label of the nearest labelled cell, -1 if none, -2 if two
// different labels are nearest at the same distance. Shells of equal squared
// distance are scanned in increasing order and the first shell holding a
// label decides: the unsigned minimum of its labels (-1 is the largest
// unsigned value) and the signed maximum (-1 is the smallest) are that
// shell's smallest and largest label, equal unless two bubbles tie. With R
// known at compile time every offset is one shared load, one min and one max.
template <int R>
__device__ __forceinline__ int nearest_label(const int* row0) {
  constexpr int W = kTX + 2 * R;
  unsigned lo = 0xffffffffu;
  int hi = -1;
#pragma unroll
  for (int S = 1; S <= R * R; ++S) {
    bool any = false;
#pragma unroll
    for (int dy = -R; dy <= R; ++dy)
#pragma unroll
      for (int dx = -R; dx <= R; ++dx)
        if (dx * dx + dy * dy == S) {
          const int l = row0[dy * W + dx];
          lo = min(lo, (unsigned)l);
          hi = max(hi, l);
          any = true;
        }
    if (any && lo != 0xffffffffu) break;
  }
  return lo == 0xffffffffu ? -1 : (hi != (int)lo ? -2 : (int)lo);
}

__global__ void __launch_bounds__(kTX * kTY) kb_owner(const RelabelBox* __restrict__ boxes,
                                                      const RelabelEntry* __restrict__ e, int m) {
  __shared__ int32_t sl[(kTY + 2 * kOMaxR) * (kTX + 2 * kOMaxR)];
  const ListWalk lw = list_walk(boxes, e, m);
  const RelabelBox& B = *lw.B;
  const int nx = B.nx, ny = B.ny, R = B.R;
  const int32_t* L = B.label;
  for (int w = lw.first; w < lw.n; w += lw.stride) {
    const int t = B.tile_list[w];
    const int tx = t % B.ntx, ty = t / B.ntx;
    const int x = tx * kTX + threadIdx.x, y = ty * kTY + threadIdx.y;
    const bool in = x < nx && y < ny;
    const size_t c = (size_t)y * nx + x;
    if (!B.tile_active[t]) {  // went quiet since the previous relabel
      if (in) B.owner[c] = -1;
      continue;
    }
    const int W = kTX + 2 * R, H = kTY + 2 * R;
    const int bx0 = tx * kTX - R, by0 = ty * kTY - R;
    __syncthreads();  // the previous tile's window is no longer read
    for (int yy = threadIdx.y; yy < H; yy += kTY) {
      const size_t row = (size_t)wrap1(by0 + yy, ny) * nx;
      for (int xx = threadIdx.x; xx < W; xx += kTX) sl[yy * W + xx] = L[row + wrap1(bx0 + xx, nx)];
    }
    __syncthreads();
    const int* row0 = sl + (threadIdx.y + R) * W + threadIdx.x + R;
    int result = row0[0];
    if (result < 0 && R == 4) {  // the default zone radius
      result = nearest_label<4>(row0);
    } else if (result < 0) {
      result = window_owner(row0, W, R);
    }
    if (in) B.owner[c] = result;
  }
}

template <bool TWO>
__global__ void __launch_bounds__(kTX * kTY) kb_rupture(const RelabelBox* __restrict__ boxes,
                                                        const RelabelEntry* __restrict__ e, int m) {
  const ListWalk lw = list_walk(boxes, e, m);
  const RelabelBox& B = *lw.B;
  const int nx = B.nx, ny = B.ny;
  const int32_t* own = B.owner;
  for (int w = lw.first; w < lw.n; w += lw.stride) {
    const int t = B.tile_list[w];
    const int act = B.tile_active[t];
    const int x = (t % B.ntx) * kTX + threadIdx.x, y = (t / B.ntx) * kTY + threadIdx.y;
    const bool in = x < nx && y < ny;
    const size_t c = (size_t)y * nx + x;
    const int o = act && in ? own[c] : -1;
    int dir = 0;
    if (o != -1) {
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const int on = own[(size_t)wrap1(y + cy(i), ny) * nx + wrap1(x + cx(i), nx)];
        if (dir == 0 && on != -1 && on != o) dir = i;
      }
    }
    int opened = 0;
    if (dir == 0) {
      if (in) B.sgn[c] = 0;
    } else {
      int ex = 0, ey = 0;
#pragma unroll
      for (int i = 1; i < Q; ++i)
        if (i == dir) {
          ex = cx(i);
          ey = cy(i);
        }
      const size_t cp = (size_t)wrap1(y + ey, ny) * nx + wrap1(x + ex, nx);
      const size_t cm = (size_t)wrap1(y - ey, ny) * nx + wrap1(x - ex, nx);
      const float pp = TWO ? B.pr[cp] : pressure_of(B.rho[cp], B.G, B.rho0);
      const float p0 = TWO ? B.pr[c] : pressure_of(B.rho[c], B.G, B.rho0);
      const float pm = TWO ? B.pr[cm] : pressure_of(B.rho[cm], B.G, B.rho0);
      const float d2 = pp - 2.0f * p0 + pm;
      const int sg = (d2 > 0.f) - (d2 < 0.f);
      const int prevs = B.sgn[c];
      if (B.eps >= 0.f && !B.open[c] && (fabsf(d2) <= B.eps || (prevs != 0 && sg != prevs))) {
        B.open[c] = 1;
        opened = 1;
      }
      B.sgn[c] = (int8_t)sg;
    }
    const int n = __syncthreads_count(opened);
    if (n && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(B.flags + FLAG_OPENED, n);
  }
}

// Also records this relabel's activity as the "previous" one of the next:
// tiles outside the list are inactive in both, so only listed tiles change.
__global__ void __launch_bounds__(kTX * kTY) kb_mask(const RelabelBox* __restrict__ boxes,
                                                     const RelabelEntry* __restrict__ e, int m) {
  const ListWalk lw = list_walk(boxes, e, m);
  const RelabelBox& B = *lw.B;
  const int nx = B.nx, ny = B.ny;
  for (int w = lw.first; w < lw.n; w += lw.stride) {
    const int t = B.tile_list[w];
    const int act = B.tile_active[t];
    const int x = (t % B.ntx) * kTX + threadIdx.x, y = (t / B.ntx) * kTY + threadIdx.y;
    const bool in = x < nx && y < ny;
    const size_t c = (size_t)y * nx + x;
    unsigned msk = 0;
    const int o = act && in ? B.owner[c] : -1;
    if (o != -1 && !B.open[c]) {
#pragma unroll
      for (int i = 1; i < Q; ++i) {
        const size_t nb = (size_t)wrap1(y + cy(i), ny) * nx + wrap1(x + cx(i), nx);
        const int on = B.owner[nb];
        if (on != -1 && on != o && !B.open[nb]) msk |= 1u << (i - 1);
      }
    }
    if (in) B.mask[c] = (uint8_t)msk;
    // tiles holding a blocked edge go to the bounce-back's list
    const int film = __syncthreads_or((msk & kCanonBits) != 0);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
      B.tile_prev[t] = (uint8_t)act;
      if (film) B.film_list[atomicAdd(B.flags + FLAG_FILM, 1)] = t;
    }
  }
}

// --- halfway bounce-back across blocked edges (the barrier of Sec. 2.1.5) ---
// The step kernels store every outgoing population in its own slot: slot
// (plane i, x) holds f_i^out(x), which the next step pulls into x + e_i. For
// a blocked edge (x, x + e_i) the wall sends it back instead: f_i^out(x)
// returns to x as population opp(i), which the next step pulls from
// x - e_opp(i) = x + e_i in plane opp(i), and f_opp(i)^out(x + e_i) returns to
// x + e_i as population i, pulled from slot (plane i, x). So after the step
// the two slots of every blocked edge trade their values. The mask is
// symmetric; each edge is handled once, from its end whose direction is
// 1, 2, 5 or 6 (mask bits 0, 1, 4, 5), and every slot belongs to one edge
// only, so no two threads touch the same slot. T is the raw storage word
// (4 or 2 bytes: the values move bit for bit); TWO: a second lattice follows
// the first nine planes.
template <typename T, bool TWO>
__device__ __forceinline__ void bounce_cell(T* __restrict__ pops, size_t N, int x, int y, int nx, int ny,
                                            unsigned m) {
  m &= kCanonBits;
  if (!m) return;
  const size_t c = (size_t)y * nx + x;
#pragma unroll
  for (int i = 1; i <= 6; ++i) {
    if (i == 3 || i == 4 || !((m >> (i - 1)) & 1u)) continue;
    const size_t a = (size_t)i * N + c;
    const size_t b = (size_t)opp(i) * N + (size_t)wrap1(y + cy(i), ny) * nx + wrap1(x + cx(i), nx);
    const T va = pops[a], vb = pops[b];
    pops[a] = vb;
    pops[b] = va;
    if (TWO) {
      const size_t a2 = a + Q * N, b2 = b + Q * N;
      const T wa = pops[a2], wb = pops[b2];
      pops[a2] = wb;
      pops[b2] = wa;
    }
  }
}

// Every cell of a box (boxes that do not use the tiled pipeline).
template <typename T, bool TWO>
__global__ void k_bounce(T* __restrict__ pops, const uint8_t* __restrict__ mask, int nx, int ny) {
  const long long N = (long long)nx * ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const unsigned m = mask[c];
    if (m & kCanonBits) bounce_cell<T, TWO>(pops, (size_t)N, (int)(c % nx), (int)(c / nx), nx, ny, m);
  }
}

// Tiled boxes: the mask phase of the latest relabel listed the tiles that
// hold a blocked edge (a short list: film tiles only). Buffer
// B.pops[B.cur ^ q] of every box in the entry list.
template <typename T, bool TWO>
__global__ void __launch_bounds__(kTX * kTY) kb_bounce(const RelabelBox* __restrict__ boxes,
                                                       const RelabelEntry* __restrict__ e, int m, int q) {
  const ListWalk lw = list_walk(boxes, e, m);
  const RelabelBox& B = *lw.B;
  T* pops = static_cast<T*>(const_cast<void*>(B.pops[B.cur ^ q]));
  const size_t N = (size_t)B.nx * B.ny;
  const int nfilm = B.flags[FLAG_FILM];
  for (int w = lw.first; w < nfilm; w += lw.stride) {
    const int t = B.film_list[w];
    const int x = (t % B.ntx) * kTX + threadIdx.x, y = (t / B.ntx) * kTY + threadIdx.y;
    if (x >= B.nx || y >= B.ny) continue;
    const unsigned msk = B.mask[(size_t)y * B.nx + x];
    if (msk & kCanonBits) bounce_cell<T, TWO>(pops, N, x, y, B.nx, B.ny, msk);
  }
}

}  // namespace

int mass_partials_needed() { return kRedBlocks * kStatVals; }

#define LBM_DISPATCH(storage, KERNEL, ...)                                  \
  switch (storage) {                                                        \
    case LBM_F32: KERNEL<LBM_F32><<<__VA_ARGS__>>>; break;                  \
    case LBM_F16_DEV: KERNEL<LBM_F16_DEV><<<__VA_ARGS__>>>; break;          \
    case LBM_BF16_DEV: KERNEL<LBM_BF16_DEV><<<__VA_ARGS__>>>; break;        \
    default: return cudaErrorInvalidValue;                                  \
  }

cudaError_t launch_density(const FieldParams& fp, float* rho, cudaStream_t s) {
  const unsigned b = blocks_for(fp.N);
  switch (fp.storage) {
    case LBM_F32: k_density<LBM_F32><<<b, kThreads, 0, s>>>(fp, rho); break;
    case LBM_F16_DEV: k_density<LBM_F16_DEV><<<b, kThreads, 0, s>>>(fp, rho); break;
    case LBM_BF16_DEV: k_density<LBM_BF16_DEV><<<b, kThreads, 0, s>>>(fp, rho); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_labels(const FieldParams& fp, const float* rho, float threshold, int32_t* label,
                          int* flags, cudaStream_t s, int32_t* keep) {
  const unsigned b = blocks_for(fp.N);
  if (keep) k_label_init_keep<<<b, kThreads, 0, s>>>(rho, fp.N, threshold, label, keep);
  else k_label_init<<<b, kThreads, 0, s>>>(rho, fp.N, threshold, label);
  k_label_union<<<b, kThreads, 0, s>>>(fp.nx, fp.ny, label, flags);
  k_label_flatten<<<b, kThreads, 0, s>>>(fp.N, label, flags);
  if (keep) k_merge_count<<<b, kThreads, 0, s>>>(fp.N, label, keep, flags);
  return cudaGetLastError();
}

cudaError_t launch_owner(int nx, int ny, int R, const int32_t* label, int32_t* owner, cudaStream_t s) {
  if (R <= kOMaxR) {
    dim3 grid((nx + kOTX - 1) / kOTX, (ny + kOTY - 1) / kOTY);
    k_owner_tiled<<<grid, dim3(kOTX, kOTY), 0, s>>>(nx, ny, R, label, owner);
  } else {
    k_owner<<<blocks_for((long long)nx * ny), kThreads, 0, s>>>(nx, ny, R, label, owner);
  }
  return cudaGetLastError();
}

cudaError_t launch_rupture(int nx, int ny, float G, float rho0, float eps, const float* rho,
                           const int32_t* owner, int8_t* sgn, uint8_t* open, int* flags,
                           cudaStream_t s) {
  k_rupture<<<blocks_for((long long)nx * ny), kThreads, 0, s>>>(nx, ny, G, rho0, eps, rho, owner, sgn,
                                                                open, flags);
  return cudaGetLastError();
}

cudaError_t launch_mask(int nx, int ny, const int32_t* owner, const uint8_t* open, uint8_t* mask,
                        cudaStream_t s) {
  k_mask<<<blocks_for((long long)nx * ny), kThreads, 0, s>>>(nx, ny, owner, open, mask);
  return cudaGetLastError();
}

cudaError_t launch_fields(const FieldParams& fp, const float* rho, const uint8_t* mask, uint32_t which,
                          float* out, cudaStream_t s) {
  const unsigned b = blocks_for(fp.N);
  switch (fp.storage) {
    case LBM_F32: k_fields<LBM_F32><<<b, kThreads, 0, s>>>(fp, rho, mask, which, out); break;
    case LBM_F16_DEV: k_fields<LBM_F16_DEV><<<b, kThreads, 0, s>>>(fp, rho, mask, which, out); break;
    case LBM_BF16_DEV: k_fields<LBM_BF16_DEV><<<b, kThreads, 0, s>>>(fp, rho, mask, which, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_pops_out(const FieldParams& fp, int plane, float* out, cudaStream_t s) {
  const unsigned b = blocks_for(fp.N);
  switch (fp.storage) {
    case LBM_F32: k_pops_out<LBM_F32><<<b, kThreads, 0, s>>>(fp, plane, out); break;
    case LBM_F16_DEV: k_pops_out<LBM_F16_DEV><<<b, kThreads, 0, s>>>(fp, plane, out); break;
    case LBM_BF16_DEV: k_pops_out<LBM_BF16_DEV><<<b, kThreads, 0, s>>>(fp, plane, out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_init_from_rho(int storage, void* pops, const double* rho, int nx, int ny,
                                 const float* wref, cudaStream_t s) {
  FieldParams fp{};
  for (int i = 0; i < Q; ++i) fp.wref[i] = wref[i];
  const unsigned b = blocks_for((long long)nx * ny);
  switch (storage) {
    case LBM_F32:
      k_init_from_rho<LBM_F32><<<b, kThreads, 0, s>>>(static_cast<float*>(pops), rho, nx, ny, fp);
      break;
    case LBM_F16_DEV:
      k_init_from_rho<LBM_F16_DEV><<<b, kThreads, 0, s>>>(static_cast<__half*>(pops), rho, nx, ny, fp);
      break;
    case LBM_BF16_DEV:
      k_init_from_rho<LBM_BF16_DEV><<<b, kThreads, 0, s>>>(static_cast<__nv_bfloat16*>(pops), rho, nx,
                                                            ny, fp);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_load_plane(int storage, void* pops, const float* f_plane, int plane, int nx, int ny,
                              const float* wref, cudaStream_t s) {
  const unsigned b = blocks_for((long long)nx * ny);
  switch (storage) {
    case LBM_F32:
      k_load_plane<LBM_F32><<<b, kThreads, 0, s>>>(static_cast<float*>(pops), f_plane, plane, nx, ny,
                                                    wref[plane]);
      break;
    case LBM_F16_DEV:
      k_load_plane<LBM_F16_DEV><<<b, kThreads, 0, s>>>(static_cast<__half*>(pops), f_plane, plane, nx, ny,
                                                        wref[plane]);
      break;
    case LBM_BF16_DEV:
      k_load_plane<LBM_BF16_DEV><<<b, kThreads, 0, s>>>(static_cast<__nv_bfloat16*>(pops), f_plane,
                                                         plane, nx, ny, wref[plane]);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_bubbles_rho(const lbm_bubble* d_bubbles, int n, double rho_l, double rho_g,
                               double width, int nx, int ny, double* rho, cudaStream_t s) {
  const unsigned tiles = (unsigned)((nx + kInitTile - 1) / kInitTile) * ((ny + kInitTile - 1) / kInitTile);
  k_bubbles_rho<<<tiles, kThreads, 0, s>>>(d_bubbles, n, rho_l, rho_g, width, nx, ny, rho);
  return cudaGetLastError();
}

cudaError_t launch_mass(const FieldParams& fp, double* partials, int nparts, double* out_dev,
                        cudaStream_t s) {
  if (nparts < kRedBlocks) return cudaErrorInvalidValue;
  switch (fp.storage) {
    case LBM_F32: k_mass_partial<LBM_F32><<<kRedBlocks, kThreads, 0, s>>>(fp, partials); break;
    case LBM_F16_DEV: k_mass_partial<LBM_F16_DEV><<<kRedBlocks, kThreads, 0, s>>>(fp, partials); break;
    case LBM_BF16_DEV: k_mass_partial<LBM_BF16_DEV><<<kRedBlocks, kThreads, 0, s>>>(fp, partials); break;
    default: return cudaErrorInvalidValue;
  }
  k_sum_partials<1><<<1, kThreads, 0, s>>>(partials, kRedBlocks, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_stats(int nx, int ny, const int32_t* label, int32_t* area, double* partials, int nparts,
                         double* out_dev, int* hist, int nbins, double dmin, double dmax, cudaStream_t s) {
  if (nparts < kRedBlocks * kStatVals || nbins > kMaxBins) return cudaErrorInvalidValue;
  const long long N = (long long)nx * ny;
  cudaError_t e = cudaMemsetAsync(area, 0, sizeof(int32_t) * N, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(int) * kMaxBins, s);
  if (e != cudaSuccess) return e;
  k_area<<<blocks_for(N), kThreads, 0, s>>>(N, label, area);
  const double ldmin = log(dmin > 0 ? dmin : 1.0);
  const double ldspan = log(dmax > dmin && dmin > 0 ? dmax : 2.0 * (dmin > 0 ? dmin : 1.0)) - ldmin;
  k_stats_partial<<<kRedBlocks, kThreads, 0, s>>>(N, label, area, nbins, ldmin, ldspan, partials, hist);
  k_sum_partials<kStatVals><<<1, kThreads, 0, s>>>(partials, kRedBlocks, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_bubble_list(int nx, int ny, const int32_t* label, int32_t* area, int32_t* list, int* count,
                               cudaStream_t s) {
  const long long N = (long long)nx * ny;
  cudaError_t e = cudaMemsetAsync(area, 0, sizeof(int32_t) * N, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_area<<<blocks_for(N), kThreads, 0, s>>>(N, label, area);
  k_bubble_list<<<blocks_for(N), kThreads, 0, s>>>(N, label, area, list, count);
  return cudaGetLastError();
}

bool relabel_tiled_ok(int nx, int ny, int R) { return nx > 2 * R && ny > 2 * R && R <= kOMaxR; }

int relabel_tile_count(int nx, int ny) { return ((nx + kTX - 1) / kTX) * ((ny + kTY - 1) / kTY); }

void relabel_entry_sizes(int nx, int ny, int* tiles, int* scan, int* list) {
  const int t = relabel_tile_count(nx, ny);
  *tiles = t;
  *scan = (t + kThreads - 1) / kThreads;
  const int cap = list_ctas();
  *list = t < cap ? t : cap;
}

cudaError_t launch_relabel_boxes(int storage, const RelabelBox* boxes, const RelabelEntry* entries, int m,
                                 const int totals[3], int parity, cudaStream_t s, bool two) {
  if (m <= 0) return cudaSuccess;
  const dim3 block(kTX, kTY);
  if (two) {  // two components: FP32 only
    if (storage != LBM_F32) return cudaErrorInvalidValue;
    kb_density_label<LBM_F32, true><<<totals[0], block, 0, s>>>(boxes, entries, m, parity);
  } else {
    switch (storage) {
      case LBM_F32: kb_density_label32<<<totals[0], dim3(kTX / 4, kTY), 0, s>>>(boxes, entries, m, parity); break;
      case LBM_F16_DEV:
        kb_density_label16<LBM_F16_DEV><<<totals[0], dim3(kTX / 4, kTY), 0, s>>>(boxes, entries, m, parity);
        break;
      case LBM_BF16_DEV:
        kb_density_label16<LBM_BF16_DEV><<<totals[0], dim3(kTX / 4, kTY), 0, s>>>(boxes, entries, m, parity);
        break;
      default: return cudaErrorInvalidValue;
    }
  }
  kb_active<<<totals[1], kThreads, 0, s>>>(boxes, entries, m);
  kb_union<<<totals[2], block, 0, s>>>(boxes, entries, m);
  kb_flatten<<<totals[2], block, 0, s>>>(boxes, entries, m);
  kb_merge<<<totals[2], block, 0, s>>>(boxes, entries, m);
  kb_owner<<<totals[2], block, 0, s>>>(boxes, entries, m);
  if (two) kb_rupture<true><<<totals[2], block, 0, s>>>(boxes, entries, m);
  else kb_rupture<false><<<totals[2], block, 0, s>>>(boxes, entries, m);
  kb_mask<<<totals[2], block, 0, s>>>(boxes, entries, m);
  return cudaGetLastError();
}

cudaError_t launch_bounce(int storage, bool two, void* pops, const uint8_t* mask, int nx, int ny, cudaStream_t s) {
  const unsigned b = blocks_for((long long)nx * ny);
  if (two) {
    if (storage != LBM_F32) return cudaErrorInvalidValue;
    k_bounce<uint32_t, true><<<b, kThreads, 0, s>>>(static_cast<uint32_t*>(pops), mask, nx, ny);
  } else if (storage == LBM_F32) {
    k_bounce<uint32_t, false><<<b, kThreads, 0, s>>>(static_cast<uint32_t*>(pops), mask, nx, ny);
  } else {
    k_bounce<uint16_t, false><<<b, kThreads, 0, s>>>(static_cast<uint16_t*>(pops), mask, nx, ny);
  }
  return cudaGetLastError();
}

cudaError_t launch_bounce_boxes(int storage, bool two, const RelabelBox* boxes, const RelabelEntry* entries, int m,
                                int total_list, int q, cudaStream_t s) {
  if (m <= 0 || total_list <= 0) return cudaSuccess;
  const dim3 block(kTX, kTY);
  if (two) {
    if (storage != LBM_F32) return cudaErrorInvalidValue;
    kb_bounce<uint32_t, true><<<total_list, block, 0, s>>>(boxes, entries, m, q);
  } else if (storage == LBM_F32) {
    kb_bounce<uint32_t, false><<<total_list, block, 0, s>>>(boxes, entries, m, q);
  } else {
    kb_bounce<uint16_t, false><<<total_list, block, 0, s>>>(boxes, entries, m, q);
  }
  return cudaGetLastError();
}

}  // namespace lbm
