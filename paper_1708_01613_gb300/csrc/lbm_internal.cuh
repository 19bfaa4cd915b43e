// Internal declarations shared by the CUDA translation units of liblbm.
// Lattice: D2Q9 (arXiv 1708.01613, Sec. 2.1.1, Eqs. 15-16), directions
// 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

constexpr int Q = 9;

__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// Opposite direction: e_opp(i) = -e_i.
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : (i <= 4 ? (i + 1) % 4 + 1 : (i - 3) % 4 + 5); }
__host__ __device__ constexpr double wq(int i) {
  return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}
__host__ __device__ constexpr float wqf(int i) {
  return i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
}

// Device flag slots (int32 each) in the workspace.
enum Flag : int {
  FLAG_NUMERIC = 0,   // NaN/Inf or rho <= 0 seen by the step kernel
  FLAG_TIMEOUT = 1,   // a bounded device loop gave up
  FLAG_OPENED = 2,    // cells opened by the latest rupture test
  FLAG_TILES = 3,     // tiles in the relabel work list
  FLAG_GAS = 4,       // gas points in the growth list
  FLAG_ITEM = 5,      // work-item counter of the dynamically scheduled step (0 between launches)
  FLAG_DONE = 6,      // CTAs of that launch that have finished (0 between launches)
  FLAG_FILM = 7,      // tiles in the list of tiles holding a blocked edge
  FLAG_MERGES = 8,    // coalescence events counted by the relabels since the last init
  FLAG_HIST = 64,     // 64 histogram counters
  FLAG_COUNT = 128
};

// Population storage: FP32 value, or a 16-bit deviation from w_i rho_ref.
// Decode and encode are explicitly rounded single operations so that every
// kernel (scalar or packed) turns a stored value into the same float.
template <int S>
struct Store;

template <>
struct Store<LBM_F32> {
  using T = float;
  static constexpr int bytes = 4;
  __device__ static __forceinline__ float load(const T* p, size_t i, float) { return __ldg(p + i); }
  __device__ static __forceinline__ float load_smem(const T* p, int i, float) { return p[i]; }
  __device__ static __forceinline__ void store(T* p, size_t i, float v, float) { p[i] = v; }
  // raw stored value (FP32: the population itself)
  __device__ static __forceinline__ float raw(const T* p, size_t i) { return __ldg(p + i); }
  __device__ static __forceinline__ float raw_smem(const T* p, int i) { return p[i]; }
  __device__ static __forceinline__ void store_raw(T* p, size_t i, float v) { p[i] = v; }
};

template <>
struct Store<LBM_F16_DEV> {
  using T = __half;
  static constexpr int bytes = 2;
  __device__ static __forceinline__ float load(const T* p, size_t i, float base) {
    return __fadd_rn(base, __half2float(__ldg(p + i)));
  }
  __device__ static __forceinline__ float load_smem(const T* p, int i, float base) {
    return __fadd_rn(base, __half2float(p[i]));
  }
  __device__ static __forceinline__ void store(T* p, size_t i, float v, float base) {
    p[i] = __float2half_rn(__fsub_rn(v, base));
  }
  // raw stored value: the deviation g = f - w_i rho_ref
  __device__ static __forceinline__ float raw(const T* p, size_t i) { return __half2float(__ldg(p + i)); }
  __device__ static __forceinline__ float raw_smem(const T* p, int i) { return __half2float(p[i]); }
  __device__ static __forceinline__ void store_raw(T* p, size_t i, float g) { p[i] = __float2half_rn(g); }
};

template <>
struct Store<LBM_BF16_DEV> {
  using T = __nv_bfloat16;
  static constexpr int bytes = 2;
  __device__ static __forceinline__ float load(const T* p, size_t i, float base) {
    return __fadd_rn(base, __bfloat162float(__ldg(p + i)));
  }
  __device__ static __forceinline__ float load_smem(const T* p, int i, float base) {
    return __fadd_rn(base, __bfloat162float(p[i]));
  }
  __device__ static __forceinline__ void store(T* p, size_t i, float v, float base) {
    p[i] = __float2bfloat16_rn(__fsub_rn(v, base));
  }
  __device__ static __forceinline__ float raw(const T* p, size_t i) { return __bfloat162float(__ldg(p + i)); }
  __device__ static __forceinline__ float raw_smem(const T* p, int i) { return __bfloat162float(p[i]); }
  __device__ static __forceinline__ void store_raw(T* p, size_t i, float g) { p[i] = __float2bfloat16_rn(g); }
};

inline int storage_bytes(int s) { return s == LBM_F32 ? 4 : 2; }

// Row-chunk height of a launch whose `resident` CTAs draw chunks (gx strips
// by ny rows) from a counter. Chunks of max_rows rows give `items48` chunks;
// if those make at least keep_waves waves (chunks / resident CTAs), the last
// wave's tail is small beside the whole and max_rows stays. Otherwise the
// height is the one that fills a whole number of waves: the fewest that
// max_rows allows, but at least min_waves once the chunks overflow one wave
// (more, shorter chunks let the fast CTAs take more). A last wave that
// fills only part of the GPU leaves the rest idle for a whole chunk time.
inline int dyn_chunk_rows(long long gx, long long ny, long long resident, int max_rows, int keep_waves,
                          int min_waves) {
  if (gx < 1 || ny < 1 || resident < 1 || max_rows < 1) return 1;
  const long long items = gx * ((ny + max_rows - 1) / max_rows);
  if (items >= (long long)keep_waves * resident) return max_rows;
  long long waves = (items + resident - 1) / resident;
  if (items > resident && waves < min_waves) waves = min_waves;
  long long per = waves * resident / gx;  // chunks per strip
  if (per < 1) per = 1;
  const long long rows = (ny + per - 1) / per;
  return (int)(rows < 1 ? 1 : (rows > max_rows ? max_rows : rows));
}

// Arguments of the fused step kernel.
struct StepParams {
  const void* src;       // populations after collision of the previous step
  void* dst;             // populations after collision of this step
  const uint8_t* mask;   // blocked-edge mask (nullptr: plain Shan-Chen)
  int* flags;            // device flag slots
  int nx, ny;
  long long N;           // nx * ny (plane stride)
  int rows_per_chunk;    // rows marched by one CTA
  int force_generic;     // kernel variant: 0 automatic, 1 plain loads, 2 one-cell staged, 3 two-cell staged,
                         // 4 two-cell staged with dynamically scheduled row chunks
  float tau, inv_tau, G, rho0, inv_rho0;
  float rho_ref;         // reference density of 16-bit deviations
  float wref[Q];         // w_i * rho_ref (16-bit deviation base)
};

// Two-component step (step2.cu): 18 FP32 planes per buffer, melt then gas.
struct Step2Params {
  const void* src;
  void* dst;
  const uint8_t* mask;  // nullptr: no barrier
  int* flags;
  int nx, ny;
  long long N;
  int rows_per_chunk;
  float tau_m, tau_g, inv_tau_m, inv_tau_g;
  float G_mm, G_mg, G_gg, rho0, inv_rho0;
};
cudaError_t launch_step2(const Step2Params& p, cudaStream_t s);
// Melt/gas densities, mixture velocity (j + F/2)/rho and pressure of the
// state in p.src; any output may be nullptr.
cudaError_t launch_fields2(const Step2Params& p, float* rho_m, float* rho_g, float* ux, float* uy, float* pr,
                           cudaStream_t s);

// One box of a batched launch (device array).
struct BatchInst {
  void* pops0;
  void* pops1;
  const uint8_t* mask;  // nullptr: plain Shan-Chen
  int* flags;
  int nx, ny;
  float tau, inv_tau, G, rho0, inv_rho0, rho_ref;
  int cur;              // buffer holding the state when parity == 0
  int pad;
};

// One work item of a batched launch: columns x0 .. x0+width, rows y0 .. y1.
struct BatchItem {
  int inst, x0, width, y0, y1;
};

// Streaming multiprocessors of the current device (queried once per device;
// 152 on a GB300 if the query fails). Grids that are sized per SM use it.
int device_sm_count();

// Launch of the fused step (step.cu). Returns a cudaError_t.
cudaError_t launch_step(int storage, const StepParams& p, cudaStream_t s);
// Launch geometry the fused step uses for a box (for tests/benchmarks).
void step_geometry(int nx, int ny, int* grid_x, int* grid_y, int* rows_per_chunk, int* block);
// Whether the TMA-staged step kernel can run on a box of width nx.
bool step_tma_allowed(int storage, int nx);
// Batched fused step (two-cell staged march over a list of work items of
// many boxes); one persistent grid drawing items from counters[parity] and
// zeroing counters[parity ^ 1]. Both counters must be zero before the
// first launch and consecutive launches must alternate parity.
// unal: the items' boxes have rows that do not start on 16-byte boundaries
// (the staging variant that bulk-copies aligned interiors and plain-loads
// the rest); one launch takes items of one kind.
cudaError_t launch_step_batch(int storage, bool masked, bool tau_one, bool unal, const BatchInst* insts,
                              const BatchItem* items, int nitems, int* counters, int parity, cudaStream_t s);
// CTAs of the batched kernel that fit the GPU at once.
int batch_resident_ctas(int storage, bool masked, bool tau_one);
// Whether the two-cell staged step kernel can run on a box of width nx with
// whole rows bulk-copied (nx % 16 == 0), or in its variant for other widths.
bool step_tma2_allowed(int storage, int nx);
bool step_tma2_unaligned_allowed(int nx);

// Barrier / field / reduction kernels (barrier.cu).
struct Workspace {
  void* pops[2];
  float* rho;          // N: density of the current state (relabel, fields)
  int32_t* label;      // N
  int32_t* owner;      // N (barrier)
  uint8_t* mask;       // N (barrier)
  uint8_t* open;       // N (barrier)
  int8_t* sgn;         // N (barrier)
  int* flags;          // FLAG_COUNT
  double* partials;    // reduction partials
  int partial_count;
};

struct FieldParams {
  const void* pops;    // current populations (post-collision of the last step)
  int storage;
  int nx, ny;
  long long N;
  float G, rho0, inv_rho0, tau;
  float wref[Q];
};

cudaError_t launch_density(const FieldParams& fp, float* rho, cudaStream_t s);
// Gas labels (4-connected, smallest index) of rho into label. With keep (the
// relabel pipeline: the owner array), each new gas cell first parks its
// label of the previous relabel there and the coalescence events are added
// to flags[FLAG_MERGES]; keep = nullptr for diagnostics.
cudaError_t launch_labels(const FieldParams& fp, const float* rho, float threshold, int32_t* label,
                          int* flags, cudaStream_t s, int32_t* keep = nullptr);
// Per-bubble areas of a label array: roots (label[c] == c) with their cell
// counts appended to list (pairs root, area) in any order; the count goes to
// *count (device). area: N int32 scratch.
cudaError_t launch_bubble_list(int nx, int ny, const int32_t* label, int32_t* area, int32_t* list, int* count,
                               cudaStream_t s);
cudaError_t launch_owner(int nx, int ny, int R, const int32_t* label, int32_t* owner, cudaStream_t s);
cudaError_t launch_rupture(int nx, int ny, float G, float rho0, float eps, const float* rho,
                           const int32_t* owner, int8_t* sgn, uint8_t* open, int* flags,
                           cudaStream_t s);
cudaError_t launch_mask(int nx, int ny, const int32_t* owner, const uint8_t* open, uint8_t* mask,
                        cudaStream_t s);
cudaError_t launch_fields(const FieldParams& fp, const float* rho, const uint8_t* mask,
                          uint32_t which, float* out, cudaStream_t s);
cudaError_t launch_pops_out(const FieldParams& fp, int plane, float* out, cudaStream_t s);
cudaError_t launch_init_from_rho(int storage, void* pops, const double* rho, int nx, int ny,
                                 const float* wref, cudaStream_t s);
cudaError_t launch_load_plane(int storage, void* pops, const float* f_plane, int plane, int nx,
                              int ny, const float* wref, cudaStream_t s);
cudaError_t launch_bubbles_rho(const lbm_bubble* d_bubbles, int n, double rho_l, double rho_g,
                               double width, int nx, int ny, double* rho, cudaStream_t s);
cudaError_t launch_mass(const FieldParams& fp, double* partials, int nparts, double* out_dev,
                        cudaStream_t s);
cudaError_t launch_stats(int nx, int ny, const int32_t* label, int32_t* area, double* partials,
                         int nparts, double* out_dev, int* hist, int nbins, double dmin, double dmax,
                         cudaStream_t s);
constexpr int kMaxHistBins = 64;
// Tiled barrier pipeline (barrier.cu): density + labels + tile flags, then
// union, flatten, owner, rupture and mask restricted to tiles near gas.
// One launch per phase serves any number of boxes.
bool relabel_tiled_ok(int nx, int ny, int R);
int relabel_tile_count(int nx, int ny);
constexpr int kRelabelTileX = 32, kRelabelTileY = 8;  // tile of the pipeline
// Launches of one relabel: density, tile scan (tiled) or label init (untiled),
// union, flatten, coalescence count, owner, rupture, mask.
constexpr int kRelabelLaunches = 8;

// A box as the pipeline sees it (device memory). Populations are read from
// pops[cur ^ parity], parity being the launch argument.
struct RelabelBox {
  const void* pops[2];
  float* rho;
  int32_t* label;
  int32_t* owner;
  int8_t* sgn;
  uint8_t* open;
  uint8_t* mask;
  uint8_t* tile_gas;
  uint8_t* tile_active;
  uint8_t* tile_prev;
  int* tile_list;
  int* film_list;  // tiles of the work list holding a blocked edge (bounce-back)
  int* flags;
  float* pr;  // two components: mixture pressure written by the density
              // phase and used by the rupture test (nullptr: one component)
  int nx, ny, ntx, nty, R, cur;
  float threshold, G, rho0, eps;
  float G_mg, G_gg;  // two components: melt-gas and gas-gas couplings
  float wref[Q];
};

// Box `box` in a launch's entry list, with the CTAs of the entries before it
// in each kind of phase (per-tile, tile-scan, tile-list). An entry list of m
// boxes has m + 1 entries: the last holds the totals.
struct RelabelEntry {
  int box, off_tiles, off_scan, off_list;
};

// Halfway bounce-back across the blocked edges of the mask (the barrier of
// Sec. 2.1.5), run on the buffer a step has just written (after the growth
// source, if any): the two slots of each blocked edge trade values, so the
// next step's pull returns every population that would cross the wall to
// its own cell in the opposite direction. `two`: 18 planes (two lattices).
// launch_bounce scans every cell; launch_bounce_boxes visits the tiles that
// the latest tiled relabel of each box in the entry list found holding a
// blocked edge, on buffer pops[cur ^ q] (total_list = the entries' list-CTA
// total).
cudaError_t launch_bounce(int storage, bool two, void* pops, const uint8_t* mask, int nx, int ny, cudaStream_t s);
cudaError_t launch_bounce_boxes(int storage, bool two, const RelabelBox* boxes, const RelabelEntry* entries, int m,
                                int total_list, int q, cudaStream_t s);

// CTAs a box takes in each kind of phase.
void relabel_entry_sizes(int nx, int ny, int* tiles, int* scan, int* list);
// The seven phases over the first m entries; totals = entries[m]'s offsets.
// two_component: the boxes are two-component (FP32; mixture pressure).
cudaError_t launch_relabel_boxes(int storage, const RelabelBox* boxes, const RelabelEntry* entries, int m,
                                 const int totals[3], int parity, cudaStream_t s, bool two_component = false);
int mass_partials_needed();

// Nucleation and growth (growth.cu). The gas census appends every cell with
// rho < threshold to `list` (order irrelevant) and sets *count. The growth
// kernel adds w_i drho to the post-collision populations of the listed
// cells, drho = min(rate, budget - released) / count, reading the released
// total from released[parity] and writing the new total to
// released[parity ^ 1] (consecutive steps alternate parity).
cudaError_t launch_gas_census(const float* rho, long long N, float threshold, int32_t* list, int* count,
                              cudaStream_t s);
cudaError_t launch_growth(int storage, void* pops, const int32_t* list, const int* count, long long N,
                          double rate, double budget, double* released, int parity, cudaStream_t s);
cudaError_t launch_nucleate(int storage, void* pops, const lbm_bubble* nuclei, int n, double rho_g, int nx,
                            int ny, const float* wref, cudaStream_t s);

}  // namespace lbm
