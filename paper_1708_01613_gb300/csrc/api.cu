// C ABI of liblbm (declared in include/lbm.h): configuration checks,
// workspace layout, and the host driver of the time loop of the extended
// Shan-Chen method (arXiv 1708.01613, Sec. 2.1.4 main flowchart: barrier
// pipeline when due, then collide+stream with the modified force).
//
// The library never allocates device memory: every device buffer is a slice
// of the caller's workspace. The population buffer that is idle between
// steps doubles as staging space for host transfers and as scratch for the
// statistics.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "handle.cuh"

using namespace lbm;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }



bool valid_config(const lbm_config* c, char* why, size_t n) {
  if (!c) return snprintf(why, n, "config is NULL"), false;
  if (c->nx < 4 || c->ny < 4) return snprintf(why, n, "nx, ny must be >= 4"), false;
  if ((long long)c->nx * c->ny > 0x7fffffffLL)
    return snprintf(why, n, "nx * ny must fit in int32"), false;
  if (c->storage < LBM_F32 || c->storage > LBM_BF16_DEV) return snprintf(why, n, "bad storage"), false;
  if (c->barrier != 0 && c->barrier != 1) return snprintf(why, n, "barrier must be 0 or 1"), false;
  if (c->relabel_every < 1) return snprintf(why, n, "relabel_every must be >= 1"), false;
  if (c->zone_radius < 0) return snprintf(why, n, "zone_radius must be >= 0"), false;
  if (c->barrier && (2 * c->zone_radius + 1 >= c->nx || 2 * c->zone_radius + 1 >= c->ny))
    return snprintf(why, n, "with the barrier on, 2 zone_radius + 1 < nx, ny"), false;
  if (c->stop_on_first_rupture != 0 && c->stop_on_first_rupture != 1)
    return snprintf(why, n, "stop_on_first_rupture must be 0 or 1"), false;
  if (c->growth != 0 && c->growth != 1) return snprintf(why, n, "growth must be 0 or 1"), false;
  if (c->components != 1 && c->components != 2) return snprintf(why, n, "components must be 1 or 2"), false;
  if (c->reserved2 != 0) return snprintf(why, n, "reserved2 must be 0"), false;
  if (c->components == 2) {
    if (c->storage != LBM_F32) return snprintf(why, n, "two components need FP32 storage"), false;
    if (c->growth) return snprintf(why, n, "two components do not take the growth source"), false;
    if (!(c->tau_g > 0.5) || !isfinite(c->tau_g)) return snprintf(why, n, "tau_g must be > 0.5"), false;
    if (!isfinite(c->G_mg) || !isfinite(c->G_gg)) return snprintf(why, n, "G_mg, G_gg must be finite"), false;
    if (c->barrier && !relabel_tiled_ok(c->nx, c->ny, c->zone_radius))
      return snprintf(why, n, "two components with the barrier need R_z <= 16"), false;
  }
  if (!(c->tau > 0.5) || !isfinite(c->tau)) return snprintf(why, n, "tau must be > 0.5"), false;
  if (!isfinite(c->G)) return snprintf(why, n, "G must be finite"), false;
  if (!(c->rho0 > 0.0) || !isfinite(c->rho0)) return snprintf(why, n, "rho0 must be > 0"), false;
  if (!isfinite(c->rho_ref) || !isfinite(c->gas_threshold) || !isfinite(c->rupture_eps))
    return snprintf(why, n, "rho_ref, gas_threshold, rupture_eps must be finite"), false;
  return true;
}

Layout layout_for(const lbm_config& c) {
  Layout L{};
  const size_t N = (size_t)c.nx * c.ny;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t eb = (size_t)storage_bytes(c.storage);
  const size_t comps = c.components == 2 ? 2 : 1;
  L.pops[0] = take(comps * Q * N * eb);
  L.pops[1] = take(comps * Q * N * eb);
  L.rho = take(4 * N);
  L.label = take(4 * N);
  if (c.barrier) {
    L.owner = take(4 * N);
    L.mask = take(N);
    L.open = take(N);
    L.sgn = take(N);
    L.ntiles = relabel_tile_count(c.nx, c.ny);
    L.tiles = take(3 * (size_t)L.ntiles);  // gas, active, previous active
    L.tile_list = take(8 * (size_t)L.ntiles);  // work list, then the tiles with a blocked edge
    L.rbox = take(sizeof(RelabelBox) + 2 * sizeof(RelabelEntry));
  }
  if (c.growth) L.gas_list = take(4 * N);
  if (c.components == 2 && c.barrier) L.pr = take(4 * N);
  L.flags = take(sizeof(int) * FLAG_COUNT);
  L.nparts = mass_partials_needed();
  L.partials = take(sizeof(double) * L.nparts);
  L.scalars = take(sizeof(double) * 16);
  L.total = off;
  return L;
}

}  // namespace



namespace {

int fail(lbm_handle* h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CUDA_TRY(h, expr)                                                               \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail((h), LBM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));             \
  } while (0)

// Buffer `buf`'s planes of component k (two-component boxes are FP32).
void* component_pops(lbm_handle* h, int buf, int k) {
  return static_cast<char*>(h->pops(buf)) + (size_t)k * Q * h->N() * storage_bytes(h->cfg.storage);
}

Step2Params step2_params(lbm_handle* h) {
  const lbm_config& c = h->cfg;
  Step2Params q{};
  q.src = h->pops(h->cur);
  q.dst = h->pops(1 - h->cur);
  q.mask = c.barrier ? h->mask() : nullptr;
  q.flags = h->flags();
  q.nx = c.nx;
  q.ny = c.ny;
  q.N = (long long)h->N();
  q.tau_m = (float)c.tau;
  q.tau_g = (float)c.tau_g;
  q.inv_tau_m = (float)(1.0 / c.tau);
  q.inv_tau_g = (float)(1.0 / c.tau_g);
  q.G_mm = (float)c.G;
  q.G_mg = (float)c.G_mg;
  q.G_gg = (float)c.G_gg;
  q.rho0 = (float)c.rho0;
  q.inv_rho0 = (float)(1.0 / c.rho0);
  return q;
}

FieldParams field_params(lbm_handle* h) {
  FieldParams fp{};
  fp.pops = h->pops(h->cur);
  fp.storage = h->cfg.storage;
  fp.nx = h->cfg.nx;
  fp.ny = h->cfg.ny;
  fp.N = (long long)h->N();
  fp.G = (float)h->cfg.G;
  fp.rho0 = (float)h->cfg.rho0;
  fp.inv_rho0 = (float)(1.0 / h->cfg.rho0);
  fp.tau = (float)h->cfg.tau;
  for (int i = 0; i < Q; ++i) fp.wref[i] = h->wref[i];
  return fp;
}

int select_device(lbm_handle* h) {
  CUDA_TRY(h, cudaSetDevice(h->device));
  return LBM_OK;
}

int check_flags(lbm_handle* h) {
  int f[3] = {0, 0, 0};
  CUDA_TRY(h, cudaMemcpyAsync(f, h->flags(), sizeof(f), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (f[FLAG_NUMERIC]) return fail(h, LBM_ENUMERIC, "NaN/Inf or rho <= 0 met by the step kernel");
  if (f[FLAG_TIMEOUT]) return fail(h, LBM_ETIMEOUT, "a bounded labelling loop gave up");
  return LBM_OK;
}

int reset_state(lbm_handle* h) {
  CUDA_TRY(h, cudaMemsetAsync(h->flags(), 0, sizeof(int) * FLAG_COUNT, h->stream));
  if (h->cfg.barrier) {
    CUDA_TRY(h, cudaMemsetAsync(h->mask(), 0, h->N(), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->open(), 0, h->N(), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->sgn(), 0, h->N(), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->owner(), 0xff, 4 * h->N(), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->label(), 0xff, 4 * h->N(), h->stream));  // no earlier bubbles
    CUDA_TRY(h, cudaMemsetAsync(h->tiles(0), 0, 3 * (size_t)h->L.ntiles, h->stream));
  }
  CUDA_TRY(h, cudaMemsetAsync(h->released(), 0, 2 * sizeof(double), h->stream));
  h->t = 0;
  h->halted = 0;
  return LBM_OK;
}

// Descriptor and one-box entry list of the tiled barrier pipeline, written
// into the workspace once (pointers into the workspace do not move).
int upload_relabel_box(lbm_handle* h) {
  if (!handle_relabel_tiled(h)) return LBM_OK;
  const RelabelBox b = handle_relabel_box(h);
  RelabelEntry e[2] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  relabel_entry_sizes(h->cfg.nx, h->cfg.ny, &e[1].off_tiles, &e[1].off_scan, &e[1].off_list);
  CUDA_TRY(h, cudaMemcpyAsync(h->rbox(), &b, sizeof(b), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->rentries(), e, sizeof(e), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // the sources live on this stack frame
  return LBM_OK;
}

// Barrier pipeline on the current populations (Sec. 2.1.5).
int relabel(lbm_handle* h) {
  const FieldParams fp = field_params(h);
  const lbm_config& c = h->cfg;
  if (handle_relabel_tiled(h)) {
    int totals[3];
    relabel_entry_sizes(c.nx, c.ny, &totals[0], &totals[1], &totals[2]);
    CUDA_TRY(h, launch_relabel_boxes(c.storage, h->rbox(), h->rentries(), 1, totals, h->cur, h->stream,
                                     h->comps() == 2));
    h->launches += kRelabelLaunches;
    return LBM_OK;
  }
  CUDA_TRY(h, launch_density(fp, h->rho(), h->stream));
  CUDA_TRY(h, launch_labels(fp, h->rho(), (float)c.gas_threshold, h->label(), h->flags(), h->stream, h->owner()));
  CUDA_TRY(h, launch_owner(c.nx, c.ny, c.zone_radius, h->label(), h->owner(), h->stream));
  CUDA_TRY(h, launch_rupture(c.nx, c.ny, (float)c.G, (float)c.rho0, (float)c.rupture_eps, h->rho(),
                             h->owner(), h->sgn(), h->open(), h->flags(), h->stream));
  CUDA_TRY(h, launch_mask(c.nx, c.ny, h->owner(), h->open(), h->mask(), h->stream));
  h->launches += kRelabelLaunches;
  return LBM_OK;
}

// Bounce-back across the blocked edges on the buffer the step just wrote
// (pops(1 - cur)), over the latest relabel's tile list where the box uses the
// tiled pipeline.
cudaError_t bounce_after_step(lbm_handle* h) {
  const lbm_config& c = h->cfg;
  const bool two = h->comps() == 2;
  if (handle_relabel_tiled(h)) {
    int totals[3];
    relabel_entry_sizes(c.nx, c.ny, &totals[0], &totals[1], &totals[2]);
    return launch_bounce_boxes(c.storage, two, h->rbox(), h->rentries(), 1, totals[2], h->cur ^ 1, h->stream);
  }
  return launch_bounce(c.storage, two, h->pops(1 - h->cur), h->mask(), c.nx, c.ny, h->stream);
}

int read_opened(lbm_handle* h, int* out) {
  CUDA_TRY(h, cudaMemcpyAsync(out, h->flags() + FLAG_OPENED, sizeof(int), cudaMemcpyDeviceToHost,
                              h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

size_t field_bytes(const lbm_handle* h, uint32_t bit) {
  const size_t N = h->N();
  switch (bit) {
    case LBM_FIELD_RHO:
    case LBM_FIELD_UX:
    case LBM_FIELD_UY:
    case LBM_FIELD_P:
    case LBM_FIELD_LABEL:
    case LBM_FIELD_OWNER: return 4 * N;
    case LBM_FIELD_MASK:
    case LBM_FIELD_OPEN: return N;
    case LBM_FIELD_POPS: return 4 * Q * N * h->comps();
    case LBM_FIELD_RHO_GAS: return 4 * N;
    default: return 0;
  }
}

constexpr uint32_t kLastField = LBM_FIELD_RHO_GAS;
constexpr uint32_t kAllFields = (kLastField << 1) - 1;

}  // namespace

namespace lbm {

int handle_fail(lbm_handle* h, int code, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

int handle_relabel(lbm_handle* h) { return relabel(h); }

bool handle_relabel_tiled(const lbm_handle* h) {
  return h->cfg.barrier && relabel_tiled_ok(h->cfg.nx, h->cfg.ny, h->cfg.zone_radius);
}

RelabelBox handle_relabel_box(lbm_handle* h) {
  const lbm_config& c = h->cfg;
  RelabelBox b;
  memset(&b, 0, sizeof(b));
  b.pops[0] = h->pops(0);
  b.pops[1] = h->pops(1);
  b.rho = h->rho();
  b.label = h->label();
  b.owner = h->owner();
  b.sgn = h->sgn();
  b.open = h->open();
  b.mask = h->mask();
  b.tile_gas = h->tiles(0);
  b.tile_active = h->tiles(1);
  b.tile_prev = h->tiles(2);
  b.tile_list = reinterpret_cast<int*>(h->ws + h->L.tile_list);
  b.film_list = b.tile_list + h->L.ntiles;
  b.flags = h->flags();
  b.pr = h->pr();
  b.G_mg = (float)c.G_mg;
  b.G_gg = (float)c.G_gg;
  b.nx = c.nx;
  b.ny = c.ny;
  b.ntx = (c.nx + kRelabelTileX - 1) / kRelabelTileX;
  b.nty = (c.ny + kRelabelTileY - 1) / kRelabelTileY;
  b.R = c.zone_radius;
  b.cur = 0;
  b.threshold = (float)c.gas_threshold;
  b.G = (float)c.G;
  b.rho0 = (float)c.rho0;
  b.eps = (float)c.rupture_eps;
  for (int i = 0; i < Q; ++i) b.wref[i] = h->wref[i];
  return b;
}

int handle_check_flags(lbm_handle* h) { return check_flags(h); }

StepParams handle_step_params(lbm_handle* h) {
  const lbm_config& c = h->cfg;
  StepParams p{};
  p.mask = c.barrier ? h->mask() : nullptr;
  p.force_generic = h->variant;
  p.flags = h->flags();
  p.nx = c.nx;
  p.ny = c.ny;
  p.N = (long long)h->N();
  p.tau = (float)c.tau;
  p.inv_tau = (float)(1.0 / c.tau);
  p.G = (float)c.G;
  p.rho0 = (float)c.rho0;
  p.inv_rho0 = (float)(1.0 / c.rho0);
  p.rho_ref = (float)c.rho_ref;
  for (int i = 0; i < Q; ++i) p.wref[i] = h->wref[i];
  return p;
}

}  // namespace lbm

extern "C" {

void lbm_config_default(lbm_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->nx = 256;
  cfg->ny = 256;
  cfg->storage = LBM_F32;
  cfg->barrier = 0;
  cfg->relabel_every = 1;
  cfg->zone_radius = 4;
  cfg->stop_on_first_rupture = 0;
  cfg->tau = 1.0;
  cfg->G = -5.5;
  cfg->rho0 = 1.0;
  cfg->rho_ref = 1.0;
  cfg->gas_threshold = log(2.0);
  cfg->rupture_eps = 1e-6;
  cfg->components = 1;
  cfg->tau_g = 1.0;
}

size_t lbm_workspace_bytes(const lbm_config* cfg) {
  char why[128];
  if (!valid_config(cfg, why, sizeof(why))) return 0;
  return layout_for(*cfg).total;
}

int lbm_create(const lbm_config* cfg, void* d_workspace, size_t bytes, void* cuda_stream,
               lbm_handle** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  char why[256];
  if (!valid_config(cfg, why, sizeof(why))) return LBM_EINVAL;
  const Layout L = layout_for(*cfg);
  if (!d_workspace || ((uintptr_t)d_workspace % kAlign) != 0) return LBM_EINVAL;
  if (bytes < L.total) return LBM_ENOMEM;
  lbm_handle* h = new (std::nothrow) lbm_handle();
  if (!h) return LBM_ENOMEM;
  h->cfg = *cfg;
  h->L = L;
  h->ws = static_cast<char*>(d_workspace);
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  h->cur = 0;
  h->err[0] = 0;
  for (int i = 0; i < Q; ++i) h->wref[i] = cfg->storage == LBM_F32 ? 0.0f : (float)(wq(i) * cfg->rho_ref);
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return LBM_ECUDA;
  }
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, d_workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    delete h;
    return LBM_EINVAL;
  }
  if (reset_state(h) != LBM_OK || upload_relabel_box(h) != LBM_OK) {
    delete h;
    return LBM_ECUDA;
  }
  *out = h;
  return LBM_OK;
}

int lbm_init_density(lbm_handle* h, const double* rho, int src_is_device) {
  if (!h) return LBM_EINVAL;
  if (!rho) return fail(h, LBM_EINVAL, "rho is NULL");
  int rc = select_device(h);
  if (rc) return rc;
  const double* src = rho;
  const int comps = h->comps();
  if (!src_is_device) {
    void* stage = h->pops(1 - h->cur);
    CUDA_TRY(h, cudaMemcpyAsync(stage, rho, 8 * h->N() * comps, cudaMemcpyHostToDevice, h->stream));
    src = static_cast<const double*>(stage);
  }
  for (int k = 0; k < comps; ++k)  // component k's planes follow the previous component's nine
    CUDA_TRY(h, launch_init_from_rho(h->cfg.storage, component_pops(h, h->cur, k), src + (size_t)k * h->N(),
                                     h->cfg.nx, h->cfg.ny, h->wref, h->stream));
  return reset_state(h);
}

int lbm_init_bubbles(lbm_handle* h, const lbm_bubble* b, int32_t n, double rho_l, double rho_g,
                     double width) {
  if (!h) return LBM_EINVAL;
  if (h->comps() != 1) return fail(h, LBM_ENOTSUP, "bubble initialisation is for one component");
  if (n < 0 || (n > 0 && !b)) return fail(h, LBM_EINVAL, "bad bubble list");
  if (!(width > 0.0) || !isfinite(rho_l) || !isfinite(rho_g))
    return fail(h, LBM_EINVAL, "width must be > 0 and densities finite");
  for (int k = 0; k < n; ++k)
    if (!isfinite(b[k].cx) || !isfinite(b[k].cy) || !isfinite(b[k].r))
      return fail(h, LBM_EINVAL, "bubble %d is not finite", k);
  const size_t bub_bytes = align_up(sizeof(lbm_bubble) * (size_t)n);
  if (bub_bytes + 8 * h->N() > h->pops_bytes())
    return fail(h, LBM_EINVAL, "too many bubbles for the staging area (%d)", n);
  int rc = select_device(h);
  if (rc) return rc;
  char* stage = static_cast<char*>(h->pops(1 - h->cur));
  lbm_bubble* d_b = reinterpret_cast<lbm_bubble*>(stage);
  double* d_rho = reinterpret_cast<double*>(stage + bub_bytes);
  if (n > 0)
    CUDA_TRY(h, cudaMemcpyAsync(d_b, b, sizeof(lbm_bubble) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, launch_bubbles_rho(d_b, n, rho_l, rho_g, width, h->cfg.nx, h->cfg.ny, d_rho, h->stream));
  CUDA_TRY(h, launch_init_from_rho(h->cfg.storage, h->pops(h->cur), d_rho, h->cfg.nx, h->cfg.ny, h->wref,
                                   h->stream));
  // the bubble list is read from pageable memory by an async copy: keep it valid
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return reset_state(h);
}

int lbm_load_populations(lbm_handle* h, const float* f, int src_is_device) {
  if (!h) return LBM_EINVAL;
  if (!f) return fail(h, LBM_EINVAL, "populations pointer is NULL");
  int rc = select_device(h);
  if (rc) return rc;
  const size_t N = h->N();
  for (int pl = 0; pl < Q * h->comps(); ++pl) {
    const float* plane = f + (size_t)pl * N;
    if (!src_is_device) {
      float* stage = static_cast<float*>(h->pops(1 - h->cur));
      CUDA_TRY(h, cudaMemcpyAsync(stage, plane, 4 * N, cudaMemcpyHostToDevice, h->stream));
      plane = stage;
    }
    CUDA_TRY(h, launch_load_plane(h->cfg.storage, component_pops(h, h->cur, pl / Q), plane, pl % Q, h->cfg.nx,
                                  h->cfg.ny, h->wref, h->stream));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->halted = 0;
  return LBM_OK;
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
  if (!h) return LBM_EINVAL;
  if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps < 0");
  if (h->in_batch) return fail(h, LBM_EINVAL, "handle belongs to a batch; step it through lbm_batch_step");
  int rc = select_device(h);
  if (rc) return rc;
  const lbm_config& c = h->cfg;
  StepParams p = handle_step_params(h);
  for (int64_t s = 0; s < nsteps && !h->halted; ++s) {
    bool stop_after = false;
    if (c.barrier && h->t % c.relabel_every == 0) {
      int before = 0;
      if (c.stop_on_first_rupture && (rc = read_opened(h, &before))) return rc;
      if ((rc = relabel(h))) return rc;
      if (c.stop_on_first_rupture) {
        int after = 0;
        if ((rc = read_opened(h, &after))) return rc;
        stop_after = after > before;
      }
    }
    const bool growing = h->growth_rate > 0.0;
    if (growing && h->t % c.relabel_every == 0) {  // gas census with the barrier pipeline
      if (!c.barrier) CUDA_TRY(h, launch_density(field_params(h), h->rho(), h->stream));
      CUDA_TRY(h, launch_gas_census(h->rho(), (long long)h->N(), (float)c.gas_threshold, h->gas_list(),
                                    h->flags() + FLAG_GAS, h->stream));
      h->launches += c.barrier ? 1 : 2;
    }
    p.src = h->pops(h->cur);
    p.dst = h->pops(1 - h->cur);
    if (c.components == 2) {
      const Step2Params q = step2_params(h);
      CUDA_TRY(h, launch_step2(q, h->stream));
    } else {
      CUDA_TRY(h, launch_step(c.storage, p, h->stream));
    }
    h->launches += 1;
    if (growing) {
      CUDA_TRY(h, launch_growth(c.storage, p.dst, h->gas_list(), h->flags() + FLAG_GAS, (long long)h->N(),
                                h->growth_rate, h->growth_budget, h->released(), (int)(h->t & 1), h->stream));
      h->launches += 1;
    }
    if (c.barrier) {  // populations that would cross a blocked edge bounce back
      CUDA_TRY(h, bounce_after_step(h));
      h->launches += 1;
    }
    h->cur ^= 1;
    h->t += 1;
    if (stop_after) h->halted = 1;
  }
  return LBM_OK;
}

int64_t lbm_steps_done(const lbm_handle* h) { return h ? h->t : -1; }

int64_t lbm_kernel_launches(const lbm_handle* h) { return h ? h->launches : -1; }

int lbm_set_step_variant(lbm_handle* h, int variant) {
  if (!h) return LBM_EINVAL;
  if (variant < 0 || variant > 4) return fail(h, LBM_EINVAL, "variant must be 0, 1, 2, 3 or 4");
  if (variant == 2 && !step_tma_allowed(h->cfg.storage, h->cfg.nx))
    return fail(h, LBM_ENOTSUP, "TMA-staged step needs nx %% 16 == 0 and nx >= 272");
  if ((variant == 3 || variant == 4) && !step_tma2_allowed(h->cfg.storage, h->cfg.nx) &&
      !step_tma2_unaligned_allowed(h->cfg.nx))
    return fail(h, LBM_ENOTSUP, "two-cell staged step needs nx >= 16");
  h->variant = variant;
  return LBM_OK;
}

int lbm_halted(const lbm_handle* h) { return h ? h->halted : 0; }

size_t lbm_fields_bytes(const lbm_handle* h, uint32_t fields) {
  if (!h || (fields & ~kAllFields)) return 0;
  size_t total = 0;
  for (uint32_t bit = 1; bit <= kLastField; bit <<= 1)
    if (fields & bit) total += field_bytes(h, bit);
  return total;
}

int lbm_read_fields(lbm_handle* h, uint32_t fields, void* dst, size_t dst_bytes, int dst_is_device) {
  if (!h) return LBM_EINVAL;
  if (!dst || fields == 0 || (fields & ~kAllFields)) return fail(h, LBM_EINVAL, "bad field selection");
  if (dst_bytes < lbm_fields_bytes(h, fields)) return fail(h, LBM_EINVAL, "dst too small");
  int rc = select_device(h);
  if (rc) return rc;
  const FieldParams fp = field_params(h);
  const size_t N = h->N();
  char* out = static_cast<char*>(dst);
  float* stage = static_cast<float*>(h->pops(1 - h->cur));
  const cudaMemcpyKind d2x = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(h, launch_density(fp, h->rho(), h->stream));
  for (uint32_t bit = 1; bit <= kLastField; bit <<= 1) {
    if (!(fields & bit)) continue;
    const size_t nb = field_bytes(h, bit);
    switch (bit) {
      case LBM_FIELD_RHO:
      case LBM_FIELD_UX:
      case LBM_FIELD_UY:
      case LBM_FIELD_P:
      case LBM_FIELD_RHO_GAS: {
        float* target = dst_is_device ? reinterpret_cast<float*>(out) : stage;
        if (h->comps() == 2) {
          const Step2Params q = step2_params(h);
          CUDA_TRY(h, launch_fields2(q, bit == LBM_FIELD_RHO ? target : nullptr,
                                     bit == LBM_FIELD_RHO_GAS ? target : nullptr, bit == LBM_FIELD_UX ? target : nullptr,
                                     bit == LBM_FIELD_UY ? target : nullptr, bit == LBM_FIELD_P ? target : nullptr,
                                     h->stream));
        } else if (bit == LBM_FIELD_RHO_GAS) {
          CUDA_TRY(h, cudaMemsetAsync(target, 0, nb, h->stream));
        } else {
          CUDA_TRY(h, launch_fields(fp, h->rho(), h->mask(), bit, target, h->stream));
        }
        if (!dst_is_device) CUDA_TRY(h, cudaMemcpyAsync(out, stage, nb, d2x, h->stream));
        break;
      }
      case LBM_FIELD_LABEL: {
        // into scratch: the relabel pipeline's own labels stay those of the
        // last relabel (the coalescence count compares the next one with them)
        int32_t* lab = dst_is_device ? reinterpret_cast<int32_t*>(out) : reinterpret_cast<int32_t*>(stage);
        CUDA_TRY(h, launch_labels(fp, h->rho(), (float)h->cfg.gas_threshold, lab, h->flags(), h->stream));
        if (!dst_is_device) CUDA_TRY(h, cudaMemcpyAsync(out, stage, nb, d2x, h->stream));
        break;
      }
      case LBM_FIELD_OWNER:
      case LBM_FIELD_MASK:
      case LBM_FIELD_OPEN: {
        const void* srcp = bit == LBM_FIELD_OWNER ? (const void*)h->owner()
                           : bit == LBM_FIELD_MASK ? (const void*)h->mask()
                                                   : (const void*)h->open();
        if (srcp) {
          CUDA_TRY(h, cudaMemcpyAsync(out, srcp, nb, d2x, h->stream));
        } else {
          const int fill = bit == LBM_FIELD_OWNER ? 0xff : 0;
          if (dst_is_device)
            CUDA_TRY(h, cudaMemsetAsync(out, fill, nb, h->stream));
          else
            memset(out, fill, nb);
        }
        break;
      }
      case LBM_FIELD_POPS:
        for (int pl = 0; pl < Q * h->comps(); ++pl) {
          FieldParams fk = fp;
          fk.pops = component_pops(h, h->cur, pl / Q);
          float* target = dst_is_device ? reinterpret_cast<float*>(out + 4 * N * pl) : stage;
          CUDA_TRY(h, launch_pops_out(fk, pl % Q, target, h->stream));
          if (!dst_is_device)
            CUDA_TRY(h, cudaMemcpyAsync(out + 4 * N * pl, stage, 4 * N, d2x, h->stream));
        }
        break;
    }
    out += nb;
  }
  return check_flags(h);
}

int lbm_nucleate(lbm_handle* h, const lbm_bubble* nuclei, int32_t n, double rho_g) {
  if (!h) return LBM_EINVAL;
  if (n < 0 || (n > 0 && !nuclei)) return fail(h, LBM_EINVAL, "bad nucleus list");
  if (!isfinite(rho_g)) return fail(h, LBM_EINVAL, "rho_g must be finite");
  for (int k = 0; k < n; ++k)
    if (!isfinite(nuclei[k].cx) || !isfinite(nuclei[k].cy) || !(nuclei[k].r >= 0.0) || !isfinite(nuclei[k].r))
      return fail(h, LBM_EINVAL, "nucleus %d: centre must be finite and 0 <= r finite", k);
  if (n == 0) return LBM_OK;
  if (sizeof(lbm_bubble) * (size_t)n > h->pops_bytes())
    return fail(h, LBM_EINVAL, "too many nuclei for the staging area (%d)", n);
  int rc = select_device(h);
  if (rc) return rc;
  lbm_bubble* d_n = static_cast<lbm_bubble*>(h->pops(1 - h->cur));  // the idle buffer stages the list
  CUDA_TRY(h, cudaMemcpyAsync(d_n, nuclei, sizeof(lbm_bubble) * n, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, launch_nucleate(h->cfg.storage, h->pops(h->cur), d_n, n, rho_g, h->cfg.nx, h->cfg.ny, h->wref,
                              h->stream));
  h->launches += 1;
  // the list is read from pageable memory by an async copy: keep it valid
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_set_growth(lbm_handle* h, double rate, double budget) {
  if (!h) return LBM_EINVAL;
  if (!h->cfg.growth) return fail(h, LBM_EINVAL, "the handle was created without config.growth");
  if (h->cfg.storage != LBM_F32)
    return fail(h, LBM_ENOTSUP, "the growth source needs FP32 storage (per-step increments fall below "
                                "the resolution of 16-bit deviations and would be lost)");
  if (!(rate >= 0.0) || !isfinite(rate) || !(budget >= 0.0) || !isfinite(budget))
    return fail(h, LBM_EINVAL, "rate and budget must be finite and >= 0");
  int rc = select_device(h);
  if (rc) return rc;
  // no census yet: nothing is released before the next one
  CUDA_TRY(h, cudaMemsetAsync(h->flags() + FLAG_GAS, 0, sizeof(int), h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->released(), 0, 2 * sizeof(double), h->stream));
  h->growth_rate = rate;
  h->growth_budget = budget;
  return LBM_OK;
}

int lbm_growth_released(lbm_handle* h, double* out) {
  if (!h) return LBM_EINVAL;
  if (!out) return fail(h, LBM_EINVAL, "out is NULL");
  int rc = select_device(h);
  if (rc) return rc;
  // the slot written by the latest step (or zeroed by lbm_set_growth)
  CUDA_TRY(h, cudaMemcpyAsync(out, h->released() + (h->t & 1), sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_mass(lbm_handle* h, double* out) {
  if (!h) return LBM_EINVAL;
  if (!out) return fail(h, LBM_EINVAL, "out is NULL");
  int rc = select_device(h);
  if (rc) return rc;
  double part[2] = {0.0, 0.0};
  for (int k = 0; k < h->comps(); ++k) {
    FieldParams fk = field_params(h);
    fk.pops = component_pops(h, h->cur, k);
    CUDA_TRY(h, launch_mass(fk, h->partials(), h->L.nparts, h->scalars(), h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(&part[k], h->scalars(), sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // the scalar slot is reused by the next component
  }
  *out = part[0] + part[1];
  return check_flags(h);
}

int lbm_bubble_stats(lbm_handle* h, lbm_stats* out, double* hist, int32_t nbins, double dmin, double dmax) {
  if (!h) return LBM_EINVAL;
  if (!out) return fail(h, LBM_EINVAL, "out is NULL");
  if (hist && (nbins < 1 || nbins > kMaxHistBins || !(dmin > 0.0) || !(dmax > dmin)))
    return fail(h, LBM_EINVAL, "histogram needs 1 <= nbins <= %d and 0 < dmin < dmax", kMaxHistBins);
  int rc = select_device(h);
  if (rc) return rc;
  const FieldParams fp = field_params(h);
  // labels and areas in the idle population buffer (>= 18 bytes per cell)
  int32_t* lab = static_cast<int32_t*>(h->pops(1 - h->cur));
  int32_t* area = lab + h->N();
  CUDA_TRY(h, launch_density(fp, h->rho(), h->stream));
  CUDA_TRY(h, launch_labels(fp, h->rho(), (float)h->cfg.gas_threshold, lab, h->flags(), h->stream));
  CUDA_TRY(h, launch_stats(h->cfg.nx, h->cfg.ny, lab, area, h->partials(), h->L.nparts, h->scalars(),
                           h->flags() + FLAG_HIST, hist ? nbins : 0, hist ? dmin : 1.0, hist ? dmax : 2.0,
                           h->stream));
  double sc[3];
  int hc[kMaxHistBins];
  int opened = 0, merges = 0;
  CUDA_TRY(h, cudaMemcpyAsync(sc, h->scalars(), sizeof(sc), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(hc, h->flags() + FLAG_HIST, sizeof(hc), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(&opened, h->flags() + FLAG_OPENED, sizeof(int), cudaMemcpyDeviceToHost,
                              h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(&merges, h->flags() + FLAG_MERGES, sizeof(int), cudaMemcpyDeviceToHost,
                              h->stream));
  if ((rc = check_flags(h))) return rc;
  double mass = 0.0;
  if ((rc = lbm_mass(h, &mass))) return rc;
  memset(out, 0, sizeof(*out));
  out->step = h->t;
  out->n_bubbles = (int32_t)llround(sc[0]);
  out->n_open = opened;
  out->gas_fraction = sc[1] / (double)h->N();
  out->mean_eq_diameter = sc[0] > 0 ? sc[2] / sc[0] : 0.0;
  out->mass = mass;
  out->n_merges = merges;
  if (hist)
    for (int b = 0; b < nbins; ++b) hist[b] = hc[b];
  return LBM_OK;
}

int lbm_bubble_areas(lbm_handle* h, int32_t capacity, int32_t* labels, double* areas, int32_t* n_out) {
  if (!h) return LBM_EINVAL;
  if (!n_out || capacity < 0 || (capacity > 0 && (!labels || !areas)))
    return fail(h, LBM_EINVAL, "need n_out, and labels and areas for capacity > 0");
  int rc = select_device(h);
  if (rc) return rc;
  const FieldParams fp = field_params(h);
  const size_t N = h->N();
  // scratch in the idle population buffer: labels, areas, (root, area) list
  // (bubbles <= N / 2: each needs a liquid neighbour or covers the box)
  int32_t* lab = static_cast<int32_t*>(h->pops(1 - h->cur));
  int32_t* area = lab + N;
  int32_t* list = area + N;
  int* count = h->flags() + FLAG_HIST;  // the histogram slots serve as scratch here
  CUDA_TRY(h, launch_density(fp, h->rho(), h->stream));
  CUDA_TRY(h, launch_labels(fp, h->rho(), (float)h->cfg.gas_threshold, lab, h->flags(), h->stream));
  CUDA_TRY(h, launch_bubble_list(h->cfg.nx, h->cfg.ny, lab, area, list, count, h->stream));
  int n = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&n, count, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  if ((rc = check_flags(h))) return rc;
  *n_out = n;
  if (n > capacity) return fail(h, LBM_EINVAL, "%d bubbles, capacity %d", n, capacity);
  std::vector<int32_t> pairs(2 * (size_t)n);
  if (n) {
    CUDA_TRY(h, cudaMemcpyAsync(pairs.data(), list, sizeof(int32_t) * 2 * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return pairs[2 * a] < pairs[2 * b]; });
  for (int k = 0; k < n; ++k) {
    labels[k] = pairs[2 * order[k]];
    areas[k] = (double)pairs[2 * order[k] + 1];
  }
  return LBM_OK;
}

int lbm_sync(lbm_handle* h) {
  if (!h) return LBM_EINVAL;
  int rc = select_device(h);
  if (rc) return rc;
  return check_flags(h);
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err : "handle is NULL"; }

void lbm_destroy(lbm_handle* h) { delete h; }

}  // extern "C"
