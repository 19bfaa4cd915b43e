// Host-side handle of liblbm, shared by the C-ABI translation units
// (api.cu for one box, batch.cu for batched launches).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "lbm_internal.cuh"

namespace lbm {

// Offsets of the slices of the caller's workspace.
struct Layout {
  size_t pops[2], rho, label, owner, mask, open, sgn, tiles, tile_list, rbox, gas_list, pr, flags, partials,
      scalars, total;
  int nparts, ntiles;
};

}  // namespace lbm

struct lbm_handle {
  lbm_config cfg;
  lbm::Layout L;
  char* ws;
  cudaStream_t stream;
  int device;
  int cur;
  int64_t t;
  int64_t launches;
  int variant;
  int halted;
  int in_batch;  // 1 while a batch drives this handle
  double growth_rate, growth_budget;  // growth source (rate 0: off)
  float wref[lbm::Q];
  char err[320];

  void* pops(int k) { return ws + L.pops[k]; }
  float* rho() { return reinterpret_cast<float*>(ws + L.rho); }
  int32_t* label() { return reinterpret_cast<int32_t*>(ws + L.label); }
  int32_t* owner() { return cfg.barrier ? reinterpret_cast<int32_t*>(ws + L.owner) : nullptr; }
  uint8_t* mask() { return cfg.barrier ? reinterpret_cast<uint8_t*>(ws + L.mask) : nullptr; }
  uint8_t* open() { return cfg.barrier ? reinterpret_cast<uint8_t*>(ws + L.open) : nullptr; }
  int8_t* sgn() { return cfg.barrier ? reinterpret_cast<int8_t*>(ws + L.sgn) : nullptr; }
  uint8_t* tiles(int k) { return reinterpret_cast<uint8_t*>(ws + L.tiles) + (size_t)k * L.ntiles; }
  int* flags() { return reinterpret_cast<int*>(ws + L.flags); }
  int32_t* gas_list() { return cfg.growth ? reinterpret_cast<int32_t*>(ws + L.gas_list) : nullptr; }
  // released growth total, two slots taking turns with the step parity
  double* released() { return reinterpret_cast<double*>(ws + L.scalars) + 14; }
  // the box's own barrier-pipeline descriptor and its one-box entry list
  lbm::RelabelBox* rbox() { return reinterpret_cast<lbm::RelabelBox*>(ws + L.rbox); }
  lbm::RelabelEntry* rentries() { return reinterpret_cast<lbm::RelabelEntry*>(rbox() + 1); }
  double* partials() { return reinterpret_cast<double*>(ws + L.partials); }
  double* scalars() { return reinterpret_cast<double*>(ws + L.scalars); }
  size_t N() const { return (size_t)cfg.nx * cfg.ny; }
  int comps() const { return cfg.components == 2 ? 2 : 1; }
  // bytes of one population buffer (all components)
  size_t pops_bytes() const { return (size_t)lbm::Q * comps() * N() * lbm::storage_bytes(cfg.storage); }
  float* pr() { return cfg.components == 2 && cfg.barrier ? reinterpret_cast<float*>(ws + L.pr) : nullptr; }
};

namespace lbm {

// Records a message on the handle and returns code.
int handle_fail(lbm_handle* h, int code, const char* fmt, ...);
// Enqueues the barrier pipeline on the handle's current populations.
int handle_relabel(lbm_handle* h);
// Synchronises the handle's stream and reports device-side faults.
int handle_check_flags(lbm_handle* h);
// Step parameters of the handle (buffers chosen by the caller).
StepParams handle_step_params(lbm_handle* h);
// True when the handle's barrier pipeline runs tiled (RelabelBox form).
bool handle_relabel_tiled(const lbm_handle* h);
// The handle's barrier-pipeline descriptor (host copy, cur = 0).
RelabelBox handle_relabel_box(lbm_handle* h);

}  // namespace lbm
