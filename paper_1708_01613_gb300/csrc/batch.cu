// Batched time stepping of many boxes (C ABI lbm_batch_*, include/lbm.h).
//
// A batch advances several independent boxes together: every step is one
// persistent launch of the two-cell staged kernel over a list of work items
// (box, column strip, row chunk) that covers all active boxes, preceded, when
// a relabel is due, by each box's barrier pipeline and followed, with the
// barrier, by the bounce-back across the boxes' blocked edges. Blocks of K steps (K =
// relabel period) are captured once as CUDA graphs and replayed. The strip
// width and chunk height of the work items are picked by lbm_batch_tune,
// which times the candidates on the batch itself. Per-cell arithmetic is the
// one of the single-box kernels, so every box evolves bitwise as it would
// alone.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <map>
#include <new>
#include <vector>

#include "handle.cuh"

using namespace lbm;

struct lbm_batch {
  std::vector<lbm_handle*> h;
  std::vector<int> active;
  std::vector<int> base_cur;   // h[i]->cur when the descriptors were uploaded
  int n = 0;
  int storage = 0, masked = 0, tau_one = 1, K = 1;
  int64_t t = 0;               // common step counter
  int par = 0;                 // steps since upload, mod 2
  cudaStream_t stream = nullptr;      // the batch's own stream (capturable)
  cudaStream_t ext = nullptr;         // the boxes' stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  BatchInst* d_insts = nullptr;
  BatchItem* d_items = nullptr;
  int* d_counter = nullptr;
  int max_items = 0;
  int nitems = 0;
  int nitems_a = 0;            // items of boxes with 16-byte rows come first; then the others
  std::vector<BatchItem> items;
  // barrier pipeline: tiled boxes relabel together, one launch per phase for
  // all boxes due at the same step; boxes are grouped by the residue of their
  // step count modulo the relabel period (relative to the batch counter)
  RelabelBox* d_rboxes = nullptr;
  RelabelEntry* d_rent = nullptr;
  struct Group {
    int start = 0;                        // first entry in d_rent
    std::vector<int> members;             // box indices, upload order
    std::vector<std::array<int, 3>> tot;  // CTA totals of the first k members
  };
  std::map<int, Group> groups;            // by residue of the step count
  std::vector<int> untiled;               // boxes relabelled one by one
  std::vector<char> lone;                 // boxes narrower than the staged kernel takes
                                          // (< 16 columns): stepped by the plain-load
                                          // kernel in the same sequence
  std::vector<char> unal;                 // rows not 16-byte multiples: the staged
                                          // kernel's variant for them (own launch)
  // bounce-back after each step: tiled boxes together (entries d_bent, in
  // stepping order), untiled boxes one by one
  RelabelEntry* d_bent = nullptr;
  std::vector<int> bounce_first;          // tiled boxes among the first k stepping boxes
  std::vector<int> bounce_ctas;           // list CTAs of the first k tiled boxes
  int strip = 512, rows = 0;
  int use_graph = 1;
  int dirty = 1;               // descriptors/items must be re-uploaded
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // K-step block starting at parity 0 / 1
  int64_t graph_launches[2] = {0, 0};             // kernels in each graph
  int64_t launches = 0;
  char err[320] = {0};
};

namespace {

constexpr size_t kAlign = 256;
constexpr int kMinItems = 64;  // work items per box, where its height allows
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int bfail(lbm_batch* b, int code, const char* fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof(b->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define BCUDA(b, expr)                                                               \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess) return bfail((b), LBM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

// Upper bound of work items for any tile choice the batch accepts.
int max_items_for(lbm_handle* const* hs, int n) {
  long long m = 0;
  for (int i = 0; i < n; ++i) m += (long long)((hs[i]->cfg.nx + 255) / 256) * hs[i]->cfg.ny;
  return m > 0x7fffffff ? 0x7fffffff : (int)m;
}

void drop_graphs(lbm_batch* b) {
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) {
      cudaGraphExecDestroy(b->graph[k]);
      b->graph[k] = nullptr;
    }
}

// Work items. A CTA walks its item row by row, each row a dependent
// load-compute-store round of a few microseconds, so a launch lasts about
// (rows per item) x (items per CTA) such rounds. While the tuned height
// gives at least four waves of items over the resident CTAs it stays;
// otherwise chunks take the smallest height whose items fill the fewest
// whole waves (at least four for FP32 once one is exceeded), as for a lone
// box: a fractional last wave idles the rest of the GPU for a chunk time,
// and with less than one wave every resident CTA gets one item. For
// multi-rate steps (`spread`) a box also gets at least kMinItems items, so
// that the launches over a few small boxes at the end of a call stay short
// too.
void build_items(lbm_batch* b, bool spread) {
  b->items.clear();
  const int res = std::max(1, batch_resident_ctas(b->storage, b->masked != 0, b->tau_one != 0));
  auto count = [&](int rows) {
    long long c = 0;
    for (int i = 0; i < b->n; ++i)
      if (b->active[i] && !b->lone[i])
        c += (long long)((b->h[i]->cfg.nx + b->strip - 1) / b->strip) * ((b->h[i]->cfg.ny + rows - 1) / rows);
    return c;
  };
  int rows_all = std::max(1, b->rows);
  const long long items_tuned = count(rows_all);
  if (items_tuned > 0 && items_tuned < 4LL * res) {
    long long waves = (items_tuned + res - 1) / res;
    if (b->storage == LBM_F32 && items_tuned > res && waves < 4) waves = 4;
    int lo = 1, hi = rows_all;  // smallest height whose items fit `waves` waves
    while (lo < hi) {
      const int mid = lo + (hi - lo) / 2;
      if (count(mid) <= waves * res) hi = mid;
      else lo = mid + 1;
    }
    rows_all = lo;
  }
  for (int i = 0; i < b->n; ++i) {
    if (!b->active[i] || b->lone[i]) continue;
    const int nx = b->h[i]->cfg.nx, ny = b->h[i]->cfg.ny;
    const int strips = (nx + b->strip - 1) / b->strip;
    const int rows = spread ? std::max(1, std::min(rows_all, (strips * ny + kMinItems - 1) / kMinItems)) : rows_all;
    for (int x0 = 0; x0 < nx; x0 += b->strip)
      for (int y0 = 0; y0 < ny; y0 += rows) {
        BatchItem it;
        it.inst = i;
        it.x0 = x0;
        it.width = std::min(b->strip, nx - x0);
        it.y0 = y0;
        it.y1 = std::min(y0 + rows, ny);
        b->items.push_back(it);
      }
  }
  // largest items first: the dynamic queue then balances like LPT scheduling
  std::stable_sort(b->items.begin(), b->items.end(), [](const BatchItem& a, const BatchItem& c) {
    return (long long)a.width * (a.y1 - a.y0) > (long long)c.width * (c.y1 - c.y0);
  });
  // boxes with 16-byte rows first (one launch), then the others (another)
  std::stable_partition(b->items.begin(), b->items.end(), [&](const BatchItem& it) { return !b->unal[it.inst]; });
  b->nitems = (int)b->items.size();
  b->nitems_a = 0;
  for (const BatchItem& it : b->items) b->nitems_a += !b->unal[it.inst];
}

// Re-uploads descriptors and items (host-synchronous copies). Boxes may be
// at different step counts: each relabels on its own phase. `order` lists
// the boxes to step, in the order their barrier entries take (empty = all
// active boxes, by index; a non-empty order means multi-rate steps).
int upload(lbm_batch* b, const std::vector<int>& order = {}) {
  if (!b->dirty) return LBM_OK;
  std::vector<BatchInst> insts(b->n);
  std::vector<RelabelBox> rboxes(b->masked ? b->n : 0);
  for (int i = 0; i < b->n; ++i) {
    lbm_handle* h = b->h[i];
    BatchInst& d = insts[i];
    memset(&d, 0, sizeof(d));
    d.pops0 = h->pops(0);
    d.pops1 = h->pops(1);
    d.mask = h->cfg.barrier ? h->mask() : nullptr;
    d.flags = h->flags();
    d.nx = h->cfg.nx;
    d.ny = h->cfg.ny;
    d.tau = (float)h->cfg.tau;
    d.inv_tau = (float)(1.0 / h->cfg.tau);
    d.G = (float)h->cfg.G;
    d.rho0 = (float)h->cfg.rho0;
    d.inv_rho0 = (float)(1.0 / h->cfg.rho0);
    d.rho_ref = (float)h->cfg.rho_ref;
    d.cur = h->cur;
    b->base_cur[i] = h->cur;
    if (b->masked && handle_relabel_tiled(h)) {
      rboxes[i] = handle_relabel_box(h);
      rboxes[i].cur = h->cur;
    }
  }
  build_items(b, !order.empty());
  if (b->nitems > b->max_items) return bfail(b, LBM_EINVAL, "too many work items (%d > %d)", b->nitems, b->max_items);
  BCUDA(b, cudaMemcpyAsync(b->d_insts, insts.data(), sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice, b->stream));
  if (b->nitems)
    BCUDA(b, cudaMemcpyAsync(b->d_items, b->items.data(), sizeof(BatchItem) * b->nitems, cudaMemcpyHostToDevice,
                             b->stream));
  BCUDA(b, cudaMemsetAsync(b->d_counter, 0, 4 * sizeof(int), b->stream));  // item counters (kind, step parity)
  b->groups.clear();
  b->untiled.clear();
  b->bounce_first.assign(1, 0);
  b->bounce_ctas.assign(1, 0);
  std::vector<RelabelEntry> ents, bents;
  if (b->masked) {
    std::vector<int> ord = order;
    if (ord.empty())
      for (int i = 0; i < b->n; ++i)
        if (b->active[i]) ord.push_back(i);
    const int r = b->h[0]->cfg.relabel_every;
    for (int i : ord) {  // bounce-back entries: the tiled boxes in stepping order
      const bool tiled = handle_relabel_tiled(b->h[i]);
      if (tiled) {
        int t0, t1, t2;
        relabel_entry_sizes(b->h[i]->cfg.nx, b->h[i]->cfg.ny, &t0, &t1, &t2);
        bents.push_back({i, 0, 0, b->bounce_ctas.back()});
        b->bounce_ctas.push_back(b->bounce_ctas.back() + t2);
      }
      b->bounce_first.push_back(b->bounce_first.back() + (tiled ? 1 : 0));
    }
    bents.push_back({-1, 0, 0, b->bounce_ctas.back()});
    for (int i : ord) {
      lbm_handle* h = b->h[i];
      if (!handle_relabel_tiled(h)) {
        b->untiled.push_back(i);
        continue;
      }
      // due at batch count T when T + (t_i - t_batch) is a multiple of r
      const int64_t o = ((h->t - b->t) % r + r) % r;
      b->groups[(int)((r - o) % r)].members.push_back(i);
    }
    for (auto& kv : b->groups) {
      lbm_batch::Group& g = kv.second;
      g.start = (int)ents.size();
      std::array<int, 3> acc = {0, 0, 0};
      g.tot.push_back(acc);
      for (int i : g.members) {
        ents.push_back({i, acc[0], acc[1], acc[2]});
        int t0, t1, t2;
        relabel_entry_sizes(b->h[i]->cfg.nx, b->h[i]->cfg.ny, &t0, &t1, &t2);
        acc = {acc[0] + t0, acc[1] + t1, acc[2] + t2};
        g.tot.push_back(acc);
      }
      ents.push_back({-1, acc[0], acc[1], acc[2]});
    }
    BCUDA(b, cudaMemcpyAsync(b->d_rboxes, rboxes.data(), sizeof(RelabelBox) * b->n, cudaMemcpyHostToDevice,
                             b->stream));
    if (!ents.empty())
      BCUDA(b, cudaMemcpyAsync(b->d_rent, ents.data(), sizeof(RelabelEntry) * ents.size(), cudaMemcpyHostToDevice,
                               b->stream));
    BCUDA(b, cudaMemcpyAsync(b->d_bent, bents.data(), sizeof(RelabelEntry) * bents.size(), cudaMemcpyHostToDevice,
                             b->stream));
  }
  BCUDA(b, cudaStreamSynchronize(b->stream));
  b->par = 0;
  b->dirty = 0;
  drop_graphs(b);
  return LBM_OK;
}

// Barrier pipeline of the boxes due at batch count b->t + j: the first
// `live` members of their residue group (all of them when live < 0) in one
// launch per phase, and the untiled boxes one by one (those for which
// `stepping` says yes). Buffers: parity `parity` since the upload.
template <class Stepping>
int enqueue_relabel(lbm_batch* b, int parity, int64_t j, int live, Stepping stepping) {
  const int r = b->h[0]->cfg.relabel_every;
  const auto it = b->groups.find((int)((b->t + j) % r));
  if (it != b->groups.end()) {
    const lbm_batch::Group& g = it->second;
    const int m = live < 0 ? (int)g.members.size() : std::min(live, (int)g.members.size());
    if (m > 0) {
      BCUDA(b, launch_relabel_boxes(b->storage, b->d_rboxes, b->d_rent + g.start, m, g.tot[m].data(), parity,
                                    b->stream));
      b->launches += kRelabelLaunches;
    }
  }
  for (int i : b->untiled) {
    lbm_handle* h = b->h[i];
    if (!stepping(i) || (h->t + j) % r != 0) continue;
    const int saved = h->cur;
    h->cur = b->base_cur[i] ^ parity;
    cudaStream_t hs = h->stream;
    h->stream = b->stream;
    const int rc = handle_relabel(h);
    h->stream = hs;
    h->cur = saved;
    if (rc) return bfail(b, rc, "relabel of box %d: %s", i, h->err);
    b->launches += kRelabelLaunches;
  }
  return LBM_OK;
}

// The batched kernels of one step: the items of boxes with 16-byte rows
// (counters 0, 1) and those of the other boxes (counters 2, 3).
int enqueue_items(lbm_batch* b, int parity, const BatchItem* items_a, int na, const BatchItem* items_u, int nu) {
  if (na > 0) {
    BCUDA(b, launch_step_batch(b->storage, b->masked != 0, b->tau_one != 0, false, b->d_insts, items_a, na,
                               b->d_counter, parity, b->stream));
    b->launches += 1;
  }
  if (nu > 0) {
    BCUDA(b, launch_step_batch(b->storage, b->masked != 0, b->tau_one != 0, true, b->d_insts, items_u, nu,
                               b->d_counter + 2, parity, b->stream));
    b->launches += 1;
  }
  return LBM_OK;
}

// The boxes outside the item list (lone) that step now: one plain-load step
// each, on the buffers of parity `parity`, on the batch stream.
template <class Stepping>
int enqueue_lone(lbm_batch* b, int parity, Stepping stepping) {
  for (int i = 0; i < b->n; ++i) {
    if (!b->lone[i] || !stepping(i)) continue;
    lbm_handle* h = b->h[i];
    StepParams p = handle_step_params(h);
    p.src = h->pops(b->base_cur[i] ^ parity);
    p.dst = h->pops(b->base_cur[i] ^ parity ^ 1);
    BCUDA(b, launch_step(b->storage, p, b->stream));
    b->launches += 1;
  }
  return LBM_OK;
}

// Bounce-back across blocked edges after the batched step of parity
// `parity`: the first `first` boxes of the stepping order (all of them when
// first < 0), on the buffers that step wrote.
template <class Stepping>
int enqueue_bounce(lbm_batch* b, int parity, int first, Stepping stepping) {
  const int total = (int)b->bounce_first.size() - 1;
  const int k = b->bounce_first[first < 0 || first > total ? total : first];
  if (k > 0) {
    BCUDA(b, launch_bounce_boxes(b->storage, false, b->d_rboxes, b->d_bent, k, b->bounce_ctas[k], parity ^ 1,
                                 b->stream));
    b->launches += 1;
  }
  for (int i : b->untiled) {
    if (!stepping(i)) continue;
    lbm_handle* h = b->h[i];
    BCUDA(b, launch_bounce(b->storage, false, h->pops(b->base_cur[i] ^ parity ^ 1), h->mask(), h->cfg.nx,
                           h->cfg.ny, b->stream));
    b->launches += 1;
  }
  return LBM_OK;
}

// Host bookkeeping after `n` steps of every active box.
void advance(lbm_batch* b, int64_t n) {
  b->t += n;
  b->par ^= (int)(n & 1);
  for (int i = 0; i < b->n; ++i)
    if (b->active[i]) {
      b->h[i]->t += n;
      b->h[i]->cur = b->base_cur[i] ^ b->par;
    }
}

// Enqueues one step `j` steps after the boxes' current state (relabel of
// every box whose own step count is then due, then the batched kernel).
int enqueue_step(lbm_batch* b, int parity, int64_t j) {
  int rc;
  if (b->masked && (rc = enqueue_relabel(b, parity, j, -1, [&](int i) { return b->active[i] != 0; })))
    return rc;
  if ((rc = enqueue_items(b, parity, b->d_items, b->nitems_a, b->d_items + b->nitems_a,
                          b->nitems - b->nitems_a)))
    return rc;
  if ((rc = enqueue_lone(b, parity, [&](int i) { return b->active[i] != 0; }))) return rc;
  if (b->masked && (rc = enqueue_bounce(b, parity, -1, [&](int i) { return b->active[i] != 0; }))) return rc;
  return LBM_OK;
}

int build_graph(lbm_batch* b, int start_parity) {
  cudaGraph_t g = nullptr;
  BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  const int64_t saved = b->launches;
  int rc = LBM_OK;
  for (int j = 0; j < b->K && rc == LBM_OK; ++j) rc = enqueue_step(b, start_parity ^ (j & 1), j);
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  b->graph_launches[start_parity] = b->launches - saved;
  b->launches = saved;  // counted again at every replay
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "stream capture: %s", cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&b->graph[start_parity], g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) return bfail(b, LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e2));
  return LBM_OK;
}

// The batch works on its own stream (the legacy default stream cannot be
// captured); events order it after earlier work on the boxes' stream and
// order later work there after it.
int enter(lbm_batch* b) {
  BCUDA(b, cudaEventRecord(b->ev_in, b->ext));
  BCUDA(b, cudaStreamWaitEvent(b->stream, b->ev_in, 0));
  return LBM_OK;
}

int leave(lbm_batch* b) {
  BCUDA(b, cudaEventRecord(b->ev_out, b->stream));
  BCUDA(b, cudaStreamWaitEvent(b->ext, b->ev_out, 0));
  return LBM_OK;
}

int active_count(const lbm_batch* b) {
  int c = 0;
  for (int i = 0; i < b->n; ++i) c += b->active[i] != 0;
  return c;
}

}  // namespace

extern "C" {

size_t lbm_batch_workspace_bytes(lbm_handle* const* handles, int32_t n) {
  if (!handles || n <= 0) return 0;
  for (int i = 0; i < n; ++i)
    if (!handles[i]) return 0;
  const int mi = max_items_for(handles, n);
  return align_up(sizeof(BatchInst) * (size_t)n) + align_up(sizeof(BatchItem) * (size_t)mi) + kAlign +
         align_up(sizeof(RelabelBox) * (size_t)n) + align_up(sizeof(RelabelEntry) * (2 * (size_t)n + 1)) +
         align_up(sizeof(RelabelEntry) * ((size_t)n + 1));
}

int lbm_batch_create(lbm_handle* const* handles, int32_t n, void* d_workspace, size_t bytes, lbm_batch** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!handles || n <= 0 || !d_workspace || ((uintptr_t)d_workspace % kAlign)) return LBM_EINVAL;
  if (bytes < lbm_batch_workspace_bytes(handles, n)) return LBM_ENOMEM;
  lbm_handle* h0 = handles[0];
  for (int i = 0; i < n; ++i) {
    lbm_handle* h = handles[i];
    for (int j = 0; j < i; ++j)
      if (handles[j] == h) return LBM_EINVAL;  // a box appears twice
    if (h->in_batch) return LBM_EINVAL;
    if (h->cfg.storage != h0->cfg.storage || h->cfg.barrier != h0->cfg.barrier) return LBM_EINVAL;
    if (h->cfg.barrier && h->cfg.relabel_every != h0->cfg.relabel_every) return LBM_EINVAL;
    if (h->cfg.stop_on_first_rupture || h->cfg.growth || h->cfg.components != 1) return LBM_ENOTSUP;
    if (h->device != h0->device || h->halted) return LBM_EINVAL;
  }
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ENOMEM;
  b->n = n;
  b->h.assign(handles, handles + n);
  b->active.assign(n, 1);
  b->base_cur.assign(n, 0);
  b->lone.assign(n, 0);
  b->unal.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const int nx = handles[i]->cfg.nx;
    b->unal[i] = !step_tma2_allowed(handles[i]->cfg.storage, nx) && step_tma2_unaligned_allowed(nx);
    b->lone[i] = !step_tma2_allowed(handles[i]->cfg.storage, nx) && !b->unal[i];
  }
  b->storage = h0->cfg.storage;
  b->masked = h0->cfg.barrier;
  // graph block: one relabel period with the barrier, else 16 steps
  b->K = h0->cfg.barrier ? h0->cfg.relabel_every : 16;
  b->t = h0->t;
  b->tau_one = 1;
  for (int i = 0; i < n; ++i) b->tau_one &= (float)handles[i]->cfg.tau == 1.0f;
  b->ext = h0->stream;
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    delete b;
    return LBM_ECUDA;
  }
  b->ws = static_cast<char*>(d_workspace);
  b->ws_bytes = bytes;
  b->max_items = max_items_for(handles, n);
  b->d_insts = reinterpret_cast<BatchInst*>(b->ws);
  b->d_items = reinterpret_cast<BatchItem*>(b->ws + align_up(sizeof(BatchInst) * (size_t)n));
  b->d_counter = reinterpret_cast<int*>(b->ws + align_up(sizeof(BatchInst) * (size_t)n) +
                                        align_up(sizeof(BatchItem) * (size_t)b->max_items));
  b->d_rboxes = reinterpret_cast<RelabelBox*>(reinterpret_cast<char*>(b->d_counter) + kAlign);
  b->d_rent = reinterpret_cast<RelabelEntry*>(reinterpret_cast<char*>(b->d_rboxes) +
                                              align_up(sizeof(RelabelBox) * (size_t)n));
  b->d_bent = reinterpret_cast<RelabelEntry*>(reinterpret_cast<char*>(b->d_rent) +
                                              align_up(sizeof(RelabelEntry) * (2 * (size_t)n + 1)));
  // default tiles: full-width strips, chunks giving ~4 items per resident CTA
  long long cells = 0;
  for (int i = 0; i < n; ++i) cells += (long long)handles[i]->cfg.nx * handles[i]->cfg.ny;
  const int res = batch_resident_ctas(b->storage, b->masked != 0, b->tau_one != 0);
  long long r = res > 0 ? cells / ((long long)512 * 4 * res) : 128;
  r = std::max(32LL, std::min(512LL, (r + 7) / 8 * 8));
  b->rows = (int)r;
  for (int i = 0; i < n; ++i) handles[i]->in_batch = 1;
  *out = b;
  return LBM_OK;
}

int lbm_batch_set_tiles(lbm_batch* b, int32_t strip_width, int32_t chunk_rows) {
  if (!b) return LBM_EINVAL;
  if (strip_width != 256 && strip_width != 512) return bfail(b, LBM_EINVAL, "strip width must be 256 or 512");
  if (chunk_rows < 8 || chunk_rows % 8) return bfail(b, LBM_EINVAL, "chunk rows must be a multiple of 8, >= 8");
  if (strip_width != b->strip || chunk_rows != b->rows) {
    b->strip = strip_width;
    b->rows = chunk_rows;
    b->dirty = 1;
  }
  return LBM_OK;
}

int lbm_batch_get_tiles(const lbm_batch* b, int32_t* strip_width, int32_t* chunk_rows) {
  if (!b) return LBM_EINVAL;
  if (strip_width) *strip_width = b->strip;
  if (chunk_rows) *chunk_rows = b->rows;
  return LBM_OK;
}

int lbm_batch_set_active(lbm_batch* b, int32_t index, int active) {
  if (!b) return LBM_EINVAL;
  if (index < 0 || index >= b->n) return bfail(b, LBM_EINVAL, "index out of range");
  const int a = active ? 1 : 0;
  if (b->active[index] != a) {
    b->active[index] = a;
    b->dirty = 1;
  }
  return LBM_OK;
}

int lbm_batch_step_one(lbm_batch* b, int32_t index, int64_t nsteps) {
  if (!b) return LBM_EINVAL;
  if (index < 0 || index >= b->n) return bfail(b, LBM_EINVAL, "index out of range");
  if (nsteps < 0) return bfail(b, LBM_EINVAL, "nsteps < 0");
  lbm_handle* h = b->h[index];
  // after the batch's earlier work, on the box's own stream; the batch's
  // later work after this (its next upload re-reads time and parity)
  BCUDA(b, cudaEventRecord(b->ev_out, b->stream));
  BCUDA(b, cudaStreamWaitEvent(h->stream, b->ev_out, 0));
  h->in_batch = 0;
  const int rc = lbm_step(h, nsteps);
  h->in_batch = 1;
  b->dirty = 1;
  drop_graphs(b);
  if (rc) return bfail(b, rc, "box %d: %s", index, h->err);
  BCUDA(b, cudaEventRecord(b->ev_in, h->stream));
  BCUDA(b, cudaStreamWaitEvent(b->stream, b->ev_in, 0));
  return LBM_OK;
}

int lbm_batch_use_graph(lbm_batch* b, int enable) {
  if (!b) return LBM_EINVAL;
  b->use_graph = enable ? 1 : 0;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps) {
  if (!b) return LBM_EINVAL;
  if (nsteps < 0) return bfail(b, LBM_EINVAL, "nsteps < 0");
  if (active_count(b) == 0 || nsteps == 0) return LBM_OK;
  int rc;
  if ((rc = enter(b))) return rc;
  rc = upload(b);
  if (rc) return rc;
  int64_t left = nsteps;
  // blocks start where the batch counter is a multiple of K; each box's
  // relabel offset to that counter is fixed while the membership is, so a
  // block's relabel schedule (captured in the graph) repeats; buffer parity
  // repeats after 2K steps (two graphs)
  while (left > 0 && b->use_graph && b->t % b->K != 0) {
    if ((rc = enqueue_step(b, b->par, 0))) return rc;
    advance(b, 1);
    --left;
  }
  while (b->use_graph && left >= b->K) {
    const int p = b->par;
    if (!b->graph[p] && (rc = build_graph(b, p))) return rc;
    BCUDA(b, cudaGraphLaunch(b->graph[p], b->stream));
    b->launches += b->graph_launches[p];
    advance(b, b->K);
    left -= b->K;
  }
  while (left > 0) {
    if ((rc = enqueue_step(b, b->par, 0))) return rc;
    advance(b, 1);
    --left;
  }
  return leave(b);
}

// Multi-rate steps: box i advances nsteps[i]. Boxes are laid out in the item
// list in descending order of their step counts, so the boxes still stepping
// at step j own a prefix of the items and step j is one launch over that
// prefix. Every box stepping at j has done exactly j steps of the call, so
// the common buffer parity j & 1 holds for all of them.
int lbm_batch_step_each(lbm_batch* b, const int64_t* nsteps, int32_t n) {
  if (!b) return LBM_EINVAL;
  if (!nsteps || n != b->n) return bfail(b, LBM_EINVAL, "need one step count per box (%d)", b->n);
  int64_t most = 0;
  for (int i = 0; i < n; ++i) {
    if (nsteps[i] < 0) return bfail(b, LBM_EINVAL, "box %d: nsteps < 0", i);
    if (nsteps[i] > 0 && !b->active[i]) return bfail(b, LBM_EINVAL, "box %d is switched off", i);
    most = std::max(most, nsteps[i]);
  }
  if (most == 0) return LBM_OK;
  int rc;
  if ((rc = enter(b))) return rc;
  std::vector<int> order;
  for (int i = 0; i < n; ++i)
    if (nsteps[i] > 0) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return nsteps[a] > nsteps[c]; });
  // item list and barrier groups in that order
  std::vector<int> keep = b->active;
  for (int i = 0; i < n; ++i) b->active[i] = nsteps[i] > 0;
  b->dirty = 1;
  rc = upload(b, order);
  b->active = keep;
  if (rc) return rc;
  // items of each kind (16-byte rows or not) in stepping order; the boxes
  // still stepping at step j own a prefix of each
  std::vector<BatchItem> sorted[2];
  std::vector<int> prefix[2];
  for (int kind = 0; kind < 2; ++kind) {
    prefix[kind].assign(order.size() + 1, 0);
    for (size_t k = 0; k < order.size(); ++k) {
      if ((b->unal[order[k]] != 0) == (kind == 1))
        for (const BatchItem& it : b->items)
          if (it.inst == order[k]) sorted[kind].push_back(it);
      prefix[kind][k + 1] = (int)sorted[kind].size();
    }
  }
  const size_t na_all = sorted[0].size();
  sorted[0].insert(sorted[0].end(), sorted[1].begin(), sorted[1].end());
  if (!sorted[0].empty())
    BCUDA(b, cudaMemcpyAsync(b->d_items, sorted[0].data(), sizeof(BatchItem) * sorted[0].size(),
                             cudaMemcpyHostToDevice, b->stream));
  std::map<int, int> glive;  // members of each barrier group still stepping
  for (const auto& kv : b->groups) glive[kv.first] = (int)kv.second.members.size();
  size_t live = order.size();
  for (int64_t j = 0; j < most; ++j) {
    while (live > 0 && nsteps[order[live - 1]] <= j) --live;
    const int parity = (int)(j & 1);
    if (b->masked) {
      const int key = (int)((b->t + j) % b->h[0]->cfg.relabel_every);
      int gl = 0;
      const auto it = b->groups.find(key);
      if (it != b->groups.end()) {
        const std::vector<int>& mem = it->second.members;
        int& c = glive[key];
        while (c > 0 && nsteps[mem[c - 1]] <= j) --c;
        gl = c;
      }
      if ((rc = enqueue_relabel(b, parity, j, gl, [&](int i) { return nsteps[i] > j; }))) return rc;
    }
    if ((rc = enqueue_items(b, parity, b->d_items, prefix[0][live], b->d_items + na_all, prefix[1][live])))
      return rc;
    if ((rc = enqueue_lone(b, parity, [&](int i) { return nsteps[i] > j; }))) return rc;
    if (b->masked && (rc = enqueue_bounce(b, parity, (int)live, [&](int i) { return nsteps[i] > j; }))) return rc;
  }
  for (int i = 0; i < n; ++i) {
    b->h[i]->t += nsteps[i];
    b->h[i]->cur ^= (int)(nsteps[i] & 1);
  }
  b->t += most;
  b->dirty = 1;  // the next lbm_batch_step re-uploads its own item list
  return leave(b);
}

int lbm_batch_tune(lbm_batch* b, int32_t trial_steps, float* best_ms_per_step) {
  if (!b) return LBM_EINVAL;
  if (trial_steps < 1) return bfail(b, LBM_EINVAL, "trial_steps must be >= 1");
  if (active_count(b) == 0) return bfail(b, LBM_EINVAL, "no active box");
  static const int strips[2] = {512, 256};
  static const int rowsc[5] = {32, 48, 64, 128, 256};  // 48: best for one large box
  const int use_graph = b->use_graph;
  b->use_graph = 0;
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  float best = 1e30f;
  int bs = b->strip, br = b->rows, rc = LBM_OK;
  for (int si = 0; si < 2 && rc == LBM_OK; ++si)
    for (int ri = 0; ri < 5 && rc == LBM_OK; ++ri) {
      if ((rc = lbm_batch_set_tiles(b, strips[si], rowsc[ri]))) break;
      if ((rc = lbm_batch_step(b, 1))) break;  // upload + warm-up
      cudaEventRecord(e0, b->stream);
      if ((rc = lbm_batch_step(b, trial_steps))) break;
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = bfail(b, LBM_ECUDA, "event synchronize failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= trial_steps;
      if (ms < best) {
        best = ms;
        bs = strips[si];
        br = rowsc[ri];
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->use_graph = use_graph;
  if (rc) return rc;
  if ((rc = lbm_batch_set_tiles(b, bs, br))) return rc;
  if (best_ms_per_step) *best_ms_per_step = best;
  return LBM_OK;
}

int lbm_batch_sync(lbm_batch* b) {
  if (!b) return LBM_EINVAL;
  BCUDA(b, cudaStreamSynchronize(b->stream));
  BCUDA(b, cudaStreamSynchronize(b->ext));
  for (int i = 0; i < b->n; ++i) {
    cudaStream_t hs = b->h[i]->stream;
    b->h[i]->stream = b->stream;
    const int rc = handle_check_flags(b->h[i]);
    b->h[i]->stream = hs;
    if (rc) return bfail(b, rc, "box %d: %s", i, b->h[i]->err);
  }
  return LBM_OK;
}

int64_t lbm_batch_steps_done(const lbm_batch* b) { return b ? b->t : -1; }

int64_t lbm_batch_kernel_launches(const lbm_batch* b) { return b ? b->launches : -1; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err : "batch is NULL"; }

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  cudaEventDestroy(b->ev_in);
  cudaEventDestroy(b->ev_out);
  cudaStreamDestroy(b->stream);
  for (lbm_handle* h : b->h) h->in_batch = 0;
  delete b;
}

}  // extern "C"
