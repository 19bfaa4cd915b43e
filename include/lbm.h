/*
 * lbm.h - C ABI of the GB300 (sm_103a) library for the time step of the
 * extended Shan-Chen lattice Boltzmann method for metal-foam bubbles
 * (Barzegari, Bayani, Mirbagheri & Shetabivash, arXiv 1708.01613).
 *
 * One handle advances one periodic D2Q9 box on one GPU. Per step it runs:
 * pull streaming (Sec. 2.1.1, Eq. 19), moments (Eq. 11), pseudopotential
 * psi = rho0 (1 - exp(-rho/rho0)) (Sec. 2.1.2, Eq. 30), the neighbour-sum
 * Shan-Chen force (Eq. 22) with the film-barrier mask, the velocity-shift
 * equilibrium u_eq = (j + tau F)/rho (Sec. 2.1.5, Eqs. 39-40; Eq. 14) and
 * BGK collision (Eq. 18). Every K steps it runs the film-barrier pipeline of
 * Sec. 2.1.5: gas labelling, nearest-bubble interaction zones, the
 * d2p/dn2 = 0 rupture test (Eq. 41) and the blocked-edge mask. The wall is
 * a barrier in both halves of the update: across a blocked edge the force
 * uses psi(x) in place of psi(x + e_i), and the population that would
 * stream across it is reflected back into its own cell in the opposite
 * direction (halfway bounce-back), so no mass crosses the wall and bubbles
 * on its two sides do not coalesce until the rupture test opens it.
 *
 * Conventions
 *  - Box: nx by ny cells, periodic on all sides, row-major, x fastest.
 *  - Directions: 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1)
 *    7:(-1,-1) 8:(1,-1); weights 4/9, 1/9 (1-4), 1/36 (5-8) (Eqs. 15-16).
 *  - Memory: the caller owns ALL device memory. lbm_create takes one
 *    caller-allocated device workspace of lbm_workspace_bytes() bytes
 *    (aligned to 256 bytes) and never allocates device memory itself. The
 *    handle owns only host state and must not outlive the workspace.
 *  - Streams: every call enqueues its work on the stream given to
 *    lbm_create (NULL = legacy default stream). lbm_step is asynchronous.
 *    lbm_read_fields, lbm_mass, lbm_bubble_stats, lbm_sync and a step with
 *    stop_on_first_rupture synchronise that stream.
 *  - Errors: every int-returning call returns an lbm_status; the library
 *    never aborts and never prints. lbm_last_error gives a message for the
 *    last failing call on that handle. A handle is not thread-safe.
 *  - Numeric faults (NaN/Inf or rho <= 0 met by the step kernel) are
 *    recorded on the device and reported as LBM_ENUMERIC by the next
 *    synchronising call.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,   /* bad config or argument */
  LBM_ENOMEM = 2,   /* workspace too small */
  LBM_ECUDA = 3,    /* a CUDA runtime call failed */
  LBM_ENUMERIC = 4, /* NaN/Inf or rho <= 0 seen on the device */
  LBM_ETIMEOUT = 5, /* a bounded device loop gave up */
  LBM_ENOTSUP = 6   /* unsupported request */
} lbm_status;

/* Population storage. F32: f_i as float. F16_DEV / BF16_DEV: the deviation
 * g_i = f_i - w_i rho_ref as IEEE half / bfloat16 (round to nearest even);
 * all arithmetic is FP32 in every mode. */
typedef enum { LBM_F32 = 0, LBM_F16_DEV = 1, LBM_BF16_DEV = 2 } lbm_storage;

/* Field selectors for lbm_read_fields / lbm_fields_bytes. Selected fields are
 * written back to back in increasing bit order, each as a full [ny][nx]
 * array (POPS: [9][ny][nx]). */
enum {
  LBM_FIELD_RHO = 1u << 0,   /* float32: rho = sum f_i (Eq. 11) */
  LBM_FIELD_UX = 1u << 1,    /* float32: (j_x + F_x / 2) / rho */
  LBM_FIELD_UY = 1u << 2,    /* float32: (j_y + F_y / 2) / rho */
  LBM_FIELD_P = 1u << 3,     /* float32: p = rho/3 + G psi^2 / 6 (Eq. 29) */
  LBM_FIELD_LABEL = 1u << 4, /* int32: bubble label (min row-major index) or -1 */
  LBM_FIELD_OWNER = 1u << 5, /* int32 (barrier on): label of the nearest bubble
                                within R_z; -1 none; -2 a wall cell, equidistant
                                from two or more bubbles */
  LBM_FIELD_MASK = 1u << 6,  /* uint8: bit i-1 set = edge (x, x+e_i) blocked:
                                owners of both ends differ, neither is -1,
                                neither end is open (symmetric) */
  LBM_FIELD_OPEN = 1u << 7,  /* uint8: 1 = cell has ruptured (barrier on) */
  LBM_FIELD_POPS = 1u << 8,  /* float32 [9][ny][nx] ([18][ny][nx] with two
                                components, melt then gas): incoming f_i of
                                the next step */
  LBM_FIELD_RHO_GAS = 1u << 9 /* float32: gas-component density (two
                                components; zeros otherwise) */
};

typedef struct {
  int32_t nx, ny;                /* box size, each >= 4 */
  int32_t storage;               /* lbm_storage */
  int32_t barrier;               /* 0: plain Shan-Chen; 1: film barrier + rupture */
  int32_t relabel_every;         /* K >= 1: barrier pipeline every K steps */
  int32_t zone_radius;           /* R_z >= 0; with the barrier on, nx, ny > 2 R_z + 1 */
  int32_t stop_on_first_rupture; /* 1: lbm_step stops after the step whose
                                    relabel first opened a cell (Sec. 2.1.4
                                    flowchart; Sec. 5 "best foaming time") */
  int32_t growth;                /* 1: reserve room (4 bytes per cell) for the
                                    growth source of lbm_set_growth; 0: none */
  double tau;                    /* BGK relaxation time > 0.5 */
  double G;                      /* Shan-Chen coupling (Eq. 22) */
  double rho0;                   /* psi scale, psi = rho0 (1 - exp(-rho/rho0)) */
  double rho_ref;                /* reference density of 16-bit deviations */
  double gas_threshold;          /* gas iff rho < this (default ln 2) */
  double rupture_eps;            /* open when |D2| <= eps; eps < 0: never */
  /* Two-component variant (Sec. 2.1.5, melt and gas lattices coupled every
   * step; Eqs. 36-40). components = 2 adds a gas lattice: tau, G above are
   * the melt's tau_m and self coupling G_mm; each component s feels
   * F_s = -psi_s(x) sum_s' G_ss' sum_i w_i psi_s'(x + e_i) e_i (barrier
   * substitution as for one component), the common velocity is
   * u' = (sum_s j_s / tau_s) / (sum_s rho_s / tau_s) and the equilibrium
   * velocity u' + tau_s F_s / rho_s. rho and the barrier act on the melt
   * density; P and the rupture test use the mixture pressure
   * (rho_m + rho_g)/3 + (G_mm psi_m^2 + 2 G_mg psi_m psi_g + G_gg psi_g^2)/6.
   * Two components need FP32 storage, growth = 0 and, with the barrier,
   * R_z <= 16; they cannot join a batch. */
  int32_t components;            /* 1 (default) or 2 */
  int32_t reserved2;             /* must be 0 */
  double tau_g;                  /* gas relaxation time > 0.5 */
  double G_mg;                   /* melt-gas coupling (symmetric) */
  double G_gg;                   /* gas self coupling */
} lbm_config;

typedef struct {
  double cx, cy, r; /* centre (cell units, cell x at coordinate x) and radius */
} lbm_bubble;

typedef struct {
  int64_t step;            /* steps done */
  int32_t n_bubbles;       /* gas components of the current density */
  int32_t reserved;
  int64_t n_open;          /* cells opened so far (barrier on) */
  double gas_fraction;     /* gas cells / all cells */
  double mean_eq_diameter; /* mean of 2 sqrt(A / pi) over bubbles */
  double mass;             /* FP64 sum of rho */
  int64_t n_merges;        /* coalescence events since the last init, counted
                              by every relabel (barrier on; 0 otherwise): the
                              components of a relabel's labelling that hold
                              gas cells of two or more components of the
                              previous relabel's (Sec. 4 merging runs, Sec. 5
                              statistics); a triple merge between two
                              relabels is one event */
} lbm_stats;

typedef struct lbm_handle lbm_handle;

/* Defaults: 256x256, F32, tau 1, G -5.5, rho0 1, rho_ref 1, barrier off,
 * K 1, R_z 4, gas threshold ln 2, eps 1e-6. */
void lbm_config_default(lbm_config* cfg);

/* Device bytes lbm_create needs for cfg (0 if cfg is invalid). */
size_t lbm_workspace_bytes(const lbm_config* cfg);

/* Validates cfg and binds the caller's device workspace (>= the size above,
 * 256-byte aligned) and CUDA stream (a cudaStream_t, may be NULL). The
 * current CUDA device must be the workspace's. On success *out is a new
 * handle; the populations are undefined until an init call. */
int lbm_create(const lbm_config* cfg, void* d_workspace, size_t bytes, void* cuda_stream,
               lbm_handle** out);

/* f_i = f_i^eq(rho, 0) = w_i rho from nx*ny FP64 densities (row-major),
 * read from host memory (src_is_device = 0) or device memory (1); with two
 * components, 2*nx*ny values: the melt densities, then the gas densities.
 * Resets the step counter, the rupture state and the error flags. */
int lbm_init_density(lbm_handle* h, const double* rho, int src_is_device);

/* Same as lbm_init_density with rho made on the device from n bubbles
 * (host array): each cell takes the bubble whose surface is nearest,
 * s = min_k (|x - c_k|_torus - r_k), and
 * rho = (rho_l + rho_g)/2 + (rho_l - rho_g)/2 tanh(s / (width / 2)),
 * computed in FP64. n = 0 gives a uniform liquid. One component only
 * (LBM_ENOTSUP with two). */
int lbm_init_bubbles(lbm_handle* h, const lbm_bubble* b, int32_t n, double rho_l, double rho_g,
                     double width);

/* Loads incoming populations f[9][ny][nx] ([18][ny][nx] with two
 * components, melt then gas; float32, host or device) as the state of the
 * next step (bitwise resume for F32 storage). */
int lbm_load_populations(lbm_handle* h, const float* f, int src_is_device);

/* Enqueues nsteps time steps (each: barrier pipeline when t % K == 0, then
 * the fused step). With stop_on_first_rupture it synchronises after each
 * relabel and stops after the step whose relabel opened the first cell;
 * lbm_steps_done tells how many steps ran. */
int lbm_step(lbm_handle* h, int64_t nsteps);

/* Kernels this handle has launched since lbm_create (host-side count). */
int64_t lbm_kernel_launches(const lbm_handle* h);

/* Selects the fused-step kernel: 0 = automatic, 1 = plain-load kernel (any
 * box), 2 = TMA-staged kernel with one cell per thread (nx % 16 == 0 and
 * nx >= 272), 3 = TMA-staged kernel with two cells per thread, one row
 * chunk per CTA (nx >= 16), 4 = the same with row chunks drawn by the
 * CTAs from a counter (nx >= 16). Variants 3 and 4 bulk-copy whole rows
 * when nx % 16 == 0, else each row's 16-byte-aligned interior, with the
 * unaligned head, tail and wrapped halo loaded plainly. Automatic picks 4
 * where the box allows (3 when the box has no more chunks than CTAs fit the
 * GPU), else 1. A variant the box does not allow returns LBM_ENOTSUP. All
 * variants compute the same operations in the same order and give bitwise
 * the same populations. The same handle must not be stepped by two streams
 * at once (variant 4 keeps its chunk counter in the handle's workspace). */
int lbm_set_step_variant(lbm_handle* h, int variant);

/* Steps done since the last init/load. */
int64_t lbm_steps_done(const lbm_handle* h);

/* 1 once a stop_on_first_rupture run has stopped, else 0. */
int lbm_halted(const lbm_handle* h);

/* Bytes lbm_read_fields writes for the selection `fields`. */
size_t lbm_fields_bytes(const lbm_handle* h, uint32_t fields);

/* Writes the selected fields of the current state to dst (host or device,
 * dst_bytes >= lbm_fields_bytes). LABEL is recomputed from the current
 * density; OWNER/MASK/OPEN are those of the last relabel. Synchronises. */
int lbm_read_fields(lbm_handle* h, uint32_t fields, void* dst, size_t dst_bytes,
                    int dst_is_device);

/* FP64 sum of rho over the box (of both components with two), reduced in
 * a fixed order. Synchronises. */
int lbm_mass(lbm_handle* h, double* out);

/* Nucleation (Sec. 2.1.3, "Random Nucleation" of the main flowchart):
 * every cell within torus distance r of a nucleus centre (cx, cy) becomes
 * gas at rest, its incoming populations set to w_i rho_g. The decision
 * dx^2 + dy^2 <= r^2 is taken in FP64 (dx, dy: torus distances along x and
 * y), like the oracle's. When and where nuclei appear is the caller's
 * choice (the paper draws them at random). nuclei: n host triples, read
 * before the call returns; n = 0 does nothing. LBM_EINVAL on non-finite
 * input or r < 0. Enqueued on the handle's stream. */
int lbm_nucleate(lbm_handle* h, const lbm_bubble* nuclei, int32_t n, double rho_g);

/* Bubble growth (Sec. 2.1.3, Eq. 34, dp/dt = A (dn/dt) / N): from the next
 * step on, every step releases `rate` of gas mass (lattice units; the
 * pressure increment taken on the ideal-gas part of the EOS, so rate =
 * 3 A dn/dt) until `budget` has been released (the last release is the
 * remainder). A release is split equally over the N gas points (rho <
 * gas_threshold) of the latest gas census, taken with the barrier pipeline
 * every K steps on the pre-collision density, and added at rest to the
 * post-collision populations: f_i^out(x) += w_i rate / N. No census exists
 * until the next step t with t % K == 0, so nothing is released before it.
 * Needs a handle created with config.growth = 1 (else LBM_EINVAL) and FP32
 * storage (LBM_ENOTSUP otherwise: a release split over many gas points adds
 * far less than half a unit in the last place of a 16-bit deviation, so it
 * would round away), rate and budget >= 0 and finite. Resets the released
 * total to 0; rate = 0 turns the source off. Not available to boxes in a
 * batch. */
int lbm_set_growth(lbm_handle* h, double rate, double budget);

/* Gas mass released so far by the growth source (FP64). Synchronises. */
int lbm_growth_released(lbm_handle* h, double* out);

/* Bubble statistics of the current density (labels recomputed) and, if
 * hist != NULL, a histogram of equivalent diameters on nbins logarithmic
 * bins over [dmin, dmax) (outliers clamped to the end bins). Synchronises. */
int lbm_bubble_stats(lbm_handle* h, lbm_stats* out, double* hist, int32_t nbins, double dmin,
                     double dmax);

/* Bubbles of the current density (labels recomputed, as in
 * lbm_bubble_stats; Sec. 5, Tab. 5 bubble sizes): *n_out = their number;
 * labels[k] (the smallest row-major index of bubble k) and areas[k] (its
 * cell count, as a double) in increasing label order, host arrays of
 * `capacity` entries. If the bubbles outnumber capacity, *n_out is still set
 * and LBM_EINVAL is returned (call again with room); capacity 0 only counts.
 * Uses the idle population buffer as scratch. Synchronises. */
int lbm_bubble_areas(lbm_handle* h, int32_t capacity, int32_t* labels, double* areas, int32_t* n_out);

/* Synchronises the stream and reports device-side faults. */
int lbm_sync(lbm_handle* h);

/* Message of the last failing call on h ("" if none). */
const char* lbm_last_error(const lbm_handle* h);

/* Frees the host handle (not the workspace). NULL is allowed. */
void lbm_destroy(lbm_handle* h);

/* ---------------------------------------------------------------------
 * Batches: many boxes advanced together. Not in the paper; it serves runs
 * of many independent foam simulations on one GPU. Every step of a batch is
 * one persistent launch of the two-cell staged kernel over a list of work
 * items (box, column strip, row chunk) of all active boxes with nx % 16 == 0,
 * one of its unaligned-row variant over the other boxes of at least 16
 * columns, and one plain-load step per narrower box,
 * preceded, when a relabel is due, by each box's barrier pipeline and
 * followed, with the barrier, by the bounce-back across blocked edges;
 * blocks of steps are captured as CUDA graphs and replayed. Each box evolves
 * bitwise as it would when stepped alone with lbm_step.
 *
 * Rules: all boxes share storage, barrier setting and relabel period, are
 * on one device, and do not stop on rupture. Boxes may be
 * at different step counts (each relabels when its own count is due). The batch works on a stream of its own (created by
 * lbm_batch_create; the legacy default stream cannot be captured into a
 * graph), ordered by events after earlier work on the first box's stream,
 * and later work on that stream is ordered after each lbm_batch_step. A box
 * in a batch may not be stepped with lbm_step. */
typedef struct lbm_batch lbm_batch;

/* Device bytes lbm_batch_create needs for these boxes (0 if invalid).
 * Boxes created with config.growth = 1 or stop_on_first_rupture = 1 cannot
 * join a batch (LBM_ENOTSUP). */
size_t lbm_batch_workspace_bytes(lbm_handle* const* handles, int32_t n);

/* Creates a batch over n handles with a caller-owned device workspace
 * (256-byte aligned). LBM_EINVAL / LBM_ENOTSUP / LBM_ENOMEM on rule or size
 * violations. */
int lbm_batch_create(lbm_handle* const* handles, int32_t n, void* d_workspace, size_t bytes, lbm_batch** out);

/* Work-item shape: strip width 256 or 512 columns, chunk height a multiple
 * of 8 rows. Changes invalidate the captured graphs. */
int lbm_batch_set_tiles(lbm_batch* b, int32_t strip_width, int32_t chunk_rows);
int lbm_batch_get_tiles(const lbm_batch* b, int32_t* strip_width, int32_t* chunk_rows);

/* Autotuner: times every (strip width, chunk height) candidate for
 * trial_steps steps on the batch itself and keeps the fastest. The boxes
 * advance by (trial_steps + 1) steps per candidate (10 candidates), as
 * ordinary steps (relabels included). */
int lbm_batch_tune(lbm_batch* b, int32_t trial_steps, float* best_ms_per_step);

/* 1 (default): replay captured graphs of whole relabel periods; 0: launch
 * step by step. Results are identical. */
int lbm_batch_use_graph(lbm_batch* b, int enable);

/* Excludes (0) or re-includes (1) box `index` from the steps that follow. */
int lbm_batch_set_active(lbm_batch* b, int32_t index, int active);

/* Enqueues nsteps steps of every active box (asynchronous). */
int lbm_batch_step(lbm_batch* b, int64_t nsteps);

/* Multi-rate steps: box i advances nsteps[i] steps (n = the batch's box
 * count; 0 = sits out; a switched-off box must get 0). Step j of the call is
 * one persistent launch over the boxes with nsteps[i] > j, so small boxes
 * can take many steps while large ones take few, as a server sharing the
 * GPU between requests wants. Relabels follow each box's own count. No
 * graphs are used; asynchronous, like lbm_batch_step. The batch's step
 * counter advances by the largest nsteps[i]. */
int lbm_batch_step_each(lbm_batch* b, const int64_t* nsteps, int32_t n);

/* Advances box `index` alone by nsteps steps through the single-box path
 * (lbm_step: its own kernels and relabels, no batch launches), ordered after
 * the batch's earlier work, with the batch's later work ordered after it; the
 * batch re-reads the box's time and buffer parity at its next step call, and
 * drops its captured graphs. For a server step in which one box of the batch
 * moves. Errors: LBM_EINVAL (index out of range, nsteps < 0), or the box's
 * own step error. Asynchronous. */
int lbm_batch_step_one(lbm_batch* b, int32_t index, int64_t nsteps);

/* Synchronises the batch stream and reports device faults of any box. */
int lbm_batch_sync(lbm_batch* b);

int64_t lbm_batch_steps_done(const lbm_batch* b);
int64_t lbm_batch_kernel_launches(const lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);

/* Frees the batch (not the workspace); the boxes can be stepped alone again. */
void lbm_batch_destroy(lbm_batch* b);

/* Allocation-free FP64 mass (sum of all populations) of a caller-held
 * population buffer: d_pops holds 9 * nx * ny values of `storage` (FP32
 * values, or 16-bit deviations from w_i rho_ref), in any cell order. The
 * paper has no counterpart: this entry point exists for callers that may not
 * allocate device memory of their own (their device memory belongs to
 * another allocator or pool, or cudaMalloc's implicit synchronisation is not
 * acceptable) and so cannot supply the workspace lbm_create needs.
 * It allocates nothing and needs no handle: the reduction's scratch is a
 * fixed 32 KiB file-scope __device__ array kept by every GPU that loads the
 * library until exit. Limit: nx * ny <= 2^28 cells; larger boxes return
 * LBM_EINVAL. The result is written to d_out (one double of device memory)
 * asynchronously on cuda_stream (NULL = legacy default stream).
 * The first call on a device, with that device current, looks up the
 * scratch's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture. All calls share the scratch: calls whose work
 * overlaps on the GPU race and may return wrong sums; order them on one
 * stream. Each call writes every scratch slot it reads, so no clearing is
 * needed. err (may be NULL) receives a message of at most err_len bytes. */
int lbm_mass_noalloc(const void* d_pops, int32_t nx, int32_t ny, int32_t storage, double rho_ref,
                     void* cuda_stream, double* d_out, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
