/*
 * Plain FP64 CPU oracle of one time step of the extended Shan-Chen lattice
 * Boltzmann method for metal-foam bubbles (Barzegari, Bayani, Mirbagheri &
 * Shetabivash, arXiv 1708.01613).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product path (the
 * CUDA library and its Python binding) never calls it, and this file shares
 * no source, header, table or helper with the CUDA path.
 *
 * Everything is FP64, written as the plain definition: one loop nest per
 * equation, no blocking, no fusion. Loops over rows run under OpenMP; every
 * cell is computed independently, so results do not depend on the thread
 * count.
 *
 * Paper passages followed (section / equation numbers of arXiv 1708.01613):
 *   moments                 Sec. 2.1.1, Eq. 11
 *   equilibrium             Sec. 2.1.1, Eq. 14
 *   D2Q9 velocities/weights Sec. 2.1.1, Eqs. 15-16
 *   BGK collision           Sec. 2.1.1, Eq. 18 (Eq. 12 is the same update
 *                           with the "- f_i" lost; Eq. 18 is used)
 *   streaming               Sec. 2.1.1, Eq. 19
 *   Shan-Chen force         Sec. 2.1.2, Eq. 22
 *   equation of state       Sec. 2.1.2, Eq. 29 (Eq. 33 drops the square)
 *   pseudopotential         Sec. 2.1.2, Eq. 30, psi = rho0 (1 - exp(-rho/rho0))
 *   velocity shift          Sec. 2.1.5, Eqs. 39-40: u = u_total + tau * F
 *                           (F per unit density here)
 *   nearest-bubble rule     Sec. 2.1.5 (interaction zones, nearest bubble,
 *                           Eq. 38 selection of one bubble's potential)
 *   barrier wall            Sec. 2.1.5, modified Shan-Chen flowchart
 *                           ("locate oxide network barrier wall ... on equal
 *                           velocity cells of each bubble interact domain",
 *                           "neglect effect from other side of barrier
 *                           wall") and the text after it: while the wall
 *                           stands the bubbles never cross it and no
 *                           coalescence occurs
 *   rupture criterion       Sec. 2.1.5, Eq. 41 (eta_m = 0 when d2p/dn2 = 0)
 *   run termination         Sec. 2.1.4 main flowchart and Sec. 5 (the foam
 *                           run ends when the first cell reaches rupture)
 *   bubble statistics       Sec. 5, Tab. 5 (counts, sizes) and the merging
 *                           runs of Sec. 4: areas, equivalent diameters and
 *                           coalescence events between relabels
 *   nucleation and growth   Sec. 2.1.3 (gas nuclei at random sites; every
 *                           step the released gas is added to the gas
 *                           points, dp/dt = A (dn/dt) / N, Eq. 34) and the
 *                           main flowchart's "Random Nucleation" and
 *                           "Bubble growth" boxes
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - direction order 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1)
 *     6:(-1,1) 7:(-1,-1) 8:(1,-1);
 *   - periodic box on all sides (the paper's "mirror" boundary, which it
 *     defines as re-entering at the opposite wall);
 *   - gas cell: rho < gas_threshold (default ln 2, the critical density of
 *     Sec. 2.1.2); bubbles are 4-connected gas components on the torus,
 *     labelled by the smallest row-major index in the component;
 *   - owner of a liquid cell: the bubble of the nearest gas cell within the
 *     zone radius R_z; none (-1) beyond R_z; a cell whose nearest gas cells
 *     belong to two or more bubbles at the same distance is a wall cell
 *     (owner -2): the wall sits on the cells equidistant from the bubbles,
 *     so it lies on a film's symmetry plane;
 *   - a blocked edge (x, x+e_i) has owners that differ, both defined (not
 *     -1; a wall cell's -2 counts as defined), and neither end opened. The
 *     other side of the wall is neglected in both halves of the update:
 *     across a blocked edge the force uses psi(x) in place of psi(x+e_i),
 *     and the population f_i^out(x) that would stream across the edge is
 *     reflected back into x as f_opp(i) (halfway bounce-back), so no mass
 *     crosses the wall;
 *   - "d2p/dn2 = 0": at a cell with a differing-owner neighbour, n is the
 *     first such lattice direction; D2 = p(x+n) - 2 p(x) + p(x-n); the cell
 *     opens (for good) when |D2| <= eps or the sign of D2 differs from the
 *     sign stored at the previous relabel; eps < 0 disables rupture;
 *   - the barrier pipeline runs on the pre-collision density at the start of
 *     every step t with t % K == 0 and the mask is held for K steps;
 *   - reported velocity u = (j + F/2) / rho; reported pressure p of Eq. 29;
 *   - growth: the pressure increment of a gas point is taken on the ideal-gas
 *     part of the equation of state, dp = c_s^2 drho with c_s^2 = 1/3, so the
 *     released gas is a density source. Each step releases growth_rate
 *     (= 3 A dn/dt in lattice units) until growth_budget is used up (the
 *     last release is the remainder); it is split equally over the N gas
 *     points (rho < gas_threshold) of the latest census, which is taken with
 *     the barrier pipeline, every K steps, on the pre-collision density, and
 *     added at rest after the collision: f_i^out(x) += w_i drho (no momentum);
 *   - nucleation: a nucleus (cx, cy, r) turns the cells within torus distance
 *     r of its centre into gas at rest: incoming f_i = w_i rho_g. When and
 *     where nuclei appear is an input (the paper's random subroutine draws
 *     them; here the seeded input generator does).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
#define OWNER_NONE (-1) /* no bubble within the zone radius */
#define OWNER_WALL (-2) /* equidistant from two or more bubbles */

static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                             1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* opposite direction: e_OPP[i] = -e_i */
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

typedef struct {
  int32_t nx, ny;
  int32_t barrier;          /* 0: plain Shan-Chen; 1: film barrier + rupture */
  int32_t relabel_every;    /* K >= 1 */
  int32_t zone_radius;      /* R_z */
  int32_t stop_on_first_rupture;
  double tau, G, rho0;
  double gas_threshold;     /* rho below this is gas */
  double rupture_eps;       /* eps for |D2| <= eps; < 0 disables rupture */
  double growth_rate;       /* gas mass released per step (0: no growth) */
  double growth_budget;     /* total gas mass of the blowing agent */
} orc_params;

typedef struct {
  double *f;       /* [9][ny][nx] incoming populations at the start of step t */
  double *f_next;  /* [9][ny][nx] scratch */
  double *rho, *jx, *jy, *psi, *Fx, *Fy; /* [ny][nx] scratch */
  int32_t *label;  /* [ny][nx] bubble label or -1 */
  int32_t *owner;  /* [ny][nx] owning bubble or -1 */
  int8_t *sgn;     /* [ny][nx] sign of D2 at the last relabel (0: none) */
  uint8_t *open;   /* [ny][nx] 1 once the cell has ruptured */
  uint8_t *mask;   /* [ny][nx] bit i-1: edge (x, x+e_i) blocked */
  int64_t t;               /* steps done */
  int64_t opened_total;    /* cells opened so far */
  int32_t opened_last;     /* cells opened at the latest relabel */
  int32_t halted;          /* 1 after the first rupture if stopping on it */
  uint8_t *gas;            /* [ny][nx] gas points of the latest census */
  int64_t n_gas;           /* their number */
  double injected;         /* gas mass released so far */
  int64_t merges_total;    /* coalescence events over all relabels so far */
} orc_state;

static inline int wrap(int a, int n) {
  a %= n;
  return a < 0 ? a + n : a;
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_lattice(int32_t *ex, int32_t *ey, double *w) {
  for (int i = 0; i < Q; ++i) {
    ex[i] = EX[i];
    ey[i] = EY[i];
    w[i] = WT[i];
  }
}

/* Eq. 30 with the scale rho0. */
double orc_psi(double rho, double rho0) { return rho0 * (1.0 - exp(-rho / rho0)); }

/* Eq. 29 with c_s^2 = 1/3. */
double orc_pressure(double rho, double G, double rho0) {
  double s = orc_psi(rho, rho0);
  return rho / 3.0 + G * s * s / 6.0;
}

/* Eq. 14 with c_s^2 = 1/3. */
void orc_equilibrium(double rho, double ux, double uy, double *feq) {
  double uu = ux * ux + uy * uy;
  for (int i = 0; i < Q; ++i) {
    double eu = EX[i] * ux + EY[i] * uy;
    feq[i] = WT[i] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
  }
}

/* Eq. 11: rho = sum f_i, j = sum e_i f_i. */
void orc_moments(const orc_params *p, const double *f, double *rho, double *jx, double *jy) {
  const int nx = p->nx, ny = p->ny;
  const size_t N = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      double r = 0.0, a = 0.0, b = 0.0;
      for (int i = 0; i < Q; ++i) {
        double fi = f[i * N + c];
        r += fi;
        a += EX[i] * fi;
        b += EY[i] * fi;
      }
      rho[c] = r;
      if (jx) jx[c] = a;
      if (jy) jy[c] = b;
    }
}

/* Eq. 22: F(x) = -G psi(x) sum_{i=1..8} w_i psi~_i e_i, where psi~_i is
 * psi(x+e_i), or psi(x) if the edge (x, x+e_i) is blocked (mask may be NULL). */
void orc_force(const orc_params *p, const double *psi, const uint8_t *mask, double *Fx,
               double *Fy) {
  const int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      double sx = 0.0, sy = 0.0;
      for (int i = 1; i < Q; ++i) {
        size_t nb = (size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
        double s = psi[nb];
        if (mask && ((mask[c] >> (i - 1)) & 1u)) s = psi[c];
        sx += WT[i] * s * EX[i];
        sy += WT[i] * s * EY[i];
      }
      Fx[c] = -p->G * psi[c] * sx;
      Fy[c] = -p->G * psi[c] * sy;
    }
}

/* Gas cells (rho < threshold) grouped into 4-connected components on the
 * torus. Cells are visited in row-major order and each unvisited gas cell
 * starts a breadth-first search that gives its whole component its own index,
 * which is therefore the smallest index in the component. Liquid: -1. */
void orc_label(const orc_params *p, const double *rho, int32_t *label) {
  const int nx = p->nx, ny = p->ny;
  const size_t N = (size_t)nx * ny;
  int32_t *queue = (int32_t *)malloc(N * sizeof(int32_t));
  for (size_t c = 0; c < N; ++c) label[c] = -1;
  for (size_t c0 = 0; c0 < N; ++c0) {
    if (!(rho[c0] < p->gas_threshold) || label[c0] >= 0) continue;
    size_t head = 0, tail = 0;
    label[c0] = (int32_t)c0;
    queue[tail++] = (int32_t)c0;
    while (head < tail) {
      int32_t c = queue[head++];
      int x = c % nx, y = c / nx;
      for (int i = 1; i <= 4; ++i) {
        size_t nb = (size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
        if (rho[nb] < p->gas_threshold && label[nb] < 0) {
          label[nb] = (int32_t)c0;
          queue[tail++] = (int32_t)nb;
        }
      }
    }
  }
  free(queue);
}

/* Interaction zones (Sec. 2.1.5): a gas cell belongs to its own bubble; a
 * liquid cell belongs to the bubble of the gas cell g nearest to it (|x-g|^2
 * on the torus) among gas cells with |x-g|^2 <= R_z^2; none (-1) if there is
 * no such cell; a wall cell (OWNER_WALL) if gas cells of two or more bubbles
 * are nearest at the same distance (the flowchart places the barrier wall on
 * the cells where the bubbles' domains are equal). Exhaustive search of the
 * window. */
void orc_owner(const orc_params *p, const int32_t *label, int32_t *owner) {
  const int nx = p->nx, ny = p->ny, R = p->zone_radius;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      if (label[c] >= 0) {
        owner[c] = label[c];
        continue;
      }
      int best_d2 = -1;
      int32_t best = -1;
      int tie = 0; /* another bubble at the best distance */
      for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
          int d2 = dx * dx + dy * dy;
          if (d2 > R * R) continue;
          int32_t l = label[(size_t)wrap(y + dy, ny) * nx + wrap(x + dx, nx)];
          if (l < 0) continue;
          if (best < 0 || d2 < best_d2) {
            best_d2 = d2;
            best = l;
            tie = 0;
          } else if (d2 == best_d2 && l != best) {
            tie = 1;
          }
        }
      owner[c] = tie ? OWNER_WALL : best;
    }
}

/* First lattice direction i (1..8) across which the owner changes between two
 * defined owners (a wall cell's owner counts as defined), or 0 if x is not on
 * a barrier. */
static int barrier_direction(const orc_params *p, const int32_t *owner, int x, int y) {
  const int nx = p->nx, ny = p->ny;
  int32_t o = owner[(size_t)y * nx + x];
  if (o == OWNER_NONE) return 0;
  for (int i = 1; i < Q; ++i) {
    int32_t on = owner[(size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx)];
    if (on != OWNER_NONE && on != o) return i;
  }
  return 0;
}

/* Rupture test of Eq. 41 under the reading given in the header, on a
 * pressure field pr. */
static void rupture_on_pressure(const orc_params *p, const double *pr, const int32_t *owner, int8_t *sgn,
                                uint8_t *open, int32_t *n_opened) {
  const int nx = p->nx, ny = p->ny;
  int32_t opened = 0;
#pragma omp parallel for schedule(static) reduction(+ : opened)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      int i = barrier_direction(p, owner, x, y);
      if (i == 0) {
        sgn[c] = 0;
        continue;
      }
      size_t cp = (size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
      size_t cm = (size_t)wrap(y - EY[i], ny) * nx + wrap(x - EX[i], nx);
      double d2 = pr[cp] - 2.0 * pr[c] + pr[cm];
      int s = (d2 > 0.0) - (d2 < 0.0);
      if (p->rupture_eps >= 0.0 && !open[c]) {
        if (fabs(d2) <= p->rupture_eps || (sgn[c] != 0 && s != sgn[c])) {
          open[c] = 1;
          opened += 1;
        }
      }
      sgn[c] = (int8_t)s;
    }
  *n_opened = opened;
}

/* Rupture test with the pressure of Eq. 29 from the density rho. */
void orc_rupture(const orc_params *p, const double *rho, const int32_t *owner, int8_t *sgn,
                 uint8_t *open, int32_t *n_opened) {
  const size_t N = (size_t)p->nx * p->ny;
  double *pr = (double *)malloc(N * sizeof(double));
  for (size_t c = 0; c < N; ++c) pr[c] = orc_pressure(rho[c], p->G, p->rho0);
  rupture_on_pressure(p, pr, owner, sgn, open, n_opened);
  free(pr);
}

/* Blocked-edge mask: bit i-1 of mask(x) is set when owner(x) and owner(x+e_i)
 * are both defined (not OWNER_NONE) and differ, and neither cell is open. The
 * relation is symmetric: bit i-1 of mask(x) equals bit OPP[i]-1 of
 * mask(x+e_i). */
void orc_mask(const orc_params *p, const int32_t *owner, const uint8_t *open, uint8_t *mask) {
  const int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      uint8_t m = 0;
      for (int i = 1; i < Q; ++i) {
        size_t nb = (size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
        if (owner[c] != OWNER_NONE && owner[nb] != OWNER_NONE && owner[c] != owner[nb] && !open[c] &&
            !open[nb])
          m |= (uint8_t)(1u << (i - 1));
      }
      mask[c] = m;
    }
}

/* Coalescence events between two labellings of the same box (bubble
 * statistics, Sec. 5 and the merging runs of Sec. 4): the number of
 * components of `now` that hold gas cells of two or more components of
 * `before`. A bubble that grows, shrinks, moves or splits is no event; a
 * triple merge within the interval is one event. Cells that are gas in only
 * one of the two labellings do not link components. */
int32_t orc_merges(const orc_params *p, const int32_t *before, const int32_t *now) {
  const size_t N = (size_t)p->nx * p->ny;
  /* first[r]: an old label seen in new component r (-1: none yet);
     merged[r]: component r already counted */
  int32_t *first = (int32_t *)malloc(N * sizeof(int32_t));
  uint8_t *merged = (uint8_t *)calloc(N, 1);
  for (size_t c = 0; c < N; ++c) first[c] = -1;
  int32_t events = 0;
  for (size_t c = 0; c < N; ++c) {
    const int32_t r = now[c], o = before[c];
    if (r < 0 || o < 0) continue;
    if (first[r] < 0) {
      first[r] = o;
    } else if (first[r] != o && !merged[r]) {
      merged[r] = 1;
      events += 1;
    }
  }
  free(first);
  free(merged);
  return events;
}

/* The barrier pipeline on the populations of the current step. */
void orc_relabel(const orc_params *p, orc_state *s) {
  const size_t N = (size_t)p->nx * p->ny;
  int32_t *before = (int32_t *)malloc(N * sizeof(int32_t));
  memcpy(before, s->label, N * sizeof(int32_t));
  orc_moments(p, s->f, s->rho, NULL, NULL);
  orc_label(p, s->rho, s->label);
  s->merges_total += orc_merges(p, before, s->label);
  free(before);
  orc_owner(p, s->label, s->owner);
  int32_t opened = 0;
  orc_rupture(p, s->rho, s->owner, s->sgn, s->open, &opened);
  orc_mask(p, s->owner, s->open, s->mask);
  s->opened_last = opened;
  s->opened_total += opened;
}

/* Gas points of the current populations: gas[c] = rho < gas_threshold, and
 * their number (the N of dp/dt = A (dn/dt) / N). */
void orc_gas_census(const orc_params *p, orc_state *s) {
  const size_t N = (size_t)p->nx * p->ny;
  orc_moments(p, s->f, s->rho, NULL, NULL);
  int64_t n = 0;
  for (size_t c = 0; c < N; ++c) {
    s->gas[c] = s->rho[c] < p->gas_threshold;
    n += s->gas[c];
  }
  s->n_gas = n;
}

/* Nucleation: every cell within torus distance r of a nucleus centre becomes
 * gas at rest, incoming f_i = w_i rho_g. nuclei: n triples (cx, cy, r). */
void orc_nucleate(const orc_params *p, orc_state *s, const double *nuclei, int32_t n, double rho_g) {
  const int nx = p->nx, ny = p->ny;
  const size_t N = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      int inside = 0;
      for (int32_t k = 0; k < n && !inside; ++k) {
        double dx = fabs((double)x - nuclei[3 * k + 0]);
        double dy = fabs((double)y - nuclei[3 * k + 1]);
        dx = fmin(dx, nx - dx);
        dy = fmin(dy, ny - dy);
        const double r = nuclei[3 * k + 2];
        inside = dx * dx + dy * dy <= r * r;
      }
      if (inside)
        for (int i = 0; i < Q; ++i) s->f[i * N + (size_t)y * nx + x] = WT[i] * rho_g;
    }
}

/* f_i = f_i^eq(rho, 0) = w_i rho, open/sign state cleared, t = 0. */
void orc_init_state(const orc_params *p, orc_state *s, const double *rho_init) {
  const size_t N = (size_t)p->nx * p->ny;
  for (int i = 0; i < Q; ++i)
    for (size_t c = 0; c < N; ++c) s->f[i * N + c] = WT[i] * rho_init[c];
  memset(s->sgn, 0, N);
  memset(s->open, 0, N);
  memset(s->mask, 0, N);
  for (size_t c = 0; c < N; ++c) s->label[c] = s->owner[c] = -1;
  s->t = 0;
  s->opened_total = 0;
  s->opened_last = 0;
  s->halted = 0;
  if (s->gas) memset(s->gas, 0, N);
  s->n_gas = 0;
  s->injected = 0.0;
  s->merges_total = 0;
}

/* One time step: barrier pipeline when due, then moments (Eq. 11),
 * pseudopotential (Eq. 30), force (Eq. 22, masked), velocity shift
 * (Eqs. 39-40), equilibrium (Eq. 14), BGK collision (Eq. 18) and streaming
 * (Eq. 19; across a blocked edge the population bounces back into its own
 * cell in the opposite direction). Returns 1 if the run is halted, else 0. */
int orc_step(const orc_params *p, orc_state *s) {
  const int nx = p->nx, ny = p->ny;
  const size_t N = (size_t)nx * ny;
  if (s->halted) return 1;
  int barrier = p->barrier != 0;
  const int growth = p->growth_rate > 0.0;
  if (s->t % p->relabel_every == 0) {
    if (barrier) orc_relabel(p, s);
    if (growth) orc_gas_census(p, s);
  }
  /* gas released this step, split over the gas points of the census */
  double drho = 0.0;
  if (growth && s->n_gas > 0) {
    double release = p->growth_rate;
    const double left = p->growth_budget - s->injected;
    if (release > left) release = left;
    if (release > 0.0) {
      drho = release / (double)s->n_gas;
      s->injected += release;
    }
  }
  orc_moments(p, s->f, s->rho, s->jx, s->jy);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      s->psi[c] = orc_psi(s->rho[c], p->rho0);
    }
  orc_force(p, s->psi, barrier ? s->mask : NULL, s->Fx, s->Fy);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t c = (size_t)y * nx + x;
      double r = s->rho[c];
      double ux = (s->jx[c] + p->tau * s->Fx[c]) / r;
      double uy = (s->jy[c] + p->tau * s->Fy[c]) / r;
      double feq[Q];
      orc_equilibrium(r, ux, uy, feq);
      const int source = drho > 0.0 && s->gas[c];
      for (int i = 0; i < Q; ++i) {
        double fi = s->f[i * N + c];
        double fout = fi - (fi - feq[i]) / p->tau;
        if (source) fout += WT[i] * drho;
        if (barrier && i > 0 && ((s->mask[c] >> (i - 1)) & 1u)) {
          /* the edge to x+e_i is blocked: bounce back into x */
          s->f_next[OPP[i] * N + c] = fout;
        } else {
          size_t dst = (size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
          s->f_next[i * N + dst] = fout;
        }
      }
    }
  memcpy(s->f, s->f_next, Q * N * sizeof(double));
  s->t += 1;
  if (barrier && p->stop_on_first_rupture && s->opened_total > 0) s->halted = 1;
  return s->halted;
}

/* Up to nsteps steps; returns the number of steps done. */
int64_t orc_run(const orc_params *p, orc_state *s, int64_t nsteps) {
  int64_t done = 0;
  while (done < nsteps && !s->halted) {
    orc_step(p, s);
    done += 1;
  }
  return done;
}

/* Diagnostics at the start of the current step (the mask last computed is
 * used for the force): rho, u = (j + F/2)/rho, and p of Eq. 29. Any output
 * pointer may be NULL. */
void orc_fields(const orc_params *p, orc_state *s, double *rho, double *ux, double *uy,
                double *pr) {
  const int nx = p->nx, ny = p->ny;
  orc_moments(p, s->f, s->rho, s->jx, s->jy);
  for (size_t c = 0; c < (size_t)nx * ny; ++c) s->psi[c] = orc_psi(s->rho[c], p->rho0);
  orc_force(p, s->psi, p->barrier ? s->mask : NULL, s->Fx, s->Fy);
  for (size_t c = 0; c < (size_t)nx * ny; ++c) {
    double r = s->rho[c];
    if (rho) rho[c] = r;
    if (ux) ux[c] = (s->jx[c] + 0.5 * s->Fx[c]) / r;
    if (uy) uy[c] = (s->jy[c] + 0.5 * s->Fy[c]) / r;
    if (pr) pr[c] = orc_pressure(r, p->G, p->rho0);
  }
}

/* One step of the update evaluated only at the listed cells: given the
 * incoming populations f of a whole box and a blocked-edge mask (may be NULL),
 * writes the incoming populations of the next step at cells[k] into
 * out[k*9 + i]. Each output is computed from its 5x5 neighbourhood with the
 * same equations as orc_step, bounce-back across blocked edges included. */
void orc_step_cells(const orc_params *p, const double *f, const uint8_t *mask,
                    const int64_t *cells, int64_t ncells, double *out) {
  const int nx = p->nx, ny = p->ny;
  const size_t N = (size_t)nx * ny;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t k = 0; k < ncells; ++k) {
    int64_t c = cells[k];
    int x = (int)(c % nx), y = (int)(c / nx);
    for (int i = 0; i < Q; ++i) {
      /* the population i arriving at x left the source cell x - e_i in
         direction i, or, if the edge (x, x - e_i) is blocked, left x itself
         in direction OPP[i] and bounced back */
      int sx = wrap(x - EX[i], nx), sy = wrap(y - EY[i], ny), d = i;
      if (mask && i > 0 && ((mask[(size_t)y * nx + x] >> (OPP[i] - 1)) & 1u)) {
        sx = x;
        sy = y;
        d = OPP[i];
      }
      size_t sc = (size_t)sy * nx + sx;
      double rho_s = 0.0, jx = 0.0, jy = 0.0;
      for (int q = 0; q < Q; ++q) {
        rho_s += f[q * N + sc];
        jx += EX[q] * f[q * N + sc];
        jy += EY[q] * f[q * N + sc];
      }
      double psi_s = orc_psi(rho_s, p->rho0);
      double sxs = 0.0, sys = 0.0;
      for (int q = 1; q < Q; ++q) {
        size_t nb = (size_t)wrap(sy + EY[q], ny) * nx + wrap(sx + EX[q], nx);
        double rn = 0.0;
        for (int r = 0; r < Q; ++r) rn += f[r * N + nb];
        double s = orc_psi(rn, p->rho0);
        if (mask && ((mask[sc] >> (q - 1)) & 1u)) s = psi_s;
        sxs += WT[q] * s * EX[q];
        sys += WT[q] * s * EY[q];
      }
      double Fx = -p->G * psi_s * sxs, Fy = -p->G * psi_s * sys;
      double ux = (jx + p->tau * Fx) / rho_s, uy = (jy + p->tau * Fy) / rho_s;
      double feq[Q];
      orc_equilibrium(rho_s, ux, uy, feq);
      double fi = f[d * N + sc];
      out[k * Q + i] = fi - (fi - feq[d]) / p->tau;
    }
  }
}

/* Initial density of round bubbles with a tanh interface: each cell takes
 * the bubble whose surface is nearest, s = min_k (d_k - r_k) with d_k the
 * torus distance from the cell centre to bubble k's centre, and
 * rho = (rho_l + rho_g)/2 + (rho_l - rho_g)/2 * tanh(s / (width / 2)).
 * With no bubbles the box is liquid. bubbles: n triples (cx, cy, r). */
void orc_init_bubbles(const orc_params *p, const double *bubbles, int32_t n, double rho_l,
                      double rho_g, double width, double *rho) {
  const int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      double best = INFINITY;
      for (int32_t k = 0; k < n; ++k) {
        double dx = fabs((double)x - bubbles[3 * k + 0]);
        double dy = fabs((double)y - bubbles[3 * k + 1]);
        dx = fmin(dx, nx - dx);
        dy = fmin(dy, ny - dy);
        double s = sqrt(dx * dx + dy * dy) - bubbles[3 * k + 2];
        if (s < best) best = s;
      }
      double v = (n > 0) ? tanh(best / (0.5 * width)) : 1.0;
      rho[(size_t)y * nx + x] = 0.5 * (rho_l + rho_g) + 0.5 * (rho_l - rho_g) * v;
    }
}

/* Bubble statistics from a label array: number of bubbles, gas fraction,
 * areas (cells) and equivalent diameters 2 sqrt(A/pi) of each bubble in
 * order of their labels, and a histogram of the diameters on nbins
 * logarithmic bins between dmin and dmax (values outside are clamped into the
 * end bins). areas/diam may be NULL; they need room for the bubble count.
 * Returns the number of bubbles. */
int32_t orc_stats(const orc_params *p, const int32_t *label, double *gas_fraction,
                  double *mean_diameter, double *areas, double *diam, double *hist,
                  int32_t nbins, double dmin, double dmax) {
  const size_t N = (size_t)p->nx * p->ny;
  int64_t *count = (int64_t *)calloc(N, sizeof(int64_t));
  int64_t gas = 0;
  for (size_t c = 0; c < N; ++c)
    if (label[c] >= 0) {
      count[label[c]] += 1;
      gas += 1;
    }
  int32_t nb = 0;
  double sum_d = 0.0;
  if (hist)
    for (int b = 0; b < nbins; ++b) hist[b] = 0.0;
  for (size_t c = 0; c < N; ++c) {
    if (count[c] == 0) continue;
    double a = (double)count[c];
    double d = 2.0 * sqrt(a / M_PI);
    if (areas) areas[nb] = a;
    if (diam) diam[nb] = d;
    sum_d += d;
    if (hist && nbins > 0) {
      double u = (log(d) - log(dmin)) / (log(dmax) - log(dmin));
      int b = (int)floor(u * nbins);
      if (b < 0) b = 0;
      if (b >= nbins) b = nbins - 1;
      hist[b] += 1.0;
    }
    nb += 1;
  }
  *gas_fraction = (double)gas / (double)N;
  *mean_diameter = nb > 0 ? sum_d / nb : 0.0;
  free(count);
  return nb;
}

/* ------------------------------------------------------------------------
 * Two-component variant (melt m and gas g lattices; Sec. 2.1.5, the
 * two-lattice description and the coupled velocities of Eqs. 36-40).
 *
 * Readings (the paper's formulas there are garbled; each is listed in the
 * design notes):
 *   - each component sigma has its own D2Q9 populations, BGK time tau_sigma
 *     and pseudopotential psi_sigma = rho0 (1 - exp(-rho_sigma / rho0));
 *   - force on sigma: F_sigma(x) = -psi_sigma(x) sum_s' G_{sigma s'} S_s'(x),
 *     S_s'(x) = sum_i w_i psi~_s'(x + e_i) e_i, with G_mm (melt cohesion, the
 *     single-component G), G_mg = G_gm (melt-gas repulsion) and G_gg, and the
 *     barrier substitution psi~ = psi_s'(x) across a blocked edge;
 *   - common velocity ("u_total", read as momentum over total density):
 *     u' = (sum_s j_s / tau_s) / (sum_s rho_s / tau_s), which is
 *     (j_m + j_g) / (rho_m + rho_g) for equal relaxation times;
 *   - equilibrium velocity of each component u_s = u' + tau_s F_s / rho_s
 *     (Eqs. 39-40; a component with rho_s = 0 has f^eq = 0 and takes u');
 *   - pressure p = (rho_m + rho_g)/3 + (1/6) sum_{s,s'} G_{ss'} psi_s psi_s'
 *     (Eq. 29 summed over the pairs; with no gas it is Eq. 29);
 *   - bubbles (for the barrier) are the 4-connected regions of melt density
 *     below gas_threshold; the rupture test uses the pressure above; both
 *     components bounce back across a blocked edge.
 * With an empty gas lattice the step is the single-component step.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t nx, ny;
  int32_t barrier, relabel_every, zone_radius, reserved;
  double tau_m, tau_g;
  double G_mm, G_mg, G_gg;
  double rho0;
  double gas_threshold; /* gas point iff melt density < this */
  double rupture_eps;
} orc2_params;

typedef struct {
  double *fm, *fg;           /* [9][ny][nx] incoming populations per component */
  double *fm_next, *fg_next; /* scratch */
  double *rm, *rg, *psim, *psig, *pr; /* [ny][nx] scratch */
  int32_t *label, *owner;
  int8_t *sgn;
  uint8_t *open, *mask;
  int64_t t, opened_total;
} orc2_state;

static orc_params orc2_as_single(const orc2_params *q) {
  orc_params p;
  memset(&p, 0, sizeof(p));
  p.nx = q->nx;
  p.ny = q->ny;
  p.barrier = q->barrier;
  p.relabel_every = q->relabel_every;
  p.zone_radius = q->zone_radius;
  p.tau = q->tau_m;
  p.G = q->G_mm;
  p.rho0 = q->rho0;
  p.gas_threshold = q->gas_threshold;
  p.rupture_eps = q->rupture_eps;
  return p;
}

/* Mixture pressure of the reading above. */
double orc2_pressure(const orc2_params *q, double rm, double rg) {
  const double a = orc_psi(rm, q->rho0), b = orc_psi(rg, q->rho0);
  return (rm + rg) / 3.0 + (q->G_mm * a * a + 2.0 * q->G_mg * a * b + q->G_gg * b * b) / 6.0;
}

/* S(x) = sum_i w_i psi~(x + e_i) e_i with the barrier substitution. */
static void neighbour_sum(int nx, int ny, const double *psi, const uint8_t *mask, size_t c, int x, int y,
                          double *sx, double *sy) {
  double ax = 0.0, ay = 0.0;
  for (int i = 1; i < Q; ++i) {
    size_t nb = (size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
    double v = psi[nb];
    if (mask && ((mask[c] >> (i - 1)) & 1u)) v = psi[c];
    ax += WT[i] * v * EX[i];
    ay += WT[i] * v * EY[i];
  }
  *sx = ax;
  *sy = ay;
}

void orc2_init_state(const orc2_params *q, orc2_state *s, const double *rho_m, const double *rho_g) {
  const size_t N = (size_t)q->nx * q->ny;
  for (int i = 0; i < Q; ++i)
    for (size_t c = 0; c < N; ++c) {
      s->fm[i * N + c] = WT[i] * rho_m[c];
      s->fg[i * N + c] = WT[i] * rho_g[c];
    }
  memset(s->sgn, 0, N);
  memset(s->open, 0, N);
  memset(s->mask, 0, N);
  for (size_t c = 0; c < N; ++c) s->label[c] = s->owner[c] = -1;
  s->t = 0;
  s->opened_total = 0;
}

/* Barrier pipeline on the melt density (labels, owners, mask) with the
 * rupture test on the mixture pressure. */
void orc2_relabel(const orc2_params *q, orc2_state *s) {
  const orc_params p = orc2_as_single(q);
  const size_t N = (size_t)q->nx * q->ny;
  orc_moments(&p, s->fm, s->rm, NULL, NULL);
  orc_moments(&p, s->fg, s->rg, NULL, NULL);
  for (size_t c = 0; c < N; ++c) s->pr[c] = orc2_pressure(q, s->rm[c], s->rg[c]);
  orc_label(&p, s->rm, s->label);
  orc_owner(&p, s->label, s->owner);
  int32_t opened = 0;
  rupture_on_pressure(&p, s->pr, s->owner, s->sgn, s->open, &opened);
  orc_mask(&p, s->owner, s->open, s->mask);
  s->opened_total += opened;
}

/* One step of both lattices. */
void orc2_step(const orc2_params *q, orc2_state *s) {
  const int nx = q->nx, ny = q->ny;
  const size_t N = (size_t)nx * ny;
  const orc_params p = orc2_as_single(q);
  const int barrier = q->barrier != 0;
  if (barrier && s->t % q->relabel_every == 0) orc2_relabel(q, s);
  const uint8_t *mask = barrier ? s->mask : NULL;
  orc_moments(&p, s->fm, s->rm, NULL, NULL);
  orc_moments(&p, s->fg, s->rg, NULL, NULL);
  for (size_t c = 0; c < N; ++c) {
    s->psim[c] = orc_psi(s->rm[c], q->rho0);
    s->psig[c] = orc_psi(s->rg[c], q->rho0);
  }
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t c = (size_t)y * nx + x;
      double rm = 0.0, rg = 0.0, jxm = 0.0, jym = 0.0, jxg = 0.0, jyg = 0.0;
      for (int i = 0; i < Q; ++i) {
        const double a = s->fm[i * N + c], b = s->fg[i * N + c];
        rm += a;
        rg += b;
        jxm += EX[i] * a;
        jym += EY[i] * a;
        jxg += EX[i] * b;
        jyg += EY[i] * b;
      }
      double smx, smy, sgx, sgy;
      neighbour_sum(nx, ny, s->psim, mask, c, x, y, &smx, &smy);
      neighbour_sum(nx, ny, s->psig, mask, c, x, y, &sgx, &sgy);
      const double Fmx = -s->psim[c] * (q->G_mm * smx + q->G_mg * sgx);
      const double Fmy = -s->psim[c] * (q->G_mm * smy + q->G_mg * sgy);
      const double Fgx = -s->psig[c] * (q->G_mg * smx + q->G_gg * sgx);
      const double Fgy = -s->psig[c] * (q->G_mg * smy + q->G_gg * sgy);
      const double den = rm / q->tau_m + rg / q->tau_g;
      const double ux = (jxm / q->tau_m + jxg / q->tau_g) / den;
      const double uy = (jym / q->tau_m + jyg / q->tau_g) / den;
      double um_x = ux, um_y = uy, ug_x = ux, ug_y = uy;
      if (rm > 0.0) {
        um_x += q->tau_m * Fmx / rm;
        um_y += q->tau_m * Fmy / rm;
      }
      if (rg > 0.0) {
        ug_x += q->tau_g * Fgx / rg;
        ug_y += q->tau_g * Fgy / rg;
      }
      double feq_m[Q], feq_g[Q];
      orc_equilibrium(rm, um_x, um_y, feq_m);
      orc_equilibrium(rg, ug_x, ug_y, feq_g);
      for (int i = 0; i < Q; ++i) {
        const double a = s->fm[i * N + c], b = s->fg[i * N + c];
        /* streaming; across a blocked edge both components bounce back */
        size_t dst = (size_t)wrap(y + EY[i], ny) * nx + wrap(x + EX[i], nx);
        int d = i;
        if (mask && i > 0 && ((mask[c] >> (i - 1)) & 1u)) {
          dst = c;
          d = OPP[i];
        }
        s->fm_next[d * N + dst] = a - (a - feq_m[i]) / q->tau_m;
        s->fg_next[d * N + dst] = b - (b - feq_g[i]) / q->tau_g;
      }
    }
  memcpy(s->fm, s->fm_next, Q * N * sizeof(double));
  memcpy(s->fg, s->fg_next, Q * N * sizeof(double));
  s->t += 1;
}

void orc2_run(const orc2_params *q, orc2_state *s, int64_t nsteps) {
  for (int64_t k = 0; k < nsteps; ++k) orc2_step(q, s);
}

/* Diagnostics at the start of the current step: component densities, the
 * physical common velocity u = (sum_s (j_s + F_s / 2)) / (rho_m + rho_g),
 * and the mixture pressure. Any output may be NULL. */
void orc2_fields(const orc2_params *q, orc2_state *s, double *rho_m, double *rho_g, double *ux, double *uy,
                 double *pr) {
  const int nx = q->nx, ny = q->ny;
  const size_t N = (size_t)nx * ny;
  const orc_params p = orc2_as_single(q);
  const uint8_t *mask = q->barrier ? s->mask : NULL;
  orc_moments(&p, s->fm, s->rm, NULL, NULL);
  orc_moments(&p, s->fg, s->rg, NULL, NULL);
  for (size_t c = 0; c < N; ++c) {
    s->psim[c] = orc_psi(s->rm[c], q->rho0);
    s->psig[c] = orc_psi(s->rg[c], q->rho0);
  }
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      const size_t c = (size_t)y * nx + x;
      double jx = 0.0, jy = 0.0;
      for (int i = 0; i < Q; ++i) {
        jx += EX[i] * (s->fm[i * N + c] + s->fg[i * N + c]);
        jy += EY[i] * (s->fm[i * N + c] + s->fg[i * N + c]);
      }
      double smx, smy, sgx, sgy;
      neighbour_sum(nx, ny, s->psim, mask, c, x, y, &smx, &smy);
      neighbour_sum(nx, ny, s->psig, mask, c, x, y, &sgx, &sgy);
      const double Fx = -s->psim[c] * (q->G_mm * smx + q->G_mg * sgx) - s->psig[c] * (q->G_mg * smx + q->G_gg * sgx);
      const double Fy = -s->psim[c] * (q->G_mm * smy + q->G_mg * sgy) - s->psig[c] * (q->G_mg * smy + q->G_gg * sgy);
      const double r = s->rm[c] + s->rg[c];
      if (rho_m) rho_m[c] = s->rm[c];
      if (rho_g) rho_g[c] = s->rg[c];
      if (ux) ux[c] = (jx + 0.5 * Fx) / r;
      if (uy) uy[c] = (jy + 0.5 * Fy) / r;
      if (pr) pr[c] = orc2_pressure(q, s->rm[c], s->rg[c]);
    }
}
