/*
 * oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE; see oracle.h).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared [-fopenmp] oracle.c -lm
 * -ffp-contract=off keeps every a*b+c as two rounded operations, so the op sequence written here is
 * the one that executes.  OpenMP (when enabled) only splits loops whose iterations are independent
 * (one agent or one voxel per iteration, no shared accumulator), so results do not depend on the
 * thread count.
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg load this file's library.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al., "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3-4):
 * ten rounds of the 4-word Philox S-box with multipliers 0xD2511F53, 0xCD9E8D57; between rounds
 * the 2-word key is bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85.  One round maps
 * (c0, c1, c2, c3) to (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)).
 * ------------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox4x32_10_n(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  for (size_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* ------------------------------------------------------------------------------------------------
 * Uniform grid (paper, "Simulation concepts", environment paragraph: equal boxes, agents assigned by
 * centre, neighbourhood = own box + 26 surrounding boxes, box size from the largest agent).
 * Reading R5: centres are quantised to a fixed-point lattice, X = round(x * 2^Q), Q = 20.  With
 * O = min X, Lq = ceil(L * 2^Q) and box coordinate (X - O) div Lq, two centres closer than R <= L
 * differ by at most Lq lattice units and so by at most one box per axis: the 27-box search is exact.
 * ------------------------------------------------------------------------------------------------ */
#define ORC_Q 20

typedef struct {
  int64_t O[3];     /* origin, lattice units            */
  int64_t Lq;       /* box length, lattice units        */
  int64_t dims[3];  /* boxes per axis                   */
  int64_t nbox;
  double R;         /* interaction (neighbour) radius   */
  double L;         /* requested box length (>= R)      */
} orc_grid_t;

static int64_t quantise(double v) { return (int64_t)llrint(ldexp(v, ORC_Q)); }

static int grid_setup(size_t n, const double* x, const double* y, const double* z, const float* diam,
                      double interaction_radius, double box_length, orc_grid_t* G) {
  if (n == 0) return -1;
  double dmax = 0.0;
  for (size_t i = 0; i < n; ++i)
    if ((double)diam[i] > dmax) dmax = (double)diam[i];
  G->R = interaction_radius > 0.0 ? interaction_radius : dmax;
  G->L = box_length > 0.0 ? box_length : G->R;
  if (!(G->R > 0.0) || G->L < G->R) return -1;
  G->Lq = (int64_t)ceil(ldexp(G->L, ORC_Q));
  const double* c[3] = {x, y, z};
  int64_t nbox = 1;
  for (int a = 0; a < 3; ++a) {
    int64_t lo = INT64_MAX, hi = INT64_MIN;
    for (size_t i = 0; i < n; ++i) {
      if (!(fabs(c[a][i]) < 1e9)) return -1; /* also rejects NaN */
      int64_t X = quantise(c[a][i]);
      if (X < lo) lo = X;
      if (X > hi) hi = X;
    }
    G->O[a] = lo;
    G->dims[a] = (hi - lo) / G->Lq + 1;
    nbox *= G->dims[a];
    if (nbox > ((int64_t)1 << 32) - 2) return -1;
  }
  G->nbox = nbox;
  return 0;
}

static void box_coords(const orc_grid_t* G, double x, double y, double z, int64_t b[3]) {
  b[0] = (quantise(x) - G->O[0]) / G->Lq;
  b[1] = (quantise(y) - G->O[1]) / G->Lq;
  b[2] = (quantise(z) - G->O[2]) / G->Lq;
}

static int64_t box_key(const orc_grid_t* G, const int64_t b[3]) {
  return b[0] + G->dims[0] * (b[1] + G->dims[1] * b[2]);
}

static void grid_vector(const orc_grid_t* G, double* g) {
  if (!g) return;
  g[0] = (double)G->O[0]; g[1] = (double)G->O[1]; g[2] = (double)G->O[2];
  g[3] = G->R; g[4] = G->L; g[5] = (double)G->Lq;
  g[6] = (double)G->dims[0]; g[7] = (double)G->dims[1]; g[8] = (double)G->dims[2];
  g[9] = (double)G->nbox;
}

int orc_grid(size_t n, const double* x, const double* y, const double* z, const float* diam,
             double interaction_radius, double box_length, double* g, uint32_t* box_id) {
  orc_grid_t G;
  if (grid_setup(n, x, y, z, diam, interaction_radius, box_length, &G)) return -1;
  grid_vector(&G, g);
  for (size_t i = 0; i < n; ++i) {
    int64_t b[3];
    box_coords(&G, x[i], y[i], z[i], b);
    box_id[i] = (uint32_t)box_key(&G, b);
  }
  return 0;
}

/* ------------------------------------------------------------------------------------------------
 * One mechanics step (agent operation "calculate mechanical forces", paper Sec. "Simulation
 * concepts"; force law reading R1-R4).  Jacobi: all forces use the positions at step start.
 * For agent i, neighbours j are visited box by box in ascending box key -- (dz, dy, dx) in
 * lexicographic order over {-1,0,1}^3 -- and by ascending id inside a box: the canonical order.
 *   neighbour:  d2 = (dx*dx + dy*dy) + dz*dz  <  R*R            (R1, strict, no sqrt)
 *   contact:    d = sqrt(d2), delta = (r_i + r_j) - d > 0, d > 0 (R2: coincident centres: no force)
 *   force:      Rr = r_i r_j / (r_i + r_j);  F = k delta - gamma sqrt(Rr delta)   (R3)
 *               S_i += (F / d) (x_i - x_j)
 *   update:     D = dt S_i; if |D| > cap then D *= cap / |D|; x_i += D        (R4)
 * ------------------------------------------------------------------------------------------------ */
int orc_mech_step(size_t n, const double* x, const double* y, const double* z, const float* diam,
                  const orc_mech_params* p, double* nx, double* ny, double* nz, uint32_t* nbr,
                  uint32_t* box_id, double* g, double* fx, double* fy, double* fz) {
  orc_grid_t G;
  if (n == 0) return 0;
  if (grid_setup(n, x, y, z, diam, p->interaction_radius, p->box_length, &G)) return -1;
  grid_vector(&G, g);

  /* Canonical order by (box, id): counting sort over ids taken in ascending order. */
  uint32_t* key = (uint32_t*)malloc(n * sizeof(uint32_t));
  uint32_t* start = (uint32_t*)calloc((size_t)G.nbox + 1, sizeof(uint32_t));
  uint32_t* order = (uint32_t*)malloc(n * sizeof(uint32_t));
  if (!key || !start || !order) {
    free(key); free(start); free(order);
    return -2;
  }
  for (size_t i = 0; i < n; ++i) {
    int64_t b[3];
    box_coords(&G, x[i], y[i], z[i], b);
    key[i] = (uint32_t)box_key(&G, b);
    start[key[i] + 1]++;
  }
  for (int64_t b = 0; b < G.nbox; ++b) start[b + 1] += start[b];
  {
    uint32_t* fill = (uint32_t*)malloc((size_t)G.nbox * sizeof(uint32_t));
    if (!fill) {
      free(key); free(start); free(order);
      return -2;
    }
    memcpy(fill, start, (size_t)G.nbox * sizeof(uint32_t));
    for (size_t i = 0; i < n; ++i) order[fill[key[i]]++] = (uint32_t)i;
    free(fill);
  }
  if (box_id) memcpy(box_id, key, n * sizeof(uint32_t));

  const double R2 = G.R * G.R;
  const double k = p->k_rep, gam = p->gamma_att, dt = p->dt, cap = p->max_disp;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1024)
#endif
  for (long long ii = 0; ii < (long long)n; ++ii) {
    size_t i = (size_t)ii;
    int64_t b[3];
    box_coords(&G, x[i], y[i], z[i], b);
    const double ri = 0.5 * (double)diam[i];
    double Sx = 0.0, Sy = 0.0, Sz = 0.0;
    uint32_t cnt = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      int64_t bz = b[2] + dz;
      if (bz < 0 || bz >= G.dims[2]) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        int64_t by = b[1] + dy;
        if (by < 0 || by >= G.dims[1]) continue;
        for (int dxb = -1; dxb <= 1; ++dxb) {
          int64_t bx = b[0] + dxb;
          if (bx < 0 || bx >= G.dims[0]) continue;
          int64_t kb = bx + G.dims[0] * (by + G.dims[1] * bz);
          for (uint32_t m = start[kb]; m < start[kb + 1]; ++m) {
            uint32_t j = order[m];
            if (j == i) continue;
            double ddx = x[i] - x[j];
            double ddy = y[i] - y[j];
            double ddz = z[i] - z[j];
            double d2 = ddx * ddx + ddy * ddy;
            d2 = d2 + ddz * ddz;
            if (d2 < R2) cnt++;
            double d = sqrt(d2);
            double rj = 0.5 * (double)diam[j];
            double delta = (ri + rj) - d;
            if (delta > 0.0 && d > 0.0) {
              double Rr = (ri * rj) / (ri + rj);
              double F = k * delta - gam * sqrt(Rr * delta);
              double s = F / d;
              Sx = Sx + s * ddx;
              Sy = Sy + s * ddy;
              Sz = Sz + s * ddz;
            }
          }
        }
      }
    }
    if (fx) { fx[i] = Sx; fy[i] = Sy; fz[i] = Sz; }
    double Dx = dt * Sx, Dy = dt * Sy, Dz = dt * Sz;
    double norm = Dx * Dx + Dy * Dy;
    norm = sqrt(norm + Dz * Dz);
    if (norm > cap) {
      double f = cap / norm;
      Dx = Dx * f; Dy = Dy * f; Dz = Dz * f;
    }
    nx[i] = x[i] + Dx;
    ny[i] = y[i] + Dy;
    nz[i] = z[i] + Dz;
    nbr[i] = cnt;
  }
  free(key); free(start); free(order);
  return 0;
}

/* ------------------------------------------------------------------------------------------------
 * Growth and division (paper Sec. "Simulation concepts": behaviours such as cell division create new
 * agents; Sec. "Performance": the cell growth and division benchmark).  Reading R7:
 *   (i)  every agent alive at step start grows: V += dv;
 *   (ii) agents with V >= vdiv divide, in ascending id; the m-th divider's daughter gets id n + m;
 *        mother and daughter keep V / 2;
 *   (iii) every agent's diameter is d = cbrt(6 V / pi) rounded to float;
 *   (iv) the division axis u comes from Philox key (seed_lo, run), counter (id, step, 2, attempt):
 *        u_k = w_k * 2^-31 - 1 for k = 0..2, accepted when 2^-20 <= |u|^2 <= 1 (at most 64 tries,
 *        else u = (0,0,1)), then normalised; the mother moves to x - o u and the daughter to x + o u
 *        with o = offset_frac * d (d of the halves).
 * ------------------------------------------------------------------------------------------------ */
/* pi rounded to double */
#define ORC_PI 3.141592653589793

static double diameter_of_volume(double v) { return (double)(float)cbrt((v * 6.0) / ORC_PI); }

static void division_axis(uint32_t id, uint32_t step, uint32_t seed_lo, uint32_t run, double u[3]) {
  const uint32_t key[2] = {seed_lo, run};
  for (uint32_t attempt = 0; attempt < 64; ++attempt) {
    const uint32_t ctr[4] = {id, step, 2u, attempt};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    double a = ldexp((double)w[0], -31) - 1.0;
    double b = ldexp((double)w[1], -31) - 1.0;
    double c = ldexp((double)w[2], -31) - 1.0;
    double q = a * a + b * b;
    q = q + c * c;
    if (q <= 1.0 && q >= ldexp(1.0, -20)) {
      double len = sqrt(q);
      u[0] = a / len; u[1] = b / len; u[2] = c / len;
      return;
    }
  }
  u[0] = 0.0; u[1] = 0.0; u[2] = 1.0;
}

int orc_grow_divide(size_t n, double* x, double* y, double* z, float* diam, double* vol,
                    double dv, double vdiv, double offset_frac, uint32_t seed_lo, uint32_t run,
                    uint32_t step, size_t* n_out) {
  size_t m = n;
  for (size_t i = 0; i < n; ++i) {
    vol[i] = vol[i] + dv;
    if (vol[i] >= vdiv) {
      double half = vol[i] * 0.5;
      double d = diameter_of_volume(half);
      double u[3];
      division_axis((uint32_t)i, step, seed_lo, run, u);
      double o = offset_frac * d;
      x[m] = x[i] + o * u[0]; y[m] = y[i] + o * u[1]; z[m] = z[i] + o * u[2];
      x[i] = x[i] - o * u[0]; y[i] = y[i] - o * u[1]; z[i] = z[i] - o * u[2];
      vol[i] = half; vol[m] = half;
      diam[i] = (float)d; diam[m] = (float)d;
      ++m;
    } else {
      diam[i] = (float)diameter_of_volume(vol[i]);
    }
  }
  *n_out = m;
  return 0;
}

/* ------------------------------------------------------------------------------------------------
 * Apoptosis (paper Sec. "Oncology use case": cell apoptosis is one of the modelled mechanisms; its
 * rate is not printed).  Reading R14: at the start of a step every agent dies with probability p:
 * Philox4x32-10 with key (seed, run) and counter (id, step, 4, 0) gives w, and the agent dies when
 * w_0 < floor(p 2^32).  Survivors keep their relative order and take the dense ids 0..m-1.
 * ------------------------------------------------------------------------------------------------ */
size_t orc_apoptosis(size_t n, double* x, double* y, double* z, float* diam, double* vol,
                     uint64_t thr, uint32_t seed_lo, uint32_t run, uint32_t step) {
  const uint32_t key[2] = {seed_lo, run};
  size_t m = 0;
  for (size_t i = 0; i < n; ++i) {
    const uint32_t ctr[4] = {(uint32_t)i, step, 4u, 0u};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    if ((uint64_t)w[0] < thr) continue;
    x[m] = x[i]; y[m] = y[i]; z[m] = z[i];
    diam[m] = diam[i];
    vol[m] = vol[i];
    ++m;
  }
  return m;
}

/* ------------------------------------------------------------------------------------------------
 * Brownian migration (paper Sec. "Oncology use case": migration is modelled as Brownian motion;
 * its amplitude is not printed).  Reading R13: after the capped mechanical update every agent moves
 * by sigma (g0, g1, g2), standard normal deviates by the Box-Muller transform of Philox4x32-10 words
 * (key (seed, run), counter (id, step, 3, 0)): with u = (w0 + 1) 2^-32, v = w1 2^-32,
 * u' = (w2 + 1) 2^-32, v' = w3 2^-32: g0 = sqrt(-2 ln u) cos(2 pi v), g1 = sqrt(-2 ln u) sin(2 pi v),
 * g2 = sqrt(-2 ln u') cos(2 pi v').  Each coordinate: x <- x + sigma g (after x <- x + D).
 * ------------------------------------------------------------------------------------------------ */
void orc_brownian(size_t n, double* x, double* y, double* z, double sigma, uint32_t seed_lo,
                  uint32_t run, uint32_t step) {
  const uint32_t key[2] = {seed_lo, run};
  for (size_t i = 0; i < n; ++i) {
    const uint32_t ctr[4] = {(uint32_t)i, step, 3u, 0u};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    const double u = ldexp((double)w[0] + 1.0, -32), v = ldexp((double)w[1], -32);
    const double u2 = ldexp((double)w[2] + 1.0, -32), v2 = ldexp((double)w[3], -32);
    const double r = sqrt(-2.0 * log(u)), r2 = sqrt(-2.0 * log(u2));
    x[i] = x[i] + sigma * (r * cos(2.0 * ORC_PI * v));
    y[i] = y[i] + sigma * (r * sin(2.0 * ORC_PI * v));
    z[i] = z[i] + sigma * (r2 * cos(2.0 * ORC_PI * v2));
  }
}

/* ------------------------------------------------------------------------------------------------
 * Secretion into a substance grid (paper Sec. "Simulation concepts": growth-factor secretion is an
 * agent behaviour acting on the extracellular substance).  Reading R8: voxel index per axis is
 * clamp(floor((x - origin) / h), 0, dims - 1); every agent adds q.
 * ------------------------------------------------------------------------------------------------ */
static int64_t voxel_of(double v, double o, double h, int64_t n) {
  double f = floor((v - o) / h);
  if (!(f >= 0.0)) return 0;
  if (f >= (double)(n - 1)) return n - 1;
  return (int64_t)f;
}

void orc_secrete(size_t n, const double* x, const double* y, const double* z, double* grid,
                 const int64_t dims[3], const double origin[3], double h, double q) {
  for (size_t i = 0; i < n; ++i) {
    int64_t a = voxel_of(x[i], origin[0], h, dims[0]);
    int64_t b = voxel_of(y[i], origin[1], h, dims[1]);
    int64_t c = voxel_of(z[i], origin[2], h, dims[2]);
    grid[a + dims[0] * (b + dims[1] * c)] += q;
  }
}

/* ------------------------------------------------------------------------------------------------
 * Chemotaxis (paper Sec. "Simulation concepts": chemotaxis is an agent behaviour that reads the
 * extracellular substance; its law is not printed).  Reading R15: after the mechanical update (and
 * migration) every agent moves by chi * grad c, the gradient of the grid as it stood at the start of
 * the step at the voxel of the agent's step-start centre (voxel as in R8).  Per axis: central
 * difference (c[v+1] - c[v-1]) / (2h) inside, one-sided (c[v+1] - c[v]) / h or (c[v] - c[v-1]) / h at
 * a wall, 0 along an axis of one voxel.
 * ------------------------------------------------------------------------------------------------ */
static double grid_derivative(const double* g, const int64_t dims[3], int64_t a, int64_t b,
                              int64_t c, int axis, double h) {
  const int64_t idx[3] = {a, b, c};
  const int64_t n = dims[axis], v = idx[axis];
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? dims[0] : dims[0] * dims[1]);
  const int64_t at = a + dims[0] * (b + dims[1] * c);
  if (n < 2) return 0.0;
  if (v == 0) return (g[at + stride] - g[at]) / h;
  if (v == n - 1) return (g[at] - g[at - stride]) / h;
  return (g[at + stride] - g[at - stride]) / (2.0 * h);
}

void orc_chemotaxis(size_t n, double* x, double* y, double* z, const double* sx, const double* sy,
                    const double* sz, const double* grid, const int64_t dims[3],
                    const double origin[3], double h, double chi) {
  for (size_t i = 0; i < n; ++i) {
    const int64_t a = voxel_of(sx[i], origin[0], h, dims[0]);
    const int64_t b = voxel_of(sy[i], origin[1], h, dims[1]);
    const int64_t c = voxel_of(sz[i], origin[2], h, dims[2]);
    x[i] = x[i] + chi * grid_derivative(grid, dims, a, b, c, 0, h);
    y[i] = y[i] + chi * grid_derivative(grid, dims, a, b, c, 1, h);
    z[i] = z[i] + chi * grid_derivative(grid, dims, a, b, c, 2, h);
  }
}

/* ------------------------------------------------------------------------------------------------
 * Diffusion of an extracellular substance (paper Sec. "Simulation concepts": standalone operation,
 * once per step).  Reading R9: explicit forward-time centred-space 7-point update,
 *   u'_v = u_v + lambda * sum_{6 faces} (u_nb - u_v) - mu_dt * u_v,  lambda = D dt / h^2,
 * zero-flux walls (a missing face neighbour contributes 0).  Mass = sum of u' in FP64, x fastest.
 * ------------------------------------------------------------------------------------------------ */
double orc_ftcs(const int64_t dims[3], const double* u, double* out, double lambda, double mu_dt) {
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (long long k = 0; k < (long long)nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t v = i + nx * (j + ny * (int64_t)k);
        double c = u[v];
        double lap = 0.0;
        if (i > 0) lap = lap + (u[v - 1] - c);
        if (i < nx - 1) lap = lap + (u[v + 1] - c);
        if (j > 0) lap = lap + (u[v - nx] - c);
        if (j < ny - 1) lap = lap + (u[v + nx] - c);
        if (k > 0) lap = lap + (u[v - nx * ny] - c);
        if (k < nz - 1) lap = lap + (u[v + nx * ny] - c);
        out[v] = (c + lambda * lap) - mu_dt * c;
      }
  double mass = 0.0;
  for (int64_t v = 0; v < nx * ny * nz; ++v) mass += out[v];
  return mass;
}

/* ------------------------------------------------------------------------------------------------
 * SIR behaviours (paper Sec. "Epidemiology use case"): infection of a susceptible agent with the
 * infection probability when an infected agent is within the infection radius; recovery of an
 * infected agent with the recovery probability each step; bounded random movement of every agent.
 * Reading R10: synchronous step on int32 fixed-point positions in a periodic cube of side L;
 *   infected-neighbour count uses states and positions at step start, minimum-image distance,
 *   d^2 < r^2 in 64-bit integers; Philox key (seed_lo, run);
 *   stream 0, counter (id, step, 0, 0): w0 < thr_inf infects a susceptible with count > 0,
 *                                       w1 < thr_rec recovers an agent infected at step start;
 *   stream 1, counter (id, step, 1, 0): move per axis ((w * (2s + 1)) >> 32) - s, wrapped into [0, L).
 * The grid is nb^3 periodic boxes of side L / nb; an axis with fewer than 3 boxes visits each box once.
 * ------------------------------------------------------------------------------------------------ */
static int64_t min_image(int64_t d, int64_t L) {
  if (d > L / 2) d -= L;
  else if (d < -(L / 2)) d += L;
  return d;
}

int orc_sir_step(size_t n, const int32_t* X, const int32_t* Y, const int32_t* Z, const uint8_t* st,
                 int32_t L, int32_t nb, int32_t r, int32_t s, uint64_t thr_inf, uint64_t thr_rec,
                 uint32_t seed_lo, uint32_t run, uint32_t step, int32_t* nX, int32_t* nY,
                 int32_t* nZ, uint8_t* nst, uint32_t* ninf, uint32_t* box_id, uint32_t counts[3]) {
  if (L <= 0 || nb <= 0 || L % nb != 0 || L / nb < r || r < 0 || s < 0 || s >= L) return -1;
  const int64_t Lb = L / nb, nbox = (int64_t)nb * nb * nb;
  uint32_t* key = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
  uint32_t* start = (uint32_t*)calloc((size_t)nbox + 1, sizeof(uint32_t));
  uint32_t* order = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
  if (!key || !start || !order) {
    free(key); free(start); free(order);
    return -2;
  }
  for (size_t i = 0; i < n; ++i) {
    if (X[i] < 0 || X[i] >= L || Y[i] < 0 || Y[i] >= L || Z[i] < 0 || Z[i] >= L) {
      free(key); free(start); free(order);
      return -1;
    }
    key[i] = (uint32_t)(X[i] / Lb + nb * (Y[i] / Lb + nb * (Z[i] / Lb)));
    start[key[i] + 1]++;
  }
  for (int64_t b = 0; b < nbox; ++b) start[b + 1] += start[b];
  {
    uint32_t* fill = (uint32_t*)malloc((size_t)nbox * sizeof(uint32_t));
    if (!fill) {
      free(key); free(start); free(order);
      return -2;
    }
    memcpy(fill, start, (size_t)nbox * sizeof(uint32_t));
    for (size_t i = 0; i < n; ++i) order[fill[key[i]]++] = (uint32_t)i;
    free(fill);
  }
  if (box_id) memcpy(box_id, key, n * sizeof(uint32_t));

  const uint32_t pkey[2] = {seed_lo, run};
  const int64_t r2 = (int64_t)r * r;
  const uint64_t span = 2u * (uint64_t)s + 1u;
  uint32_t cS = 0, cI = 0, cR = 0;
  for (size_t i = 0; i < n; ++i) {
    int64_t b[3] = {X[i] / Lb, Y[i] / Lb, Z[i] / Lb};
    /* Distinct neighbour box coordinates per axis (periodic). */
    int64_t nbx[3][3];
    int cntx[3];
    for (int a = 0; a < 3; ++a) {
      cntx[a] = 0;
      for (int d = -1; d <= 1; ++d) {
        int64_t c = ((b[a] + d) % nb + nb) % nb;
        int dup = 0;
        for (int q = 0; q < cntx[a]; ++q) dup |= (nbx[a][q] == c);
        if (!dup) nbx[a][cntx[a]++] = c;
      }
    }
    uint32_t infected = 0;
    for (int qz = 0; qz < cntx[2]; ++qz)
      for (int qy = 0; qy < cntx[1]; ++qy)
        for (int qx = 0; qx < cntx[0]; ++qx) {
          int64_t kb = nbx[0][qx] + nb * (nbx[1][qy] + nb * nbx[2][qz]);
          for (uint32_t m = start[kb]; m < start[kb + 1]; ++m) {
            uint32_t j = order[m];
            if (j == i || st[j] != 1) continue;
            int64_t dx = min_image((int64_t)X[i] - X[j], L);
            int64_t dy = min_image((int64_t)Y[i] - Y[j], L);
            int64_t dz = min_image((int64_t)Z[i] - Z[j], L);
            if (dx * dx + dy * dy + dz * dz < r2) infected++;
          }
        }
    ninf[i] = infected;
    uint32_t w[4], mv[4];
    const uint32_t c0[4] = {(uint32_t)i, step, 0u, 0u};
    const uint32_t c1[4] = {(uint32_t)i, step, 1u, 0u};
    orc_philox4x32_10(c0, pkey, w);
    orc_philox4x32_10(c1, pkey, mv);
    uint8_t ns = st[i];
    if (st[i] == 0 && infected > 0 && (uint64_t)w[0] < thr_inf) ns = 1;
    if (st[i] == 1 && (uint64_t)w[1] < thr_rec) ns = 2;
    nst[i] = ns;
    cS += (ns == 0); cI += (ns == 1); cR += (ns == 2);
    const int32_t* P[3] = {X, Y, Z};
    int32_t* NP[3] = {nX, nY, nZ};
    for (int a = 0; a < 3; ++a) {
      int64_t step_a = (int64_t)(((uint64_t)mv[a] * span) >> 32) - s;
      int64_t v = (int64_t)P[a][i] + step_a;
      if (v < 0) v += L;
      else if (v >= L) v -= L;
      NP[a][i] = (int32_t)v;
    }
  }
  counts[0] = cS; counts[1] = cI; counts[2] = cR;
  free(key); free(start); free(order);
  return 0;
}

/* ------------------------------------------------------------------------------------------------
 * Neurite mechanics (paper Sec. "Neuroscience module": neurite elements are cylinders, modelled as a
 * spring with a point mass at the distal end, connected as a binary tree so that forces travel
 * along the chain; Sec. "Simulation concepts": sphere or cylinder geometry).  The paper prints no
 * force law for cylinders; readings R16-R20:
 *   R16 agent a is a soma (mother[a] < 0; a sphere at p_a) or a neurite element (a cylinder from
 *       the proximal point q_a = p_{mother[a]} + o_a to the distal point p_a), radius r_a = d_a / 2;
 *   R17 spring: v = p_e - q_e, l = |v|, T = k_s (l - l0_e) / l0_e; the distal point takes -T v / l,
 *       the mother +T v / l (nothing when l = 0);
 *   R18 contact between the bodies of i and j (not excluded): closest points c_i, c_j (a soma's is
 *       its centre; an element's lies on its axis at parameter s_i in [0, 1], 0 proximal), then the
 *       sphere law of R3 between them: dv = c_i - c_j, d = |dv|, delta = (r_i + r_j) - d; when
 *       delta > 0 and d > 0, f = (F / d) dv with F = k delta - gamma sqrt(rho delta).  A soma takes
 *       f; an element takes s_i f at its distal point and passes (1 - s_i) f to its mother;
 *   R19 excluded pairs (they share an end point): an element and its mother, an element and its
 *       daughters, two elements with the same mother;
 *   R20 neighbours: binning point b_a = p_a (soma) or 0.5 (q_a + p_a) (element); extent e_a = d_a or
 *       l_a + d_a; radius L = max_a e_a (or a larger fixed value); a neighbour of i is j != i with
 *       |b_i - b_j|^2 < L^2.  Every contact pair is a neighbour pair: |b_i - b_j| <= l_i/2 + l_j/2 +
 *       |c_i - c_j| < e_i/2 + e_j/2 <= L.
 *   update (R4): D = dt (own share + sum over daughters of what they pass up), capped, p += D.
 * This oracle takes every pair (brute force over all j), so it does not depend on any grid.
 * ------------------------------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) {
  return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/* Closest points of segments P(s) = P0 + s u and Q(t) = Q0 + t v, s, t in [0, 1] (a zero-length
 * segment is a point): the argmin of f(s, t) = |P(s) - Q(t)|^2 over the unit square, written out from
 * its definition.  f is a convex quadratic, so its minimum over the square lies either at the
 * stationary point of the two infinite lines (when that point is inside the square) or on one of
 * the four edges, and on an edge at the clamped minimiser of a one-variable quadratic.  The
 * candidates are therefore
 *   s = 0 with t = clamp(E / C),        s = 1 with t = clamp((B + E) / C),
 *   t = 0 with s = clamp(-D / A),       t = 1 with s = clamp((B - D) / A),
 *   the stationary point s = (B E - C D) / den, t = (A E - B D) / den  (den = |u x v|^2 > 0),
 * with w = P0 - Q0, A = u.u, B = u.v, C = v.v, D = u.w, E = v.w; each is scored by its own distance
 * |P(s) - Q(t)|, evaluated directly.  Tie rule (reading R18): the first candidate in the order above
 * whose distance is within 1e-12 (|u| + |v| + |w|) of the smallest; only parallel segments have
 * tied candidates (their minimum is not unique), and the stationary point, listed last, then does
 * not exist.  A point segment (A = 0 or C = 0) takes the clamped minimiser of the other parameter. */
static double seg_pair_dist(const double P0[3], const double u[3], const double Q0[3],
                            const double v[3], double s, double t) {
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = (P0[k] + s * u[k]) - (Q0[k] + t * v[k]);
  return sqrt(dot3(d, d));
}

void orc_segment_closest(const double P0[3], const double u[3], const double Q0[3],
                         const double v[3], double* s_out, double* t_out) {
  double w[3] = {P0[0] - Q0[0], P0[1] - Q0[1], P0[2] - Q0[2]};
  double A = dot3(u, u), B = dot3(u, v), C = dot3(v, v), D = dot3(u, w), E = dot3(v, w);
  if (A <= 0.0 || C <= 0.0) {
    *s_out = A <= 0.0 ? 0.0 : clamp01(-D / A);
    *t_out = A <= 0.0 ? (C <= 0.0 ? 0.0 : clamp01(E / C)) : 0.0;
    return;
  }
  double cs[5], ct[5];
  int nc = 0;
  cs[nc] = 0.0; ct[nc] = clamp01(E / C); ++nc;
  cs[nc] = 1.0; ct[nc] = clamp01((B + E) / C); ++nc;
  cs[nc] = clamp01(-D / A); ct[nc] = 0.0; ++nc;
  cs[nc] = clamp01((B - D) / A); ct[nc] = 1.0; ++nc;
  double cr[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
  double den = dot3(cr, cr);
  if (den > 0.0) {
    double ss = (B * E - C * D) / den, tt = (A * E - B * D) / den;
    if (ss >= 0.0 && ss <= 1.0 && tt >= 0.0 && tt <= 1.0) {
      cs[nc] = ss; ct[nc] = tt; ++nc;
    }
  }
  double dist[5], dmin = INFINITY;
  for (int c = 0; c < nc; ++c) {
    dist[c] = seg_pair_dist(P0, u, Q0, v, cs[c], ct[c]);
    if (dist[c] < dmin) dmin = dist[c];
  }
  double tol = 1e-12 * ((sqrt(A) + sqrt(C)) + sqrt(dot3(w, w)));
  int pick = 0;
  while (dist[pick] > dmin + tol) ++pick;
  *s_out = cs[pick];
  *t_out = ct[pick];
}

typedef struct {
  double p[3], q[3], ax[3];  /* distal point, proximal point, axis p - q (zero for a soma) */
  double r, len;             /* radius, axis length                                       */
  int64_t mother;
} orc_body_t;

static void neurite_body(size_t a, const double* x, const double* y, const double* z,
                         const double* diam, const int32_t* mother, const double* ox,
                         const double* oy, const double* oz, orc_body_t* B) {
  B->p[0] = x[a]; B->p[1] = y[a]; B->p[2] = z[a];
  B->r = 0.5 * diam[a];
  B->mother = mother[a];
  if (mother[a] < 0) {
    for (int k = 0; k < 3; ++k) { B->q[k] = B->p[k]; B->ax[k] = 0.0; }
    B->len = 0.0;
  } else {
    size_t m = (size_t)mother[a];
    B->q[0] = x[m] + ox[a]; B->q[1] = y[m] + oy[a]; B->q[2] = z[m] + oz[a];
    for (int k = 0; k < 3; ++k) B->ax[k] = B->p[k] - B->q[k];
    B->len = sqrt(dot3(B->ax, B->ax));
  }
}

/* Own and passed-up shares of the force on agent i and its neighbour count (R17-R20), over every
 * other agent j in ascending id. */
static void neurite_shares(size_t n, size_t i, const orc_body_t* B, const double* bin,
                           const double* rest, const orc_neurite_params* p, double L2,
                           double keep[3], double pass[3], uint32_t* cnt_out) {
  const orc_body_t* bi = &B[i];
  const double k = p->k_rep, gam = p->gamma_att;
  uint32_t cnt = 0;
  for (int c = 0; c < 3; ++c) { keep[c] = 0.0; pass[c] = 0.0; }
  if (bi->mother >= 0 && bi->len > 0.0) {  /* R17 */
    double T = p->k_spring * (bi->len - rest[i]) / rest[i];
    for (int c = 0; c < 3; ++c) {
      double f = T * (bi->ax[c] / bi->len);
      keep[c] -= f;
      pass[c] += f;
    }
  }
  for (size_t j = 0; j < n; ++j) {
    if (j == i) continue;
    const orc_body_t* bj = &B[j];
    double db[3] = {bin[3 * i] - bin[3 * j], bin[3 * i + 1] - bin[3 * j + 1],
                    bin[3 * i + 2] - bin[3 * j + 2]};
    double d2 = db[0] * db[0] + db[1] * db[1];
    d2 = d2 + db[2] * db[2];
    if (d2 < L2) cnt++;
    /* R19 */
    if (bi->mother == (int64_t)j || bj->mother == (int64_t)i) continue;
    if (bi->mother >= 0 && bi->mother == bj->mother) continue;
    double s = 0.0, t = 0.0;
    orc_segment_closest(bi->q, bi->ax, bj->q, bj->ax, &s, &t);
    double dv[3];
    for (int c = 0; c < 3; ++c) dv[c] = (bi->q[c] + s * bi->ax[c]) - (bj->q[c] + t * bj->ax[c]);
    double d = sqrt(dot3(dv, dv));
    double delta = (bi->r + bj->r) - d;
    if (delta > 0.0 && d > 0.0) {
      double rho = (bi->r * bj->r) / (bi->r + bj->r);
      double F = k * delta - gam * sqrt(rho * delta);
      for (int c = 0; c < 3; ++c) {
        double f = (F / d) * dv[c];
        if (bi->mother < 0) {
          keep[c] += f;
        } else {
          keep[c] += s * f;
          pass[c] += (1.0 - s) * f;
        }
      }
    }
  }
  *cnt_out = cnt;
}

/* R4 update of one agent from its summed force. */
static void neurite_update(double x, double y, double z, const double S[3],
                           const orc_neurite_params* p, double* nx, double* ny, double* nz) {
  double Dx = p->dt * S[0], Dy = p->dt * S[1], Dz = p->dt * S[2];
  double norm = Dx * Dx + Dy * Dy;
  norm = sqrt(norm + Dz * Dz);
  if (norm > p->max_disp) {
    double f = p->max_disp / norm;
    Dx = Dx * f; Dy = Dy * f; Dz = Dz * f;
  }
  *nx = x + Dx;
  *ny = y + Dy;
  *nz = z + Dz;
}

/* Validates the agents, builds every body and binning point and the radius L. */
static int neurite_setup(size_t n, const double* x, const double* y, const double* z,
                         const double* diam, const double* rest, const int32_t* mother,
                         const double* ox, const double* oy, const double* oz,
                         const orc_neurite_params* p, orc_body_t** B_out, double** bin_out,
                         double* L_out) {
  for (size_t a = 0; a < n; ++a) {
    if (mother[a] >= (int64_t)a || mother[a] < -1) return -1;
    if (!(diam[a] > 0.0)) return -1;
    if (mother[a] >= 0 && !(rest[a] > 0.0)) return -1;
  }
  orc_body_t* B = (orc_body_t*)malloc((n ? n : 1) * sizeof(orc_body_t));
  double* bin = (double*)malloc((n ? 3 * n : 1) * sizeof(double));
  if (!B || !bin) {
    free(B); free(bin);
    return -2;
  }
  double L = p->interaction_radius;
  for (size_t a = 0; a < n; ++a) {
    neurite_body(a, x, y, z, diam, mother, ox, oy, oz, &B[a]);
    double e = B[a].len + diam[a];
    if (e > L) L = e;
    for (int k = 0; k < 3; ++k)
      bin[3 * a + k] = mother[a] < 0 ? B[a].p[k] : 0.5 * (B[a].q[k] + B[a].p[k]);
  }
  *B_out = B;
  *bin_out = bin;
  *L_out = L;
  return 0;
}

int orc_neurite_step(size_t n, const double* x, const double* y, const double* z,
                     const double* diam, const double* rest, const int32_t* mother,
                     const double* ox, const double* oy, const double* oz,
                     const orc_neurite_params* p, double* nx, double* ny, double* nz,
                     uint32_t* nbr, double* L_out, double* fx, double* fy, double* fz) {
  if (n == 0) return 0;
  orc_body_t* B = NULL;
  double* bin = NULL;
  double L = 0.0;
  int rc = neurite_setup(n, x, y, z, diam, rest, mother, ox, oy, oz, p, &B, &bin, &L);
  if (rc) return rc;
  double* up = (double*)calloc(3 * n, sizeof(double));   /* what each element passes to its mother */
  double* own = (double*)calloc(3 * n, sizeof(double));  /* what each agent keeps                  */
  if (!up || !own) {
    free(B); free(bin); free(up); free(own);
    return -2;
  }
  const double L2 = L * L;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256)
#endif
  for (long long ii = 0; ii < (long long)n; ++ii) {
    size_t i = (size_t)ii;
    neurite_shares(n, i, B, bin, rest, p, L2, &own[3 * i], &up[3 * i], &nbr[i]);
  }
  /* daughters pass their share to the mother, taken in ascending daughter id */
  for (size_t a = 0; a < n; ++a) {
    if (mother[a] < 0) continue;
    size_t m = (size_t)mother[a];
    for (int c = 0; c < 3; ++c) own[3 * m + c] += up[3 * a + c];
  }
  for (size_t a = 0; a < n; ++a) {
    const double* S = &own[3 * a];
    if (fx) { fx[a] = S[0]; fy[a] = S[1]; fz[a] = S[2]; }
    neurite_update(x[a], y[a], z[a], S, p, &nx[a], &ny[a], &nz[a]);
  }
  if (L_out) *L_out = L;
  free(B); free(bin); free(up); free(own);
  return 0;
}

/* The same step for the m agents listed in idx only (their daughters' shares included): new
 * positions and neighbour counts of those agents, O(m N).  For checks at sizes where the full
 * O(N^2) step is out of reach. */
int orc_neurite_sample(size_t n, const double* x, const double* y, const double* z,
                       const double* diam, const double* rest, const int32_t* mother,
                       const double* ox, const double* oy, const double* oz,
                       const orc_neurite_params* p, size_t m, const int64_t* idx, double* nx,
                       double* ny, double* nz, uint32_t* nbr, double* L_out) {
  orc_body_t* B = NULL;
  double* bin = NULL;
  double L = 0.0;
  for (size_t k = 0; k < m; ++k)
    if (idx[k] < 0 || (size_t)idx[k] >= n) return -1;
  int rc = neurite_setup(n, x, y, z, diam, rest, mother, ox, oy, oz, p, &B, &bin, &L);
  if (rc) return rc;
  const double L2 = L * L;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (long long kk = 0; kk < (long long)m; ++kk) {
    size_t a = (size_t)idx[kk];
    double S[3], pass[3], kd[3], pd[3];
    uint32_t cnt = 0, cd = 0;
    neurite_shares(n, a, B, bin, rest, p, L2, S, pass, &cnt);
    for (size_t c = a + 1; c < n; ++c) {  /* daughters have larger ids */
      if (mother[c] != (int32_t)a) continue;
      neurite_shares(n, c, B, bin, rest, p, L2, kd, pd, &cd);
      for (int q = 0; q < 3; ++q) S[q] += pd[q];
    }
    neurite_update(x[a], y[a], z[a], S, p, &nx[kk], &ny[kk], &nz[kk]);
    nbr[kk] = cnt;
  }
  if (L_out) *L_out = L;
  free(B); free(bin);
  return 0;
}
