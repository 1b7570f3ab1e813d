// mbatch.cu -- served mechanics simulations advanced together: a pool of simulation slots with
// continuous admission (C ABI in include/bdm.h, "Batched mechanics").
//
// BioDynaMo (arXiv 2006.06775), Sec. "Simulation concepts": every step, every agent of a simulation
// is assigned to the uniform grid and its mechanical force is summed over the 27 boxes around it
// (readings R1-R6).  A served simulation of a few thousand agents runs each step as a dozen launches
// of a few microseconds, so launches, not the GPU, set its pace.  The pool holds `slots`
// simulations of up to `slot_capacity` agents each, at fixed places: slot s owns agents
// [s * cap, s * cap + n_s) of every per-agent array and boxes [s * boxcap, s * boxcap + nbox_s) of
// the box arrays, with its own grid (DevGrid) and constants.  Every kernel of a step covers all
// active slots at once through a work list of (slot, 256-agent tile) pairs, so a step is one
// sequence of nine launches (captured in a CUDA graph) whatever the number of simulations.  The box
// histogram of all slots is scanned in one pass; a slot's box starts are made local by subtracting
// the start of its first box, so each slot's agents stay in its own range.
//
// Each slot computes exactly what a single handle (bdm_create) computes for the same simulation:
// the same grid (grid_from_bounds), the same canonical (box, id) order, and per pair the same
// operations in the same order (one thread per agent walking its 27 boxes in ascending key, the
// contacts summed in that order, with the explicitly rounded FP32 helpers of mechcore.cuh) -- bit
// for bit on both paths.  A slot admitted with a step target advances until it reaches it; its
// state stays in place until it is read out and released.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "bdm.h"
#include "common.cuh"
#include "gridcore.cuh"
#include "mechcore.cuh"

void bdm_count_launches(unsigned long long k);  // api.cu

namespace bdm {
namespace {

constexpr int kMT = 256;  // agents per tile = threads per block

struct Slot {        // one slot's place in the pool and its progress (device copy)
  unsigned off;      // first agent
  unsigned n;        // agents (0: free)
  unsigned boff;     // first box
  unsigned active;   // 1 while steps remain
  unsigned steps;    // steps completed
  unsigned target;   // steps to run
  unsigned par;      // attribute buffer holding the slot's agents (it stays put once the slot stops)
};

struct Tile {
  unsigned slot, first;  // agents first .. first + 255 of the slot (local indices)
};

struct MbDev {
  Slot* slot;
  DevGrid* grid;
  MechConsts* consts;
  Tile* tiles;
  unsigned* ntiles;
  double *px, *py, *pz;  // centres, in the order of the last step (the force kernel writes here)
  double *sx, *sy, *sz;  // centres gathered into this step's canonical order
  float* diam[2];
  unsigned* id[2];       // ids local to the slot (0 .. n - 1, insertion order)
  float4* p4;            // mixed: FP32 offsets from the box's lower corner + radius
  unsigned *key, *rank, *perm, *skey, *nbr;
  unsigned *count, *start;
  unsigned long long* scan_tiles;
  unsigned* scan_ctr;
  unsigned* scan_items;
  unsigned* err;
  unsigned nslots, max_scan_tiles;
};

// ---- kernels (a block takes whole tiles; a tile's agents belong to one slot) ------------------

// Per-slot bounds of the centres and the largest diameter (reading R5), into the slot's grid.
__global__ void __launch_bounds__(kMT) k_mb_bounds(MbDev d, int cur) {
  const unsigned nt = *d.ntiles;
  for (unsigned tl = blockIdx.x; tl < nt; tl += gridDim.x) {
    const Tile T = d.tiles[tl];
    const Slot S = d.slot[T.slot];
    if (!S.active) continue;  // the same for the whole block
    const unsigned k = T.first + threadIdx.x;
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    unsigned md = 0;
    if (k < S.n) {
      const unsigned i = S.off + k;
      const double v[3] = {d.px[i], d.py[i], d.pz[i]};
      for (int a = 0; a < 3; ++a) {
        const unsigned long long e = enc_double(v[a]);
        mn[a] = e;
        mx[a] = e;
      }
      md = __float_as_uint(d.diam[cur][i]);
    }
    block_commit_bounds<kMT>(mn, mx, md, &d.grid[T.slot]);
    __syncthreads();  // the reduction's shared memory is read before the next tile reuses it
  }
}

// Each active slot's grid from its bounds; then the bounds are reset for the next step.  A slot
// whose grid fails (radius, extent or box capacity) stops with the error bit in its grid.
__global__ void k_mb_finalize(MbDev d) {
  const unsigned s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0) *d.scan_ctr = 0u;
  if (s >= d.nslots) return;
  Slot& S = d.slot[s];
  if (!S.active) return;
  DevGrid* g = &d.grid[s];
  g->n = S.n;
  grid_from_bounds(g, d.consts[s]);
  for (int a = 0; a < 3; ++a) {
    g->acc_min[a] = ~0ull;
    g->acc_max[a] = 0ull;
  }
  g->acc_maxdiam = 0u;
  if (!g->nbox) S.active = 0u;
}

// Box of each agent (global key = slot's first box + local key) and its arrival rank.
__global__ void __launch_bounds__(kMT) k_mb_key_hist(MbDev d) {
  const unsigned nt = *d.ntiles;
  for (unsigned tl = blockIdx.x; tl < nt; tl += gridDim.x) {
    const Tile T = d.tiles[tl];
    const Slot S = d.slot[T.slot];
    const unsigned k = T.first + threadIdx.x;
    if (!S.active || k >= S.n) continue;
    const DevGrid* g = &d.grid[T.slot];
    const unsigned i = S.off + k;
    const long long Lq = g->Lq;
    const float inv = g->invLq;
    const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
    int ix = box_div(quantise(d.px[i]) - g->O[0], Lq, inv);
    int iy = box_div(quantise(d.py[i]) - g->O[1], Lq, inv);
    int iz = box_div(quantise(d.pz[i]) - g->O[2], Lq, inv);
    if (ix >= d0 || iy >= d1 || iz >= d2) {  // impossible by construction of the bounds
      atomicOr(d.err, (unsigned)ERR_BOUNDS);
      ix = min(ix, d0 - 1);
      iy = min(iy, d1 - 1);
      iz = min(iz, d2 - 1);
    }
    const unsigned gk = S.boff + (unsigned)ix + (unsigned)d0 * ((unsigned)iy + (unsigned)d1 * (unsigned)iz);
    d.key[i] = gk;
    d.rank[i] = atomicAdd(&d.count[gk], 1u);
  }
}

// Counting-sort scatter within the slot: local slot = box start - slot's first start + rank.
__global__ void __launch_bounds__(kMT) k_mb_scatter(MbDev d) {
  const unsigned nt = *d.ntiles;
  for (unsigned tl = blockIdx.x; tl < nt; tl += gridDim.x) {
    const Tile T = d.tiles[tl];
    const Slot S = d.slot[T.slot];
    const unsigned k = T.first + threadIdx.x;
    if (!S.active || k >= S.n) continue;
    const unsigned i = S.off + k, base = d.start[S.boff];
    d.perm[S.off + (d.start[d.key[i]] - base) + d.rank[i]] = i;
  }
}

// Canonicalise and gather (reading R6): within a box ascending id; the payload moves into the
// canonical order (attributes from buffer cur to cur ^ 1), with the box key local to the slot and,
// for the mixed path, each agent's FP32 offset from its box's lower corner.
template <bool MIXED>
__global__ void __launch_bounds__(kMT) k_mb_gather(MbDev d, int cur) {
  const unsigned nt = *d.ntiles;
  for (unsigned tl = blockIdx.x; tl < nt; tl += gridDim.x) {
    const Tile T = d.tiles[tl];
    const Slot S = d.slot[T.slot];
    const unsigned kk = T.first + threadIdx.x;
    if (!S.active || kk >= S.n) continue;
    const DevGrid* g = &d.grid[T.slot];
    const unsigned base = d.start[S.boff];
    const unsigned k = S.off + kk;
    const unsigned s = d.perm[k];
    const unsigned b = d.key[s];
    const unsigned lo = d.start[b] - base + S.off, hi = d.start[b + 1] - base + S.off;
    const unsigned myid = d.id[cur][s];
    unsigned dst = lo;
    if (hi - lo > 1)
      for (unsigned m = lo; m < hi; ++m)
        if (m != k) dst += d.id[cur][d.perm[m]] < myid ? 1u : 0u;
    const double x = d.px[s], y = d.py[s], z = d.pz[s];
    const float di = d.diam[cur][s];
    const unsigned lb = b - S.boff;
    d.sx[dst] = x;
    d.sy[dst] = y;
    d.sz[dst] = z;
    d.diam[cur ^ 1][dst] = di;
    d.id[cur ^ 1][dst] = myid;
    d.skey[dst] = lb;
    if (MIXED) {
      const unsigned d0 = (unsigned)g->dims[0], d1 = (unsigned)g->dims[1];
      const long long Lq = g->Lq;
      const unsigned ix = lb % d0, t = lb / d0;
      const unsigned iy = t % d1, iz = t / d1;
      const float ox = (float)(int)(quantise(x) - g->O[0] - (long long)ix * Lq) * kQInv;
      const float oy = (float)(int)(quantise(y) - g->O[1] - (long long)iy * Lq) * kQInv;
      const float oz = (float)(int)(quantise(z) - g->O[2] - (long long)iz * Lq) * kQInv;
      d.p4[dst] = make_float4(ox, oy, oz, 0.5f * di);
    }
  }
}

// Force + capped update, one thread per agent in canonical order: the nine row runs of its 27 boxes
// in ascending key, each run's agents in canonical order.  FP64: the single handle's FP64 pair
// (explicitly rounded intrinsics in the oracle's order), contacts summed in candidate order.  Mixed:
// FP32 d^2 from the box-relative offsets, the count exact (FP32 outside the +-2^-12 band around R^2,
// the oracle's FP64 expression inside it), contact_force in candidate order, then the FP64 centre
// += the capped FP32 displacement.  The new centres go to (px, py, pz) in canonical order.
template <bool MIXED>
__global__ void __launch_bounds__(kMT) k_mb_force(MbDev d, int cur) {
  const unsigned nt = *d.ntiles;
  for (unsigned tl = blockIdx.x; tl < nt; tl += gridDim.x) {
    const Tile T = d.tiles[tl];
    const Slot S = d.slot[T.slot];
    const unsigned kk = T.first + threadIdx.x;
    if (!S.active || kk >= S.n) continue;
    const DevGrid* g = &d.grid[T.slot];
    const MechConsts c = d.consts[T.slot];
    const unsigned base = d.start[S.boff], i = S.off + kk;
    const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
    const unsigned lb = d.skey[i];
    const int ix = (int)(lb % (unsigned)d0);
    const unsigned q0 = lb / (unsigned)d0;
    const int iy = (int)(q0 % (unsigned)d1), iz = (int)(q0 / (unsigned)d1);
    const int xl = ix > 0 ? ix - 1 : 0, xh = ix + 1 < d0 ? ix + 1 : ix;
    const double xi = d.sx[i], yi = d.sy[i], zi = d.sz[i];
    const double R2 = g->R2;
    unsigned cnt = 0;
    double nx, ny, nz;
    if (!MIXED) {
      const double ri = 0.5 * (double)d.diam[cur][i];
      double Sx = 0.0, Sy = 0.0, Sz = 0.0;
      for (int sg = 0; sg < 9; ++sg) {
        const int jz = iz + sg / 3 - 1, jy = iy + sg % 3 - 1;
        if (jz < 0 || jz >= d2 || jy < 0 || jy >= d1) continue;
        const unsigned row = S.boff + ((unsigned)jz * (unsigned)d1 + (unsigned)jy) * (unsigned)d0;
        const unsigned a = d.start[row + xl] - base + S.off, e = d.start[row + xh + 1] - base + S.off;
        for (unsigned j = a; j < e; ++j) {
          if (j == i) continue;
          const double ax = __dsub_rn(xi, d.sx[j]), ay = __dsub_rn(yi, d.sy[j]), az = __dsub_rn(zi, d.sz[j]);
          const double e2 =
              __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
          cnt += e2 < R2 ? 1u : 0u;
          const double dd = __dsqrt_rn(e2);
          const double rj = 0.5 * (double)d.diam[cur][j];
          const double delta = __dsub_rn(__dadd_rn(ri, rj), dd);
          if (delta > 0.0 && dd > 0.0) {
            const double rho = __ddiv_rn(__dmul_rn(ri, rj), __dadd_rn(ri, rj));
            const double F = __dsub_rn(__dmul_rn(c.k, delta),
                                       __dmul_rn(c.gamma, __dsqrt_rn(__dmul_rn(rho, delta))));
            const double sc = __ddiv_rn(F, dd);
            Sx = __dadd_rn(Sx, __dmul_rn(sc, ax));
            Sy = __dadd_rn(Sy, __dmul_rn(sc, ay));
            Sz = __dadd_rn(Sz, __dmul_rn(sc, az));
          }
        }
      }
      double Dx = __dmul_rn(c.dt, Sx), Dy = __dmul_rn(c.dt, Sy), Dz = __dmul_rn(c.dt, Sz);
      double nrm = __dadd_rn(__dmul_rn(Dx, Dx), __dmul_rn(Dy, Dy));
      nrm = __dsqrt_rn(__dadd_rn(nrm, __dmul_rn(Dz, Dz)));
      if (nrm > c.cap) {
        const double f = __ddiv_rn(c.cap, nrm);
        Dx = __dmul_rn(Dx, f);
        Dy = __dmul_rn(Dy, f);
        Dz = __dmul_rn(Dz, f);
      }
      nx = __dadd_rn(xi, Dx);
      ny = __dadd_rn(yi, Dy);
      nz = __dadd_rn(zi, Dz);
    } else {
      const float Lf = g->Lf, R2lo = g->R2lo, R2hi = g->R2hi;
      const float4 pi = d.p4[i];
      const float pxm = pi.x + Lf, px0 = pi.x, pxp = pi.x - Lf;  // neighbour box at x-1, x, x+1
      float Fx = 0.f, Fy = 0.f, Fz = 0.f;
      for (int sg = 0; sg < 9; ++sg) {
        const int jz = iz + sg / 3 - 1, jy = iy + sg % 3 - 1;
        if (jz < 0 || jz >= d2 || jy < 0 || jy >= d1) continue;
        const unsigned row = S.boff + ((unsigned)jz * (unsigned)d1 + (unsigned)jy) * (unsigned)d0;
        const unsigned a = d.start[row + xl] - base + S.off;
        const unsigned m1 = ix > 0 ? d.start[row + ix] - base + S.off : a;  // end of box x-1
        const unsigned m2 = d.start[row + ix + 1] - base + S.off;           // end of box x
        const unsigned e = d.start[row + xh + 1] - base + S.off;            // end of the run
        const float py = pi.y - (float)(sg % 3 - 1) * Lf, pz = pi.z - (float)(sg / 3 - 1) * Lf;
        for (unsigned j = a; j < e; ++j) {
          const float4 q = d.p4[j];
          const unsigned bx = j < m1 ? 0u : (j < m2 ? 1u : 2u);
          const float ex = (bx == 0 ? pxm : (bx == 1 ? px0 : pxp)) - q.x;
          const float ey = py - q.y;
          const float ez = pz - q.z;
          const float dd = pair_d2(ex, ey, ez);
          if (dd < R2lo) ++cnt;
          else if (dd <= R2hi) cnt += fp64_within(i, j, d.sx, d.sy, d.sz, R2);
          const float rs = pi.w + q.w;
          if (dd < rs * rs && dd > 0.f) contact_force(Fx, Fy, Fz, ex, ey, ez, pi.w, q.w, c.kf, c.gammaf);
        }
      }
      cnt -= 1u;  // the agent itself
      float Dx, Dy, Dz;
      capped_displacement(Fx, Fy, Fz, c.dtf, c.capf, Dx, Dy, Dz);
      nx = __dadd_rn(xi, f2d_exact(Dx));
      ny = __dadd_rn(yi, f2d_exact(Dy));
      nz = __dadd_rn(zi, f2d_exact(Dz));
    }
    d.px[i] = nx;
    d.py[i] = ny;
    d.pz[i] = nz;
    d.nbr[i] = cnt;
  }
}

// One step done for every active slot (its attributes are now in buffer `written`); a slot
// reaching its target stops.
__global__ void k_mb_step_done(MbDev d, int written) {
  const unsigned s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= d.nslots) return;
  Slot& S = d.slot[s];
  if (!S.active) return;
  S.par = (unsigned)written;
  S.steps += 1u;
  d.grid[s].step += 1ull;
  if (S.steps >= S.target) S.active = 0u;
}

// Upload of a slot's agents: validate, dense ids 0 .. n - 1, cleared outputs.
__global__ void __launch_bounds__(kMT) k_mb_prepare(MbDev d, unsigned slot, int cur) {
  const Slot S = d.slot[slot];
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < S.n; k += gridDim.x * blockDim.x) {
    const unsigned i = S.off + k;
    const double x = d.px[i], y = d.py[i], z = d.pz[i];
    const float dm = d.diam[cur][i];
    if (!(dm > 0.f && fabs(x) < 1e9 && fabs(y) < 1e9 && fabs(z) < 1e9))  // NaN fails
      atomicOr(&d.grid[slot].err, (unsigned)ERR_BOUNDS);
    d.id[cur][i] = k;
    d.nbr[i] = 0u;
    d.skey[i] = 0u;
  }
}

// Read-out of one slot in id order into the gathered-centre buffers at the slot's offset.
__global__ void __launch_bounds__(kMT) k_mb_unsort(MbDev d, unsigned slot, float* odiam,
                                                   unsigned* onbr, unsigned* obox) {
  const Slot S = d.slot[slot];
  const int cur = (int)S.par;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < S.n; k += gridDim.x * blockDim.x) {
    const unsigned i = S.off + k, id = d.id[cur][i];
    if (id >= S.n) {
      atomicOr(d.err, (unsigned)ERR_BOUNDS);
      continue;
    }
    d.sx[S.off + id] = d.px[i];
    d.sy[S.off + id] = d.py[i];
    d.sz[S.off + id] = d.pz[i];
    odiam[S.off + id] = d.diam[cur][i];
    onbr[S.off + id] = d.nbr[i];
    obox[S.off + id] = d.skey[i];
  }
}

}  // namespace
}  // namespace bdm

using namespace bdm;

struct bdm_mbatch {
  int precision = BDM_MIXED;
  unsigned slots = 0;
  size_t cap = 0, boxcap = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  std::vector<void*> allocs;
  MbDev dev{};
  std::vector<Slot> hslot;          // host view of the slots
  std::vector<DevGrid> hgrid;
  Slot* pin_slot = nullptr;         // pinned staging
  DevGrid* pin_grid = nullptr;
  int cur = 0;                      // attribute buffer holding the agents
  int blocks = 0;
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;  // (steps, attribute parity)
};

namespace {

int mfail(bdm_mbatch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  return code;
}

#define MCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return mfail(b, BDM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

template <typename T>
int malloc_n(bdm_mbatch* b, T** p, size_t n) {
  const size_t bytes = std::max<size_t>(256, (n * sizeof(T) + 255) & ~size_t(255));
  void* q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return mfail(b, BDM_ENOMEM, "device allocation of %zu bytes failed", bytes);
  }
  b->allocs.push_back(q);
  *p = (T*)q;
  return BDM_OK;
}

int upload_tiles(bdm_mbatch* b) {
  std::vector<Tile> tiles;
  for (unsigned s = 0; s < b->slots; ++s)
    for (unsigned f = 0; f < b->hslot[s].n; f += kMT) tiles.push_back(Tile{s, f});
  const unsigned nt = (unsigned)tiles.size();
  if (nt) MCK(cudaMemcpyAsync(b->dev.tiles, tiles.data(), sizeof(Tile) * nt, cudaMemcpyHostToDevice, b->stream));
  MCK(cudaMemcpyAsync(b->dev.ntiles, &nt, sizeof(unsigned), cudaMemcpyHostToDevice, b->stream));
  MCK(cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
  return BDM_OK;
}

int enqueue_step(bdm_mbatch* b) {
  cudaStream_t s = b->stream;
  MbDev& D = b->dev;
  const int cur = b->cur;
  const unsigned sb = (b->slots + 127) / 128;
  k_mb_bounds<<<b->blocks, kMT, 0, s>>>(D, cur);
  k_mb_finalize<<<sb, 128, 0, s>>>(D);
  MCK(cudaMemsetAsync(D.scan_tiles, 0, sizeof(unsigned long long) * D.max_scan_tiles, s));
  k_mb_key_hist<<<b->blocks, kMT, 0, s>>>(D);
  launch_scan(s, D.count, D.start, D.scan_items, D.scan_tiles, D.scan_ctr, D.err, 1, b->blocks);
  k_mb_scatter<<<b->blocks, kMT, 0, s>>>(D);
  if (b->precision == BDM_MIXED) {
    k_mb_gather<true><<<b->blocks, kMT, 0, s>>>(D, cur);
    k_mb_force<true><<<b->blocks, kMT, 0, s>>>(D, cur ^ 1);
  } else {
    k_mb_gather<false><<<b->blocks, kMT, 0, s>>>(D, cur);
    k_mb_force<false><<<b->blocks, kMT, 0, s>>>(D, cur ^ 1);
  }
  k_mb_step_done<<<sb, 128, 0, s>>>(D, cur ^ 1);
  b->cur ^= 1;
  MCK(cudaGetLastError());
  return BDM_OK;
}

constexpr unsigned long long kMbLaunchesPerStep = 9;

bool valid_slot_params(const bdm_params* p, int precision) {
  return p && p->struct_size == sizeof(bdm_params) && p->kind == BDM_MECHANICS &&
         p->precision == precision && p->skin == 0.0 && !p->growth_enabled && !p->diffusion_enabled &&
         p->brownian_sigma == 0.0 && p->p_apoptosis == 0.0 && p->chemotaxis == 0.0 &&
         std::isfinite(p->dt) && p->dt >= 0.0 && std::isfinite(p->max_displacement) &&
         p->max_displacement >= 0.0 && std::isfinite(p->repulsion) && p->repulsion >= 0.0 &&
         std::isfinite(p->attraction) && p->attraction >= 0.0 && p->interaction_radius >= 0.0 &&
         p->box_length >= 0.0 &&
         (p->box_length == 0.0 || p->interaction_radius == 0.0 || p->box_length >= p->interaction_radius);
}

}  // namespace

extern "C" {

int bdm_mbatch_create(int precision, int slots, size_t slot_capacity, void* stream, bdm_mbatch** out) {
  if (!out) return BDM_EINVAL;
  *out = nullptr;
  bdm_mbatch* b = new (std::nothrow) bdm_mbatch();
  if (!b) return BDM_ENOMEM;
  *out = b;
  if ((precision != BDM_FP64 && precision != BDM_MIXED) || slots <= 0 || slot_capacity == 0 ||
      (unsigned long long)slots * slot_capacity > 0x7FFFFFFFull)
    return mfail(b, BDM_EINVAL, "precision must be BDM_FP64 or BDM_MIXED, slots and capacity positive, "
                                "slots x capacity below 2^31");
  b->precision = precision;
  b->slots = (unsigned)slots;
  b->cap = slot_capacity;
  b->boxcap = 2 * slot_capacity + 4096;
  if ((unsigned long long)slots * b->boxcap + 1 > 0xF0000000ull)
    return mfail(b, BDM_EINVAL, "slots x box capacity exceeds 32-bit box indices");
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return mfail(b, BDM_ECUDA, "cudaStreamCreate failed (no CUDA device?)");
    }
    b->own_stream = true;
  }
  const size_t A = (size_t)slots * slot_capacity, Bx = (size_t)slots * b->boxcap + 1;
  MbDev& D = b->dev;
  int rc;
  if ((rc = malloc_n(b, &D.slot, b->slots)) || (rc = malloc_n(b, &D.grid, b->slots)) ||
      (rc = malloc_n(b, &D.consts, b->slots)) ||
      (rc = malloc_n(b, &D.tiles, (size_t)slots * ((slot_capacity + kMT - 1) / kMT))) ||
      (rc = malloc_n(b, &D.ntiles, 1)) || (rc = malloc_n(b, &D.px, A)) || (rc = malloc_n(b, &D.py, A)) ||
      (rc = malloc_n(b, &D.pz, A)) || (rc = malloc_n(b, &D.sx, A)) || (rc = malloc_n(b, &D.sy, A)) ||
      (rc = malloc_n(b, &D.sz, A)) || (rc = malloc_n(b, &D.diam[0], A)) || (rc = malloc_n(b, &D.diam[1], A)) ||
      (rc = malloc_n(b, &D.id[0], A)) || (rc = malloc_n(b, &D.id[1], A)) ||
      (rc = malloc_n(b, &D.key, A)) || (rc = malloc_n(b, &D.rank, A)) || (rc = malloc_n(b, &D.perm, A)) ||
      (rc = malloc_n(b, &D.skey, A)) || (rc = malloc_n(b, &D.nbr, A)) || (rc = malloc_n(b, &D.count, Bx)) ||
      (rc = malloc_n(b, &D.start, Bx)) || (rc = malloc_n(b, &D.scan_ctr, 1)) ||
      (rc = malloc_n(b, &D.scan_items, 1)) || (rc = malloc_n(b, &D.err, 1)))
    return rc;
  if (precision == BDM_MIXED && (rc = malloc_n(b, &D.p4, A))) return rc;
  D.max_scan_tiles = (unsigned)((Bx + kScanTile - 1) / kScanTile + 1);
  if ((rc = malloc_n(b, &D.scan_tiles, D.max_scan_tiles))) return rc;
  D.nslots = b->slots;
  b->hslot.assign(b->slots, Slot{});
  b->hgrid.assign(b->slots, DevGrid{});
  for (unsigned s = 0; s < b->slots; ++s) {
    b->hslot[s].off = (unsigned)(s * slot_capacity);
    b->hslot[s].boff = (unsigned)(s * b->boxcap);
  }
  MCK(cudaMallocHost((void**)&b->pin_slot, sizeof(Slot) * b->slots));
  MCK(cudaMallocHost((void**)&b->pin_grid, sizeof(DevGrid)));
  cudaStream_t s = b->stream;
  const unsigned items = (unsigned)Bx, zero = 0;
  MCK(cudaMemcpyAsync(D.slot, b->hslot.data(), sizeof(Slot) * b->slots, cudaMemcpyHostToDevice, s));
  MCK(cudaMemsetAsync(D.grid, 0, sizeof(DevGrid) * b->slots, s));
  MCK(cudaMemsetAsync(D.count, 0, sizeof(unsigned) * Bx, s));
  MCK(cudaMemsetAsync(D.start, 0, sizeof(unsigned) * Bx, s));
  MCK(cudaMemcpyAsync(D.scan_items, &items, sizeof(unsigned), cudaMemcpyHostToDevice, s));
  MCK(cudaMemcpyAsync(D.ntiles, &zero, sizeof(unsigned), cudaMemcpyHostToDevice, s));
  MCK(cudaMemsetAsync(D.err, 0, sizeof(unsigned), s));
  MCK(cudaStreamSynchronize(s));
  int dev = 0, sms = 0;
  MCK(cudaGetDevice(&dev));
  MCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  b->blocks = sms * 8;
  return BDM_OK;
}

int bdm_mbatch_load(bdm_mbatch* b, int slot, const bdm_params* p, size_t n, const double* x,
                    const double* y, const double* z, const float* diameter, int steps) {
  if (!b) return BDM_EINVAL;
  if (slot < 0 || (unsigned)slot >= b->slots) return mfail(b, BDM_EINVAL, "no slot %d", slot);
  if (b->hslot[slot].n) return mfail(b, BDM_ESTATE, "slot %d is occupied", slot);
  if (!valid_slot_params(p, b->precision))
    return mfail(b, BDM_EINVAL, "slot %d: parameters must be plain mechanics of the pool's precision "
                                "(no skin, growth, diffusion or oncology behaviours)", slot);
  if (n == 0 || n > b->cap) return mfail(b, BDM_EINVAL, "slot %d: %zu agents (1 .. %zu)", slot, n, b->cap);
  if (!x || !y || !z || !diameter) return mfail(b, BDM_EINVAL, "NULL agent arrays");
  if (steps < 0) return mfail(b, BDM_EINVAL, "negative step count");
  cudaStream_t s = b->stream;
  MbDev& D = b->dev;
  Slot& S = b->hslot[slot];
  const size_t off = S.off;
  MCK(cudaMemcpyAsync(D.px + off, x, n * sizeof(double), cudaMemcpyHostToDevice, s));
  MCK(cudaMemcpyAsync(D.py + off, y, n * sizeof(double), cudaMemcpyHostToDevice, s));
  MCK(cudaMemcpyAsync(D.pz + off, z, n * sizeof(double), cudaMemcpyHostToDevice, s));
  MCK(cudaMemcpyAsync(D.diam[b->cur] + off, diameter, n * sizeof(float), cudaMemcpyHostToDevice, s));
  S.n = (unsigned)n;
  S.active = steps > 0 ? 1u : 0u;
  S.steps = 0;
  S.target = (unsigned)steps;
  S.par = (unsigned)b->cur;
  DevGrid G{};
  for (int a = 0; a < 3; ++a) G.acc_min[a] = ~0ull;
  G.nbox1 = 1;
  G.n = (unsigned)n;
  b->hgrid[slot] = G;
  MechConsts c{};
  c.dt = p->dt;
  c.k = p->repulsion;
  c.gamma = p->attraction;
  c.cap = p->max_displacement;
  c.dtf = (float)p->dt;
  c.kf = (float)p->repulsion;
  c.gammaf = (float)p->attraction;
  c.capf = (float)p->max_displacement;
  c.interaction_radius = p->interaction_radius;
  c.box_length = p->box_length;
  c.box_capacity = (unsigned)b->boxcap;
  c.capacity = (unsigned)b->cap;
  c.skin = 0.0;
  c.max_cadence = 1;
  c.mixed = b->precision == BDM_MIXED ? 1 : 0;
  *b->pin_slot = S;
  *b->pin_grid = G;
  MCK(cudaMemcpyAsync(D.slot + slot, b->pin_slot, sizeof(Slot), cudaMemcpyHostToDevice, s));
  MCK(cudaMemcpyAsync(D.grid + slot, b->pin_grid, sizeof(DevGrid), cudaMemcpyHostToDevice, s));
  MCK(cudaMemcpyAsync(D.consts + slot, &c, sizeof(MechConsts), cudaMemcpyHostToDevice, s));
  k_mb_prepare<<<std::max<int>(1, std::min<int>(b->blocks, (int)((n + kMT - 1) / kMT))), kMT, 0, s>>>(D, (unsigned)slot, b->cur);
  MCK(cudaGetLastError());
  bdm_count_launches(1);
  MCK(cudaStreamSynchronize(s));  // the caller's arrays and the staging are free again
  MCK(cudaMemcpy(b->pin_grid, D.grid + slot, sizeof(DevGrid), cudaMemcpyDeviceToHost));
  if (b->pin_grid->err) {
    S = Slot{S.off, 0, S.boff, 0, 0, 0, 0};
    *b->pin_slot = S;
    MCK(cudaMemcpy(D.slot + slot, b->pin_slot, sizeof(Slot), cudaMemcpyHostToDevice));
    return mfail(b, BDM_EINVAL, "slot %d: diameters must be > 0 and |position| < 1e9", slot);
  }
  return upload_tiles(b);
}

int bdm_mbatch_step(bdm_mbatch* b, int n) {
  if (!b) return BDM_EINVAL;
  if (n < 0) return mfail(b, BDM_EINVAL, "negative step count");
  if (n == 0) return BDM_OK;
  const auto key = std::make_pair(n, b->cur);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    const int c0 = b->cur;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    MCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = BDM_OK;
    for (int k = 0; k < n && rc == BDM_OK; ++k) rc = enqueue_step(b);
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
    b->cur = c0;
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ce != cudaSuccess) return mfail(b, BDM_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return mfail(b, BDM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
    it = b->graphs.emplace(key, exec).first;
  }
  MCK(cudaGraphLaunch(it->second, b->stream));
  bdm_count_launches(kMbLaunchesPerStep * (unsigned long long)n);
  b->cur ^= (n & 1);
  return BDM_OK;
}

int bdm_mbatch_poll(bdm_mbatch* b, int32_t* steps_done) {
  if (!b) return BDM_EINVAL;
  MCK(cudaMemcpyAsync(b->pin_slot, b->dev.slot, sizeof(Slot) * b->slots, cudaMemcpyDeviceToHost, b->stream));
  MCK(cudaStreamSynchronize(b->stream));
  for (unsigned s = 0; s < b->slots; ++s) {
    b->hslot[s].steps = b->pin_slot[s].steps;
    b->hslot[s].active = b->pin_slot[s].active;
    if (steps_done) steps_done[s] = b->hslot[s].n ? (int32_t)b->pin_slot[s].steps : -1;
  }
  return BDM_OK;
}

int bdm_mbatch_get_state(bdm_mbatch* b, int slot, bdm_state* st) {
  if (!b || !st) return BDM_EINVAL;
  if (st->struct_size != sizeof(bdm_state)) return mfail(b, BDM_EINVAL, "state.struct_size mismatch");
  if (slot < 0 || (unsigned)slot >= b->slots) return mfail(b, BDM_EINVAL, "no slot %d", slot);
  const Slot S = b->hslot[slot];
  cudaStream_t s = b->stream;
  MbDev& D = b->dev;
  MCK(cudaMemcpyAsync(b->pin_grid, D.grid + slot, sizeof(DevGrid), cudaMemcpyDeviceToHost, s));
  MCK(cudaMemcpyAsync(b->pin_slot + slot, D.slot + slot, sizeof(Slot), cudaMemcpyDeviceToHost, s));
  MCK(cudaStreamSynchronize(s));
  const DevGrid& G = *b->pin_grid;
  if (G.err & ERR_GRID_OVERFLOW)
    return mfail(b, BDM_ENOMEM, "slot %d: grid needs more boxes than the slot holds", slot);
  if (G.err) return mfail(b, BDM_ESTATE, "slot %d: invalid grid (error bits 0x%x)", slot, G.err);
  st->n = S.n;
  st->step = b->pin_slot[slot].steps;
  st->mass_total = 0.0;
  for (int k = 0; k < 3; ++k) {
    st->sir_counts[k] = 0;
    st->grid_origin_q[k] = G.O[k];
    st->grid_dims[k] = G.dims[k];
  }
  st->grid_box_q = G.Lq;
  st->grid_rebuilds = (uint32_t)b->pin_slot[slot].steps;
  st->list_entries = 0;
  st->stationary_skipped = 0;
  if (S.n && (st->x || st->y || st->z || st->diameter || st->neighbour_count || st->box_id)) {
    float* odiam = (float*)D.rank;  // scratch of the pool's size, free between steps
    unsigned* onbr = D.key;
    unsigned* obox = D.perm;
    k_mb_unsort<<<std::max<int>(1, std::min<int>(b->blocks, (int)((S.n + kMT - 1) / kMT))), kMT, 0, s>>>(
        D, (unsigned)slot, odiam, onbr, obox);
    MCK(cudaGetLastError());
    bdm_count_launches(1);
    const size_t off = S.off, n = S.n;
    if (st->x) MCK(cudaMemcpyAsync(st->x, D.sx + off, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (st->y) MCK(cudaMemcpyAsync(st->y, D.sy + off, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (st->z) MCK(cudaMemcpyAsync(st->z, D.sz + off, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (st->diameter) MCK(cudaMemcpyAsync(st->diameter, odiam + off, n * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (st->neighbour_count)
      MCK(cudaMemcpyAsync(st->neighbour_count, onbr + off, n * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    if (st->box_id) MCK(cudaMemcpyAsync(st->box_id, obox + off, n * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
    unsigned e = 0;
    MCK(cudaMemcpy(&e, D.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (e) return mfail(b, BDM_ESTATE, "device index check failed (error bits 0x%x)", e);
  }
  return BDM_OK;
}

int bdm_mbatch_release(bdm_mbatch* b, int slot) {
  if (!b) return BDM_EINVAL;
  if (slot < 0 || (unsigned)slot >= b->slots) return mfail(b, BDM_EINVAL, "no slot %d", slot);
  Slot& S = b->hslot[slot];
  S.n = 0;
  S.active = 0;
  S.steps = S.target = 0;
  *b->pin_slot = S;
  MCK(cudaMemcpyAsync(b->dev.slot + slot, b->pin_slot, sizeof(Slot), cudaMemcpyHostToDevice, b->stream));
  return upload_tiles(b);  // synchronises: the staging is free again
}

void bdm_mbatch_destroy(bdm_mbatch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  for (void* q : b->allocs) cudaFree(q);
  if (b->pin_slot) cudaFreeHost(b->pin_slot);
  if (b->pin_grid) cudaFreeHost(b->pin_grid);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  cudaGetLastError();
  delete b;
}

const char* bdm_mbatch_last_error(const bdm_mbatch* b) { return b ? b->err.c_str() : "NULL handle"; }

}  // extern "C"
