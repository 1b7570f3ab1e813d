// sir.cu -- random-walk SIR model (BioDynaMo, arXiv 2006.06775, Sec. "Epidemiology use case": a
// susceptible person becomes infected with the infection probability when an infected person is
// within the infection radius; an infected person recovers with the recovery probability each
// step; every person moves randomly by a bounded distance; an operation counts S, I and R).
// Reading R10: synchronous integer step on a 2^-10 um lattice, periodic cube, Philox4x32-10 keyed
// by (seed, run) with counters (id, step, stream, 0).
//
// Agents stay in id order and are updated in place.  A step is:
//   scan     exclusive scan of the box histogram (built by the previous step's update)
//   index    agents into box order (perm); infected agents into a compact source list
//   push     every infected agent visits the agents of its 27 boxes and adds 1 to the infected-
//            neighbour count of each one within the radius (minimum image)
//   update   infection / recovery / move of every agent from its count, and the next step's box,
//            rank and histogram entry
// Only the few infected agents search the grid, so the per-agent work is a handful of streaming
// accesses and two Philox blocks.  The counts are integer sums, so the order of the atomic
// additions does not matter and every result equals the pull-form definition exactly.  One run
// uses four kernels per step; a batch of runs uses ONE persistent kernel per step whose phases
// are separated by a bounded grid barrier.
#include "common.cuh"
#include "scan.cuh"
#include "sir.cuh"

namespace bdm {

// floor(X / Lb) for 0 <= X < L < 2^31 and at most 1625 boxes per axis: the float estimate is within
// one of the quotient (relative error ~3 * 2^-24), one integer comparison makes it exact.
__device__ __forceinline__ int box_coord(int X, const SirRun& r) {
  int q = __float2int_rz(__int2float_rn(X) * r.invLb);
  const int t = q * r.Lb;
  if (t > X) --q;
  else if (X - t >= r.Lb) ++q;
  return q;
}

__device__ __forceinline__ unsigned sir_box(int X, int Y, int Z, const SirRun& r) {
  return (unsigned)box_coord(X, r) +
         (unsigned)r.nb * ((unsigned)box_coord(Y, r) + (unsigned)r.nb * (unsigned)box_coord(Z, r));
}

// Distinct periodic neighbours {c, c+1, c-1} of box coordinate c on an axis of nb boxes.
__device__ __forceinline__ int neighbour_boxes(int c, int nb, int out[3]) {
  if (nb == 1) {
    out[0] = 0;
    return 1;
  }
  out[0] = c;
  out[1] = (c + 1) % nb;
  if (nb == 2) return 2;
  out[2] = (c + nb - 1) % nb;
  return 3;
}

// The x-neighbours of box coordinate c as at most two half-open runs of consecutive boxes.
__device__ __forceinline__ int neighbour_runs(int c, int nb, int lo[2], int hi[2]) {
  if (nb <= 3) {
    lo[0] = 0;
    hi[0] = nb;
    return 1;
  }
  if (c == 0) {
    lo[0] = 0, hi[0] = 2;
    lo[1] = nb - 1, hi[1] = nb;
    return 2;
  }
  if (c == nb - 1) {
    lo[0] = 0, hi[0] = 1;
    lo[1] = nb - 2, hi[1] = nb;
    return 2;
  }
  lo[0] = c - 1;
  hi[0] = c + 2;
  return 1;
}

__device__ __forceinline__ long long min_image(long long d, long long L) {
  if (d > L / 2) d -= L;
  else if (d < -(L / 2)) d += L;
  return d;
}

// index phase for agent p of run ri (every lane of the warp calls; `valid` masks padding): place p
// in box order, clear its count, and append it to the source list if infected.  The bounds keep a
// step whose scan or barrier was cut short by a timeout inside the arrays.
__device__ __forceinline__ void sir_index(unsigned p, bool valid, unsigned ri, const SirState a,
                                          const unsigned* __restrict__ kn,
                                          const unsigned* __restrict__ rk,
                                          const unsigned* __restrict__ start,
                                          unsigned* __restrict__ perm, unsigned* __restrict__ ninf,
                                          uint2* __restrict__ src, unsigned* nsrc, unsigned total) {
  bool inf = false;
  if (valid) {
    const unsigned d = start[kn[p]] + rk[p];
    if (d < total) perm[d] = p;
    ninf[p] = 0u;
    inf = a.st[p] == 1;
  }
  const unsigned m = __ballot_sync(0xFFFFFFFFu, inf);
  if (m) {
    const unsigned lane = threadIdx.x & 31u;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(nsrc, (unsigned)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    const unsigned k = base + (unsigned)__popc(m & ((1u << lane) - 1u));
    if (inf && k < total) src[k] = make_uint2(p, ri);
  }
}

// push phase for infected agent j of run r.
__device__ __forceinline__ void sir_push(unsigned j, const SirRun& r, const SirState a,
                                         const unsigned* __restrict__ start,
                                         const unsigned* __restrict__ perm,
                                         unsigned* __restrict__ ninf, unsigned total) {
  const int Xj = a.X[j], Yj = a.Y[j], Zj = a.Z[j];
  const long long L = r.L;
  const int nb = r.nb;
  int cy[3], cz[3], xlo[2], xhi[2];
  const int ny = neighbour_boxes(box_coord(Yj, r), nb, cy);
  const int nz = neighbour_boxes(box_coord(Zj, r), nb, cz);
  const int nr = neighbour_runs(box_coord(Xj, r), nb, xlo, xhi);
  for (int qz = 0; qz < nz; ++qz)
    for (int qy = 0; qy < ny; ++qy) {
      const unsigned row = r.box_off + (unsigned)nb * ((unsigned)cy[qy] + (unsigned)nb * (unsigned)cz[qz]);
      for (int k = 0; k < nr; ++k) {
        const unsigned m0 = start[row + (unsigned)xlo[k]];
        const unsigned m1 = min(start[row + (unsigned)xhi[k]], total);
        for (unsigned m = m0; m < m1; ++m) {
          const unsigned i = perm[m];
          if (i == j || i >= total) continue;
          const long long dx = min_image((long long)a.X[i] - Xj, L);
          const long long dy = min_image((long long)a.Y[i] - Yj, L);
          const long long dz = min_image((long long)a.Z[i] - Zj, L);
          if (dx * dx + dy * dy + dz * dz < r.r2) atomicAdd(&ninf[i], 1u);
        }
      }
    }
}

// Infection, recovery and move of agent p of run r from its infected-neighbour count `cnt`; writes
// the new position and state in place and returns the state.
__device__ __forceinline__ unsigned char sir_advance(unsigned p, const SirRun& r, SirState a,
                                                     unsigned cnt, unsigned step, int NP[3]) {
  const int P[3] = {a.X[p], a.Y[p], a.Z[p]};
  const unsigned char si = a.st[p];
  const unsigned id = p - r.agent_off;
  unsigned char ns = si;
  if ((si == 0 && cnt > 0) || si == 1) {  // the only cases in which this draw decides anything
    const uint4 w = philox10(make_uint4(id, step, 0u, 0u), r.key);
    if (si == 0 && (unsigned long long)w.x < r.thr_inf) ns = 1;
    if (si == 1 && (unsigned long long)w.y < r.thr_rec) ns = 2;
  }
  const uint4 mv = philox10(make_uint4(id, step, 1u, 0u), r.key);
  const unsigned W[3] = {mv.x, mv.y, mv.z};
  const long long L = r.L;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    long long v = (long long)P[k] + ((long long)(((unsigned long long)W[k] * r.span) >> 32) - r.s);
    if (v < 0) v += L;
    else if (v >= L) v -= L;
    NP[k] = (int)v;
  }
  a.X[p] = NP[0];
  a.Y[p] = NP[1];
  a.Z[p] = NP[2];
  a.st[p] = ns;
  return ns;
}

// update phase for agent p of run r: draws, move, read-outs, next box / rank / histogram entry.
__device__ __forceinline__ unsigned char sir_update(unsigned p, const SirRun& r, SirState a,
                                                    const unsigned* __restrict__ ninf,
                                                    unsigned* __restrict__ box,
                                                    unsigned* __restrict__ kn,
                                                    unsigned* __restrict__ rk,
                                                    unsigned* __restrict__ count, unsigned step) {
  int NP[3];
  const unsigned char ns = sir_advance(p, r, a, ninf[p], step, NP);
  box[p] = kn[p];
  const unsigned b2 = r.box_off + sir_box(NP[0], NP[1], NP[2], r);
  kn[p] = b2;
  rk[p] = atomicAdd(&count[b2], 1u);
  return ns;
}

// Per-block S/I/R sums committed with three atomics (all threads call; `valid` masks padding).
__device__ __forceinline__ void commit_counts(unsigned char ns, bool valid, unsigned* dst) {
  __shared__ unsigned s_c[3];
  if (threadIdx.x < 3) s_c[threadIdx.x] = 0;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31;
  for (int c = 0; c < 3; ++c) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, valid && ns == c);
    if (lane == 0 && m) atomicAdd(&s_c[c], (unsigned)__popc(m));
  }
  __syncthreads();
  if (threadIdx.x < 3 && s_c[threadIdx.x]) atomicAdd(&dst[threadIdx.x], s_c[threadIdx.x]);
}

// ---- one run: [init] ; scan -> index -> push -> update ---------------------------------------
__global__ void __launch_bounds__(kBlock) k_sir_init(SirState a, unsigned* __restrict__ kn,
                                                     unsigned* __restrict__ rk,
                                                     unsigned* __restrict__ box,
                                                     unsigned* __restrict__ count, SirRun r,
                                                     unsigned lo, unsigned hi) {
  for (unsigned p = lo + blockIdx.x * blockDim.x + threadIdx.x; p < hi; p += gridDim.x * blockDim.x) {
    const unsigned b = r.box_off + sir_box(a.X[p], a.Y[p], a.Z[p], r);
    kn[p] = b;
    box[p] = b;
    rk[p] = atomicAdd(&count[b], 1u);
  }
}

__global__ void __launch_bounds__(kBlock) k_sir_index(SirState a, const unsigned* __restrict__ kn,
                                                      const unsigned* __restrict__ rk,
                                                      const unsigned* __restrict__ start,
                                                      unsigned* __restrict__ perm,
                                                      unsigned* __restrict__ ninf,
                                                      uint2* __restrict__ src, unsigned n,
                                                      DevGrid* g) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // the scan has finished: ready its counter
    g->scan_ctr[0] = 0;
    g->sir_counts[0] = g->sir_counts[1] = g->sir_counts[2] = 0;
  }
  for (unsigned base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const unsigned p = base + threadIdx.x;
    sir_index(p, p < n, 0u, a, kn, rk, start, perm, ninf, src, &g->sir_sources, n);
  }
}

__global__ void __launch_bounds__(kBlock) k_sir_push(SirState a, const unsigned* __restrict__ start,
                                                     const unsigned* __restrict__ perm,
                                                     unsigned* __restrict__ ninf,
                                                     const uint2* __restrict__ src, SirRun r,
                                                     unsigned n, const DevGrid* g) {
  const unsigned ns = min(g->sir_sources, n);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x)
    sir_push(src[i].x, r, a, start, perm, ninf, n);
}

__global__ void __launch_bounds__(kBlock) k_sir_update(SirState a, const unsigned* __restrict__ ninf,
                                                       unsigned* __restrict__ box,
                                                       unsigned* __restrict__ kn,
                                                       unsigned* __restrict__ rk,
                                                       unsigned* __restrict__ count, SirRun r,
                                                       DevGrid* g) {
  const unsigned n = r.agent_n;
  const unsigned step = (unsigned)g->step;
  if (blockIdx.x == 0 && threadIdx.x == 0) g->sir_sources = 0;  // the push has read it
  for (unsigned base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const unsigned p = base + threadIdx.x;
    unsigned char ns = 0;
    if (p < n) ns = sir_update(p, r, a, ninf, box, kn, rk, count, step);
    commit_counts(ns, p < n, g->sir_counts);
  }
}

// ---- batch of runs: one persistent launch per step --------------------------------------------
// Bounded grid barrier (generation counter).  A timeout sets ERR_TIMEOUT and lets the block go on;
// the step's results are then invalid and the host reports BDM_ETIMEOUT.
__device__ __forceinline__ void grid_barrier(unsigned* ctr, volatile unsigned* gen,
                                             unsigned nblocks, unsigned* err, unsigned limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(ctr, 1u) + 1u;
    if (arrived == nblocks) {
      *ctr = 0u;
      __threadfence();
      atomicAdd((unsigned*)gen, 1u);
    } else {
      unsigned spins = 0;
      while (*gen == g0) {
        if (++spins > limit) {
          atomicOr(err, (unsigned)ERR_TIMEOUT);
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kBlock) k_sir_init_batch(SirBatchDev B) {
  for (unsigned t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const SirRun r = B.run[B.tile_run[t]];
    const unsigned p = B.tile_start[t] + threadIdx.x;
    if (p < r.agent_off + r.agent_n) {
      const unsigned b = r.box_off + sir_box(B.a.X[p], B.a.Y[p], B.a.Z[p], r);
      B.kn[p] = b;
      B.box[p] = b;
      B.rk[p] = atomicAdd(&B.count[b], 1u);
    }
  }
}

// On entry: the histogram of the agents' boxes is in `count`; the scan's tile flags, its counter
// and the source counter are zero.
__global__ void __launch_bounds__(kBlock) k_sir_ensemble(SirBatchDev B, DevGrid* g,
                                                          unsigned barrier_blocks,
                                                          unsigned spin_limit) {
  const unsigned step = (unsigned)g->step;
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nthreads = gridDim.x * blockDim.x;
  unsigned* slot = B.hist + (size_t)(step % B.hist_len) * B.runs * 3u;
  // P1: global exclusive scan over all runs' boxes (clears the histogram)
  scan_tiles(B.count, B.start, B.total_boxes + 1u, B.tiles, &g->scan_ctr[0], &g->err, 1);
  grid_barrier(&B.bar[0], &B.bar[1], barrier_blocks, &g->err, spin_limit);
  // every block read the step before the barrier; the scan's flags are free again
  if (tid == 0) {
    g->step += 1ull;
    g->scan_ctr[0] = 0u;
  }
  for (unsigned t = tid; t < B.max_tiles; t += nthreads) B.tiles[t] = 0ull;
  for (unsigned t = tid; t < B.runs * 3u; t += nthreads) slot[t] = 0u;
  // P2: box order and source list
  for (unsigned t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const unsigned ri = B.tile_run[t];
    const SirRun r = B.run[ri];
    const unsigned p = B.tile_start[t] + threadIdx.x;
    sir_index(p, p < r.agent_off + r.agent_n, ri, B.a, B.kn, B.rk, B.start, B.perm, B.ninf, B.src,
              &g->sir_sources, B.total_agents);
  }
  grid_barrier(&B.bar[0], &B.bar[1], barrier_blocks, &g->err, spin_limit);
  // P3: infected agents push into their neighbours' counts
  {
    const unsigned ns = min(*(volatile unsigned*)&g->sir_sources, B.total_agents);
    for (unsigned i = tid; i < ns; i += nthreads) {
      const uint2 e = B.src[i];
      sir_push(e.x, B.run[e.y < B.runs ? e.y : 0u], B.a, B.start, B.perm, B.ninf, B.total_agents);
    }
  }
  grid_barrier(&B.bar[0], &B.bar[1], barrier_blocks, &g->err, spin_limit);
  if (tid == 0) g->sir_sources = 0u;  // every block has read it
  // P4: infection, recovery, move, next histogram; per-run S/I/R counts of this step
  for (unsigned t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const unsigned ri = B.tile_run[t];
    const SirRun r = B.run[ri];
    const unsigned p = B.tile_start[t] + threadIdx.x;
    const bool valid = p < r.agent_off + r.agent_n;
    unsigned char ns = 0;
    if (valid) ns = sir_update(p, r, B.a, B.ninf, B.box, B.kn, B.rk, B.count, step);
    commit_counts(ns, valid, slot + 3u * ri);
  }
}

// ---- batch of runs, one CTA per run -------------------------------------------------------------
// When every run's box array and infected-neighbour counts fit in shared memory ((nb^3 + 1 + agents)
// words), each run is advanced by one CTA per step: histogram, scan and counts live in shared memory,
// the phases are separated by __syncthreads, and there is neither a grid barrier nor a global scan.
// Same phases and the same integer arithmetic as the persistent kernel, so the same results (the
// order of agents inside a box and of the pushes does not enter any result).
constexpr int kSR = 1024;

// Exclusive prefix sum of v[0..m) in place; every thread of the block calls (v in shared memory).
__device__ void block_exclusive_scan(unsigned* v, unsigned m) {
  __shared__ unsigned s_w[kSR / 32];
  const unsigned t = threadIdx.x, lane = t & 31u, w = t >> 5;
  const unsigned per = (m + kSR - 1u) / kSR;
  const unsigned lo = min(t * per, m), hi = min(lo + per, m);
  unsigned sum = 0;
  for (unsigned k = lo; k < hi; ++k) sum += v[k];
  unsigned incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  if (lane == 31u) s_w[w] = incl;
  __syncthreads();
  if (w == 0) {
    const unsigned x = s_w[lane];
    unsigned xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, xi, o);
      if ((int)lane >= o) xi += y;
    }
    s_w[lane] = xi - x;
  }
  __syncthreads();
  unsigned acc = s_w[w] + incl - sum;
  for (unsigned k = lo; k < hi; ++k) {
    const unsigned x = v[k];
    v[k] = acc;
    acc += x;
  }
  __syncthreads();
}

// push of infected agent j of run r over the run-local box starts and counts in shared memory.
__device__ __forceinline__ void sir_push_local(unsigned j, const SirRun& r, const SirState a,
                                               const unsigned* s_start,
                                               const unsigned* __restrict__ perm, unsigned off,
                                               unsigned* s_cnt) {
  const int Xj = a.X[j], Yj = a.Y[j], Zj = a.Z[j];
  const long long L = r.L;
  const int nb = r.nb;
  int cy[3], cz[3], xlo[2], xhi[2];
  const int ny = neighbour_boxes(box_coord(Yj, r), nb, cy);
  const int nz = neighbour_boxes(box_coord(Zj, r), nb, cz);
  const int nr = neighbour_runs(box_coord(Xj, r), nb, xlo, xhi);
  for (int qz = 0; qz < nz; ++qz)
    for (int qy = 0; qy < ny; ++qy) {
      const unsigned row = (unsigned)nb * ((unsigned)cy[qy] + (unsigned)nb * (unsigned)cz[qz]);
      for (int k = 0; k < nr; ++k) {
        const unsigned m1 = s_start[row + (unsigned)xhi[k]];
        for (unsigned m = s_start[row + (unsigned)xlo[k]]; m < m1; ++m) {
          const unsigned i = perm[off + m];
          if (i == j) continue;
          const long long dx = min_image((long long)a.X[i] - Xj, L);
          const long long dy = min_image((long long)a.Y[i] - Yj, L);
          const long long dz = min_image((long long)a.Z[i] - Zj, L);
          if (dx * dx + dy * dy + dz * dz < r.r2) atomicAdd(&s_cnt[i - off], 1u);
        }
      }
    }
}

__global__ void __launch_bounds__(kSR) k_sir_runs(SirBatchDev B, DevGrid* g) {
  extern __shared__ unsigned s_dyn[];
  __shared__ unsigned s_nsrc, s_c[3];
  const unsigned ri = blockIdx.x;
  const SirRun r = B.run[ri];
  const unsigned n = r.agent_n, off = r.agent_off;
  const unsigned nbox = (unsigned)r.nb * (unsigned)r.nb * (unsigned)r.nb;
  unsigned* s_box = s_dyn;              // histogram, then box starts (nbox + 1)
  unsigned* s_cnt = s_dyn + nbox + 1u;  // infected neighbours of each agent of the run
  const unsigned t = threadIdx.x;
  const unsigned step = (unsigned)g->step;  // advanced by a separate launch after this one
  for (unsigned k = t; k <= nbox; k += kSR) s_box[k] = 0u;
  if (t == 0) {
    s_nsrc = 0u;
    s_c[0] = s_c[1] = s_c[2] = 0u;
  }
  __syncthreads();
  // boxes of the step-start positions (also the read-out) and ranks inside them
  for (unsigned q = t; q < n; q += kSR) {
    const unsigned p = off + q;
    const unsigned b = sir_box(B.a.X[p], B.a.Y[p], B.a.Z[p], r);
    B.kn[p] = b;
    B.rk[p] = atomicAdd(&s_box[b], 1u);
    B.box[p] = r.box_off + b;
    s_cnt[q] = 0u;
  }
  __syncthreads();
  block_exclusive_scan(s_box, nbox + 1u);
  // box order; infected agents to the source list
  for (unsigned q = t; q < n; q += kSR) {
    const unsigned p = off + q;
    B.perm[off + s_box[B.kn[p]] + B.rk[p]] = p;
    if (B.a.st[p] == 1) B.src[off + atomicAdd(&s_nsrc, 1u)] = make_uint2(p, ri);
  }
  __syncthreads();
  // infected agents push into their neighbours' counts
  const unsigned ns = s_nsrc;
  for (unsigned k = t; k < ns; k += kSR) sir_push_local(B.src[off + k].x, r, B.a, s_box, B.perm, off, s_cnt);
  __syncthreads();
  // infection, recovery, move; S/I/R counts of this step
  unsigned c0 = 0u, c1 = 0u, c2 = 0u;
  for (unsigned q = t; q < n; q += kSR) {
    const unsigned p = off + q;
    int NP[3];
    const unsigned cnt = s_cnt[q];
    const unsigned char st = sir_advance(p, r, B.a, cnt, step, NP);
    B.ninf[p] = cnt;
    c0 += st == 0 ? 1u : 0u;
    c1 += st == 1 ? 1u : 0u;
    c2 += st == 2 ? 1u : 0u;
  }
  auto add = [](unsigned a, unsigned b) { return a + b; };
  c0 = warp_reduce(c0, add);
  c1 = warp_reduce(c1, add);
  c2 = warp_reduce(c2, add);
  if ((t & 31u) == 0) {
    if (c0) atomicAdd(&s_c[0], c0);
    if (c1) atomicAdd(&s_c[1], c1);
    if (c2) atomicAdd(&s_c[2], c2);
  }
  __syncthreads();
  if (t < 3) B.hist[(size_t)(step % B.hist_len) * B.runs * 3u + 3u * ri + t] = s_c[t];
}

// Evaluate the device Philox generator on n (counter, key) pairs.
__global__ void k_philox(unsigned n, const uint4* __restrict__ ctr, const uint2* __restrict__ key,
                         uint4* __restrict__ out) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = philox10(ctr[i], key[i]);
}

// ---- launch wrappers ---------------------------------------------------------------------------
void launch_philox(cudaStream_t s, unsigned n, const uint4* ctr, const uint2* key, uint4* out) {
  const unsigned blocks = n ? (n + kBlock - 1) / kBlock : 1u;
  k_philox<<<blocks < 4096u ? blocks : 4096u, kBlock, 0, s>>>(n, ctr, key, out);
}

void launch_sir_init(cudaStream_t s, const SirSingle& S, unsigned lo, unsigned hi, int grid_blocks) {
  if (hi <= lo) return;
  const unsigned need = (hi - lo + kBlock - 1) / kBlock;
  k_sir_init<<<need < (unsigned)grid_blocks ? need : (unsigned)grid_blocks, kBlock, 0, s>>>(
      S.a, S.kn, S.rk, S.box, S.count, S.run, lo, hi);
}

void launch_sir_init_batch(cudaStream_t s, const SirBatchDev& B, int grid_blocks) {
  if (!B.ntiles) return;
  k_sir_init_batch<<<B.ntiles < (unsigned)grid_blocks ? B.ntiles : (unsigned)grid_blocks, kBlock, 0, s>>>(B);
}

void launch_sir_step(cudaStream_t s, const SirSingle& S, DevGrid* g, int grid_blocks, int scan_blocks) {
  const unsigned n = S.run.agent_n;
  cudaMemsetAsync(S.tiles, 0, sizeof(unsigned long long) * S.max_tiles, s);
  launch_scan(s, S.count, S.start, &g->nbox1, S.tiles, &g->scan_ctr[0], &g->err, 1, scan_blocks);
  k_sir_index<<<grid_blocks, kBlock, 0, s>>>(S.a, S.kn, S.rk, S.start, S.perm, S.ninf, S.src, n, g);
  k_sir_push<<<grid_blocks, kBlock, 0, s>>>(S.a, S.start, S.perm, S.ninf, S.src, S.run, n, g);
  k_sir_update<<<grid_blocks, kBlock, 0, s>>>(S.a, S.ninf, S.box, S.kn, S.rk, S.count, S.run, g);
  launch_step_done(s, g);
}

cudaError_t launch_sir_ensemble(cudaStream_t s, const SirBatchDev& B, DevGrid* g, int blocks,
                                unsigned barrier_extra, unsigned spin_limit, bool cooperative) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kBlock);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = cooperative ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_sir_ensemble, B, g, (unsigned)blocks + barrier_extra,
                            spin_limit);
}

// Dynamic shared memory of the per-run kernel for runs of up to `words` (nb^3 + 1 + agents) words;
// 0 when it does not fit on this device.
size_t sir_runs_smem_bytes(size_t words) {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  const size_t bytes = words * sizeof(unsigned);
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k_sir_runs) != cudaSuccess) return 0;
  if (bytes + fa.sharedSizeBytes > (size_t)optin) return 0;
  if (cudaFuncSetAttribute(k_sir_runs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    return 0;
  return bytes;
}

void launch_sir_runs(cudaStream_t s, const SirBatchDev& B, DevGrid* g, size_t smem_bytes) {
  k_sir_runs<<<B.runs, kSR, smem_bytes, s>>>(B, g);
  launch_step_done(s, g);
}

int sir_ensemble_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sir_ensemble, kBlock, 0);
  return nb;
}

}  // namespace bdm
