// sir.cu -- random-walk SIR model (BioDynaMo, arXiv 2006.06775, Sec. "Epidemiology use case": a
// susceptible person becomes infected with the infection probability when an infected person is
// within the infection radius; an infected person recovers with the recovery probability each
// step; every person moves randomly by a bounded distance; an operation counts S, I and R).
// Reading R10: synchronous integer step on a 2^-10 um lattice, periodic cube, Philox4x32-10 keyed
// by (seed, run) with counters (id, step, stream, 0).
//
// Agents stay in id order.  Every agent's box id is computed each step, and the uniform grid index
// (box -> agent ids, rebuilt by counting sort) holds the INFECTED agents only: the infection rule and
// the infected-neighbour count only ever look at infected agents, so searching the 27 boxes of this
// index gives exactly the counts of a full index at a fraction of the candidates.  One run uses four
// kernels per step; a batch of runs uses ONE persistent kernel per step whose phases are separated
// by a bounded grid barrier.
#include "common.cuh"
#include "scan.cuh"
#include "sir.cuh"

namespace bdm {

__device__ __forceinline__ unsigned sir_box(int X, int Y, int Z, const SirRun& r) {
  return (unsigned)(X / r.Lb) + (unsigned)r.nb * ((unsigned)(Y / r.Lb) + (unsigned)r.nb * (unsigned)(Z / r.Lb));
}

__device__ __forceinline__ int neighbour_boxes(int b, int nb, int out[3]) {
  if (nb == 1) {
    out[0] = 0;
    return 1;
  }
  out[0] = b;
  out[1] = (b + 1) % nb;
  if (nb == 2) return 2;
  out[2] = (b + nb - 1) % nb;
  return 3;
}

__device__ __forceinline__ long long min_image(long long d, long long L) {
  if (d > L / 2) d -= L;
  else if (d < -(L / 2)) d += L;
  return d;
}

// Update of agent a (global index; id within its run = a - r.agent_off).  Returns the new state.
__device__ __forceinline__ unsigned char sir_update(unsigned a, const SirRun& r, const SirState cur,
                                                    SirState nxt, const unsigned* __restrict__ start,
                                                    const unsigned* __restrict__ perm,
                                                    unsigned* __restrict__ ninf, unsigned step) {
  const int Xi = cur.X[a], Yi = cur.Y[a], Zi = cur.Z[a];
  const unsigned char si = cur.st[a];
  const long long L = r.L;
  int cx[3], cy[3], cz[3];
  const int nx = neighbour_boxes(Xi / r.Lb, r.nb, cx);
  const int ny = neighbour_boxes(Yi / r.Lb, r.nb, cy);
  const int nz = neighbour_boxes(Zi / r.Lb, r.nb, cz);
  unsigned cnt = 0;
  for (int qz = 0; qz < nz; ++qz)
    for (int qy = 0; qy < ny; ++qy)
      for (int qx = 0; qx < nx; ++qx) {
        const unsigned b = r.box_off + (unsigned)cx[qx] +
                           (unsigned)r.nb * ((unsigned)cy[qy] + (unsigned)r.nb * (unsigned)cz[qz]);
        const unsigned e = start[b + 1];
        for (unsigned m = start[b]; m < e; ++m) {
          const unsigned j = perm[m];  // an infected agent
          if (j == a) continue;
          const long long dx = min_image((long long)Xi - cur.X[j], L);
          const long long dy = min_image((long long)Yi - cur.Y[j], L);
          const long long dz = min_image((long long)Zi - cur.Z[j], L);
          cnt += (dx * dx + dy * dy + dz * dz < r.r2) ? 1u : 0u;
        }
      }
  const unsigned id = a - r.agent_off;
  const uint4 w = philox10(make_uint4(id, step, 0u, 0u), r.key);
  unsigned char ns = si;
  if (si == 0 && cnt > 0 && (unsigned long long)w.x < r.thr_inf) ns = 1;
  if (si == 1 && (unsigned long long)w.y < r.thr_rec) ns = 2;
  const uint4 mv = philox10(make_uint4(id, step, 1u, 0u), r.key);
  const int P[3] = {Xi, Yi, Zi};
  const unsigned W[3] = {mv.x, mv.y, mv.z};
  int NP[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    long long v = (long long)P[k] + ((long long)(((unsigned long long)W[k] * r.span) >> 32) - r.s);
    if (v < 0) v += L;
    else if (v >= L) v -= L;
    NP[k] = (int)v;
  }
  nxt.X[a] = NP[0];
  nxt.Y[a] = NP[1];
  nxt.Z[a] = NP[2];
  nxt.st[a] = ns;
  ninf[a] = cnt;
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

// ---- one run: keyhist -> scan -> scatter -> update ------------------------------------------
__global__ void __launch_bounds__(kBlock) k_sir_keyhist(SirState cur, unsigned* __restrict__ key,
                                                        unsigned* __restrict__ rank,
                                                        unsigned* __restrict__ count, SirRun r,
                                                        DevGrid* g) {
  const unsigned n = r.agent_n;
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    g->scan_ctr[0] = 0;
    g->sir_counts[0] = g->sir_counts[1] = g->sir_counts[2] = 0;
  }
  for (unsigned a = tid; a < n; a += gridDim.x * blockDim.x) {
    const unsigned b = sir_box(cur.X[a], cur.Y[a], cur.Z[a], r);
    key[a] = b;
    if (cur.st[a] == 1) rank[a] = atomicAdd(&count[b], 1u);
  }
}

__global__ void __launch_bounds__(kBlock) k_sir_scatter(const unsigned* __restrict__ key,
                                                        const unsigned* __restrict__ rank,
                                                        const unsigned char* __restrict__ st,
                                                        const unsigned* __restrict__ start,
                                                        unsigned* __restrict__ perm, unsigned n) {
  for (unsigned a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x)
    if (st[a] == 1) perm[start[key[a]] + rank[a]] = a;
}

__global__ void __launch_bounds__(kBlock) k_sir_update(SirState cur, SirState nxt,
                                                       const unsigned* __restrict__ start,
                                                       const unsigned* __restrict__ perm,
                                                       unsigned* __restrict__ ninf, SirRun r,
                                                       DevGrid* g) {
  const unsigned n = r.agent_n;
  const unsigned step = (unsigned)g->step;
  for (unsigned base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const unsigned a = base + threadIdx.x;
    unsigned char ns = 0;
    if (a < n) ns = sir_update(a, r, cur, nxt, start, perm, ninf, step);
    commit_counts(ns, a < n, g->sir_counts);
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

__global__ void __launch_bounds__(kBlock) k_sir_ensemble(SirBatchDev B, DevGrid* g,
                                                          unsigned barrier_blocks,
                                                          unsigned spin_limit) {
  const unsigned step = (unsigned)g->step;
  const int par = (int)(g->step & 1ull);
  const SirState cur = B.state[par], nxt = B.state[par ^ 1];
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nthreads = gridDim.x * blockDim.x;
  // P1: reset the scan and this step's count slot; box id + histogram
  for (unsigned t = tid; t < B.max_tiles; t += nthreads) B.tiles[t] = 0ull;
  unsigned* slot = B.hist + (size_t)(step % B.hist_len) * B.runs * 3u;
  for (unsigned t = tid; t < B.runs * 3u; t += nthreads) slot[t] = 0u;
  if (tid == 0) g->scan_ctr[0] = 0u;
  for (unsigned t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const SirRun r = B.run[B.tile_run[t]];
    const unsigned a = B.tile_start[t] + threadIdx.x;
    if (a < r.agent_off + r.agent_n) {
      const unsigned b = r.box_off + sir_box(cur.X[a], cur.Y[a], cur.Z[a], r);
      B.key[a] = b;
      if (cur.st[a] == 1) B.rank[a] = atomicAdd(&B.count[b], 1u);
    }
  }
  grid_barrier(&B.bar[0], &B.bar[1], barrier_blocks, &g->err, spin_limit);
  if (tid == 0) g->step += 1ull;  // every block read the step before the barrier
  // P2: global exclusive scan over all runs' boxes (clears the histogram)
  scan_tiles(B.count, B.start, B.total_boxes + 1u, B.tiles, &g->scan_ctr[0], &g->err, 1);
  grid_barrier(&B.bar[0], &B.bar[1], barrier_blocks, &g->err, spin_limit);
  // P3: scatter agent indices into box order
  for (unsigned a = tid; a < B.total_agents; a += nthreads)
    if (cur.st[a] == 1) B.perm[B.start[B.key[a]] + B.rank[a]] = a;
  grid_barrier(&B.bar[0], &B.bar[1], barrier_blocks, &g->err, spin_limit);
  // P4: infection, recovery, move; per-run S/I/R counts of this step
  for (unsigned t = blockIdx.x; t < B.ntiles; t += gridDim.x) {
    const unsigned ri = B.tile_run[t];
    const SirRun r = B.run[ri];
    const unsigned a = B.tile_start[t] + threadIdx.x;
    const bool valid = a < r.agent_off + r.agent_n;
    unsigned char ns = 0;
    if (valid) ns = sir_update(a, r, cur, nxt, B.start, B.perm, B.ninf, step);
    commit_counts(ns, valid, slot + 3u * ri);
  }
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

void launch_sir_step(cudaStream_t s, const SirSingle& S, DevGrid* g, int par, int grid_blocks,
                     int scan_blocks) {
  const SirState cur = S.state[par], nxt = S.state[par ^ 1];
  k_sir_keyhist<<<grid_blocks, kBlock, 0, s>>>(cur, S.key, S.rank, S.count, S.run, g);
  cudaMemsetAsync(S.tiles, 0, sizeof(unsigned long long) * S.max_tiles, s);
  launch_scan(s, S.count, S.start, &g->nbox1, S.tiles, &g->scan_ctr[0], &g->err, 1, scan_blocks);
  k_sir_scatter<<<grid_blocks, kBlock, 0, s>>>(S.key, S.rank, cur.st, S.start, S.perm, S.run.agent_n);
  k_sir_update<<<grid_blocks, kBlock, 0, s>>>(cur, nxt, S.start, S.perm, S.ninf, S.run, g);
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

int sir_ensemble_blocks_per_sm() {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sir_ensemble, kBlock, 0);
  return nb;
}

}  // namespace bdm
