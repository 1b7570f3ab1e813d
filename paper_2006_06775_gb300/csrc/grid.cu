// grid.cu -- uniform-grid rebuild of one step (BioDynaMo, arXiv 2006.06775, Sec. "Simulation
// concepts", environment paragraph: equal boxes, agents assigned to boxes by centre, box size from
// the largest agent).  GPU form: per-axis bounds -> grid finalize -> box id + histogram -> single-pass
// prefix scan -> scatter -> canonicalising gather into (box, id) order (readings R5, R6).
#include "common.cuh"
#include "gridcore.cuh"
#include "scan.cuh"

namespace bdm {

__global__ void __launch_bounds__(kBlock) k_bounds(const double* __restrict__ x,
                                                   const double* __restrict__ y,
                                                   const double* __restrict__ z,
                                                   const float* __restrict__ diam, DevGrid* g) {
  const unsigned n = g->n;
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  unsigned md = 0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v[3] = {x[i], y[i], z[i]};
    for (int a = 0; a < 3; ++a) {
      unsigned long long e = enc_double(v[a]);
      mn[a] = e < mn[a] ? e : mn[a];
      mx[a] = e > mx[a] ? e : mx[a];
    }
    if (diam) {
      unsigned d = __float_as_uint(diam[i]);
      md = d > md ? d : md;
    }
  }
  block_commit_bounds(mn, mx, md, g);
}

// Turn the accumulated bounds into this step's grid (reading R5), then reset the accumulators and
// the scan tile counter for the next producer.  One thread.
__global__ void k_finalize(DevGrid* g, MechConsts c) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const unsigned n = g->n;
  g->scan_ctr[0] = 0;
  g->scan_ctr[1] = 0;
  g->n_eval = 0;
  grid_from_bounds(g, c);
  // Rebuild the grid this step, or evaluate the neighbour lists of the last rebuild (skin > 0).  A
  // pair within R now was within R + skin at the last rebuild while no agent has moved more than
  // skin / 2 since, so its lists still hold every neighbour and contact.
  unsigned rebuild = 1u;
  if (c.skin > 0.0 && g->nbox && g->list_valid && !g->list_overflow && g->Lf == g->Lf_list &&
      __uint_as_float(g->max_disp) <= c.skin_half && g->since_rebuild + 1u < c.max_cadence)
    rebuild = 0u;
  g->rebuild = rebuild;
  g->n_step = g->nbox ? n : 0u;
  if (rebuild) {
    g->n_sort = g->nbox ? n : 0u;
    g->nbox1_sort = g->nbox1;
    g->list_valid = c.skin > 0.0 && g->nbox ? 1u : 0u;
    g->list_overflow = 0u;
    g->max_disp = 0u;
    g->since_rebuild = 0u;
    g->Lf_list = g->Lf;
    g->rebuilds += 1u;
    g->list_entries = 0ull;
  } else {
    g->n_sort = 0u;
    g->nbox1_sort = 0u;
    g->since_rebuild += 1u;
  }
  for (int a = 0; a < 3; ++a) {
    g->acc_min[a] = ~0ull;
    g->acc_max[a] = 0ull;
  }
  g->acc_maxdiam = 0u;
}

// Box id of each agent (current order) and its arrival rank in the box histogram.
__global__ void __launch_bounds__(kBlock) k_key_hist(const double* __restrict__ x,
                                                     const double* __restrict__ y,
                                                     const double* __restrict__ z,
                                                     unsigned* __restrict__ key,
                                                     unsigned* __restrict__ rank,
                                                     unsigned* __restrict__ count,
                                                     const unsigned* __restrict__ id,
                                                     PackedAgent* __restrict__ pack, DevGrid* g) {
  const unsigned n = g->nbox ? g->n_sort : 0u;
  const bool packing = pack && g->fresh;
  const long long O0 = g->O[0], O1 = g->O[1], O2 = g->O[2], Lq = g->Lq;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const float inv = g->invLq;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int ix = box_div(quantise(x[i]) - O0, Lq, inv);
    int iy = box_div(quantise(y[i]) - O1, Lq, inv);
    int iz = box_div(quantise(z[i]) - O2, Lq, inv);
    if (ix >= d0 || iy >= d1 || iz >= d2) {  // impossible by construction of the bounds
      atomicOr(&g->err, (unsigned)ERR_BOUNDS);
      ix = min(ix, d0 - 1); iy = min(iy, d1 - 1); iz = min(iz, d2 - 1);
    }
    unsigned k = (unsigned)ix + (unsigned)d0 * ((unsigned)iy + (unsigned)d1 * (unsigned)iz);
    key[i] = k;
    rank[i] = atomicAdd(&count[k], 1u);
    if (packing) {
      PackedAgent a;
      a.x = x[i];
      a.y = y[i];
      a.z = z[i];
      a.id = id[i];
      a.key = k;
      pack[i] = a;
    }
  }
}

// Exclusive scan of *n_items values (box histogram -> box starts, or division flags -> ranks).
__global__ void __launch_bounds__(kBlock) k_scan(unsigned* __restrict__ in,
                                                 unsigned* __restrict__ out,
                                                 const unsigned* n_items,
                                                 unsigned long long* tiles, unsigned* tile_ctr,
                                                 unsigned* err, int zero_input) {
  scan_tiles(in, out, *n_items, tiles, tile_ctr, err, zero_input);
}

// Counting-sort scatter: slot = box start + arrival rank.
__global__ void __launch_bounds__(kBlock) k_scatter(const unsigned* __restrict__ key,
                                                    const unsigned* __restrict__ rank,
                                                    const unsigned* __restrict__ start,
                                                    unsigned* __restrict__ perm, DevGrid* g) {
  const unsigned n = g->nbox ? g->n_sort : 0u;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    perm[start[key[i]] + rank[i]] = i;
}

// Canonicalise and gather: the arrival order inside a box is replaced by ascending id (R6), and the
// agent payload moves into the canonical order.  The mixed-precision path also writes each agent's
// FP32 offset from its box's lower corner (exact lattice difference, then one rounding) and radius.
// With neighbour lists (XSORT) a box's agents are ordered by their lattice x coordinate instead, ties
// by id: a row of three boxes is then sorted along x, and the list build stops walking a row where
// its candidates leave the agent's x window.  The lists' order (and so the FP32 force sums) follows
// this order; counts and box ids do not depend on it.
template <bool MIXED, bool XSORT>
__global__ void __launch_bounds__(kBlock) k_gather(
    const unsigned* __restrict__ perm, const unsigned* __restrict__ key,
    const unsigned* __restrict__ start, const double* __restrict__ sx,
    const double* __restrict__ sy, const double* __restrict__ sz, AgentArrays src,
    double* __restrict__ dx, double* __restrict__ dy, double* __restrict__ dz, AgentArrays dst,
    unsigned* __restrict__ skey, float4* __restrict__ p4, const PackedAgent* __restrict__ pack,
    DevGrid* g) {
  const unsigned n = g->nbox ? g->n_sort : 0u;
  const long long O0 = g->O[0], O1 = g->O[1], O2 = g->O[2], Lq = g->Lq;
  const unsigned d0 = (unsigned)g->dims[0], d1 = (unsigned)g->dims[1];
  const bool packed = pack && g->fresh;  // the same for every thread
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned s = perm[k];
    PackedAgent a;
    if (packed) {
      a = pack[s];
    } else {
      a.key = key[s];
      a.id = src.id[s];
    }
    const unsigned b = a.key;
    const unsigned lo = start[b], hi = start[b + 1];
    const unsigned myid = a.id;
    if (!packed) {
      a.x = sx[s];
      a.y = sy[s];
      a.z = sz[s];
    }
    unsigned d = lo;
    if (hi - lo > 1) {
      if (XSORT) {
        // x order through the order-preserving integer encoding (the lattice x, and so the FP32
        // offset, never decreases along it)
        const unsigned long long qm = enc_double(a.x);
        for (unsigned m = lo; m < hi; ++m) {
          if (m == k) continue;
          const unsigned s2 = perm[m];
          const unsigned long long q2 = enc_double(packed ? pack[s2].x : sx[s2]);
          const unsigned id2 = packed ? pack[s2].id : src.id[s2];
          d += (q2 < qm || (q2 == qm && id2 < myid)) ? 1u : 0u;
        }
      } else {
        for (unsigned m = lo; m < hi; ++m)
          if (m != k) d += (packed ? pack[perm[m]].id : src.id[perm[m]]) < myid ? 1u : 0u;
      }
    }
    const double x = a.x, y = a.y, z = a.z;
    const float di = src.diam[s];
    dx[d] = x;
    dy[d] = y;
    dz[d] = z;
    dst.diam[d] = di;
    dst.id[d] = myid;
    if (src.vol) dst.vol[d] = src.vol[s];
    skey[d] = b;
    if (MIXED) {
      const unsigned ix = b % d0, t = b / d0;
      const unsigned iy = t % d1, iz = t / d1;
      const float ox = (float)(int)(quantise(x) - O0 - (long long)ix * Lq) * kQInv;
      const float oy = (float)(int)(quantise(y) - O1 - (long long)iy * Lq) * kQInv;
      const float oz = (float)(int)(quantise(z) - O2 - (long long)iz * Lq) * kQInv;
      p4[d] = make_float4(ox, oy, oz, 0.5f * di);
    }
  }
}

// ---- launch wrappers -------------------------------------------------------------------------
void launch_bounds(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                   int grid_blocks) {
  k_bounds<<<grid_blocks, kBlock, 0, s>>>(b.pos.x, b.pos.y, b.pos.z, attr.diam, g);
}

void launch_finalize(cudaStream_t s, DevGrid* g, MechConsts c) { k_finalize<<<1, 32, 0, s>>>(g, c); }

void launch_key_hist(cudaStream_t s, const MechBuffers& b, const unsigned* id, DevGrid* g,
                     int grid_blocks) {
  k_key_hist<<<grid_blocks, kBlock, 0, s>>>(b.pos.x, b.pos.y, b.pos.z, b.key, b.rank, b.count, id,
                                            b.pack, g);
}

void launch_scan(cudaStream_t s, unsigned* in, unsigned* out, const unsigned* n_items,
                 unsigned long long* tiles, unsigned* tile_ctr, unsigned* err, int zero_input,
                 int grid_blocks) {
  k_scan<<<grid_blocks, kBlock, 0, s>>>(in, out, n_items, tiles, tile_ctr, err, zero_input);
}

void launch_scatter(cudaStream_t s, const MechBuffers& b, DevGrid* g, int grid_blocks) {
  k_scatter<<<grid_blocks, kBlock, 0, s>>>(b.key, b.rank, b.start, b.perm, g);
}

void launch_gather(cudaStream_t s, const MechBuffers& b, const AgentArrays& src_attr,
                   const AgentArrays& dst_attr, DevGrid* g, bool mixed, bool xsort, int grid_blocks) {
  if (mixed && xsort)
    k_gather<true, true><<<grid_blocks, kBlock, 0, s>>>(b.perm, b.key, b.start, b.pos.x, b.pos.y,
                                                        b.pos.z, src_attr, b.sorted.x, b.sorted.y,
                                                        b.sorted.z, dst_attr, b.skey, b.p4, b.pack, g);
  else if (mixed)
    k_gather<true, false><<<grid_blocks, kBlock, 0, s>>>(b.perm, b.key, b.start, b.pos.x, b.pos.y,
                                                         b.pos.z, src_attr, b.sorted.x, b.sorted.y,
                                                         b.sorted.z, dst_attr, b.skey, b.p4, b.pack, g);
  else
    k_gather<false, false><<<grid_blocks, kBlock, 0, s>>>(b.perm, b.key, b.start, b.pos.x, b.pos.y,
                                                          b.pos.z, src_attr, b.sorted.x, b.sorted.y,
                                                          b.sorted.z, dst_attr, b.skey, b.p4, b.pack, g);
}

}  // namespace bdm
