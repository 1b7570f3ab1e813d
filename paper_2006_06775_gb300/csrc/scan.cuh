// scan.cuh -- single-pass exclusive prefix scan (decoupled look-back) used by the grid rebuild.
#pragma once
#include "common.cuh"

namespace bdm {

// ---------------------------------------------------------------------------------------------
// Single-pass exclusive scan with decoupled look-back.  Tiles of 4096 items are claimed in order
// through a counter, so a tile only ever waits on tiles already owned by running blocks; every wait
// is bounded and sets ERR_TIMEOUT instead of hanging.  out[i] = sum_{j<i} in[i] for i < items;
// with zero_input the inputs are cleared as they are read (the box histogram is then ready for the
// next step).  Tile status word: bits 62-63 flag (1 aggregate, 2 inclusive prefix), low 32 value.
// ---------------------------------------------------------------------------------------------
// Called by every thread of a block of kBlock threads; returns when no tile is left.
__device__ __forceinline__ void scan_tiles(unsigned* __restrict__ in, unsigned* __restrict__ out,
                                           const unsigned items, unsigned long long* tiles,
                                           unsigned* tile_ctr, unsigned* err, int zero_input) {
  __shared__ unsigned s_tile;
  __shared__ unsigned s_warp[kBlock / 32];
  __shared__ unsigned s_exclusive;
  __shared__ unsigned s_items[kScanTile + kScanTile / 32];  // striped -> blocked, padded
  const unsigned ntiles = (items + kScanTile - 1) / kScanTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  volatile unsigned long long* vt = tiles;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    __syncthreads();
    const unsigned tile = s_tile;
    if (tile >= ntiles) {
      __syncthreads();  // everyone has read s_tile before a later call may overwrite it
      return;
    }
    const unsigned tbase = tile * kScanTile;
    // coalesced striped load (item k * 256 + t), stored blocked per thread through shared memory
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const unsigned li = (unsigned)k * kBlock + threadIdx.x;
      const unsigned idx = tbase + li;
      s_items[li + (li >> 5)] = idx < items ? in[idx] : 0u;
    }
    __syncthreads();
    unsigned v[kScanItems];
    unsigned sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const unsigned li = threadIdx.x * kScanItems + k;
      v[k] = s_items[li + (li >> 5)];
      sum += v[k];
    }
    // block-wide exclusive scan of the per-thread sums
    unsigned incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned w = lane < kBlock / 32 ? s_warp[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned t = __shfl_up_sync(0xFFFFFFFFu, w, o);
        if (lane >= o) w += t;
      }
      if (lane < kBlock / 32) s_warp[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    const unsigned warp_excl = warp ? s_warp[warp - 1] : 0u;
    const unsigned aggregate = s_warp[kBlock / 32 - 1];
    unsigned thread_excl = warp_excl + incl - sum;
    // look-back (warp 0)
    if (warp == 0) {
      unsigned exclusive = 0;
      if (tile == 0) {
        if (lane == 0) vt[0] = (2ull << 62) | aggregate;
      } else {
        if (lane == 0) vt[tile] = (1ull << 62) | aggregate;
        int pred = (int)tile - 1;
        unsigned spins = 0;
        bool timed_out = false;
        while (pred >= 0) {
          int t = pred - lane;
          unsigned long long st = t >= 0 ? vt[t] : (2ull << 62);
          unsigned flag = (unsigned)(st >> 62);
          if (__any_sync(0xFFFFFFFFu, flag == 0)) {
            if (++spins > kSpinLimit) {
              timed_out = true;
              break;
            }
            __nanosleep(64);
            continue;
          }
          unsigned incl_mask = __ballot_sync(0xFFFFFFFFu, flag == 2);
          unsigned val = (unsigned)(st & 0xFFFFFFFFull);
          if (incl_mask) {
            int first = __ffs(incl_mask) - 1;  // nearest tile with an inclusive prefix
            unsigned contrib = lane <= first ? val : 0u;
            exclusive += warp_reduce(contrib, [](unsigned a, unsigned b) { return a + b; });
            break;
          }
          exclusive += warp_reduce(val, [](unsigned a, unsigned b) { return a + b; });
          pred -= 32;
        }
        if (timed_out && lane == 0) atomicOr(err, (unsigned)ERR_TIMEOUT);
        if (lane == 0) vt[tile] = (2ull << 62) | (unsigned)(exclusive + aggregate);
      }
      if (lane == 0) s_exclusive = exclusive;
    }
    __syncthreads();
    unsigned run = s_exclusive + thread_excl;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const unsigned li = threadIdx.x * kScanItems + k;
      s_items[li + (li >> 5)] = run;
      run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
      const unsigned li = (unsigned)k * kBlock + threadIdx.x;
      const unsigned idx = tbase + li;
      if (idx < items) {
        out[idx] = s_items[li + (li >> 5)];
        if (zero_input) in[idx] = 0u;
      }
    }
    __syncthreads();  // shared memory is reused by the next tile
  }
}

}  // namespace bdm
