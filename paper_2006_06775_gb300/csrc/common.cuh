// common.cuh -- shared definitions of the libbdm CUDA kernels (sm_103a).
//
// Everything here is device plumbing for the hot path of the BioDynaMo step (arXiv 2006.06775,
// Sec. "Simulation concepts"): the device-resident grid description, error bits, exact integer
// helpers for the grid lattice (reading R5), and a Philox4x32-10 generator written from its
// published definition (Salmon et al., SC'11).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bdm.h"

namespace bdm {

constexpr int kQ = 20;                        // grid lattice: 2^-20 um (reading R5)
constexpr double kQScale = 1048576.0;         // 2^20
constexpr float kQInv = 1.0f / 1048576.0f;    // 2^-20, exact
constexpr int kBlock = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kBlock * kScanItems; // 4096 items per scan tile
constexpr unsigned kSpinLimit = 1u << 22;      // bounded waits: ~0.5 s with 100 ns sleeps

enum ErrBit : unsigned {
  ERR_GRID_OVERFLOW = 1u,   // grid needs more boxes than box_capacity
  ERR_CAPACITY = 2u,        // division would exceed agent capacity
  ERR_TIMEOUT = 4u,         // a bounded spin-wait gave up
  ERR_RADIUS = 8u,          // box length below interaction radius / bad extent
  ERR_BOUNDS = 16u,         // an index check failed (never expected)
};

// Device-resident description of the current step's grid and counters.  Written by the finalize
// kernel, read by every kernel of the step, so that a step needs no host round trip and a whole
// n-step sequence can be captured in one CUDA graph.
struct DevGrid {
  unsigned long long acc_min[3];  // order-preserving encodings of the per-axis minimum centre
  unsigned long long acc_max[3];
  unsigned acc_maxdiam;           // float bits of the largest diameter (diameters are positive)
  unsigned n;                     // agents
  long long O[3];                 // origin, lattice units
  long long Lq;                   // box length, lattice units
  int dims[3];                    // boxes per axis
  unsigned nbox;
  unsigned nbox1;                 // nbox + 1: items of the box scan
  unsigned ndiv1;                 // n_old + 1: items of the division scan
  double R;                       // interaction radius (um)
  double R2;                      // R * R
  float Lf;                       // box length in um (float of Lq * 2^-20)
  float R2f;                      // float(R2)
  float R2lo, R2hi;               // FP32 band around R2 inside which the FP64 test decides
  float invLq;                    // float(1 / Lq): estimate for the box division
  unsigned scan_ctr[2];           // dynamic tile counters of the two scans
  unsigned err;                   // ErrBit flags
  unsigned sir_counts[3];         // S, I, R after the last SIR step
  unsigned sir_sources;           // entries of this SIR step's list of infected agents
  unsigned long long step;        // steps completed (Philox counters)
  unsigned bad_input;             // first rejected agent of the last upload (~0u: none)
  double mass;                    // FP64 substance total after the last diffusion step
  // neighbour lists (mixed precision with a skin): which part of the step runs is decided here by
  // the finalize kernel, so one captured step serves rebuild and list steps alike
  unsigned n_sort;                // agents the grid rebuild sorts this step (n, or 0 on list steps)
  unsigned nbox1_sort;            // items of this step's box scan (nbox + 1, or 0 on list steps)
  unsigned rebuild;               // 1: this step rebuilds the grid and the lists
  unsigned list_valid;            // lists describe the current agents (cleared by uploads)
  unsigned list_overflow;         // an agent had more listed candidates than the list holds
  unsigned max_disp;              // float bits: max over agents of |moves| since the last rebuild
  unsigned since_rebuild;         // steps since the last rebuild
  unsigned rebuilds;              // rebuilds so far
  unsigned long long list_entries;  // listed candidates of the last rebuild
  float list_L2f;                 // list radius squared (R + skin)^2, widened by 2^-10
  float Lf_list;                  // box length (um) of the grid the lists were built on
  unsigned n_step;                // agents the last step moved (a list step's box-id read-out)
  unsigned long long skipped;     // agent evaluations skipped as stationary (list steps)
  unsigned n_eval;                // stationary skip: warps listed for evaluation this step
  unsigned fresh;                 // agents were uploaded since the last step (arbitrary order)
};

struct MechConsts {               // per-simulation constants passed by value
  double dt, k, gamma, cap;
  float dtf, kf, gammaf, capf;
  double interaction_radius, box_length;
  unsigned box_capacity, capacity;
  int force_variant;              // 0: one thread per agent, 1: warp-shared pairs
  double skin;                    // neighbour-list skin (um); 0: grid walk every step
  float skin_half;                // rebuild when an agent may have moved more than this
  unsigned max_cadence;           // rebuild at least every this many steps (bounds FP32 drift)
  int skip_stationary;            // list steps skip agents that, with their listed neighbours, stood still
  int mixed;                      // mixed precision: contacts are searched within R only
};

// ---- exact helpers -------------------------------------------------------------------------

// Order-preserving map of a (non-NaN) double to uint64: a < b  <=>  enc(a) < enc(b).
__device__ __forceinline__ unsigned long long enc_double(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dec_double(unsigned long long e) {
  unsigned long long b = (e >> 63) ? (e & 0x7FFFFFFFFFFFFFFFull) : ~e;
  return __longlong_as_double((long long)b);
}

// round(v * 2^20) with ties to even, using integer operations on the IEEE-754 bits (no FP64 pipe).
// Valid for |v| < 2^40 um; the result equals llrint(ldexp(v, 20)).
__device__ __forceinline__ long long quantise(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;                                    // zero / subnormal -> 0
  unsigned long long m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  int sh = e - 1075 + kQ;                                  // v * 2^20 = m * 2^sh
  unsigned long long q;
  if (sh >= 0) {
    q = m << sh;                                           // sh <= 8 for |v| < 2^40
  } else if (sh < -54) {
    q = 0;                                                 // |v * 2^20| < 1/2
  } else {
    int s = -sh;                                           // 1..54
    unsigned long long rem = m & ((1ull << s) - 1ull);
    unsigned long long half = 1ull << (s - 1);
    q = m >> s;
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  return (b >> 63) ? -(long long)q : (long long)q;
}

// Exact float -> double conversion with integer operations only (GB300's conversion instruction
// runs on the slow FP64 pipe): zeros, subnormals (normalised with a leading-zero count) and normal
// numbers; the displacements it converts are finite.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long bits;
  if (e != 0u) {  // normal: rebias the exponent 127 -> 1023, widen the mantissa
    bits = ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (m != 0u) {  // subnormal m * 2^-149 with its leading one at bit p
    const int p = 31 - __clz((int)m);
    bits = ((unsigned long long)(p + 874) << 52) |
           (((unsigned long long)m << (52 - p)) & 0x000FFFFFFFFFFFFFull);
  } else {
    bits = 0ull;
  }
  return __longlong_as_double((long long)(sign | bits));
}

// floor(D / Lq) for 0 <= D < 2^51, 0 < Lq < 2^40: a float estimate corrected by exact products.
// The estimate converts two 32-bit halves (64-bit integer -> float conversions run on GB300's slow
// conversion pipe).
__device__ __forceinline__ int box_div(long long D, long long Lq, float invLq) {
  float df = (float)(int)(D >> 20) * 1048576.0f + (float)(int)(D & 0xFFFFF);
  long long q = (long long)(int)(df * invLq);
  if (q < 0) q = 0;
  while (q > 0 && q * Lq > D) --q;
  while ((q + 1) * Lq <= D) ++q;
  return (int)q;
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ------------------------------------
// Round: (c0,c1,c2,c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)) with
// M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by (0x9E3779B9, 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// ---- asynchronous global -> shared copies (per thread; completion by commit / wait groups) ------
// Both addresses must be aligned to the copy size.  A thread reads what it copied only after a
// wait that covers the copy's group.
template <int B>
__device__ __forceinline__ void cp_async_n(void* smem, const void* gmem) {
  static_assert(B == 4 || B == 8 || B == 16, "cp.async copies 4, 8 or 16 bytes");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- block reductions -------------------------------------------------------------------------
template <typename T, typename Op>
__device__ __forceinline__ T warp_reduce(T v, Op op) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

// ---------------------------------------------------------------------------------------------
// Block-wide bounds commit: min/max of order-preserving centre encodings and the largest diameter
// bits, one atomic per quantity per block.  Every thread of the block must call it.
// ---------------------------------------------------------------------------------------------
template <int NT = kBlock>
__device__ __forceinline__ void block_commit_bounds(unsigned long long mn[3], unsigned long long mx[3],
                                    unsigned md, DevGrid* g) {
  __shared__ unsigned long long s_mn[3][NT / 32], s_mx[3][NT / 32];
  __shared__ unsigned s_md[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  auto umin = [](unsigned long long a, unsigned long long b) { return a < b ? a : b; };
  auto umax = [](unsigned long long a, unsigned long long b) { return a > b ? a : b; };
  for (int a = 0; a < 3; ++a) {
    mn[a] = warp_reduce(mn[a], umin);
    mx[a] = warp_reduce(mx[a], umax);
  }
  md = warp_reduce(md, [](unsigned a, unsigned b) { return a > b ? a : b; });
  if (lane == 0) {
    for (int a = 0; a < 3; ++a) {
      s_mn[a][warp] = mn[a];
      s_mx[a][warp] = mx[a];
    }
    s_md[warp] = md;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; ++w) {
      for (int a = 0; a < 3; ++a) {
        s_mn[a][0] = umin(s_mn[a][0], s_mn[a][w]);
        s_mx[a][0] = umax(s_mx[a][0], s_mx[a][w]);
      }
      s_md[0] = s_md[0] > s_md[w] ? s_md[0] : s_md[w];
    }
    for (int a = 0; a < 3; ++a) {
      if (s_mn[a][0] != ~0ull) atomicMin(&g->acc_min[a], s_mn[a][0]);
      if (s_mx[a][0] != 0ull) atomicMax(&g->acc_max[a], s_mx[a][0]);
    }
    if (s_md[0]) atomicMax(&g->acc_maxdiam, s_md[0]);
  }
}

}  // namespace bdm

// ---- launch wrappers (defined in the .cu files, called by the C ABI layer) ---------------------
namespace bdm {

struct WarpBounds {              // bounds of a warp-sized group of agents (stationary skip)
  unsigned long long mn[3], mx[3];  // order-preserving encodings of the per-axis min / max centre
  unsigned md;                      // float bits of the largest diameter
  float dm;                         // largest move since the last rebuild
};

struct AgentArrays {             // one SoA buffer of agents
  double *x, *y, *z;
  float* diam;
  unsigned* id;
  double* vol;                   // growth only (else nullptr)
};

struct alignas(32) PackedAgent {  // one agent's centre, id and box in one 32-byte sector
  double x, y, z;
  unsigned id, key;
};

struct MechBuffers {
  AgentArrays pos;               // current positions (x,y,z used); with a skin = pset[current]
  AgentArrays sorted;            // positions gathered into canonical order (x,y,z used)
  // skin > 0: two position sets that alternate every step (x,y,z and the offsets p4set), the
  // list kernels read one and write the other; without a skin pset[0] = pos and p4set[0] = p4
  AgentArrays pset[2];
  float4* p4set[2];
  AgentArrays attr[2];           // diam/id/vol, ping-pong by step parity
  unsigned *key, *rank, *perm, *skey, *nbr, *count, *start;
  float4* p4;                    // mixed: box-relative offsets + radius (= p4set[current])
  // the first rebuild after an upload: the agents packed by the key kernel, so the gather reads one
  // sector per agent from the arbitrary upload order instead of one per field
  PackedAgent* pack;
  unsigned long long* tiles[2];  // scan tile states (box scan, division scan)
  unsigned* flag;                // growth: divide flags by id; also the division rank array
  unsigned* drank;
  unsigned max_tiles;
  // neighbour lists (skin > 0): kListCap entries per agent, interleaved per group of 32 agents;
  // an entry is (j << 5) | (row * 3 + box x) in the sorted order and grid of the last rebuild
  unsigned* list;
  unsigned* list_n;
  float* disp;                   // |moves| of each agent since the last rebuild
  // stationary skip, per warp-sized group of agents (32 consecutive in the sorted order): a bit per
  // agent, set if it moved (alternate like pset); its bounds, largest diameter and move since the
  // rebuild as of its last evaluation; and, from the last rebuild, for each of the nine neighbour
  // rows two ranges [first, end) of agents holding every candidate of its agents (row-major: row
  // sg of group w at sg * wstride + w)
  unsigned* wmoved[2];
  struct WarpBounds* wbounds;
  uint4* wrows;
  size_t wstride;
  unsigned* evl;                 // warps listed for evaluation on a list step
};

// grid.cu
void launch_bounds(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                   int grid_blocks);
void launch_finalize(cudaStream_t s, DevGrid* g, MechConsts c);
void launch_key_hist(cudaStream_t s, const MechBuffers& b, const unsigned* id, DevGrid* g,
                     int grid_blocks);
void launch_scan(cudaStream_t s, unsigned* in, unsigned* out, const unsigned* n_items,
                 unsigned long long* tiles, unsigned* tile_ctr, unsigned* err, int zero_input,
                 int grid_blocks);
void launch_scatter(cudaStream_t s, const MechBuffers& b, DevGrid* g, int grid_blocks);
void launch_gather(cudaStream_t s, const MechBuffers& b, const AgentArrays& src_attr,
                   const AgentArrays& dst_attr, DevGrid* g, bool mixed, bool xsort, int grid_blocks);
// mechanics.cu
void launch_force(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                  MechConsts c, bool mixed, int grid_blocks);
int force_mixed_blocks_per_sm(int variant);
int force_fp64_blocks(size_t capacity, int sms);  // grid of the FP64 force kernel
constexpr unsigned kListCap = 32;  // listed candidates per agent (R + skin)
// neighbour-list steps (mechanics.cu): the list build of a rebuild step, the list-driven force (or
// the walk when a list overflowed), the in-place update, and the attribute copy that keeps one
// attribute buffer current
void launch_force_skin(cudaStream_t s, const MechBuffers& b, int cur, DevGrid* g, MechConsts c,
                       bool build, int grid_blocks);
void launch_list_build(cudaStream_t s, const MechBuffers& b, DevGrid* g, int grid_blocks);
void launch_still_warps(cudaStream_t s, const MechBuffers& b, int cur, DevGrid* g, int grid_blocks);
void launch_attr_copy(cudaStream_t s, const AgentArrays& src, const AgentArrays& dst, DevGrid* g,
                      int grid_blocks);
int force_skin_blocks_per_sm(bool build);
int list_build_blocks_per_sm();
void launch_apoptosis_flags(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                            unsigned long long thr, uint2 key, int grid_blocks);
void launch_apoptosis_compact(cudaStream_t s, const MechBuffers& b, const AgentArrays& src,
                              const AgentArrays& dst, DevGrid* g, int grid_blocks);
void launch_brownian(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                     double sigma, uint2 key, bool fp64, int grid_blocks);
void launch_chemotaxis(cudaStream_t s, const MechBuffers& b, DevGrid* g, const float* grid,
                       const int dims[3], const double origin[3], double h, double chi,
                       int grid_blocks);
void launch_readout_box(cudaStream_t s, const AgentArrays& start_pos, unsigned* skey, DevGrid* g,
                        int grid_blocks);
void launch_grow(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                 double dv, double vdiv, int grid_blocks);
void launch_divide(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                   double offset_frac, uint2 key, unsigned capacity, int grid_blocks);
void launch_secrete(cudaStream_t s, const MechBuffers& b, DevGrid* g, float* grid,
                    const int dims[3], const double origin[3], double h, float q,
                    int grid_blocks);
void launch_unsort(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                   double* ox, double* oy, double* oz, float* odiam, double* ovol,
                   unsigned* onbr, unsigned* obox, int grid_blocks);
void launch_unsort_axis(cudaStream_t s, const double* src, const unsigned* id, double* dst, DevGrid* g,
                        int grid_blocks);
void launch_step_done(cudaStream_t s, DevGrid* g);
void launch_prepare_agents(cudaStream_t s, unsigned n0, unsigned n, const double* x, const double* y,
                           const double* z, const float* diam, unsigned* id, double* vol,
                           bool derive_volume, unsigned* nbr, unsigned* skey, DevGrid* g,
                           int grid_blocks);
// diffusion.cu
void launch_ftcs(cudaStream_t s, const float* u, float* out, const int dims[3], float lambda,
                 float mu_dt, double* partials, DevGrid* g);
// Block partials of one FTCS step (an upper bound for both kernels), in 64-bit arithmetic.
long long ftcs_partials_needed(const int dims[3]);
// The FTCS launches fit the grid-dimension limits and their block count fits an int.
bool ftcs_launchable(const int dims[3]);
void launch_grid_mass(cudaStream_t s, const float* u, const int dims[3], double* partials, DevGrid* g);
void launch_ftcs_mass_to(cudaStream_t s, const float* u, float* out, const int dims[3],
                         float lambda, float mu_dt, double* partials, double* mass);

}  // namespace bdm
