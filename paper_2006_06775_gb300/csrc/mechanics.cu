// mechanics.cu -- mechanical interaction of spherical agents and the behaviours that change them
// (BioDynaMo, arXiv 2006.06775, Sec. "Simulation concepts": agent operations "calculate mechanical
// forces" and behaviours such as growth, division and secretion; force law and update: readings
// R1-R4, sum order R6, growth/division R7, secretion R8).
#include <type_traits>

#include "common.cuh"
#include "mechcore.cuh"

namespace bdm {

// ---------------------------------------------------------------------------------------------
// Force + capped update, FP64 check path: one warp per agent in canonical order.  The agent's
// candidates are read box by box in ascending key -- for each (dz, dy) the up-to-three boxes along x
// are contiguous in the sorted arrays -- which is exactly the oracle's (box, id) order.  The lanes
// take the candidates 32 at a time and each evaluates one pair with explicitly rounded FP64
// intrinsics in the oracle's order (no contraction); the pair forces are then added in candidate
// order, one after another, by every lane (shuffles), so the sum is the oracle's bit for bit while
// the long FP64 division and square-root chains of different pairs run side by side.  The epilogue
// folds the new centres into the bounds of the next step's grid.
// ---------------------------------------------------------------------------------------------
constexpr int kF64 = 128;  // threads per block: four agents at a time

__global__ void __launch_bounds__(kF64) k_force_fp64(
    const double* __restrict__ sx, const double* __restrict__ sy, const double* __restrict__ sz,
    const float* __restrict__ diam, const unsigned* __restrict__ skey,
    const unsigned* __restrict__ start, double* __restrict__ ox, double* __restrict__ oy,
    double* __restrict__ oz, unsigned* __restrict__ nbr, DevGrid* g, MechConsts c) {
  const unsigned n = g->nbox ? g->n : 0u;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const double R2 = g->R2;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned warps = gridDim.x * (blockDim.x >> 5);
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  unsigned md = 0;
  for (unsigned i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const unsigned b = skey[i];
    const int ix = (int)(b % (unsigned)d0);
    const unsigned t = b / (unsigned)d0;
    const int iy = (int)(t % (unsigned)d1), iz = (int)(t / (unsigned)d1);
    const double xi = sx[i], yi = sy[i], zi = sz[i];
    const double ri = 0.5 * (double)diam[i];
    // row runs: lane r < 9 holds row r's candidate range [ra, ra + len)
    unsigned ra = 0, len = 0;
    if (lane < 9u) {
      const int jz = iz + (int)lane / 3 - 1, jy = iy + (int)lane % 3 - 1;
      if (jz >= 0 && jz < d2 && jy >= 0 && jy < d1) {
        const unsigned row = ((unsigned)jz * (unsigned)d1 + (unsigned)jy) * (unsigned)d0;
        const int xlo = ix > 0 ? ix - 1 : 0, xhi = ix < d0 - 1 ? ix + 1 : d0 - 1;
        ra = start[row + xlo];
        len = start[row + xhi + 1] - ra;
      }
    }
    unsigned incl = len;  // inclusive scan of the run lengths over lanes 0..8
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if ((int)lane >= o) incl += v;
    }
    const unsigned total = __shfl_sync(0xFFFFFFFFu, incl, 8);
    unsigned cnt = 0;
    double Sx = 0.0, Sy = 0.0, Sz = 0.0;
    for (unsigned c0 = 0; c0 < total; c0 += 32u) {
      const unsigned ci = c0 + lane;
      // the run holding candidate ci, and its index j
      unsigned j = 0;
      for (int r = 0; r < 9; ++r) {
        const unsigned e = __shfl_sync(0xFFFFFFFFu, incl, r);
        const unsigned a = __shfl_sync(0xFFFFFFFFu, ra, r);
        const unsigned l = __shfl_sync(0xFFFFFFFFu, len, r);
        if (ci < e && ci >= e - l) j = a + (ci - (e - l));
      }
      bool within = false, contact = false;
      double fx = 0.0, fy = 0.0, fz = 0.0;
      if (ci < total && j != i) {
        const double ax = __dsub_rn(xi, sx[j]), ay = __dsub_rn(yi, sy[j]), az = __dsub_rn(zi, sz[j]);
        const double e2 =
            __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
        within = e2 < R2;
        const double d = __dsqrt_rn(e2);
        const double rj = 0.5 * (double)diam[j];
        const double delta = __dsub_rn(__dadd_rn(ri, rj), d);
        if (delta > 0.0 && d > 0.0) {
          const double rho = __ddiv_rn(__dmul_rn(ri, rj), __dadd_rn(ri, rj));
          const double F = __dsub_rn(__dmul_rn(c.k, delta),
                                     __dmul_rn(c.gamma, __dsqrt_rn(__dmul_rn(rho, delta))));
          const double sc = __ddiv_rn(F, d);
          fx = __dmul_rn(sc, ax);
          fy = __dmul_rn(sc, ay);
          fz = __dmul_rn(sc, az);
          contact = true;
        }
      }
      cnt += (unsigned)__popc(__ballot_sync(0xFFFFFFFFu, within));
      // the contacts' forces added in candidate order
      unsigned cm = __ballot_sync(0xFFFFFFFFu, contact);
      while (cm) {
        const int l = __ffs(cm) - 1;
        cm &= cm - 1u;
        Sx = __dadd_rn(Sx, __shfl_sync(0xFFFFFFFFu, fx, l));
        Sy = __dadd_rn(Sy, __shfl_sync(0xFFFFFFFFu, fy, l));
        Sz = __dadd_rn(Sz, __shfl_sync(0xFFFFFFFFu, fz, l));
      }
    }
    if (lane == 0u) {
      double Dx = __dmul_rn(c.dt, Sx), Dy = __dmul_rn(c.dt, Sy), Dz = __dmul_rn(c.dt, Sz);
      double nrm = __dadd_rn(__dmul_rn(Dx, Dx), __dmul_rn(Dy, Dy));
      nrm = __dsqrt_rn(__dadd_rn(nrm, __dmul_rn(Dz, Dz)));
      if (nrm > c.cap) {
        const double f = __ddiv_rn(c.cap, nrm);
        Dx = __dmul_rn(Dx, f); Dy = __dmul_rn(Dy, f); Dz = __dmul_rn(Dz, f);
      }
      const double nx = __dadd_rn(xi, Dx), ny = __dadd_rn(yi, Dy), nz = __dadd_rn(zi, Dz);
      ox[i] = nx;
      oy[i] = ny;
      oz[i] = nz;
      nbr[i] = cnt;
      const unsigned long long e0 = enc_double(nx), e1 = enc_double(ny), e2 = enc_double(nz);
      mn[0] = e0 < mn[0] ? e0 : mn[0]; mx[0] = e0 > mx[0] ? e0 : mx[0];
      mn[1] = e1 < mn[1] ? e1 : mn[1]; mx[1] = e1 > mx[1] ? e1 : mx[1];
      mn[2] = e2 < mn[2] ? e2 : mn[2]; mx[2] = e2 > mx[2] ? e2 : mx[2];
      const unsigned dbits = __float_as_uint(diam[i]);
      md = dbits > md ? dbits : md;
    }
  }
  block_commit_bounds<kF64>(mn, mx, md, g);
}

// ---------------------------------------------------------------------------------------------
// Force + capped update, mixed precision.  One thread per agent in canonical order (grid-stride).
// The nine row segments (dz, dy in {-1,0,1}) of its 27-box neighbourhood are contiguous runs of the
// canonical order; each run is split by two box boundaries into its x-1, x, x+1 boxes (which give
// the x shift of a candidate's box-relative offset).  Per candidate the loop only evaluates FP32
// d^2 and writes the candidate branch-free into slot nc of a shared-memory list, advancing nc when
// d^2 <= R^2 (1 + 2^-12): every neighbour, band candidate and contact is listed (about 5 of 26
// candidates at 0.3 volume fraction).  A flush then takes the listed candidates in order: the
// neighbour count, the band queue and, for contacts, the force law, so none of that runs masked in
// every iteration of the candidate loop.  In a dense row run (more than kDenseBox agents per box
// somewhere in the warp) every active lane flushes as soon as one lane's list is full, so the
// flushes of the warp run side by side.  Contacts are summed in the canonical (box, id) order.
// Loads go through L1: consecutive agents share almost all of their neighbourhood.
//
// Neighbour predicate d^2 < R^2: FP32 outside a +-2^-12 relative band, the oracle's FP64 expression
// inside it, so counts stay exact.  Band candidates are queued (kBQ per thread) and decided in FP64
// after the loop; if more turn up, a second pass recounts every candidate from one d^2.  The agent
// meets itself once (d^2 = 0): counted, then removed.  The displacement is added to the FP64 centre
// (exact conversion, one FP64 add per axis).
// ---------------------------------------------------------------------------------------------
constexpr int kFT = 256;   // threads per CTA
constexpr int kCL = 16;    // candidate list length per thread
constexpr int kBQ = 8;     // band queue length per thread
constexpr unsigned kDenseBox = 8;  // agents per box above which a row run is treated as dense
constexpr unsigned kSkipSpan = 16;  // stationary skip: a row range over more warps is evaluated

// FP64 decision of one band candidate, as a real call: a conditional call inside a loop cannot be
// if-converted, so the loop never occupies GB300's slow FP64 pipe for candidates outside the band.
__device__ __noinline__ unsigned fp64_within_call(unsigned i, unsigned j, const double* __restrict__ sx,
                                                  const double* __restrict__ sy,
                                                  const double* __restrict__ sz, double R2) {
  return fp64_within(i, j, sx, sy, sz, R2);
}

// Neighbour count of agent i from a second pass over its 27 boxes: FP32 below the band, the oracle's
// FP64 expression inside it.  Used when more band candidates turned up than the per-thread queue
// holds; it replaces the first pass's count, so every candidate is decided by one d^2.
__device__ __noinline__ unsigned band_rescan(
    unsigned i, const double* __restrict__ sx, const double* __restrict__ sy,
    const double* __restrict__ sz, const float4* __restrict__ p4, const unsigned* __restrict__ start,
    int ix, int iy, int iz, int d0, int d1, int d2, float4 pi, float Lf, float R2lo, float R2hi,
    double R2) {
  unsigned k = 0;
  const int xl = ix > 0 ? ix - 1 : 0, xh = ix + 1 < d0 ? ix + 1 : ix;
  for (int sg = 0; sg < 9; ++sg) {
    const int jz = iz + sg / 3 - 1, jy = iy + sg % 3 - 1;
    if (jz < 0 || jz >= d2 || jy < 0 || jy >= d1) continue;
    const unsigned row = ((unsigned)jz * (unsigned)d1 + (unsigned)jy) * (unsigned)d0;
    const unsigned a = start[row + xl], e = start[row + xh + 1];
    const unsigned m1 = ix > 0 ? start[row + ix] : a, m2 = start[row + ix + 1];
    const float py = pi.y - (float)(sg % 3 - 1) * Lf, pz = pi.z - (float)(sg / 3 - 1) * Lf;
    for (unsigned j = a; j < e; ++j) {
      const float4 q = p4[j];
      const float px = pi.x - (j < m1 ? -Lf : (j < m2 ? 0.f : Lf));
      const float ex = px - q.x, ey = py - q.y, ez = pz - q.z;
      const float dd = pair_d2(ex, ey, ez);
      if (dd < R2lo) ++k;
      else if (dd <= R2hi) k += fp64_within_call(i, j, sx, sy, sz, R2);
    }
  }
  return k;
}

__global__ void __launch_bounds__(kFT, 3) k_force_mixed(
    const double* __restrict__ sx, const double* __restrict__ sy, const double* __restrict__ sz,
    const float4* __restrict__ p4, const unsigned* __restrict__ skey,
    const unsigned* __restrict__ start, double* __restrict__ ox, double* __restrict__ oy,
    double* __restrict__ oz, unsigned* __restrict__ nbr, DevGrid* g, MechConsts c) {
  __shared__ unsigned s_cj[kCL][kFT];       // candidate list: index
  __shared__ unsigned char s_cc[kCL][kFT];  // candidate list: row segment * 3 + box x
  __shared__ unsigned s_bq[kBQ][kFT];       // band queue: candidates decided in FP64 after the loop
  const unsigned n = g->nbox ? g->n : 0u;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const double R2 = g->R2;
  const float Lf = g->Lf, R2lo = g->R2lo, R2hi = g->R2hi;
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  unsigned md = 0;
  // candidate offset shift of each box code (row * 3 + box x): exact multiples of the box length
  __shared__ float4 s_shift[27];
  if (threadIdx.x < 27) {
    const int row = threadIdx.x / 3, bx = threadIdx.x % 3;
    s_shift[threadIdx.x] = make_float4(-(float)(bx - 1) * Lf, -(float)(row % 3 - 1) * Lf,
                                       -(float)(row / 3 - 1) * Lf, 0.f);
  }
  __syncthreads();
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned b = __ldg(skey + i);
    const int ix = (int)(b % (unsigned)d0);
    const unsigned q0 = b / (unsigned)d0;
    const int iy = (int)(q0 % (unsigned)d1), iz = (int)(q0 / (unsigned)d1);
    const int xl = ix > 0 ? ix - 1 : 0, xh = ix + 1 < d0 ? ix + 1 : ix;
    const float4 pi = __ldg(p4 + i);
    const double xi = sx[i], yi = sy[i], zi = sz[i];
    const float pxm = pi.x + Lf, px0 = pi.x, pxp = pi.x - Lf;  // neighbour box at x-1, x, x+1
    unsigned cnt = 0;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    int nc = 0;
    // candidates with d^2 within 2^-12 of R^2 (decided in FP64 after the loop, so the FP64 code
    // never runs predicated inside the candidate loop)
    unsigned nband = 0;
    const int t = threadIdx.x;
    auto flush = [&]() {  // count, band queue and force law over the listed candidates, in order
      for (int k = 0; k < nc; ++k) {
        const unsigned cj = s_cj[k][t], cc = s_cc[k][t];
        const float4 q = __ldg(p4 + cj);
        const float4 sh = s_shift[cc];
        const float ex = (pi.x + sh.x) - q.x;
        const float ey = (pi.y + sh.y) - q.y;
        const float ez = (pi.z + sh.z) - q.z;
        const float dd = pair_d2(ex, ey, ez);
        if (dd < R2lo) {
          ++cnt;
        } else {  // near R: queued for the FP64 decision after the loop
          if (nband < (unsigned)kBQ) s_bq[nband][t] = cj;
          ++nband;
        }
        const float rs = pi.w + q.w;
        if (dd < rs * rs && dd > 0.f) contact_force(Fx, Fy, Fz, ex, ey, ez, pi.w, q.w, c.kf, c.gammaf);
      }
      nc = 0;
    };
#pragma unroll 1
    for (int sg = 0; sg < 9; ++sg) {
      const int jz = iz + sg / 3 - 1, jy = iy + sg % 3 - 1;
      if (jz < 0 || jz >= d2 || jy < 0 || jy >= d1) continue;
      const unsigned row = ((unsigned)jz * (unsigned)d1 + (unsigned)jy) * (unsigned)d0;
      const unsigned a = __ldg(start + row + xl);
      const unsigned m1 = ix > 0 ? __ldg(start + row + ix) : a;  // end of box x-1
      const unsigned m2 = __ldg(start + row + ix + 1);           // end of box x
      const unsigned e = __ldg(start + row + xh + 1);            // end of the run
      const float py = pi.y - (float)(sg % 3 - 1) * Lf, pz = pi.z - (float)(sg / 3 - 1) * Lf;
      auto run = [&](auto dense) {
        for (unsigned j = a; j < e; ++j) {
          const float4 q = __ldg(p4 + j);
          const unsigned bx = j < m1 ? 0u : (j < m2 ? 1u : 2u);
          const float ex = (bx == 0 ? pxm : (bx == 1 ? px0 : pxp)) - q.x;
          const float ey = py - q.y;
          const float ez = pz - q.z;
          const float dd = pair_d2(ex, ey, ez);
          s_cj[nc][t] = j;  // kept only if within R (every neighbour, band candidate and contact)
          s_cc[nc][t] = (unsigned char)(sg * 3 + (int)bx);
          nc += dd <= R2hi ? 1 : 0;
          if constexpr (decltype(dense)::value) {
            // dense rows: a full list is flushed by every active lane at once, so the lanes'
            // force evaluations run side by side instead of one lane at a time
            if (__any_sync(__activemask(), nc == kCL)) flush();
          } else {
            if (nc == kCL) flush();
          }
        }
      };
      if (__any_sync(__activemask(), e - a > 3u * kDenseBox)) run(std::true_type{});
      else run(std::false_type{});
    }
    flush();
    if (nband > (unsigned)kBQ) {
      cnt = band_rescan(i, sx, sy, sz, p4, start, ix, iy, iz, d0, d1, d2, pi, Lf, R2lo, R2hi, R2);
    } else {
      for (unsigned k = 0; k < nband; ++k) cnt += fp64_within(i, s_bq[k][t], sx, sy, sz, R2);
    }
    cnt -= 1u;  // the agent itself
    float Dx, Dy, Dz;
    capped_displacement(Fx, Fy, Fz, c.dtf, c.capf, Dx, Dy, Dz);
    const double nx = __dadd_rn(xi, f2d_exact(Dx));
    const double ny = __dadd_rn(yi, f2d_exact(Dy));
    const double nz = __dadd_rn(zi, f2d_exact(Dz));
    ox[i] = nx;
    oy[i] = ny;
    oz[i] = nz;
    nbr[i] = cnt;
    const unsigned long long e0 = enc_double(nx), e1 = enc_double(ny), e2 = enc_double(nz);
    mn[0] = e0 < mn[0] ? e0 : mn[0]; mx[0] = e0 > mx[0] ? e0 : mx[0];
    mn[1] = e1 < mn[1] ? e1 : mn[1]; mx[1] = e1 > mx[1] ? e1 : mx[1];
    mn[2] = e2 < mn[2] ? e2 : mn[2]; mx[2] = e2 > mx[2] ? e2 : mx[2];
    const unsigned dbits = __float_as_uint(2.0f * pi.w);
    md = dbits > md ? dbits : md;
  }
  block_commit_bounds<kFT>(mn, mx, md, g);
}

// ---------------------------------------------------------------------------------------------
// Neighbour-list steps (skin > 0).  A rebuild step lists, per agent, every candidate within R + skin
// found by the 27-box walk on a grid whose box length is at least R + skin ((j << 5) |
// (row * 3 + box x), in the rebuild's box order: k_list_build).  Every step then evaluates the
// lists (k_force_skin<false>): while no agent has moved more than skin / 2 since the rebuild, every
// pair within R was within R + skin at the rebuild, so every neighbour and contact is listed.
// Counts use the same FP32 band + FP64 decision as the walk, so they stay exact; the FP32 force sums
// follow the list (the box order of the last rebuild).  If a list overflowed, that step's
// forces come from the walk itself (k_force_skin<true>) and the next step rebuilds.  Both apply the
// capped displacement themselves, into the other of two alternating position sets.
// ---------------------------------------------------------------------------------------------

// List layout: the entries of the 32 agents of one warp-sized group are interleaved, entry k of agent
// i at (i / 32) * 32 * kListCap + k * 32 + i % 32, so entry k of a warp's agents is one 128-byte
// line and every line read is fully used.
__device__ __forceinline__ size_t list_at(unsigned i, unsigned k) {
  return (size_t)(i >> 5) * (32u * kListCap) + (size_t)k * 32u + (i & 31u);
}

// Neighbour count of agent i over its m listed candidates, each decided from one d^2 (used when the
// band queue overflows).
__device__ __noinline__ unsigned list_rescan(unsigned i, unsigned m, const unsigned* __restrict__ list,
                                             const double* __restrict__ sx,
                                             const double* __restrict__ sy,
                                             const double* __restrict__ sz,
                                             const float4* __restrict__ p4, float4 pi, float Lf,
                                             float R2lo, float R2hi, double R2) {
  unsigned k = 0;
  for (unsigned e = 0; e < m; ++e) {
    const unsigned v = list[list_at(i, e)];
    const unsigned j = v >> 5, cc = v & 31u;
    const float4 q = p4[j];
    const int sgk = (int)(cc / 3u), bxk = (int)(cc % 3u);
    const float ex = (pi.x - (float)(bxk - 1) * Lf) - q.x;
    const float ey = pi.y - (float)(sgk % 3 - 1) * Lf - q.y;
    const float ez = pi.z - (float)(sgk / 3 - 1) * Lf - q.z;
    const float dd = pair_d2(ex, ey, ez);
    if (dd < R2lo) ++k;
    else if (dd <= R2hi) k += fp64_within_call(i, j, sx, sy, sz, R2);
  }
  return k;
}

// Positions of a list step live in two sets that alternate every step (centres FP64, offsets FP32):
// the kernel reads the current set and writes the next, so every neighbour read sees step-start
// values while each agent's own update is written at once (no separate update pass).  On a rebuild
// step the centres come from the gather's set and the offsets from the current set's offset buffer,
// which the gather has overwritten in box order.
template <bool BUILD, bool SKIP = false>
__global__ void __launch_bounds__(kFT, BUILD ? 3 : 4) k_force_skin(
    const double* __restrict__ gx, const double* __restrict__ gy, const double* __restrict__ gz,
    const double* __restrict__ px, const double* __restrict__ py, const double* __restrict__ pz,
    const float4* __restrict__ p4, double* __restrict__ ox, double* __restrict__ oy,
    double* __restrict__ oz, float4* __restrict__ op4, unsigned* __restrict__ skey,
    const unsigned* __restrict__ start, unsigned* __restrict__ list, unsigned* __restrict__ list_n,
    float* __restrict__ disp, unsigned* __restrict__ nbr,
    unsigned* __restrict__ wnext, WarpBounds* __restrict__ wcache,
    const unsigned* __restrict__ evl, double* __restrict__ rx, double* __restrict__ ry,
    double* __restrict__ rz, DevGrid* g, MechConsts c) {
  // BUILD: the walk with forces, only on a rebuild step whose lists overflowed; otherwise the lists
  // (built by k_list_build on a rebuild step) give the forces
  if (BUILD ? !(g->rebuild && g->list_overflow) : g->list_overflow != 0u) return;
  __shared__ unsigned s_cj[kCL][kFT];       // candidate list: index
  __shared__ unsigned char s_cc[kCL][kFT];  // candidate list: row segment * 3 + box x
  __shared__ unsigned s_bq[kBQ][kFT];       // band queue: candidates decided in FP64 after the loop
  // per-thread bounds of the new centres, largest diameter and move since the rebuild (kept in
  // shared memory: the loop already uses every register the occupancy target allows)
  __shared__ unsigned long long s_mn[3][kFT], s_mx[3][kFT];
  __shared__ unsigned s_md[kFT];
  __shared__ float s_dm[kFT];
  // list steps: the next agent's offsets, list length and first four entries are copied ahead
  // (double-buffered), and this agent's FP64 centre and move arrive during its force loop
  __shared__ float4 s_pi[2][kFT];
  __shared__ unsigned s_m[2][kFT];
  __shared__ unsigned s_v[2][4][kFT];
  __shared__ double s_c[3][kFT];
  __shared__ float s_d[kFT];
  const unsigned n = g->nbox ? g->n : 0u;
  const bool rb = g->rebuild != 0u;
  // step-start centres: gathered on a rebuild step, the current set otherwise
  const double* __restrict__ sx = rb ? gx : px;
  const double* __restrict__ sy = rb ? gy : py;
  const double* __restrict__ sz = rb ? gz : pz;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const double R2 = g->R2;
  const float Lf = BUILD ? g->Lf : g->Lf_list, R2lo = g->R2lo, R2hi = g->R2hi, L2 = g->list_L2f;
  const int t = threadIdx.x;
  // candidate offset shift of each box code (row * 3 + box x): exact multiples of the box length
  __shared__ float4 s_shift[27];
  if (t < 27) {
    const int row = t / 3, bx = t % 3;
    s_shift[t] = make_float4(-(float)(bx - 1) * Lf, -(float)(row % 3 - 1) * Lf,
                             -(float)(row / 3 - 1) * Lf, 0.f);
  }
  for (int a = 0; a < 3; ++a) {
    s_mn[a][t] = ~0ull;
    s_mx[a][t] = 0ull;
  }
  s_md[t] = 0u;
  s_dm[t] = 0.f;
  __syncthreads();
  const unsigned stride = gridDim.x * blockDim.x;
  auto prefetch = [&](unsigned a, int b) {  // list step: agent a's offsets, list length, entries 0-3
    cp_async_n<16>(&s_pi[b][t], p4 + a);
    cp_async_n<4>(&s_m[b][t], list_n + a);
#pragma unroll
    for (int u = 0; u < 4; ++u) cp_async_n<4>(&s_v[b][u][t], list + list_at(a, (unsigned)u));
  };
  int buf = 0;
  // The agents this launch evaluates: every agent, or with the stationary skip the warps (32
  // consecutive agents) that k_still_warps listed.  There a lane past the last agent repeats the
  // last agent, so the warp stays whole and writes the same values twice.
  const unsigned lane = (unsigned)t & 31u;
  unsigned k = SKIP ? (blockIdx.x * blockDim.x + threadIdx.x) >> 5 : blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned kstep = SKIP ? stride >> 5 : stride;
  const unsigned kend = SKIP ? (n ? g->n_eval : 0u) : n;
  auto agent = [&](unsigned w) -> unsigned {
    const unsigned a = w * 32u + lane;
    return a < n ? a : n - 1u;
  };
  // listed warps of this and the next iteration (loaded one iteration ahead of their use)
  unsigned wcur = 0, wnxt = 0, wnn = 0;
  if constexpr (SKIP) {
    if (k < kend) wcur = __ldg(evl + k);
    if (k + kstep < kend) wnxt = __ldg(evl + k + kstep);
  }
  if constexpr (!BUILD) {
    if (k < kend) prefetch(SKIP ? agent(wcur) : k, 0);
    cp_async_commit();
  }
  for (; k < kend; k += kstep, wcur = wnxt, wnxt = wnn) {
    const unsigned i = SKIP ? agent(wcur) : k;
    if constexpr (SKIP) wnn = k + 2u * kstep < kend ? __ldg(evl + k + 2u * kstep) : 0u;
    float4 pi;
    double x0 = 0.0, y0 = 0.0, z0 = 0.0;  // this agent's step-start centre
    float dprev = 0.f;
    if constexpr (BUILD) {
      pi = __ldg(p4 + i);
    } else {
      cp_async_n<8>(&s_c[0][t], sx + i);
      cp_async_n<8>(&s_c[1][t], sy + i);
      cp_async_n<8>(&s_c[2][t], sz + i);
      cp_async_n<4>(&s_d[t], disp + i);
      cp_async_commit();
      if (k + kstep < kend) prefetch(SKIP ? agent(wnxt) : i + stride, buf ^ 1);
      cp_async_commit();
      cp_async_wait<2>();  // this agent's prefetch (issued one iteration earlier) has landed
      pi = s_pi[buf][t];
    }
    const float pxm = pi.x + Lf, px0 = pi.x, pxp = pi.x - Lf;  // neighbour box at x-1, x, x+1
    unsigned cnt = 0;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    int nc = 0;
    unsigned nband = 0;
    auto flush = [&]() {  // count, band queue and force law over the staged candidates, in order
      for (int k = 0; k < nc; ++k) {
        const unsigned cj = s_cj[k][t], cc = s_cc[k][t];
        const float4 q = __ldg(p4 + cj);
        const int sgk = (int)(cc / 3u), bxk = (int)(cc % 3u);
        const float ex = (bxk == 0 ? pxm : (bxk == 1 ? px0 : pxp)) - q.x;
        const float ey = pi.y - (float)(sgk % 3 - 1) * Lf - q.y;
        const float ez = pi.z - (float)(sgk / 3 - 1) * Lf - q.z;
        const float dd = pair_d2(ex, ey, ez);
        if (dd < R2lo) {
          ++cnt;
        } else {  // near R: queued for the FP64 decision after the loop
          if (nband < (unsigned)kBQ) s_bq[nband][t] = cj;
          ++nband;
        }
        const float rs = pi.w + q.w;
        if (dd < rs * rs && dd > 0.f) contact_force(Fx, Fy, Fz, ex, ey, ez, pi.w, q.w, c.kf, c.gammaf);
      }
      nc = 0;
    };
    if constexpr (BUILD) {
      const unsigned b = __ldg(skey + i);
      const int ix = (int)(b % (unsigned)d0);
      const unsigned q0 = b / (unsigned)d0;
      const int iy = (int)(q0 % (unsigned)d1), iz = (int)(q0 / (unsigned)d1);
      const int xl = ix > 0 ? ix - 1 : 0, xh = ix + 1 < d0 ? ix + 1 : ix;
      unsigned ln = 0;
#pragma unroll 1
      for (int sg = 0; sg < 9; ++sg) {
        const int jz = iz + sg / 3 - 1, jy = iy + sg % 3 - 1;
        if (jz < 0 || jz >= d2 || jy < 0 || jy >= d1) continue;
        const unsigned row = ((unsigned)jz * (unsigned)d1 + (unsigned)jy) * (unsigned)d0;
        const unsigned a = __ldg(start + row + xl);
        const unsigned m1 = ix > 0 ? __ldg(start + row + ix) : a;  // end of box x-1
        const unsigned m2 = __ldg(start + row + ix + 1);           // end of box x
        const unsigned e = __ldg(start + row + xh + 1);            // end of the run
        const float py = pi.y - (float)(sg % 3 - 1) * Lf, pz = pi.z - (float)(sg / 3 - 1) * Lf;
        auto run = [&](auto dense) {
          for (unsigned j = a; j < e; ++j) {
            const float4 q = __ldg(p4 + j);
            const unsigned bx = j < m1 ? 0u : (j < m2 ? 1u : 2u);
            const float ex = (bx == 0 ? pxm : (bx == 1 ? px0 : pxp)) - q.x;
            const float ey = py - q.y;
            const float ez = pz - q.z;
            const float dd = pair_d2(ex, ey, ez);
            const unsigned code = (unsigned)(sg * 3 + (int)bx);
            if (dd <= L2 && j != i) {  // within R + skin: listed for the steps until the rebuild
              if (ln < kListCap) list[list_at(i, ln)] = (j << 5) | code;
              ++ln;
            }
            s_cj[nc][t] = j;  // kept only if within R (every neighbour, band candidate and contact)
            s_cc[nc][t] = (unsigned char)code;
            nc += dd <= R2hi ? 1 : 0;
            if constexpr (decltype(dense)::value) {
              if (__any_sync(__activemask(), nc == kCL)) flush();
            } else {
              if (nc == kCL) flush();
            }
          }
        };
        if (__any_sync(__activemask(), e - a > 3u * kDenseBox)) run(std::true_type{});
        else run(std::false_type{});
      }
      flush();
      if (nband > (unsigned)kBQ) {
        cnt = band_rescan(i, sx, sy, sz, p4, start, ix, iy, iz, d0, d1, d2, pi, Lf, R2lo, R2hi, R2);
      } else {
        for (unsigned k = 0; k < nband; ++k) cnt += fp64_within(i, s_bq[k][t], sx, sy, sz, R2);
      }
      cnt -= 1u;  // the agent itself
      list_n[i] = ln < kListCap ? ln : kListCap;
      if (ln > kListCap) g->list_overflow = 1u;  // the next step rebuilds again
    } else {
      // four entries at a time, their loads and their candidates' loads issued together, so the loop
      // does not wait on one dependent load pair per entry
      const unsigned m = s_m[buf][t];
      // the warp runs to its longest list (a uniform bound: no lane leaves the loop early; slots
      // past a lane's list are evaluated as far away and add nothing)
      const unsigned mw = __reduce_max_sync(__activemask(), m);  // lanes past n have left the loop
      for (unsigned k0 = 0; k0 < mw; k0 += 4) {
        unsigned v[4];
        if (k0 == 0) {
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = s_v[buf][u][t];
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            v[u] = k0 + (unsigned)u < m ? __ldg(list + list_at(i, k0 + u)) : 0u;
        }
        float4 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          q[u] = k0 + (unsigned)u < m ? __ldg(p4 + (v[u] >> 5)) : make_float4(3.0e4f, 3.0e4f, 3.0e4f, 0.f);
        // the four entries are evaluated without branches (a slot past the list is far away, so it
        // neither counts nor touches), two at a time through the paired FP32 instructions (the same
        // per-component rounding as the scalar ones); contributions are added in list order
        const float2 pxy = make_float2(pi.x, pi.y), m1 = make_float2(-1.f, -1.f);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int a = 2 * hh, b = 2 * hh + 1;
          const float4 sa = s_shift[k0 + (unsigned)a < m ? v[a] & 31u : 13u];
          const float4 sb = s_shift[k0 + (unsigned)b < m ? v[b] & 31u : 13u];
          const float2 exa = __ffma2_rn(make_float2(q[a].x, q[a].y), m1, __fadd2_rn(pxy, make_float2(sa.x, sa.y)));
          const float2 exb = __ffma2_rn(make_float2(q[b].x, q[b].y), m1, __fadd2_rn(pxy, make_float2(sb.x, sb.y)));
          const float eza = (pi.z + sa.z) - q[a].z, ezb = (pi.z + sb.z) - q[b].z;
          const float2 dd = make_float2(pair_d2(exa.x, exa.y, eza), pair_d2(exb.x, exb.y, ezb));
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float d = e ? dd.y : dd.x;
            cnt += d < R2lo ? 1u : 0u;
            if (d >= R2lo && d <= R2hi) {  // near R: queued for the FP64 decision after the loop
              if (nband < (unsigned)kBQ) s_bq[nband][t] = v[e ? b : a] >> 5;
              ++nband;
            }
          }
          const float2 rs = make_float2(pi.w + q[a].w, pi.w + q[b].w);
          const float2 rinv = make_float2(rsqrtf(dd.x), rsqrtf(dd.y));
          const float2 delta = __ffma2_rn(make_float2(-dd.x, -dd.y), rinv, rs);
          // sqrt(rho delta) = sqrt(ri rj delta / rs) = p rsqrt(p rs) with p = ri rj delta
          const float2 pp = __fmul2_rn(make_float2(pi.w * q[a].w, pi.w * q[b].w), delta);
          const float2 tt = __fmul2_rn(pp, rs);
          const float2 gv = __fmul2_rn(make_float2(c.gammaf, c.gammaf),
                                       __fmul2_rn(pp, make_float2(rsqrtf(tt.x), rsqrtf(tt.y))));
          const float2 sc = __fmul2_rn(__ffma2_rn(make_float2(c.kf, c.kf), delta, make_float2(-gv.x, -gv.y)), rinv);
          const float2 rs2 = __fmul2_rn(rs, rs);
          const bool ta = dd.x <= R2hi && dd.x < rs2.x && dd.x > 0.f && delta.x > 0.f;
          const bool tb = dd.y <= R2hi && dd.y < rs2.y && dd.y > 0.f && delta.y > 0.f;
          Fx = ta ? fmaf(sc.x, exa.x, Fx) : Fx;
          Fy = ta ? fmaf(sc.x, exa.y, Fy) : Fy;
          Fz = ta ? fmaf(sc.x, eza, Fz) : Fz;
          Fx = tb ? fmaf(sc.y, exb.x, Fx) : Fx;
          Fy = tb ? fmaf(sc.y, exb.y, Fy) : Fy;
          Fz = tb ? fmaf(sc.y, ezb, Fz) : Fz;
        }
      }
      if (nband > (unsigned)kBQ) {
        cnt = list_rescan(i, m, list, sx, sy, sz, p4, pi, Lf, R2lo, R2hi, R2);
      } else {
        for (unsigned k = 0; k < nband; ++k) cnt += fp64_within(i, s_bq[k][t], sx, sy, sz, R2);
      }
    }
    float Dx, Dy, Dz;
    capped_displacement(Fx, Fy, Fz, c.dtf, c.capf, Dx, Dy, Dz);
    nbr[i] = cnt;
    const bool moved = Dx != 0.f || Dy != 0.f || Dz != 0.f;
    // update: FP64 centre += displacement (exact conversion, one FP64 add), FP32 offset +=
    // displacement, move since the rebuild (a list step's box ids are derived on read-out:
    // k_readout_box)
    if constexpr (BUILD) {
      x0 = sx[i];
      y0 = sy[i];
      z0 = sz[i];
    } else {
      cp_async_wait<1>();  // this agent's centre and move (the newest group is the next prefetch)
      x0 = s_c[0][t];
      y0 = s_c[1][t];
      z0 = s_c[2][t];
      dprev = s_d[t];
      buf ^= 1;
    }
    const double nx = __dadd_rn(x0, f2d_exact(Dx));
    const double ny = __dadd_rn(y0, f2d_exact(Dy));
    const double nz = __dadd_rn(z0, f2d_exact(Dz));
    ox[i] = nx;
    oy[i] = ny;
    oz[i] = nz;
    if constexpr (SKIP && !BUILD) {
      // a rebuild step's centres go into both position sets (the current one was consumed by the
      // gather), so on the next step a stationary warp needs no copy: its offsets did not change
      // either (an unmoved agent's offset plus a zero displacement is the same value)
      if (rb) {
        rx[i] = nx;
        ry[i] = ny;
        rz[i] = nz;
      }
    }
    op4[i] = make_float4(pi.x + Dx, pi.y + Dy, pi.z + Dz, pi.w);
    const float D = (rb ? 0.f : dprev) + sqrtf(Dx * Dx + Dy * Dy + Dz * Dz);
    disp[i] = D;
    s_dm[t] = fmaxf(s_dm[t], D);
    const unsigned long long e0 = enc_double(nx), e1 = enc_double(ny), e2 = enc_double(nz);
    s_mn[0][t] = e0 < s_mn[0][t] ? e0 : s_mn[0][t];
    s_mx[0][t] = e0 > s_mx[0][t] ? e0 : s_mx[0][t];
    s_mn[1][t] = e1 < s_mn[1][t] ? e1 : s_mn[1][t];
    s_mx[1][t] = e1 > s_mx[1][t] ? e1 : s_mx[1][t];
    s_mn[2][t] = e2 < s_mn[2][t] ? e2 : s_mn[2][t];
    s_mx[2][t] = e2 > s_mx[2][t] ? e2 : s_mx[2][t];
    const unsigned dbits = __float_as_uint(2.0f * pi.w);
    s_md[t] = dbits > s_md[t] ? dbits : s_md[t];
    if constexpr (SKIP && !BUILD) {
      // the warp's cache: bounds of its new centres, its largest diameter and move (lanes past n
      // have left the loop; the active lanes are a prefix of the warp)
      // (the warp is whole: a lane past the last agent repeats the last agent)
      const unsigned am = 0xFFFFFFFFu;
      const unsigned ee[3] = {(unsigned)(e0 >> 32), (unsigned)(e1 >> 32), (unsigned)(e2 >> 32)};
      const unsigned el[3] = {(unsigned)e0, (unsigned)e1, (unsigned)e2};
      WarpBounds wb;
#pragma unroll
      for (int a = 0; a < 3; ++a) {  // 64-bit min / max from two 32-bit warp reductions each
        const unsigned hn = __reduce_min_sync(am, ee[a]), hx = __reduce_max_sync(am, ee[a]);
        const unsigned ln = __reduce_min_sync(am, ee[a] == hn ? el[a] : ~0u);
        const unsigned lx = __reduce_max_sync(am, ee[a] == hx ? el[a] : 0u);
        wb.mn[a] = ((unsigned long long)hn << 32) | ln;
        wb.mx[a] = ((unsigned long long)hx << 32) | lx;
      }
      wb.md = __reduce_max_sync(am, dbits);
      wb.dm = __uint_as_float(__reduce_max_sync(am, __float_as_uint(D)));  // D >= 0
      const unsigned anymoved = __ballot_sync(am, moved);
      if ((t & 31) == 0) {
        wcache[i >> 5] = wb;
        wnext[i >> 5] = anymoved;  // lane l: agent 32 (i >> 5) + l (a repeated last agent adds
                                   // its own bit again or a bit past the last agent, never read)
      }
    }
  }
  if constexpr (!BUILD) cp_async_wait<0>();
  __shared__ unsigned s_dmax;
  if (t == 0) s_dmax = 0u;
  __syncthreads();
  // non-negative floats order like their bits
  const unsigned wmax =
      warp_reduce(__float_as_uint(s_dm[t]), [](unsigned a, unsigned b) { return a > b ? a : b; });
  if ((t & 31) == 0 && wmax) atomicMax(&s_dmax, wmax);
  unsigned long long mn[3] = {s_mn[0][t], s_mn[1][t], s_mn[2][t]};
  unsigned long long mx[3] = {s_mx[0][t], s_mx[1][t], s_mx[2][t]};
  block_commit_bounds<kFT>(mn, mx, s_md[t], g);  // contains a __syncthreads
  if (t == 0 && s_dmax) atomicMax(&g->max_disp, s_dmax);
}

// Lists of a rebuild step: the 27-box walk on a grid of box length >= R + skin, keeping
// every candidate within R + skin (no forces; the list kernel computes them from the lists).  The
// nine row runs of an agent (each its boxes x-1, x, x+1, contiguous in the box order) are
// first collected into a per-thread table in shared memory, all 36 run bounds loaded at once; the
// candidates of all runs are then visited in ONE loop, so a warp's lanes, whose runs differ in
// length, wait only for the lane with the most candidates in total rather than for the longest run
// of every row.  Entries are written in the box order (boxes by key, a box's agents along x).
constexpr int kLB = 256;  // threads per block of the list build

__global__ void __launch_bounds__(kLB) k_list_build(const float4* __restrict__ p4,
                                                    const unsigned* __restrict__ skey,
                                                    const unsigned* __restrict__ start,
                                                    unsigned* __restrict__ list,
                                                    unsigned* __restrict__ list_n, DevGrid* g) {
  if (!g->rebuild) return;
  // non-empty row runs: (first | row << 27, end of box x-1, end of box x, end of run)
  __shared__ uint4 s_run[9][kLB];
  const unsigned n = g->nbox ? g->n : 0u;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const float Lf = g->Lf, L2 = g->list_L2f;
  const int t = threadIdx.x;
  unsigned overflow = 0, listed = 0;
  for (unsigned i = blockIdx.x * kLB + (unsigned)t; i < n; i += gridDim.x * kLB) {
    const unsigned b = __ldg(skey + i);
    const int ix = (int)(b % (unsigned)d0);
    const unsigned q0 = b / (unsigned)d0;
    const int iy = (int)(q0 % (unsigned)d1), iz = (int)(q0 / (unsigned)d1);
    const float4 pi = __ldg(p4 + i);
    unsigned nr = 0, pb1 = 0, pb2 = 0;  // runs in all, before the dz = 0 plane, before dz = +1
#pragma unroll
    for (int sg = 0; sg < 9; ++sg) {
      if (sg == 3) pb1 = nr;
      if (sg == 6) pb2 = nr;
      const int jz = iz + sg / 3 - 1, jy = iy + sg % 3 - 1;
      if (jz < 0 || jz >= d2 || jy < 0 || jy >= d1) continue;
      const unsigned row = ((unsigned)jz * (unsigned)d1 + (unsigned)jy) * (unsigned)d0 + (unsigned)ix;
      const unsigned e1 = __ldg(start + row), e2 = __ldg(start + row + 1);
      const unsigned e0 = ix > 0 ? __ldg(start + row - 1) : e1;
      const unsigned e3 = ix + 1 < d0 ? __ldg(start + row + 2) : e2;
      if (e3 > e0) s_run[nr++][t] = make_uint4(e0 | ((unsigned)sg << 27), e1, e2, e3);
    }
    unsigned ln = 0;
    // one loop per z plane of three rows: the warp's lanes stay within the same three row ranges
    // (shared cache lines), and wait only for the lane with the most candidates in the plane
    for (int pl = 0; pl < 3; ++pl) {
      unsigned r = pl == 0 ? 0u : (pl == 1 ? pb1 : pb2);
      const unsigned r1 = pl == 0 ? pb1 : (pl == 1 ? pb2 : nr);
      if (r == r1) continue;
      uint4 run = s_run[r][t];
      unsigned j = run.x & 0x7FFFFFFu, cb = (run.x >> 27) * 3u;
      float py = pi.y - (float)((int)(run.x >> 27) % 3 - 1) * Lf;
      float pz = pi.z - (float)((int)(run.x >> 27) / 3 - 1) * Lf;
      for (;;) {
        const float4 q = __ldg(p4 + j);
        const unsigned bx = (j >= run.y ? 1u : 0u) + (j >= run.z ? 1u : 0u);
        const float ex = (pi.x - (float)((int)bx - 1) * Lf) - q.x;
        const float ey = py - q.y;
        const float ez = pz - q.z;
        const float dd = pair_d2(ex, ey, ez);
        if (dd <= L2 && j != i) {
          if (ln < (unsigned)kListCap) list[list_at(i, ln)] = (j << 5) | (cb + bx);
          ++ln;
        }
        if (++j == run.w) {  // next row run of the plane
          if (++r == r1) break;
          run = s_run[r][t];
          j = run.x & 0x7FFFFFFu;
          cb = (run.x >> 27) * 3u;
          py = pi.y - (float)((int)(run.x >> 27) % 3 - 1) * Lf;
          pz = pi.z - (float)((int)(run.x >> 27) / 3 - 1) * Lf;
        }
      }
    }
    list_n[i] = ln < (unsigned)kListCap ? ln : (unsigned)kListCap;
    overflow |= ln > (unsigned)kListCap ? 1u : 0u;
    listed += ln < (unsigned)kListCap ? ln : (unsigned)kListCap;
  }
  if (overflow) g->list_overflow = 1u;  // this step's forces come from the walk, the next rebuilds
  listed = warp_reduce(listed, [](unsigned a, unsigned b) { return a + b; });
  if ((threadIdx.x & 31) == 0 && listed) atomicAdd(&g->list_entries, (unsigned long long)listed);
}

// Stationary skip, before the list kernel of every step: which warps (32 consecutive agents in the
// sorted order) the list kernel evaluates.  On a list step a warp is left out when its agents and
// every agent of its row ranges kept their positions in the previous step (no moved bit set): its
// agents' force inputs are those of the previous step, so their evaluation would repeat it (zero
// displacement, the same counts).  Nothing of a left-out warp is rewritten: both position sets
// hold its centres and offsets (a rebuild step writes its centres into both), its counts stay, its
// bounds come from its cache, and its moved bits are cleared.  A rebuild renumbers the agents, so a
// rebuild step lists every warp and records the row ranges of the new order.  Box keys grow along
// a warp; for the neighbour row at (dy, dz) the warp's agents in the first agent's row of boxes
// have their candidates between the first agent's box shifted by (-1, dy, dz) and the end of that
// row shifted by (dy, dz), and those in the last agent's row between that row's start shifted and
// the last agent's box shifted by (+1, dy, dz); a warp spanning more rows gets one range from first
// to last.  Clamping at the grid's faces only widens a range.  One thread per warp; the listed
// warps are appended in block order (their order enters no result).
constexpr int kStillT = 256;
__device__ __forceinline__ uint2 row_range(const unsigned* __restrict__ start, long long ka,
                                           long long ke, long long nbox) {
  ka = min(max(ka, 0ll), nbox);
  ke = min(max(ke, 0ll), nbox);
  return make_uint2(__ldg(start + ka), __ldg(start + ke));
}

__global__ void __launch_bounds__(kStillT) k_still_warps(
    const unsigned* __restrict__ skey, const unsigned* __restrict__ start, uint4* __restrict__ wrows,
    size_t ws, const unsigned* __restrict__ wprev, unsigned* __restrict__ wnext,
    const WarpBounds* __restrict__ wcache, unsigned* __restrict__ evl, DevGrid* g) {
  if (g->list_overflow) return;  // this step's forces come from the walk
  const unsigned n = g->nbox ? g->n : 0u;
  const unsigned nw = (n + 31u) / 32u;
  const bool rb = g->rebuild != 0u;
  const long long nbox = (long long)g->nbox, d0 = g->dims[0], d1 = g->dims[1];
  __shared__ unsigned s_cnt[kStillT / 32];
  __shared__ unsigned s_base;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  unsigned md = 0u, skipped = 0u;
  for (unsigned W0 = blockIdx.x * kStillT; W0 < nw; W0 += gridDim.x * kStillT) {  // block-uniform
    const unsigned W = W0 + (unsigned)t;  // this thread's group; a warp takes 32 consecutive ones
    const bool live = W < nw;
    bool ev = live;
    if (rb) {  // the row ranges of the new order (two per row: the first and last agent's)
      if (live) {
        const long long kf = __ldg(skey + W * 32u), kl = __ldg(skey + min(W * 32u + 31u, n - 1u));
        const long long rf = kf / d0, rl = kl / d0;
#pragma unroll
        for (int sg = 0; sg < 9; ++sg) {
          const long long off = ((long long)(sg / 3 - 1) * d1 + (long long)(sg % 3 - 1)) * d0;
          uint2 r0, r1 = make_uint2(1u, 0u);
          if (rl == rf || rl > rf + 1) {
            r0 = row_range(start, kf + off - 1, kl + off + 2, nbox);
          } else {
            r0 = row_range(start, kf + off - 1, (rf + 1) * d0 + off, nbox);
            r1 = row_range(start, rl * d0 + off, kl + off + 2, nbox);
          }
          wrows[sg * ws + W] = make_uint4(r0.x, r0.y, r1.x, r1.y);
        }
      }
    } else {
      // The warp's 32 groups have their candidates of one row within a window of 64 moved words
      // (2048 agents) from the lowest of their ranges: loaded once by the warp, each lane tests
      // the bits of its two ranges (a range over more than three words, or past the window, counts
      // as moved).  The nine rows' loads are issued together.
      bool dirty = false;
      uint4 rr[9];
#pragma unroll
      for (int sg = 0; sg < 9; ++sg) rr[sg] = live ? wrows[sg * ws + W] : make_uint4(1u, 0u, 1u, 0u);
      unsigned wmin[9], M0[9], M1[9];
#pragma unroll
      for (int sg = 0; sg < 9; ++sg) {
        const unsigned lo0 = rr[sg].y > rr[sg].x ? rr[sg].x : ~0u;
        const unsigned lo1 = rr[sg].w > rr[sg].z ? rr[sg].z : ~0u;
        wmin[sg] = __reduce_min_sync(0xFFFFFFFFu, min(lo0, lo1)) >> 5;  // 2^27 - 1 if all empty
      }
#pragma unroll
      for (int sg = 0; sg < 9; ++sg) {
        M0[sg] = wmin[sg] + lane < nw ? __ldg(wprev + wmin[sg] + lane) : 0u;
        M1[sg] = wmin[sg] + 32u + lane < nw ? __ldg(wprev + wmin[sg] + 32u + lane) : 0u;
      }
#pragma unroll
      for (int sg = 0; sg < 9; ++sg) {
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const unsigned lo = part ? rr[sg].z : rr[sg].x, hi = part ? rr[sg].w : rr[sg].y;
          const bool has = hi > lo;
          const unsigned a = has ? (lo >> 5) - wmin[sg] : 0u;
          const unsigned b = has ? ((hi - 1u) >> 5) - wmin[sg] : 0u;
          if (has && (b - a > 2u || b >= 64u)) dirty = true;
#pragma unroll
          for (unsigned j = 0; j < 3u; ++j) {
            const unsigned wi = min(a + j, 63u);
            const unsigned v0 = __shfl_sync(0xFFFFFFFFu, M0[sg], (int)(wi & 31u));
            const unsigned v1 = __shfl_sync(0xFFFFFFFFu, M1[sg], (int)(wi & 31u));
            if (has && a + j <= b && b < 64u) {
              const unsigned base = (wmin[sg] + a + j) * 32u;
              const unsigned s0 = max(lo, base) - base, s1 = min(hi, base + 32u) - base;
              const unsigned mask = (s1 >= 32u ? ~0u : (1u << s1) - 1u) & ~((1u << s0) - 1u);
              if ((wi < 32u ? v0 : v1) & mask) dirty = true;
            }
          }
        }
      }
      ev = live && dirty;
      if (live && !dirty) {
        wnext[W] = 0u;
        const WarpBounds wb = wcache[W];
        for (int a = 0; a < 3; ++a) {
          mn[a] = wb.mn[a] < mn[a] ? wb.mn[a] : mn[a];
          mx[a] = wb.mx[a] > mx[a] ? wb.mx[a] : mx[a];
        }
        md = wb.md > md ? wb.md : md;
        skipped += min(32u, n - W * 32u);
      }
    }
    // listed groups in thread order, after those other blocks listed before them
    const unsigned m = __ballot_sync(0xFFFFFFFFu, ev);
    if (lane == 0) s_cnt[wid] = (unsigned)__popc(m);
    __syncthreads();
    if (t == 0) {
      unsigned tot = 0;
      for (int w = 0; w < kStillT / 32; ++w) {
        const unsigned c = s_cnt[w];
        s_cnt[w] = tot;
        tot += c;
      }
      s_base = tot ? atomicAdd(&g->n_eval, tot) : 0u;
    }
    __syncthreads();
    if (ev) evl[s_base + s_cnt[wid] + (unsigned)__popc(m & ((1u << lane) - 1u))] = W;
    __syncthreads();  // s_cnt and s_base are rewritten by the next iteration
  }
  // one commit per block (same-address atomics from every warp would queue at L2)
  __shared__ unsigned s_sk[kStillT / 32];
  skipped = warp_reduce(skipped, [](unsigned a, unsigned b) { return a + b; });
  if (lane == 0) s_sk[wid] = skipped;
  block_commit_bounds<kStillT>(mn, mx, md, g);  // contains a __syncthreads
  if (t == 0) {
    unsigned long long tot = 0;
    for (int w = 0; w < kStillT / 32; ++w) tot += s_sk[w];
    if (tot) atomicAdd(&g->skipped, tot);
  }
}

// Box-id read-out after a list step: the box of each agent's step-start centre on that step's grid
// (after a rebuild step the gather has written it).  The step-start centres are the position set
// the step read, the one that is not current after it.  Only agents that took part in the step.
__global__ void __launch_bounds__(kBlock) k_readout_box(const double* __restrict__ x,
                                                        const double* __restrict__ y,
                                                        const double* __restrict__ z,
                                                        unsigned* __restrict__ skey, DevGrid* g) {
  if (g->rebuild) return;
  const unsigned n = g->n_step;
  const long long O0 = g->O[0], O1 = g->O[1], O2 = g->O[2], Lq = g->Lq;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const float inv = g->invLq;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int bx = box_div(quantise(x[i]) - O0, Lq, inv);
    int by = box_div(quantise(y[i]) - O1, Lq, inv);
    int bz = box_div(quantise(z[i]) - O2, Lq, inv);
    if (bx >= d0 || by >= d1 || bz >= d2) {  // impossible by construction of the bounds
      atomicOr(&g->err, (unsigned)ERR_BOUNDS);
      bx = min(bx, d0 - 1); by = min(by, d1 - 1); bz = min(bz, d2 - 1);
    }
    skey[i] = (unsigned)bx + (unsigned)d0 * ((unsigned)by + (unsigned)d1 * (unsigned)bz);
  }
}

// Keep one attribute buffer current: a rebuild's gather writes the canonical order into the other.
__global__ void __launch_bounds__(kBlock) k_attr_copy(AgentArrays src, AgentArrays dst, DevGrid* g) {
  const unsigned n = g->nbox ? g->n_sort : 0u;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    dst.diam[i] = src.diam[i];
    dst.id[i] = src.id[i];
  }
}

// ---------------------------------------------------------------------------------------------
// Force + capped update, mixed precision, warp-shared pairs (tunable alternative to one thread per
// agent).  A warp owns 32 consecutive agents; for each of the nine rows the (agent, candidate)
// pairs of all 32 agents are dealt out evenly over the lanes (owner table in shared memory), so
// lanes stay busy regardless of how candidate counts vary between agents.  Counts are tallied with
// shared-memory integer atomics; contacts are appended in pair order (ballot), which keeps each
// agent's contacts in the canonical order, and each lane then evaluates its own contacts.  Same
// arithmetic and outputs as k_force_mixed.
// ---------------------------------------------------------------------------------------------
constexpr int kPW = kFT / 32;     // warps per CTA
constexpr int kPairCap = 256;     // pairs per chunk of a row (owner table)
constexpr int kConCap = 256;      // contact list per warp
constexpr int kMyCap = 12;        // per-lane contact slots during a flush
constexpr int kBandCap = 32;      // band list per warp

__global__ void __launch_bounds__(kFT, 3) k_force_mixed_pairs(
    const double* __restrict__ sx, const double* __restrict__ sy, const double* __restrict__ sz,
    const float4* __restrict__ p4, const unsigned* __restrict__ skey,
    const unsigned* __restrict__ start, double* __restrict__ ox, double* __restrict__ oy,
    double* __restrict__ oz, unsigned* __restrict__ nbr, DevGrid* g, MechConsts c) {
  __shared__ unsigned char s_own[kPW][kPairCap];
  __shared__ uint4 s_run[kPW][32];
  __shared__ float4 s_pi[kPW][32];
  __shared__ unsigned s_cnt[kPW][32];
  __shared__ unsigned s_cj[kPW][kConCap];
  __shared__ unsigned short s_cinfo[kPW][kConCap];
  __shared__ unsigned short s_my[kPW][kMyCap][32];
  __shared__ unsigned s_bj[kPW][kBandCap];
  __shared__ unsigned char s_bo[kPW][kBandCap];
  __shared__ unsigned s_nb[kPW];
  const unsigned n = g->nbox ? g->n : 0u;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const double R2 = g->R2;
  const float Lf = g->Lf, R2lo = g->R2lo, R2hi = g->R2hi;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  unsigned md = 0;
  const unsigned nwarps = gridDim.x * kPW;
  for (unsigned base = (blockIdx.x * kPW + w) * 32u; base < n; base += nwarps * 32u) {
    const unsigned i = base + lane;
    const bool valid = i < n;
    int ix = 0, iy = 0, iz = 0;
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
      const unsigned b = __ldg(skey + i);
      ix = (int)(b % (unsigned)d0);
      const unsigned q0 = b / (unsigned)d0;
      iy = (int)(q0 % (unsigned)d1);
      iz = (int)(q0 / (unsigned)d1);
      pi = __ldg(p4 + i);
    }
    s_pi[w][lane] = pi;
    s_cnt[w][lane] = 0u;
    if (lane == 0) s_nb[w] = 0u;
    unsigned nc = 0;  // contacts in the list (warp-uniform)
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;
    const int xl = ix > 0 ? ix - 1 : 0, xh = ix + 1 < d0 ? ix + 1 : ix;
    // Force law over the listed contacts: each lane collects its own entries (list order = the
    // canonical order of its candidates) and evaluates them; the list is then empty.
    auto flush = [&]() {
      __syncwarp();
      unsigned k = 0;
      for (unsigned e = 0; e < nc; ++e) {
        const unsigned info = s_cinfo[w][e];
        if ((int)(info & 31u) == lane) {
          if (k == (unsigned)kMyCap) {  // full: evaluate the slots, keep collecting
            for (unsigned t = 0; t < k; ++t) {
              const unsigned ee = s_my[w][t][lane];
              const unsigned inf = s_cinfo[w][ee], cj = s_cj[w][ee];
              const unsigned code = inf >> 5, sgk = code / 3u, bxk = code % 3u;
              const float4 q = __ldg(p4 + cj);
              const float ex = fmaf(-((float)bxk - 1.f), Lf, pi.x) - q.x;
              const float ey = (pi.y - (float)((int)(sgk % 3u) - 1) * Lf) - q.y;
              const float ez = (pi.z - (float)((int)(sgk / 3u) - 1) * Lf) - q.z;
              contact_force(Fx, Fy, Fz, ex, ey, ez, pi.w, q.w, c.kf, c.gammaf);
            }
            k = 0;
          }
          s_my[w][k++][lane] = (unsigned short)e;
        }
      }
      for (unsigned t = 0; t < k; ++t) {
        const unsigned ee = s_my[w][t][lane];
        const unsigned inf = s_cinfo[w][ee], cj = s_cj[w][ee];
        const unsigned code = inf >> 5, sgk = code / 3u, bxk = code % 3u;
        const float4 q = __ldg(p4 + cj);
        const float ex = fmaf(-((float)bxk - 1.f), Lf, pi.x) - q.x;
        const float ey = (pi.y - (float)((int)(sgk % 3u) - 1) * Lf) - q.y;
        const float ez = (pi.z - (float)((int)(sgk / 3u) - 1) * Lf) - q.z;
        contact_force(Fx, Fy, Fz, ex, ey, ez, pi.w, q.w, c.kf, c.gammaf);
      }
      nc = 0;
      __syncwarp();
    };
    __syncwarp();
#pragma unroll 1
    for (int sg = 0; sg < 9; ++sg) {
      const int jz = iz + sg / 3 - 1, jy = iy + sg % 3 - 1;
      uint4 r = make_uint4(0u, 0u, 0u, 0u);  // a, end of box x-1, end of box x, end
      if (valid && jz >= 0 && jz < d2 && jy >= 0 && jy < d1) {
        const unsigned row = ((unsigned)jz * (unsigned)d1 + (unsigned)jy) * (unsigned)d0;
        r.x = __ldg(start + row + xl);
        r.y = ix > 0 ? __ldg(start + row + ix) : r.x;
        r.z = __ldg(start + row + ix + 1);
        r.w = __ldg(start + row + xh + 1);
      }
      const unsigned len = r.w - r.x;
      unsigned P = len;  // inclusive scan over the warp
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xFFFFFFFFu, P, o);
        if (lane >= o) P += t;
      }
      const unsigned T = __shfl_sync(0xFFFFFFFFu, P, 31);
      P -= len;  // exclusive
      s_run[w][lane] = make_uint4(r.x, r.y, r.z, P);
      const float shy = (float)(sg % 3 - 1) * Lf, shz = (float)(sg / 3 - 1) * Lf;
      for (unsigned c0 = 0; c0 < T; c0 += kPairCap) {
        // owner table of pairs [c0, c0 + kPairCap)
        const unsigned lo = P > c0 ? P : c0, hi = min(P + len, c0 + kPairCap);
        for (unsigned p = lo; p < hi; ++p) s_own[w][p - c0] = (unsigned char)lane;
        __syncwarp();
        const unsigned cend = min(T, c0 + kPairCap);
        for (unsigned p0 = c0; p0 < cend; p0 += 32) {
          if (nc + 32u > (unsigned)kConCap) flush();
          const unsigned p = p0 + lane;
          const bool act = p < cend;
          const unsigned o = act ? s_own[w][p - c0] : 0u;
          const uint4 ro = s_run[w][o];
          const float4 po = s_pi[w][o];
          const unsigned j = ro.x + (p - ro.w);
          bool con = false;
          unsigned bx = 0;
          if (act) {
            const float4 q = __ldg(p4 + j);
            bx = j < ro.y ? 0u : (j < ro.z ? 1u : 2u);
            const float ex = fmaf(-((float)bx - 1.f), Lf, po.x) - q.x;
            const float ey = (po.y - shy) - q.y;
            const float ez = (po.z - shz) - q.z;
            const float dd = pair_d2(ex, ey, ez);
            if (dd < R2lo) atomicAdd(&s_cnt[w][o], 1u);
            else if (dd <= R2hi) {
              const unsigned pos = atomicAdd(&s_nb[w], 1u);
              if (pos < (unsigned)kBandCap) {
                s_bj[w][pos] = j;
                s_bo[w][pos] = (unsigned char)o;
              }
            }
            const float rs = po.w + q.w;
            con = dd < rs * rs && dd > 0.f;
          }
          const unsigned M = __ballot_sync(0xFFFFFFFFu, con);
          if (con) {
            const unsigned pos = nc + __popc(M & lt_mask);
            s_cj[w][pos] = j;
            s_cinfo[w][pos] = (unsigned short)(o | ((unsigned)(sg * 3 + (int)bx) << 5));
          }
          nc += __popc(M);
        }
        __syncwarp();
      }
    }
    flush();
    // neighbour count: own tally minus the agent itself, plus band candidates decided in FP64
    unsigned cnt = s_cnt[w][lane] - 1u;
    const unsigned nb = s_nb[w];
    if (nb > (unsigned)kBandCap) {
      // band list overflowed (very rare): every agent of the warp recounts its neighbours, deciding
      // every candidate from one d^2
      if (valid) cnt = band_rescan(i, sx, sy, sz, p4, start, ix, iy, iz, d0, d1, d2,
                                   pi, Lf, R2lo, R2hi, R2) - 1u;
    } else {
      for (unsigned e = 0; e < nb; ++e)
        if (s_bo[w][e] == (unsigned char)lane) cnt += fp64_within(i, s_bj[w][e], sx, sy, sz, R2);
    }
    __syncwarp();
    if (valid) {
      const double xi = sx[i], yi = sy[i], zi = sz[i];
      float Dx, Dy, Dz;
      capped_displacement(Fx, Fy, Fz, c.dtf, c.capf, Dx, Dy, Dz);
      const double nx = __dadd_rn(xi, f2d_exact(Dx));
      const double ny = __dadd_rn(yi, f2d_exact(Dy));
      const double nz = __dadd_rn(zi, f2d_exact(Dz));
      ox[i] = nx;
      oy[i] = ny;
      oz[i] = nz;
      nbr[i] = cnt;
      const unsigned long long e0 = enc_double(nx), e1 = enc_double(ny), e2 = enc_double(nz);
      mn[0] = e0 < mn[0] ? e0 : mn[0]; mx[0] = e0 > mx[0] ? e0 : mx[0];
      mn[1] = e1 < mn[1] ? e1 : mn[1]; mx[1] = e1 > mx[1] ? e1 : mx[1];
      mn[2] = e2 < mn[2] ? e2 : mn[2]; mx[2] = e2 > mx[2] ? e2 : mx[2];
      const unsigned dbits = __float_as_uint(2.0f * pi.w);
      md = dbits > md ? dbits : md;
    }
  }
  block_commit_bounds<kFT>(mn, mx, md, g);
}

int force_fp64_blocks(size_t capacity, int sms) {
  const size_t need = (capacity + kF64 / 32 - 1) / (kF64 / 32);  // one warp per agent
  const size_t cap = (size_t)sms * 16;
  return (int)(need < 1 ? 1 : (need < cap ? need : cap));
}

int force_mixed_blocks_per_sm(int variant) {
  int nb = 0;
  if (variant == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_mixed_pairs, kFT, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_mixed, kFT, 0);
  return nb > 0 ? nb : 1;
}

// ---------------------------------------------------------------------------------------------
// Growth (R7 i, iii): every agent grows by dv; agents reaching vdiv are flagged by id and keep
// their diameter until the division kernel halves them.  Also prepares the division scan.
// ---------------------------------------------------------------------------------------------
constexpr double kPi = 3.141592653589793;

__device__ __forceinline__ float diameter_of(double v) {
  return (float)cbrt(__ddiv_rn(__dmul_rn(v, 6.0), kPi));
}

__global__ void __launch_bounds__(kBlock) k_grow(float* __restrict__ diam,
                                                 const unsigned* __restrict__ id,
                                                 double* __restrict__ vol,
                                                 unsigned* __restrict__ flag, DevGrid* g,
                                                 double dv, double vdiv) {
  const unsigned n = g->n;
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    g->ndiv1 = n + 1;
    g->scan_ctr[1] = 0;
    flag[n] = 0u;
  }
  for (unsigned k = tid; k < n; k += gridDim.x * blockDim.x) {
    const double v = __dadd_rn(vol[k], dv);
    vol[k] = v;
    const bool divides = v >= vdiv;
    flag[id[k]] = divides ? 1u : 0u;
    if (!divides) diam[k] = diameter_of(v);
  }
}

// ---------------------------------------------------------------------------------------------
// Oncology behaviours (readings R13, R14).  Apoptosis at step start: each agent dies with probability
// p (Philox counter (id, step, 4, 0)); survivors keep their relative id order and take the dense ids
// 0..m-1 (scan of the survival flags in id order), and move to the slot of their new id.  Brownian
// migration after the capped mechanical update: sigma times standard normal deviates from the
// Box-Muller transform of Philox words (counter (id, step, 3, 0)), evaluated in FP32 and added to
// the FP64 centre.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_apo_flag(const unsigned* __restrict__ id,
                                                     unsigned* __restrict__ flag, DevGrid* g,
                                                     unsigned long long thr, uint2 key) {
  const unsigned n = g->n;
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid == 0) {
    g->ndiv1 = n + 1;
    g->scan_ctr[1] = 0;
    flag[n] = 0u;
  }
  const unsigned step = (unsigned)g->step;
  for (unsigned k = tid; k < n; k += gridDim.x * blockDim.x) {
    const unsigned myid = id[k];
    const uint4 w = philox10(make_uint4(myid, step, 4u, 0u), key);
    flag[myid] = (unsigned long long)w.x >= thr ? 1u : 0u;
  }
}

__global__ void __launch_bounds__(kBlock) k_apo_compact(
    const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
    AgentArrays src, double* __restrict__ ox, double* __restrict__ oy, double* __restrict__ oz,
    AgentArrays dst, const unsigned* __restrict__ flag, const unsigned* __restrict__ drank,
    DevGrid* g) {
  const unsigned n_old = g->ndiv1 - 1;
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  for (unsigned k = tid; k < n_old; k += gridDim.x * blockDim.x) {
    const unsigned myid = src.id[k];
    if (!flag[myid]) continue;
    const unsigned m = drank[myid];
    ox[m] = x[k];
    oy[m] = y[k];
    oz[m] = z[k];
    dst.diam[m] = src.diam[k];
    dst.id[m] = m;
    if (src.vol) dst.vol[m] = src.vol[k];
  }
  if (tid == 0) g->n = drank[n_old];
}

__global__ void __launch_bounds__(kBlock) k_apo_copy(const double* __restrict__ x,
                                                     const double* __restrict__ y,
                                                     const double* __restrict__ z,
                                                     double* __restrict__ ox, double* __restrict__ oy,
                                                     double* __restrict__ oz, const DevGrid* g) {
  const unsigned n = g->n;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    ox[k] = x[k];
    oy[k] = y[k];
    oz[k] = z[k];
  }
}

// FP64: the deviates in double precision, in the oracle's expressions (the FP64 check path keeps
// its positions within 1e-9 relative); mixed precision: in FP32.
template <bool FP64>
__global__ void __launch_bounds__(kBlock) k_brownian(double* __restrict__ x, double* __restrict__ y,
                                                     double* __restrict__ z,
                                                     const unsigned* __restrict__ id,
                                                     const DevGrid* g, double sigma, uint2 key) {
  const unsigned n = g->nbox ? g->n : 0u;
  const unsigned step = (unsigned)g->step;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint4 w = philox10(make_uint4(id[k], step, 3u, 0u), key);
    if constexpr (FP64) {
      const double u = ((double)w.x + 1.0) * 0x1p-32, v = (double)w.y * 0x1p-32;
      const double u2 = ((double)w.z + 1.0) * 0x1p-32, v2 = (double)w.w * 0x1p-32;
      const double r = sqrt(-2.0 * log(u)), r2 = sqrt(-2.0 * log(u2));
      const double pi2 = 2.0 * 3.141592653589793;
      x[k] = x[k] + sigma * (r * cos(pi2 * v));
      y[k] = y[k] + sigma * (r * sin(pi2 * v));
      z[k] = z[k] + sigma * (r2 * cos(pi2 * v2));
    } else {
      const float u = ((float)w.x + 1.0f) * 0x1p-32f, v = (float)w.y * 0x1p-32f;
      const float u2 = ((float)w.z + 1.0f) * 0x1p-32f, v2 = (float)w.w * 0x1p-32f;
      const float r = sqrtf(-2.0f * logf(u)), r2 = sqrtf(-2.0f * logf(u2));
      float sn, cs;
      sincospif(2.0f * v, &sn, &cs);
      const float cs2 = cospif(2.0f * v2);
      const float sg = (float)sigma;
      x[k] = __dadd_rn(x[k], (double)(sg * (r * cs)));
      y[k] = __dadd_rn(y[k], (double)(sg * (r * sn)));
      z[k] = __dadd_rn(z[k], (double)(sg * (r2 * cs2)));
    }
  }
}

// Division (R7 ii, iv): the m-th divider in id order gets daughter id/slot n_old + m.
__global__ void __launch_bounds__(kBlock) k_divide(double* __restrict__ x, double* __restrict__ y,
                                                   double* __restrict__ z, float* __restrict__ diam,
                                                   unsigned* __restrict__ id,
                                                   double* __restrict__ vol,
                                                   const unsigned* __restrict__ flag,
                                                   const unsigned* __restrict__ drank, DevGrid* g,
                                                   double offset_frac, uint2 key,
                                                   unsigned capacity) {
  const unsigned n_old = g->ndiv1 - 1;
  const unsigned total = drank[n_old];
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  if ((unsigned long long)n_old + total > capacity) {
    if (tid == 0) atomicOr(&g->err, (unsigned)ERR_CAPACITY);
    return;
  }
  const unsigned step = (unsigned)g->step;
  for (unsigned k = tid; k < n_old; k += gridDim.x * blockDim.x) {
    const unsigned myid = id[k];
    if (!flag[myid]) continue;
    const unsigned m = n_old + drank[myid];
    const double half = __dmul_rn(vol[k], 0.5);
    const float df = diameter_of(half);
    double u0 = 0.0, u1 = 0.0, u2 = 1.0;
    for (unsigned attempt = 0; attempt < 64; ++attempt) {
      const uint4 w = philox10(make_uint4(myid, step, 2u, attempt), key);
      const double a = __dsub_rn((double)w.x * 0x1p-31, 1.0);  // w * 2^-31 - 1
      const double bb = __dsub_rn((double)w.y * 0x1p-31, 1.0);
      const double cc = __dsub_rn((double)w.z * 0x1p-31, 1.0);
      const double q = __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(bb, bb)), __dmul_rn(cc, cc));
      if (q <= 1.0 && q >= 0x1p-20) {
        const double len = __dsqrt_rn(q);
        u0 = __ddiv_rn(a, len);
        u1 = __ddiv_rn(bb, len);
        u2 = __ddiv_rn(cc, len);
        break;
      }
    }
    const double o = __dmul_rn(offset_frac, (double)df);
    const double px = x[k], py = y[k], pz = z[k];
    x[m] = __dadd_rn(px, __dmul_rn(o, u0));
    y[m] = __dadd_rn(py, __dmul_rn(o, u1));
    z[m] = __dadd_rn(pz, __dmul_rn(o, u2));
    x[k] = __dsub_rn(px, __dmul_rn(o, u0));
    y[k] = __dsub_rn(py, __dmul_rn(o, u1));
    z[k] = __dsub_rn(pz, __dmul_rn(o, u2));
    vol[k] = half;
    vol[m] = half;
    diam[k] = df;
    diam[m] = df;
    id[m] = m;
  }
  if (tid == 0) g->n = n_old + total;
}

// Secretion (R8): every agent adds q to the voxel holding its centre, clamped into the grid.
__device__ __forceinline__ int voxel_of(double v, double o, double h, int n) {
  const double f = floor(__ddiv_rn(__dsub_rn(v, o), h));
  if (!(f >= 0.0)) return 0;
  if (f >= (double)(n - 1)) return n - 1;
  return (int)f;
}

// Chemotaxis (reading R15): x += chi * grad c, the gradient of the step-start grid at the voxel of
// the step-start centre (central differences inside, one-sided at walls, 0 along a one-voxel axis),
// in FP64 in the oracle's expressions.
__device__ __forceinline__ double grid_derivative(const float* __restrict__ u, int a, int b, int c,
                                                  int nx, int ny, int nz, int axis, double h) {
  const int n = axis == 0 ? nx : (axis == 1 ? ny : nz);
  const int v = axis == 0 ? a : (axis == 1 ? b : c);
  const size_t stride = axis == 0 ? 1u : (axis == 1 ? (size_t)nx : (size_t)nx * (size_t)ny);
  const size_t at = (size_t)a + (size_t)nx * ((size_t)b + (size_t)ny * (size_t)c);
  if (n < 2) return 0.0;
  if (v == 0) return ((double)u[at + stride] - (double)u[at]) / h;
  if (v == n - 1) return ((double)u[at] - (double)u[at - stride]) / h;
  return ((double)u[at + stride] - (double)u[at - stride]) / (2.0 * h);
}

__global__ void __launch_bounds__(kBlock) k_chemotaxis(double* __restrict__ x, double* __restrict__ y,
                                                       double* __restrict__ z,
                                                       const double* __restrict__ sx,
                                                       const double* __restrict__ sy,
                                                       const double* __restrict__ sz,
                                                       const float* __restrict__ grid, const DevGrid* g,
                                                       int nx, int ny, int nz, double ox, double oy,
                                                       double oz, double h, double chi) {
  const unsigned n = g->nbox ? g->n : 0u;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int a = voxel_of(sx[k], ox, h, nx), b = voxel_of(sy[k], oy, h, ny), c = voxel_of(sz[k], oz, h, nz);
    x[k] = x[k] + chi * grid_derivative(grid, a, b, c, nx, ny, nz, 0, h);
    y[k] = y[k] + chi * grid_derivative(grid, a, b, c, nx, ny, nz, 1, h);
    z[k] = z[k] + chi * grid_derivative(grid, a, b, c, nx, ny, nz, 2, h);
  }
}

__global__ void __launch_bounds__(kBlock) k_secrete(const double* __restrict__ x,
                                                    const double* __restrict__ y,
                                                    const double* __restrict__ z,
                                                    float* __restrict__ grid, DevGrid* g, int n0,
                                                    int n1, int n2, double o0, double o1,
                                                    double o2, double h, float q) {
  const unsigned n = g->n;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int a = voxel_of(x[k], o0, h, n0), b = voxel_of(y[k], o1, h, n1),
              c = voxel_of(z[k], o2, h, n2);
    atomicAdd(&grid[(size_t)a + (size_t)n0 * ((size_t)b + (size_t)n1 * (size_t)c)], q);
  }
}

// Read-out in agent-id order.
__global__ void __launch_bounds__(kBlock) k_unsort(
    const double* __restrict__ x, const double* __restrict__ y, const double* __restrict__ z,
    AgentArrays attr, const unsigned* __restrict__ nbr, const unsigned* __restrict__ skey,
    double* __restrict__ ox, double* __restrict__ oy, double* __restrict__ oz,
    float* __restrict__ odiam, double* __restrict__ ovol, unsigned* __restrict__ onbr,
    unsigned* __restrict__ obox, DevGrid* g) {
  const unsigned n = g->n;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned i = attr.id[k];
    if (i >= n) {
      atomicOr(&g->err, (unsigned)ERR_BOUNDS);
      continue;
    }
    if (ox) { ox[i] = x[k]; oy[i] = y[k]; oz[i] = z[k]; }
    if (odiam) odiam[i] = attr.diam[k];
    if (ovol && attr.vol) ovol[i] = attr.vol[k];
    if (onbr) onbr[i] = nbr[k];
    if (obox) obox[i] = skey[k];
  }
}

// Read-out of one coordinate into agent-id order (a read-out of the three runs as three launches, so
// that each coordinate's copy to the host overlaps the next coordinate's permutation).
__global__ void __launch_bounds__(kBlock) k_unsort_axis(const double* __restrict__ src,
                                                        const unsigned* __restrict__ id,
                                                        double* __restrict__ dst, DevGrid* g) {
  const unsigned n = g->n;
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned i = id[k];
    if (i >= n) {
      atomicOr(&g->err, (unsigned)ERR_BOUNDS);
      continue;
    }
    dst[i] = src[k];
  }
}

// Upload of new agents (slots n0 .. n0 + n - 1): validate, assign dense ids, derive volumes
// ((pi/6) d^3 in the order ((pi/6 * d) * d) * d) and clear the per-agent outputs.  The first
// rejected agent (diameter <= 0, non-finite centre, |centre| >= 1e9 um) is recorded in bad_input.
__global__ void __launch_bounds__(kBlock) k_prepare_agents(
    unsigned n0, unsigned n, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const float* __restrict__ diam, unsigned* __restrict__ id,
    double* __restrict__ vol, int derive_volume, unsigned* __restrict__ nbr,
    unsigned* __restrict__ skey, DevGrid* g) {
  if (blockIdx.x == 0 && threadIdx.x == 0) g->fresh = 1u;  // the next rebuild gathers packed agents
  for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const unsigned i = n0 + k;
    const double px = x[i], py = y[i], pz = z[i];
    const float d = diam[i];
    const bool ok = d > 0.0f && fabs(px) < 1e9 && fabs(py) < 1e9 && fabs(pz) < 1e9;  // NaN fails
    if (!ok) atomicMin(&g->bad_input, k);
    id[i] = i;
    if (derive_volume) {
      const double dd = (double)d;
      vol[i] = __dmul_rn(__dmul_rn(__dmul_rn(0.5235987755982988, dd), dd), dd);
    }
    nbr[i] = 0u;
    skey[i] = 0u;
  }
}

__global__ void k_step_done(DevGrid* g) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    g->step += 1ull;
    g->fresh = 0u;
  }
}

// ---- launch wrappers -------------------------------------------------------------------------
void launch_force(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                  MechConsts c, bool mixed, int grid_blocks) {
  if (mixed && c.force_variant == 1)
    k_force_mixed_pairs<<<grid_blocks, kFT, 0, s>>>(b.sorted.x, b.sorted.y, b.sorted.z, b.p4,
                                                    b.skey, b.start, b.pos.x, b.pos.y, b.pos.z,
                                                    b.nbr, g, c);
  else if (mixed)
    k_force_mixed<<<grid_blocks, kFT, 0, s>>>(b.sorted.x, b.sorted.y, b.sorted.z, b.p4, b.skey,
                                              b.start, b.pos.x, b.pos.y, b.pos.z, b.nbr, g, c);
  else
    k_force_fp64<<<grid_blocks, kF64, 0, s>>>(b.sorted.x, b.sorted.y, b.sorted.z, attr.diam,
                                                b.skey, b.start, b.pos.x, b.pos.y, b.pos.z, b.nbr,
                                                g, c);
}

void launch_force_skin(cudaStream_t s, const MechBuffers& b, int cur, DevGrid* g, MechConsts c,
                       bool build, int grid_blocks) {
  const AgentArrays& P = b.pset[cur];
  const AgentArrays& N = b.pset[cur ^ 1];
  if (build)
    k_force_skin<true><<<grid_blocks, kFT, 0, s>>>(b.sorted.x, b.sorted.y, b.sorted.z, P.x, P.y, P.z,
                                                   b.p4set[cur], N.x, N.y, N.z, b.p4set[cur ^ 1],
                                                   b.skey, b.start, b.list, b.list_n, b.disp, b.nbr,
                                                   nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                   g, c);
  else if (c.skip_stationary)
    k_force_skin<false, true><<<grid_blocks, kFT, 0, s>>>(b.sorted.x, b.sorted.y, b.sorted.z, P.x, P.y,
                                                          P.z, b.p4set[cur], N.x, N.y, N.z,
                                                          b.p4set[cur ^ 1], b.skey, b.start, b.list,
                                                          b.list_n, b.disp, b.nbr, b.wmoved[cur ^ 1],
                                                          b.wbounds, b.evl, P.x, P.y, P.z, g, c);
  else
    k_force_skin<false><<<grid_blocks, kFT, 0, s>>>(b.sorted.x, b.sorted.y, b.sorted.z, P.x, P.y, P.z,
                                                    b.p4set[cur], N.x, N.y, N.z, b.p4set[cur ^ 1],
                                                    b.skey, b.start, b.list, b.list_n, b.disp, b.nbr,
                                                    nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                    g, c);
}

void launch_list_build(cudaStream_t s, const MechBuffers& b, DevGrid* g, int grid_blocks) {
  k_list_build<<<grid_blocks, kLB, 0, s>>>(b.p4, b.skey, b.start, b.list, b.list_n, g);
}

void launch_still_warps(cudaStream_t s, const MechBuffers& b, int cur, DevGrid* g, int grid_blocks) {
  // a quarter of the streaming grid: fewer blocks, fewer commits; each block's rows overlap
  k_still_warps<<<grid_blocks / 4 > 0 ? grid_blocks / 4 : 1, kStillT, 0, s>>>(b.skey, b.start, b.wrows, b.wstride, b.wmoved[cur],
                                                b.wmoved[cur ^ 1], b.wbounds, b.evl, g);
}

void launch_readout_box(cudaStream_t s, const AgentArrays& start_pos, unsigned* skey, DevGrid* g,
                        int grid_blocks) {
  k_readout_box<<<grid_blocks, kBlock, 0, s>>>(start_pos.x, start_pos.y, start_pos.z, skey, g);
}

void launch_attr_copy(cudaStream_t s, const AgentArrays& src, const AgentArrays& dst, DevGrid* g,
                      int grid_blocks) {
  k_attr_copy<<<grid_blocks, kBlock, 0, s>>>(src, dst, g);
}

int list_build_blocks_per_sm() {
  int a = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_list_build, kLB, 0);
  return a > 0 ? a : 1;
}

int force_skin_blocks_per_sm(bool build) {
  int a = 0;
  if (build) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_force_skin<true>, kFT, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_force_skin<false>, kFT, 0);
  return a > 0 ? a : 1;
}

void launch_apoptosis_flags(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                            unsigned long long thr, uint2 key, int grid_blocks) {
  k_apo_flag<<<grid_blocks, kBlock, 0, s>>>(attr.id, b.flag, g, thr, key);
}

void launch_apoptosis_compact(cudaStream_t s, const MechBuffers& b, const AgentArrays& src,
                              const AgentArrays& dst, DevGrid* g, int grid_blocks) {
  k_apo_compact<<<grid_blocks, kBlock, 0, s>>>(b.pos.x, b.pos.y, b.pos.z, src, b.sorted.x, b.sorted.y,
                                               b.sorted.z, dst, b.flag, b.drank, g);
  k_apo_copy<<<grid_blocks, kBlock, 0, s>>>(b.sorted.x, b.sorted.y, b.sorted.z, b.pos.x, b.pos.y,
                                            b.pos.z, g);
}

void launch_brownian(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                     double sigma, uint2 key, bool fp64, int grid_blocks) {
  if (fp64) k_brownian<true><<<grid_blocks, kBlock, 0, s>>>(b.pos.x, b.pos.y, b.pos.z, attr.id, g, sigma, key);
  else k_brownian<false><<<grid_blocks, kBlock, 0, s>>>(b.pos.x, b.pos.y, b.pos.z, attr.id, g, sigma, key);
}

void launch_grow(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                 double dv, double vdiv, int grid_blocks) {
  k_grow<<<grid_blocks, kBlock, 0, s>>>(attr.diam, attr.id, attr.vol, b.flag, g, dv, vdiv);
}

void launch_divide(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                   double offset_frac, uint2 key, unsigned capacity, int grid_blocks) {
  k_divide<<<grid_blocks, kBlock, 0, s>>>(b.pos.x, b.pos.y, b.pos.z, attr.diam, attr.id, attr.vol,
                                          b.flag, b.drank, g, offset_frac, key, capacity);
}

void launch_chemotaxis(cudaStream_t s, const MechBuffers& b, DevGrid* g, const float* grid,
                       const int dims[3], const double origin[3], double h, double chi,
                       int grid_blocks) {
  k_chemotaxis<<<grid_blocks, kBlock, 0, s>>>(b.pos.x, b.pos.y, b.pos.z, b.sorted.x, b.sorted.y,
                                              b.sorted.z, grid, g, dims[0], dims[1], dims[2],
                                              origin[0], origin[1], origin[2], h, chi);
}

void launch_secrete(cudaStream_t s, const MechBuffers& b, DevGrid* g, float* grid,
                    const int dims[3], const double origin[3], double h, float q,
                    int grid_blocks) {
  k_secrete<<<grid_blocks, kBlock, 0, s>>>(b.pos.x, b.pos.y, b.pos.z, grid, g, dims[0], dims[1],
                                           dims[2], origin[0], origin[1], origin[2], h, q);
}

void launch_unsort(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                   double* ox, double* oy, double* oz, float* odiam, double* ovol,
                   unsigned* onbr, unsigned* obox, int grid_blocks) {
  k_unsort<<<grid_blocks, kBlock, 0, s>>>(b.pos.x, b.pos.y, b.pos.z, attr, b.nbr, b.skey, ox, oy,
                                          oz, odiam, ovol, onbr, obox, g);
}

void launch_unsort_axis(cudaStream_t s, const double* src, const unsigned* id, double* dst, DevGrid* g,
                        int grid_blocks) {
  k_unsort_axis<<<grid_blocks, kBlock, 0, s>>>(src, id, dst, g);
}

void launch_step_done(cudaStream_t s, DevGrid* g) { k_step_done<<<1, 32, 0, s>>>(g); }

void launch_prepare_agents(cudaStream_t s, unsigned n0, unsigned n, const double* x, const double* y,
                           const double* z, const float* diam, unsigned* id, double* vol,
                           bool derive_volume, unsigned* nbr, unsigned* skey, DevGrid* g,
                           int grid_blocks) {
  k_prepare_agents<<<grid_blocks, kBlock, 0, s>>>(n0, n, x, y, z, diam, id, vol,
                                                  derive_volume ? 1 : 0, nbr, skey, g);
}

}  // namespace bdm
