// neurite.cu -- neurite mechanics: somata (spheres) and neurite elements (cylinders joined as trees)
// on the uniform grid, and the C ABI of include/bdm_neurite.h.
//
// BioDynaMo (arXiv 2006.06775), Sec. "Neuroscience module": an element is a spring with a point
// mass at its distal end, and forces travel along the chain of elements; Sec. "Simulation
// concepts": sphere or cylinder geometry and the uniform grid sized by the largest agent.  The
// force law is the reading stated in include/bdm_neurite.h (R16-R20).
//
// One step, all on the handle's stream (captured once per position parity into a CUDA graph):
//   k_nr_prepare   id order: proximal point, binning point, extent and spring of every agent, and
//                  per-block bounds / largest extent    (reads 84 B, writes 56 B mixed / 72 B FP64)
//   k_nr_finalize  one block: origin, L, box length, boxes per axis
//   k_nr_key       box key + arrival rank (histogram atomics)
//   k_scan         exclusive scan of the histogram (shared with the sphere grid; clears it)
//   k_nr_scatter   each agent's records into box order: mixed, a dense 16 B box-relative binning
//                  point + bound and a 32 B (axis, radius, id, mother) sector; FP64, end points
//                  (64 + 8 B)
//   k_nr_force     one thread per box-ordered slot: the 27 boxes around it (9 runs of 3), neighbour
//                  count, contacts with the lever split, spring; own and passed-up shares in id
//                  order, one 32 B (mixed) or 64 B (FP64) record per agent
//   k_nr_update    id order: own share + daughters' passed-up shares (ascending daughter id),
//                  capped displacement (mixed: FP32, then one FP64 add per axis), new FP64
//                  positions (ping-pong)
// With a skin (mixed precision) the finalize kernel decides on the device whether the step
// rebuilds: a rebuild step bins on boxes of L + skin and k_nr_list_build lists every agent within
// L + skin of each slot; on the other steps k_nr_key and the scan do nothing, the scatter refreshes
// the records in the slots of the last rebuild, and k_nr_force_list evaluates the lists.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "bdm.h"
#include "bdm_neurite.h"
#include "common.cuh"

void bdm_count_launches(unsigned long long k);

using namespace bdm;

namespace {

constexpr int kNrBlock = 256;
constexpr int kNrForceBlock = 128;
constexpr int kNrList = 24;           // contact candidates a thread defers to the second pass
constexpr unsigned kNrSlotBits = 27;  // mixed path: slot index bits of a deferred entry
constexpr int kNrMaxPartials = 2048;  // blocks of the prepare kernel (one bounds record each)
constexpr int kNrPartialWords = 7;    // min xyz, max xyz, largest extent
constexpr unsigned kNrListCap = 128;   // listed agents per slot (skin > 0)
constexpr unsigned kNrListFull = 0xFFFFFFFFu;  // list length of a slot whose list overflowed
constexpr unsigned kNrMaxCadence = 64;  // a rebuild at least every 64 steps

struct NrGrid {
  double origin[3];
  double L, L2, Lbox, invLbox;
  float Lf, L2lo, L2hi, pad;
  int dims[3];
  unsigned nbox, nbox1;
  unsigned scan_ctr[2];
  unsigned err;
  // neighbour lists (mixed precision, skin > 0), decided by the finalize kernel every step
  double L_list;               // L of the last rebuild
  unsigned rebuild;            // 1: this step rebuilds the grid and the lists
  unsigned nbox1_sort;         // items of this step's box scan (nbox + 1, or 0 on list steps)
  unsigned list_valid;         // the lists describe the current agents (cleared by set_agents)
  unsigned since_rebuild;      // steps since the last rebuild
  unsigned max_disp;           // float bits: largest summed move of a point since the rebuild
  float list_L2f;              // (L_list + skin)^2, widened by 2^-10
  unsigned pad2;
  unsigned long long rebuilds, list_entries;
};

struct alignas(32) Dbl4 {
  double x, y, z, w;
};

__device__ __forceinline__ double dot3_rn(double a0, double a1, double a2, double b0, double b1,
                                          double b2) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a0, b0), __dmul_rn(a1, b1)), __dmul_rn(a2, b2));
}

template <typename T>
__device__ __forceinline__ T clamp01(T v) {
  return v < T(0) ? T(0) : (v > T(1) ? T(1) : v);
}

// Closest points of segments P0 + s u and Q0 + t v (s, t in [0, 1]), the argmin of |P(s) - Q(t)|^2
// on the unit square.  Non-parallel segments have a unique minimiser, found by clamping the line
// minimiser in s, taking t optimal for that s, and re-optimising s if t was clamped (Ericson,
// Real-Time Collision Detection, Sec. 5.1.9); den = |u x v|^2 (with FP32 from the cross product,
// which keeps its accuracy for nearly parallel segments).  Segments with den <= 1e-12 |u|^2 |v|^2
// are treated as parallel: the candidates are the four edge minimisers (s = 0, s = 1, t = 0,
// t = 1, each with the clamped optimal other parameter), and the first in that order whose distance
// is within a rounding tolerance of the smallest is taken.  That is reading R18's tie rule for
// parallel segments, whose minimum is not unique.
// Edge minimiser c of the parallel case: s = 0, s = 1, t = 0, t = 1 (c = 0 .. 3), each with the
// clamped optimal other parameter.
template <typename T>
__device__ __forceinline__ void edge_minimiser(int c, T A, T B, T C, T D, T E, T& s, T& t) {
  if (c < 2) {
    s = c == 0 ? T(0) : T(1);
    t = clamp01((c == 0 ? E : B + E) / C);
  } else {
    t = c == 2 ? T(0) : T(1);
    s = clamp01((c == 2 ? -D : B - D) / A);
  }
}

template <typename T>
__device__ __forceinline__ void closest_params(const T P0[3], const T u[3], const T Q0[3],
                                               const T v[3], T& s, T& t) {
  const T w0 = P0[0] - Q0[0], w1 = P0[1] - Q0[1], w2 = P0[2] - Q0[2];
  const T A = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
  const T B = (u[0] * v[0] + u[1] * v[1]) + u[2] * v[2];
  const T C = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
  const T D = (u[0] * w0 + u[1] * w1) + u[2] * w2;
  const T E = (v[0] * w0 + v[1] * w1) + v[2] * w2;
  if (A <= T(0) && C <= T(0)) {
    s = T(0);
    t = T(0);
  } else if (A <= T(0)) {
    s = T(0);
    t = clamp01(E / C);
  } else if (C <= T(0)) {
    t = T(0);
    s = clamp01(-D / A);
  } else {
    T den;
    if (sizeof(T) == 4) {
      const T c0 = u[1] * v[2] - u[2] * v[1], c1 = u[2] * v[0] - u[0] * v[2],
              c2 = u[0] * v[1] - u[1] * v[0];
      den = (c0 * c0 + c1 * c1) + c2 * c2;
    } else {
      den = A * C - B * B;
    }
    if (!(den > T(1e-12) * (A * C))) {
      // parallel (rare): the smallest distance over the four edge minimisers, then the first of
      // them within a rounding tolerance of it (two compact passes, not unrolled, so the force
      // kernel's registers are not spent on this branch)
      const T tol = (sizeof(T) == 4 ? T(1e-5) : T(1e-12)) *
                    ((sqrt(A) + sqrt(C)) + sqrt((w0 * w0 + w1 * w1) + w2 * w2));
      T dmin = T(0);
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
          edge_minimiser<T>(c, A, B, C, D, E, s, t);
          const T d0 = (w0 + s * u[0]) - t * v[0];
          const T d1 = (w1 + s * u[1]) - t * v[1];
          const T d2 = (w2 + s * u[2]) - t * v[2];
          const T dist = sqrt((d0 * d0 + d1 * d1) + d2 * d2);
          if (pass == 0) {
            dmin = c == 0 || dist < dmin ? dist : dmin;
          } else if (dist <= dmin + tol) {
            return;  // s, t of the first edge minimiser within the tolerance
          }
        }
      }
      return;  // not reached: the smallest one is within the tolerance of itself
    }
    s = clamp01((B * E - C * D) / den);
    t = (B * s + E) / C;
    if (t < T(0)) {
      t = T(0);
      s = clamp01(-D / A);
    } else if (t > T(1)) {
      t = T(1);
      s = clamp01((B - D) / A);
    }
  }
}

// Contact of body i (segment qi + s ai, radius ri) with body j: adds the own and passed-up shares of
// the force on i (R18).  Returns nothing when the bodies do not overlap.
template <typename T>
__device__ __forceinline__ void contact(const T qi[3], const T ai[3], T ri, bool i_is_element,
                                        const T qj[3], const T aj[3], T rj, T k, T gam, T keep[3],
                                        T pass[3]) {
  T s, t;
  closest_params(qi, ai, qj, aj, s, t);
  T dv[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) dv[c] = (qi[c] + s * ai[c]) - (qj[c] + t * aj[c]);
  const T d = sqrt((dv[0] * dv[0] + dv[1] * dv[1]) + dv[2] * dv[2]);
  const T delta = (ri + rj) - d;
  if (!(delta > T(0) && d > T(0))) return;
  const T rho = (ri * rj) / (ri + rj);
  const T F = k * delta - gam * sqrt(rho * delta);
  const T w = F / d;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T f = w * dv[c];
    if (i_is_element) {
      keep[c] += s * f;
      pass[c] += (T(1) - s) * f;
    } else {
      keep[c] += f;
    }
  }
}

// mixed records of one box-ordered slot: A = (binning point - box corner, half extent bound) in a
// dense array (the sweep reads only A), and one 32 B sector holding B = (axis p - q, radius) and the
// (id, mother) pair, which only contacts and exclusions read
struct alignas(32) NrRecB {
  float4 B;
  int2 C;
  int2 pad;
};

struct NrRecords {
  Dbl4* A64;     // FP64: (q, r)
  Dbl4* B64;     // FP64: (p, half extent bound)
  float4* A32;   // mixed: A records
  NrRecB* RB;    // mixed: B + (id, mother) records
  int2* C;       // FP64: (id, mother)
};

// ---- per-step kernels ---------------------------------------------------------------------------
// GB300's FP64 pipe is narrow: the streaming kernels keep FP64 to what the exact results need
// (proximal and binning points, lengths -- they decide L and the neighbour counts -- and the
// positions), with one division per agent at most.
// MIXED: the spring force is evaluated in FP32 (from the FP64 axis and length) and stored in spr;
// FP64: it is evaluated in FP64 and stored in spr64.
template <bool MIXED>
__global__ void __launch_bounds__(kNrBlock) k_nr_prepare(
    unsigned n, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const double* __restrict__ diam,
    const double* __restrict__ inv_rest, const int* __restrict__ mother,
    const double* __restrict__ ox, const double* __restrict__ oy, const double* __restrict__ oz,
    double k_spring, double* __restrict__ bx, double* __restrict__ by, double* __restrict__ bz,
    float4* __restrict__ spr, Dbl4* __restrict__ spr64, float4* __restrict__ axr,
    double* __restrict__ partials, const NrGrid* g, const unsigned* __restrict__ key,
    const unsigned* __restrict__ rank, const unsigned* __restrict__ start, NrRecords rec) {
  // with neighbour lists (rec.A32 given) the records also go straight into the slots of the last
  // rebuild: a list step then needs no scatter, and a rebuild step's scatter overwrites them
  const bool direct = MIXED && rec.A32 != nullptr && g->nbox != 0 && g->list_valid;
  const int gd0 = g->dims[0], gd1 = g->dims[1];
  const double Lbox = g->Lbox;
  // bounds in the order-preserving integer encoding of doubles (integer compares; GB300's FP64
  // pipe is narrow)
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull}, ext = 0ull;
  for (unsigned a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
    const double px = x[a], py = y[a], pz = z[a];
    const int m = mother[a];
    double b[3] = {px, py, pz};
    float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
    Dbl4 f64{0.0, 0.0, 0.0, 0.0};
    const double d = diam[a];
    double e = d, len = 0.0;
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (m >= 0) {
      const double qx = __dadd_rn(x[m], ox[a]), qy = __dadd_rn(y[m], oy[a]),
                   qz = __dadd_rn(z[m], oz[a]);
      ax = __dsub_rn(px, qx);
      ay = __dsub_rn(py, qy);
      az = __dsub_rn(pz, qz);
      len = __dsqrt_rn(dot3_rn(ax, ay, az, ax, ay, az));
      b[0] = __dmul_rn(0.5, __dadd_rn(qx, px));
      b[1] = __dmul_rn(0.5, __dadd_rn(qy, py));
      b[2] = __dmul_rn(0.5, __dadd_rn(qz, pz));
      e = __dadd_rn(len, e);
      if (len > 0.0) {
        // spring (R17): T v / l with T = k (l / l0 - 1)
        if constexpr (MIXED) {
          const float lf = (float)len;
          const float w = (float)k_spring * ((float)(len * inv_rest[a]) - 1.f) / lf;
          f = make_float4(w * (float)ax, w * (float)ay, w * (float)az, 0.f);
        } else {
          const double w = k_spring * (len * inv_rest[a] - 1.0) / len;
          f64 = Dbl4{w * ax, w * ay, w * az, 0.0};
        }
      }
    }
    // half extent (half length + radius) rounded up: the contact test's bound
    f.w = __double2float_ru(0.5 * len + 0.5 * d);
    bx[a] = b[0];
    by[a] = b[1];
    bz[a] = b[2];
    spr[a] = f;
    if constexpr (MIXED) {
      const float4 B = make_float4((float)ax, (float)ay, (float)az, (float)(0.5 * d));
      axr[a] = B;
      if (direct) {  // as k_nr_scatter computes them, in the rebuild's slot and box
        const unsigned k = key[a];
        const unsigned slot = start[k] + rank[a];
        const unsigned ix = k % (unsigned)gd0, iy = (k / (unsigned)gd0) % (unsigned)gd1,
                       iz = k / ((unsigned)gd0 * (unsigned)gd1);
        rec.A32[slot] = make_float4((float)(b[0] - (g->origin[0] + (double)ix * Lbox)),
                                    (float)(b[1] - (g->origin[1] + (double)iy * Lbox)),
                                    (float)(b[2] - (g->origin[2] + (double)iz * Lbox)), f.w);
        rec.RB[slot].B = B;
      }
    } else {
      spr64[a] = f64;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const unsigned long long eb = enc_double(b[c]);
      mn[c] = eb < mn[c] ? eb : mn[c];
      mx[c] = eb > mx[c] ? eb : mx[c];
    }
    const unsigned long long ee = enc_double(e);
    ext = ee > ext ? ee : ext;
  }
  __shared__ unsigned long long s_red[kNrBlock / 32][kNrPartialWords];
  unsigned long long v[kNrPartialWords] = {mn[0], mn[1], mn[2], mx[0], mx[1], mx[2], ext};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < kNrPartialWords; ++k) {
      const unsigned long long w = __shfl_down_sync(0xffffffffu, v[k], o);
      v[k] = k < 3 ? (w < v[k] ? w : v[k]) : (w > v[k] ? w : v[k]);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int k = 0; k < kNrPartialWords; ++k) s_red[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x < kNrPartialWords) {
    const int k = threadIdx.x;
    unsigned long long r = s_red[0][k];
    for (int w = 1; w < kNrBlock / 32; ++w) {
      const unsigned long long q = s_red[w][k];
      r = k < 3 ? (q < r ? q : r) : (q > r ? q : r);
    }
    // empty blocks leave the identities: +inf / -inf / 0 once decoded
    partials[blockIdx.x * kNrPartialWords + k] =
        r == ~0ull ? INFINITY : (r == 0ull ? (k < 6 ? -INFINITY : 0.0) : dec_double(r));
  }
}

// One block of kNrBlock threads: reduces the prepare kernel's bounds records and sets up the grid.
// With a skin it first decides whether the step rebuilds: every pair of binning points within L
// now was within L + 2 m at the last rebuild, m the largest summed move of an agent's point since
// then (a binning point, a soma's centre or an element's midpoint, moves at most as far as the
// points that define it), so while 2 m + L - L_rebuild <= skin the lists hold every neighbour and
// every contact, and the grid and slots of the rebuild stay.
__global__ void __launch_bounds__(kNrBlock) k_nr_finalize(const double* __restrict__ partials,
                                                          int nblk, unsigned n, double R,
                                                          unsigned long long box_cap, double skin,
                                                          NrGrid* g) {
  __shared__ double s_red[kNrBlock / 32][kNrPartialWords];
  double v[kNrPartialWords] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < kNrPartialWords; ++k) {
      const double w = partials[b * kNrPartialWords + k];
      v[k] = k < 3 ? fmin(v[k], w) : fmax(v[k], w);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < kNrPartialWords; ++k) {
      const double w = __shfl_down_sync(0xffffffffu, v[k], o);
      v[k] = k < 3 ? fmin(v[k], w) : fmax(v[k], w);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int k = 0; k < kNrPartialWords; ++k) s_red[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < kNrBlock / 32; ++w)
    for (int k = 0; k < kNrPartialWords; ++k)
      s_red[0][k] = k < 3 ? fmin(s_red[0][k], s_red[w][k]) : fmax(s_red[0][k], s_red[w][k]);
  const double* s_v = s_red[0];
  g->scan_ctr[0] = 0;
  g->scan_ctr[1] = 0;
  const double L = fmax(R, s_v[6]);
  g->L = L;
  g->L2 = __dmul_rn(L, L);
  g->L2lo = (float)(g->L2 * (1.0 - 0x1p-14));
  g->L2hi = (float)(g->L2 * (1.0 + 0x1p-14));
  if (n == 0 || !(L > 0.0) || !isfinite(L)) {
    g->nbox = 0;
    g->nbox1 = 0;
    g->nbox1_sort = 0;
    g->rebuild = 0;
    if (n) g->err |= ERR_RADIUS;
    return;
  }
  if (skin > 0.0) {
    if (g->list_valid && g->nbox != 0 && g->since_rebuild + 1u < kNrMaxCadence &&
        2.0 * (double)__uint_as_float(g->max_disp) + (L - g->L_list) <= skin * (1.0 - 1e-6)) {
      g->rebuild = 0u;  // a list step: the grid and the slots of the last rebuild stay
      g->nbox1_sort = 0u;
      g->since_rebuild += 1u;
      return;
    }
    g->L_list = L;
    g->list_valid = 1u;
    g->max_disp = 0u;
    g->since_rebuild = 0u;
    g->rebuilds += 1ull;
    g->list_entries = 0ull;
    g->list_L2f = (float)((L + skin) * (L + skin)) * (1.0f + 1.0f / 1024.0f);
  }
  g->rebuild = 1u;
  g->nbox = 0;
  g->nbox1 = 0;
  g->nbox1_sort = 0;
  const double Lbox = (L + skin) * (1.0 + 0x1p-20);
  double nb = 1.0;
  int dims[3];
  for (int k = 0; k < 3; ++k) {
    const double span = s_v[3 + k] - s_v[k];
    const double c = floor(span / Lbox) + 1.0;
    if (!(c >= 1.0 && c < 2147483647.0)) {
      g->err |= ERR_GRID_OVERFLOW;
      return;
    }
    dims[k] = (int)c;
    nb *= c;
  }
  if (nb > (double)box_cap) {
    g->err |= ERR_GRID_OVERFLOW;
    return;
  }
  for (int k = 0; k < 3; ++k) {
    g->origin[k] = s_v[k];
    g->dims[k] = dims[k];
  }
  g->Lbox = Lbox;
  g->invLbox = 1.0 / Lbox;
  g->Lf = (float)Lbox;
  g->nbox = (unsigned)nb;
  g->nbox1 = (unsigned)nb + 1u;
  g->nbox1_sort = (unsigned)nb + 1u;
}

// Box coordinate: (v - o) / Lbox by the reciprocal.  Its error (a few ulp of at most `dims` box
// units) is far below the 2^-20 widening of the box, so binning points closer than L still land in
// the same or adjacent boxes.
__device__ __forceinline__ int nr_box_coord(double v, double o, double invL, int dim) {
  const int i = (int)floor((v - o) * invL);
  return min(max(i, 0), dim - 1);
}

__global__ void __launch_bounds__(kNrBlock) k_nr_key(unsigned n, const double* __restrict__ bx,
                                                     const double* __restrict__ by,
                                                     const double* __restrict__ bz,
                                                     const NrGrid* g, unsigned* __restrict__ key,
                                                     unsigned* __restrict__ rank,
                                                     unsigned* __restrict__ count) {
  if (g->nbox == 0 || !g->rebuild) return;  // a list step keeps the keys and ranks of the rebuild
  const double invL = g->invLbox;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const double o0 = g->origin[0], o1 = g->origin[1], o2 = g->origin[2];
  for (unsigned a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
    const int ix = nr_box_coord(bx[a], o0, invL, d0);
    const int iy = nr_box_coord(by[a], o1, invL, d1);
    const int iz = nr_box_coord(bz[a], o2, invL, d2);
    const unsigned k = (unsigned)ix + (unsigned)d0 * ((unsigned)iy + (unsigned)d1 * (unsigned)iz);
    key[a] = k;
    rank[a] = atomicAdd(&count[k], 1u);
  }
}

// (id, mother) of a box-ordered slot
template <bool MIXED>
__device__ __forceinline__ int2 rec_c(const NrRecords& rec, unsigned u) {
  if constexpr (MIXED) return rec.RB[u].C;
  else return rec.C[u];
}

template <bool MIXED>
__global__ void __launch_bounds__(kNrBlock) k_nr_scatter(
    unsigned n, const unsigned* __restrict__ key, const unsigned* __restrict__ rank,
    const unsigned* __restrict__ start, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, const double* __restrict__ diam, const int* __restrict__ mother,
    const double* __restrict__ ox, const double* __restrict__ oy, const double* __restrict__ oz,
    const double* __restrict__ bx, const double* __restrict__ by, const double* __restrict__ bz,
    const float4* __restrict__ spr, const float4* __restrict__ axr, const NrGrid* g,
    NrRecords rec, int lists) {
  // with neighbour lists a list step's records were written by k_nr_prepare
  if (g->nbox == 0 || (lists && !g->rebuild)) return;
  const int d0 = g->dims[0], d1 = g->dims[1];
  const double Lbox = g->Lbox;
  for (unsigned a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
    const unsigned k = key[a];
    const unsigned slot = start[k] + rank[a];
    const int m = mother[a];
    if constexpr (MIXED) {
      const unsigned ix = k % (unsigned)d0, iy = (k / (unsigned)d0) % (unsigned)d1,
                     iz = k / ((unsigned)d0 * (unsigned)d1);
      const float o0 = (float)(bx[a] - (g->origin[0] + (double)ix * Lbox));
      const float o1 = (float)(by[a] - (g->origin[1] + (double)iy * Lbox));
      const float o2 = (float)(bz[a] - (g->origin[2] + (double)iz * Lbox));
      rec.A32[slot] = make_float4(o0, o1, o2, spr[a].w);
      NrRecB r;
      r.B = axr[a];
      r.C = make_int2((int)a, m);
      r.pad = make_int2(0, 0);
      rec.RB[slot] = r;
      continue;
    }
    const double p[3] = {x[a], y[a], z[a]};
    double q[3] = {p[0], p[1], p[2]};
    if (m >= 0) {
      q[0] = __dadd_rn(x[m], ox[a]);
      q[1] = __dadd_rn(y[m], oy[a]);
      q[2] = __dadd_rn(z[m], oz[a]);
    }
    const double r = 0.5 * diam[a];
    const float h = spr[a].w;
    rec.C[slot] = make_int2((int)a, m);
    rec.A64[slot] = Dbl4{q[0], q[1], q[2], r};
    rec.B64[slot] = Dbl4{p[0], p[1], p[2], (double)h};
  }
}

// Force kernel output, one record per agent in id order: own share (w: neighbour count) and the
// share passed up to the mother.
struct alignas(32) NrOut32 {
  float4 keep, pass;
};
struct alignas(64) NrOut64 {
  Dbl4 keep, pass;
};

// One thread per box-ordered slot t: agent i = (id of slot t).  The 27 boxes around i's box are
// visited as 9 runs of 3 boxes adjacent in x, whose slots are contiguous.  Neighbours are counted in
// FP64 (R20; the mixed kernel decides in FP32 outside a 2^-14 band around L^2 and re-tests inside it
// in FP64).  A candidate whose binning point is farther than the sum of the two half extents cannot
// touch and skips the closest-point test.  The mixed kernel is held to 64 registers (twice the
// resident warps of its natural allocation).
template <bool MIXED>
__global__ void __launch_bounds__(kNrForceBlock, MIXED ? 8 : 1) k_nr_force(
    unsigned n, const unsigned* __restrict__ start, const unsigned* __restrict__ key,
    const NrGrid* g, NrRecords rec, const double* __restrict__ bx, const double* __restrict__ by,
    const double* __restrict__ bz, const float4* __restrict__ spr, const Dbl4* __restrict__ spr64,
    double k_rep, double gamma, NrOut32* __restrict__ out32, NrOut64* __restrict__ out64) {
  if (g->nbox == 0) return;
  using T = typename std::conditional<MIXED, float, double>::type;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const double L2 = g->L2;
  const float Lf = g->Lf, L2lo = g->L2lo, L2hi = g->L2hi;
  const T k = (T)k_rep, gam = (T)gamma;
  __shared__ unsigned s_def[MIXED ? kNrList : 1][kNrForceBlock];
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int2 ci = rec_c<MIXED>(rec, t);
    const int i = ci.x, mi = ci.y;
    const unsigned kb = key[i];
    const int ix = (int)(kb % (unsigned)d0), iy = (int)((kb / (unsigned)d0) % (unsigned)d1),
              iz = (int)(kb / ((unsigned)d0 * (unsigned)d1));
    const float4 sp = spr[i];
    T keep[3], pass[3];
    if constexpr (MIXED) {
      keep[0] = -sp.x; keep[1] = -sp.y; keep[2] = -sp.z;
      pass[0] = sp.x; pass[1] = sp.y; pass[2] = sp.z;
    } else {
      const Dbl4 s64 = spr64[i];
      keep[0] = -s64.x; keep[1] = -s64.y; keep[2] = -s64.z;
      pass[0] = s64.x; pass[1] = s64.y; pass[2] = s64.z;
    }
    unsigned cnt = 0;
    T qi[3], ai[3], ri;
    const float hi = sp.w;
    float bfi[3] = {0.f, 0.f, 0.f};  // mixed: binning point relative to the box corner
    double bi[3];  // FP64 binning point (FP64 kernel: always; mixed: loaded when a test needs it)
    bool have_bi = false;
    if constexpr (MIXED) {
      const float4 A = rec.A32[t], B = rec.RB[t].B;
      ai[0] = B.x; ai[1] = B.y; ai[2] = B.z; ri = B.w;
      bfi[0] = A.x; bfi[1] = A.y; bfi[2] = A.z;
      // geometry relative to the box corner: q = b - a / 2
      qi[0] = A.x - 0.5f * B.x; qi[1] = A.y - 0.5f * B.y; qi[2] = A.z - 0.5f * B.z;
    } else {
      const Dbl4 A = rec.A64[t], B = rec.B64[t];
      qi[0] = A.x; qi[1] = A.y; qi[2] = A.z; ri = A.w;
      ai[0] = __dsub_rn(B.x, A.x); ai[1] = __dsub_rn(B.y, A.y); ai[2] = __dsub_rn(B.z, A.z);
      bi[0] = __dmul_rn(0.5, __dadd_rn(A.x, B.x));
      bi[1] = __dmul_rn(0.5, __dadd_rn(A.y, B.y));
      bi[2] = __dmul_rn(0.5, __dadd_rn(A.z, B.z));
      have_bi = true;
    }
    const int x0 = max(ix - 1, 0), x1 = min(ix + 1, d0 - 1);
    int ndef = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      const int bz2 = iz + dz;
      if (bz2 < 0 || bz2 >= d2) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int by2 = iy + dy;
        if (by2 < 0 || by2 >= d1) continue;
        const unsigned row = (unsigned)d0 * ((unsigned)by2 + (unsigned)d1 * (unsigned)bz2) + (unsigned)x0;
        // slots of boxes x0..x1 of this row are contiguous: box b of the run holds [s_b, s_b+1);
        // missing boxes (at the grid's x faces) repeat the last bound, so the run ends at s3
        const int nb = x1 - x0 + 1;
        const unsigned s0 = start[row], s1 = start[row + 1];
        const unsigned s2 = nb >= 2 ? start[row + 2] : s1;
        const unsigned s3 = nb >= 3 ? start[row + 3] : s2;
        const float shy = (float)dy * Lf, shz = (float)dz * Lf;
        int bxc = 0;  // box of the run the slot u is in
        unsigned nxt = s1;
        if constexpr (MIXED) {
          // i's binning point minus the candidate box's corner shift: e = ebase - A.xyz
          float ex = bfi[0] - (float)(x0 - ix) * Lf;
          const float ey = bfi[1] - shy, ez = bfi[2] - shz;
          // software-pipelined: the next candidate's record is requested before this one is
          // tested, so each lane keeps two loads in flight
          float4 An = s0 < s3 ? rec.A32[s0] : make_float4(0.f, 0.f, 0.f, 0.f);
          for (unsigned u = s0; u < s3; ++u) {
            const float4 A = An;
            if (u + 1 < s3) An = rec.A32[u + 1];
            while (u >= nxt) {
              ++bxc;
              nxt = bxc == 1 ? s2 : s3;
              ex = bfi[0] - (float)(x0 + bxc - ix) * Lf;
            }
            const float e0 = ex - A.x, e1 = ey - A.y, e2 = ez - A.z;
            const float d2f = (e0 * e0 + e1 * e1) + e2 * e2;
            // beyond L (widened by the FP32 band) j is neither a neighbour nor, by R20, a contact
            if (d2f >= L2hi) continue;
            // i itself has d2f = 0 exactly: it is counted here and taken off after the sweep
            if (d2f < L2lo) {
              ++cnt;
            } else {
              if (!have_bi) {
                bi[0] = bx[i]; bi[1] = by[i]; bi[2] = bz[i];
                have_bi = true;
              }
              const int j = rec_c<MIXED>(rec, u).x;
              const double e[3] = {__dsub_rn(bi[0], bx[j]), __dsub_rn(bi[1], by[j]),
                                   __dsub_rn(bi[2], bz[j])};
              if (dot3_rn(e[0], e[1], e[2], e[0], e[1], e[2]) < L2) ++cnt;
            }
            const float hs = (hi + A.w) * 1.0001f + 1e-4f;
            if (d2f >= hs * hs || u == t) continue;
            const int2 cj = rec_c<MIXED>(rec, u);
            if (mi == cj.x || cj.y == i || (mi >= 0 && mi == cj.y)) continue;
            const int dx = x0 + bxc - ix;
            if (ndef < kNrList) {
              // deferred: evaluated with the warp's other contacts after the sweep
              s_def[ndef][threadIdx.x] = u | ((unsigned)((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)) << kNrSlotBits);
              ++ndef;
              continue;
            }
            const float4 B = rec.RB[u].B;
            const float rel[3] = {A.x + (float)dx * Lf, A.y + shy, A.z + shz};
            const float aj[3] = {B.x, B.y, B.z};
            const float qj[3] = {rel[0] - 0.5f * B.x, rel[1] - 0.5f * B.y, rel[2] - 0.5f * B.z};
            contact<float>(qi, ai, ri, mi >= 0, qj, aj, B.w, k, gam, keep, pass);
          }
        } else {
          for (unsigned u = s0; u < s3; ++u) {
            while (u >= nxt) {
              ++bxc;
              nxt = bxc == 1 ? s2 : s3;
            }
            if (u == t) continue;
            const Dbl4 A = rec.A64[u], B = rec.B64[u];
            const double bj0 = __dmul_rn(0.5, __dadd_rn(A.x, B.x));
            const double bj1 = __dmul_rn(0.5, __dadd_rn(A.y, B.y));
            const double bj2 = __dmul_rn(0.5, __dadd_rn(A.z, B.z));
            const double e0 = __dsub_rn(bi[0], bj0), e1 = __dsub_rn(bi[1], bj1),
                         e2 = __dsub_rn(bi[2], bj2);
            const double dd = dot3_rn(e0, e1, e2, e0, e1, e2);
            if (dd < L2) ++cnt;
            const double hs = (double)hi + B.w;
            if (dd > hs * hs * (1.0 + 1e-12)) continue;
            const int2 cj = rec.C[u];
            if (mi == cj.x || cj.y == i || (mi >= 0 && mi == cj.y)) continue;
            const double qj[3] = {A.x, A.y, A.z};
            const double aj[3] = {__dsub_rn(B.x, A.x), __dsub_rn(B.y, A.y), __dsub_rn(B.z, A.z)};
            contact<double>(qi, ai, ri, mi >= 0, qj, aj, A.w, k, gam, keep, pass);
          }
        }
      }
    }
    if constexpr (MIXED) {
      cnt -= 1u;  // i itself
      // second pass: the deferred contacts (the sweep above only counted and filtered, so lanes
      // run this with far less divergence than contacts evaluated inside the sweep)
      for (int e = 0; e < ndef; ++e) {
        const unsigned w = s_def[e][threadIdx.x];
        const unsigned u = w & ((1u << kNrSlotBits) - 1u), code = w >> kNrSlotBits;
        const int dx = (int)(code % 3u) - 1, dy = (int)((code / 3u) % 3u) - 1, dz = (int)(code / 9u) - 1;
        const float4 A = rec.A32[u], B = rec.RB[u].B;
        const float rel[3] = {A.x + (float)dx * Lf, A.y + (float)dy * Lf, A.z + (float)dz * Lf};
        const float aj[3] = {B.x, B.y, B.z};
        const float qj[3] = {rel[0] - 0.5f * B.x, rel[1] - 0.5f * B.y, rel[2] - 0.5f * B.z};
        contact<float>(qi, ai, ri, mi >= 0, qj, aj, B.w, k, gam, keep, pass);
      }
      NrOut32 o;
      o.keep = make_float4(keep[0], keep[1], keep[2], __uint_as_float(cnt));
      o.pass = make_float4(pass[0], pass[1], pass[2], 0.f);
      out32[i] = o;
    } else {
      NrOut64 o;
      o.keep = Dbl4{keep[0], keep[1], keep[2], (double)cnt};
      o.pass = Dbl4{pass[0], pass[1], pass[2], 0.0};
      out64[i] = o;
    }
  }
}

// Neighbour lists (mixed precision, skin > 0).  Slot t's list holds the slots u != t whose binning
// points lie within L + skin of t's (FP32 box-relative offsets, the radius widened by 2^-10), each
// as u | (box code << 27) in the sweep's order (rows by z then y, boxes by x, slots ascending);
// the entries of 32 consecutive slots are interleaved (entry k of slot t at (t / 32) 32 cap +
// 32 k + t % 32) so that entry k of a warp's slots is one line.
__device__ __forceinline__ size_t nr_list_at(unsigned t, unsigned k) {
  return (size_t)(t >> 5) * (32u * kNrListCap) + (size_t)k * 32u + (t & 31u);
}

// A rebuild step's lists: the 27 boxes around each slot (9 runs of 3 boxes adjacent in x), as the
// sweep visits them.  A slot with more than kNrListCap entries (in a dense region) gets the length
// kNrListFull: the list kernel sweeps its boxes every step instead.
__global__ void __launch_bounds__(kNrForceBlock) k_nr_list_build(
    unsigned n, const unsigned* __restrict__ start, const unsigned* __restrict__ key, NrGrid* g,
    NrRecords rec, unsigned* __restrict__ list, unsigned* __restrict__ list_n) {
  if (g->nbox == 0 || !g->rebuild) return;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const float Lf = g->Lf, LL2 = g->list_L2f;
  unsigned listed = 0u;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int i = rec.RB[t].C.x;
    const unsigned kb = key[i];
    const int ix = (int)(kb % (unsigned)d0), iy = (int)((kb / (unsigned)d0) % (unsigned)d1),
              iz = (int)(kb / ((unsigned)d0 * (unsigned)d1));
    const float4 Ai = rec.A32[t];
    const int x0 = max(ix - 1, 0), x1 = min(ix + 1, d0 - 1);
    unsigned ln = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      const int bz2 = iz + dz;
      if (bz2 < 0 || bz2 >= d2) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int by2 = iy + dy;
        if (by2 < 0 || by2 >= d1) continue;
        const unsigned row = (unsigned)d0 * ((unsigned)by2 + (unsigned)d1 * (unsigned)bz2) + (unsigned)x0;
        const int nb = x1 - x0 + 1;
        const unsigned s0 = start[row], s1 = start[row + 1];
        const unsigned s2 = nb >= 2 ? start[row + 2] : s1;
        const unsigned s3 = nb >= 3 ? start[row + 3] : s2;
        const float ey = Ai.y - (float)dy * Lf, ez = Ai.z - (float)dz * Lf;
        int bxc = 0;
        unsigned nxt = s1;
        float ex = Ai.x - (float)(x0 - ix) * Lf;
        float4 An = s0 < s3 ? rec.A32[s0] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (unsigned u = s0; u < s3; ++u) {
          const float4 A = An;
          if (u + 1 < s3) An = rec.A32[u + 1];
          while (u >= nxt) {
            ++bxc;
            nxt = bxc == 1 ? s2 : s3;
            ex = Ai.x - (float)(x0 + bxc - ix) * Lf;
          }
          const float e0 = ex - A.x, e1 = ey - A.y, e2 = ez - A.z;
          const float d2f = (e0 * e0 + e1 * e1) + e2 * e2;
          if (d2f <= LL2 && u != t) {
            const int dx = x0 + bxc - ix;
            if (ln < kNrListCap)
              list[nr_list_at(t, ln)] = u | ((unsigned)((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)) << kNrSlotBits);
            ++ln;
          }
        }
      }
    }
    list_n[t] = ln <= kNrListCap ? ln : kNrListFull;
    listed += ln <= kNrListCap ? ln : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) listed += __shfl_xor_sync(0xffffffffu, listed, o);
  if ((threadIdx.x & 31) == 0 && listed) atomicAdd(&g->list_entries, (unsigned long long)listed);
}

// Every step with a skin: the neighbour count, contacts and spring of slot t from its list, with
// the sweep's tests in the same order -- FP32 outside a 2^-14 band around L^2 (the step's L), FP64
// inside it; a candidate farther than the sum of the half extents cannot touch; R19's exclusions;
// contacts deferred to a second pass over the lane's deferred entries.  A slot whose list
// overflowed (list length kNrListFull) sweeps its 27 boxes instead, in the same order.
__global__ void __launch_bounds__(kNrForceBlock, 8) k_nr_force_list(
    unsigned n, const unsigned* __restrict__ start, const unsigned* __restrict__ key,
    const NrGrid* g, NrRecords rec, const double* __restrict__ bx, const double* __restrict__ by,
    const double* __restrict__ bz, const float4* __restrict__ spr, double k_rep, double gamma,
    const unsigned* __restrict__ list, const unsigned* __restrict__ list_n,
    NrOut32* __restrict__ out32) {
  if (g->nbox == 0) return;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const double L2 = g->L2;
  const float Lf = g->Lf, L2lo = g->L2lo, L2hi = g->L2hi;
  const float k = (float)k_rep, gam = (float)gamma;
  __shared__ unsigned s_def[kNrList][kNrForceBlock];
  __shared__ float4 s_sh[27];  // candidate shift of each box code: -(dx, dy, dz) L
  if (threadIdx.x < 27) {
    const int c = (int)threadIdx.x;
    s_sh[c] = make_float4(-(float)(c % 3 - 1) * Lf, -(float)((c / 3) % 3 - 1) * Lf,
                          -(float)(c / 9 - 1) * Lf, 0.f);
  }
  __syncthreads();
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int2 ci = rec.RB[t].C;
    const int i = ci.x, mi = ci.y;
    const float4 sp = spr[i];
    float keep[3] = {-sp.x, -sp.y, -sp.z}, pass[3] = {sp.x, sp.y, sp.z};
    unsigned cnt = 0;
    const float hi = sp.w;
    const float4 A = rec.A32[t], B = rec.RB[t].B;
    const float ai[3] = {B.x, B.y, B.z}, ri = B.w;
    const float qi[3] = {A.x - 0.5f * B.x, A.y - 0.5f * B.y, A.z - 0.5f * B.z};
    double bi[3];
    bool have_bi = false;
    int ndef = 0;
    // one candidate: w = u | (box code << 27), Au its A record
    auto consider = [&](unsigned w, const float4& Au) {
      const unsigned u = w & ((1u << kNrSlotBits) - 1u), code = w >> kNrSlotBits;
      const int dx = (int)(code % 3u) - 1, dy = (int)((code / 3u) % 3u) - 1, dz = (int)(code / 9u) - 1;
      const float e0 = (A.x - (float)dx * Lf) - Au.x, e1 = (A.y - (float)dy * Lf) - Au.y,
                  e2 = (A.z - (float)dz * Lf) - Au.z;
      const float d2f = (e0 * e0 + e1 * e1) + e2 * e2;
      if (d2f >= L2hi) return;
      if (d2f < L2lo) {
        ++cnt;
      } else {
        if (!have_bi) {
          bi[0] = bx[i]; bi[1] = by[i]; bi[2] = bz[i];
          have_bi = true;
        }
        const int j = rec.RB[u].C.x;
        const double ed[3] = {__dsub_rn(bi[0], bx[j]), __dsub_rn(bi[1], by[j]), __dsub_rn(bi[2], bz[j])};
        if (dot3_rn(ed[0], ed[1], ed[2], ed[0], ed[1], ed[2]) < L2) ++cnt;
      }
      const float hs = (hi + Au.w) * 1.0001f + 1e-4f;
      if (d2f >= hs * hs) return;
      const int2 cj = rec.RB[u].C;
      if (mi == cj.x || cj.y == i || (mi >= 0 && mi == cj.y)) return;
      if (ndef < kNrList) {
        s_def[ndef][threadIdx.x] = w;
        ++ndef;
        return;
      }
      const float4 Bu = rec.RB[u].B;
      const float rel[3] = {Au.x + (float)dx * Lf, Au.y + (float)dy * Lf, Au.z + (float)dz * Lf};
      const float aj[3] = {Bu.x, Bu.y, Bu.z};
      const float qj[3] = {rel[0] - 0.5f * Bu.x, rel[1] - 0.5f * Bu.y, rel[2] - 0.5f * Bu.z};
      contact<float>(qi, ai, ri, mi >= 0, qj, aj, Bu.w, k, gam, keep, pass);
    };
    const unsigned m0 = list_n[t];
    const bool full = m0 == kNrListFull;
    const unsigned m = full ? 0u : m0;
    // Four entries at a time, their loads issued together; the warp runs to its longest list (a
    // slot past a lane's list reads nothing and tests false).  Counts are taken here; entries
    // close enough to touch are deferred (R19's exclusions are checked with the contacts).
    const unsigned mw = __reduce_max_sync(__activemask(), m);
    for (unsigned k0 = 0; k0 < mw; k0 += 4) {
      unsigned w[4];
      float4 Au[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) w[q] = k0 + (unsigned)q < m ? list[nr_list_at(t, k0 + (unsigned)q)] : 0u;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        Au[q] = k0 + (unsigned)q < m ? rec.A32[w[q] & ((1u << kNrSlotBits) - 1u)]
                                     : make_float4(3.0e4f, 3.0e4f, 3.0e4f, 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool ok = k0 + (unsigned)q < m;
        const float4 sh = s_sh[ok ? w[q] >> kNrSlotBits : 13u];
        const float e0 = (A.x + sh.x) - Au[q].x, e1 = (A.y + sh.y) - Au[q].y,
                    e2 = (A.z + sh.z) - Au[q].z;
        const float d2f = (e0 * e0 + e1 * e1) + e2 * e2;
        cnt += ok && d2f < L2lo ? 1u : 0u;
        if (ok && d2f >= L2lo && d2f < L2hi) {  // inside the band: FP64 decides (rare)
          if (!have_bi) {
            bi[0] = bx[i]; bi[1] = by[i]; bi[2] = bz[i];
            have_bi = true;
          }
          const int j = rec.RB[w[q] & ((1u << kNrSlotBits) - 1u)].C.x;
          const double ed[3] = {__dsub_rn(bi[0], bx[j]), __dsub_rn(bi[1], by[j]), __dsub_rn(bi[2], bz[j])};
          if (dot3_rn(ed[0], ed[1], ed[2], ed[0], ed[1], ed[2]) < L2) ++cnt;
        }
        const float hs = (hi + Au[q].w) * 1.0001f + 1e-4f;
        if (ok && d2f < L2hi && d2f < hs * hs) {
          if (ndef < kNrList) {
            s_def[ndef][threadIdx.x] = w[q];
            ++ndef;
          } else {  // the deferred entries are full: this one now (rare)
            const unsigned u = w[q] & ((1u << kNrSlotBits) - 1u);
            const int2 cj = rec.RB[u].C;
            if (!(mi == cj.x || cj.y == i || (mi >= 0 && mi == cj.y))) {
              const float4 Bu = rec.RB[u].B;
              const float rel[3] = {Au[q].x - sh.x, Au[q].y - sh.y, Au[q].z - sh.z};
              const float aj[3] = {Bu.x, Bu.y, Bu.z};
              const float qj[3] = {rel[0] - 0.5f * Bu.x, rel[1] - 0.5f * Bu.y, rel[2] - 0.5f * Bu.z};
              contact<float>(qi, ai, ri, mi >= 0, qj, aj, Bu.w, k, gam, keep, pass);
            }
          }
        }
      }
    }
    if (full) {  // the list overflowed: the 27 boxes, as the list build visits them
      const unsigned kb = key[i];
      const int ix = (int)(kb % (unsigned)d0), iy = (int)((kb / (unsigned)d0) % (unsigned)d1),
                iz = (int)(kb / ((unsigned)d0 * (unsigned)d1));
      const int x0 = max(ix - 1, 0), x1 = min(ix + 1, d0 - 1);
      for (int dz = -1; dz <= 1; ++dz) {
        const int bz2 = iz + dz;
        if (bz2 < 0 || bz2 >= d2) continue;
        for (int dy = -1; dy <= 1; ++dy) {
          const int by2 = iy + dy;
          if (by2 < 0 || by2 >= d1) continue;
          const unsigned row = (unsigned)d0 * ((unsigned)by2 + (unsigned)d1 * (unsigned)bz2) + (unsigned)x0;
          const int nb = x1 - x0 + 1;
          const unsigned s0 = start[row], s1 = start[row + 1];
          const unsigned s2 = nb >= 2 ? start[row + 2] : s1;
          const unsigned s3 = nb >= 3 ? start[row + 3] : s2;
          int bxc = 0;
          unsigned nxt = s1;
          for (unsigned u = s0; u < s3; ++u) {
            while (u >= nxt) {
              ++bxc;
              nxt = bxc == 1 ? s2 : s3;
            }
            if (u == t) continue;
            const int dx = x0 + bxc - ix;
            consider(u | ((unsigned)((dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)) << kNrSlotBits), rec.A32[u]);
          }
        }
      }
    }
    for (int e = 0; e < ndef; ++e) {
      const unsigned w = s_def[e][threadIdx.x];
      const unsigned u = w & ((1u << kNrSlotBits) - 1u);
      const int2 cj = rec.RB[u].C;
      if (mi == cj.x || cj.y == i || (mi >= 0 && mi == cj.y)) continue;  // R19
      const float4 sh = s_sh[w >> kNrSlotBits];
      const float4 Au = rec.A32[u], Bu = rec.RB[u].B;
      const float rel[3] = {Au.x - sh.x, Au.y - sh.y, Au.z - sh.z};
      const float aj[3] = {Bu.x, Bu.y, Bu.z};
      const float qj[3] = {rel[0] - 0.5f * Bu.x, rel[1] - 0.5f * Bu.y, rel[2] - 0.5f * Bu.z};
      contact<float>(qi, ai, ri, mi >= 0, qj, aj, Bu.w, k, gam, keep, pass);
    }
    NrOut32 o;
    o.keep = make_float4(keep[0], keep[1], keep[2], __uint_as_float(cnt));
    o.pass = make_float4(pass[0], pass[1], pass[2], 0.f);
    out32[i] = o;
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(kNrBlock) k_nr_update(
    unsigned n, const double* __restrict__ x, const double* __restrict__ y,
    const double* __restrict__ z, double* __restrict__ nx, double* __restrict__ ny,
    double* __restrict__ nz, const NrOut32* __restrict__ out32, const NrOut64* __restrict__ out64,
    const unsigned* __restrict__ cstart, const unsigned* __restrict__ clist,
    unsigned* __restrict__ nbr, NrGrid* g, double dt, double cap, float* __restrict__ disp) {
  if (g->nbox == 0) return;
  const double cap2 = cap * cap;
  const float dtf = (float)dt, capf = (float)cap, cap2f = capf * capf;
  // with neighbour lists: each point's summed move since the rebuild, and its largest value
  const bool rb = g->rebuild != 0u;
  float dmax = 0.f;
  for (unsigned a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
    if constexpr (MIXED) {
      // FP32 sum and cap (the shares are FP32), exact conversion, one FP64 add per axis
      const float4 kp = out32[a].keep;
      float F0 = kp.x, F1 = kp.y, F2 = kp.z;
      const unsigned c1 = cstart[a + 1];
      for (unsigned c = cstart[a]; c < c1; ++c) {
        const float4 ps = out32[clist[c]].pass;
        F0 += ps.x; F1 += ps.y; F2 += ps.z;
      }
      float D0 = dtf * F0, D1 = dtf * F1, D2 = dtf * F2;
      const float nn = (D0 * D0 + D1 * D1) + D2 * D2;
      if (nn > cap2f) {
        const float f = capf * rsqrtf(nn);
        D0 *= f; D1 *= f; D2 *= f;
      }
      nx[a] = __dadd_rn(x[a], f2d_exact(D0));
      ny[a] = __dadd_rn(y[a], f2d_exact(D1));
      nz[a] = __dadd_rn(z[a], f2d_exact(D2));
      nbr[a] = __float_as_uint(kp.w);
      if (disp) {
        const float Dm = (rb ? 0.f : disp[a]) + sqrtf((D0 * D0 + D1 * D1) + D2 * D2);
        disp[a] = Dm;
        dmax = fmaxf(dmax, Dm);
      }
      continue;
    }
    double S0, S1, S2;
    unsigned cnt;
    if constexpr (MIXED) {
      const float4 kp = out32[a].keep;
      S0 = kp.x; S1 = kp.y; S2 = kp.z;
      cnt = __float_as_uint(kp.w);
    } else {
      const Dbl4 kp = out64[a].keep;
      S0 = kp.x; S1 = kp.y; S2 = kp.z;
      cnt = (unsigned)kp.w;
    }
    const unsigned c1 = cstart[a + 1];
    for (unsigned c = cstart[a]; c < c1; ++c) {
      const unsigned d = clist[c];
      if constexpr (MIXED) {
        const float4 ps = out32[d].pass;
        S0 += ps.x; S1 += ps.y; S2 += ps.z;
      } else {
        const Dbl4 ps = out64[d].pass;
        S0 += ps.x; S1 += ps.y; S2 += ps.z;
      }
    }
    double D0 = dt * S0, D1 = dt * S1, D2 = dt * S2;
    const double nn = (D0 * D0 + D1 * D1) + D2 * D2;
    if (nn > cap2) {
      const double f = cap / sqrt(nn);
      D0 *= f;
      D1 *= f;
      D2 *= f;
    }
    nx[a] = x[a] + D0;
    ny[a] = y[a] + D1;
    nz[a] = z[a] + D2;
    nbr[a] = cnt;
  }
  if (disp) {  // non-negative floats order like their bits
    unsigned b = __float_as_uint(dmax);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned v = __shfl_xor_sync(0xffffffffu, b, o);
      b = v > b ? v : b;
    }
    if ((threadIdx.x & 31) == 0 && b) atomicMax(&g->max_disp, b);
  }
}

}  // namespace

// ---- handle -------------------------------------------------------------------------------------
struct bdm_neurite {
  bdm_neurite_params p{};
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool poisoned = false;
  bool mixed = true;
  int sms = 152;
  size_t capacity = 0, box_capacity = 0, n = 0;
  NrGrid* g = nullptr;
  NrGrid* gh = nullptr;  // pinned mirror
  double *x[2] = {nullptr, nullptr}, *y[2] = {nullptr, nullptr}, *z[2] = {nullptr, nullptr};
  int cur = 0;
  double *diam = nullptr, *inv_rest = nullptr, *ox = nullptr, *oy = nullptr, *oz = nullptr;
  int* mother = nullptr;
  double *bx = nullptr, *by = nullptr, *bz = nullptr;
  float4* spr = nullptr;  // spring force (xyz, mixed) and half-extent bound (w), id order
  Dbl4* spr64 = nullptr;  // spring force of the FP64 path
  float4* axr = nullptr;  // mixed path: element axis p - q (xyz) and radius (w), id order
  double* partials = nullptr;
  unsigned *key = nullptr, *rank = nullptr, *count = nullptr, *start = nullptr;
  unsigned long long* tiles = nullptr;
  unsigned max_tiles = 0;
  unsigned *cstart = nullptr, *clist = nullptr, *nbr = nullptr;
  unsigned *list = nullptr, *list_n = nullptr;  // skin > 0: neighbour lists by slot
  float* disp = nullptr;                         // skin > 0: summed move since the rebuild
  NrRecords rec{};
  NrOut32* out32 = nullptr;
  NrOut64* out64 = nullptr;
  std::vector<void*> allocs;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  unsigned long long graph_kernels = 0;
  bool capturing = false;
  unsigned long long capture_kernels = 0;
  int blocks_stream = 1216, blocks_prep = 1216, blocks_force = 1216, blocks_scan = 608;
  // profiling
  bool prof = false;
  struct Stat {
    std::string name;
    uint64_t launches = 0;
    double total_ms = 0.0;
  };
  struct Pending {
    int stat;
    cudaEvent_t a, b;
  };
  std::vector<Stat> stats;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
};

namespace {

int nfail(bdm_neurite* s, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (s) s->err = buf;
  return code;
}

#define NCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return nfail(s, BDM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int nalloc(bdm_neurite* s, T** ptr, size_t count) {
  size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  bytes = (bytes + 255) & ~size_t(255);
  void* q = nullptr;
  if (cudaMalloc(&q, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nfail(s, BDM_ENOMEM, "device allocation of %zu bytes failed", bytes);
  }
  s->allocs.push_back(q);
  *ptr = (T*)q;
  return BDM_OK;
}

cudaEvent_t prof_event(bdm_neurite* s) {
  if (!s->free_events.empty()) {
    cudaEvent_t e = s->free_events.back();
    s->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

template <typename F>
int nrun(bdm_neurite* s, const char* name, F&& f) {
  int stat = -1;
  cudaEvent_t a = nullptr, b = nullptr;
  if (s->prof && !s->capturing) {
    for (size_t k = 0; k < s->stats.size(); ++k)
      if (s->stats[k].name == name) stat = (int)k;
    if (stat < 0) {
      s->stats.push_back(bdm_neurite::Stat{name, 0, 0.0});
      stat = (int)s->stats.size() - 1;
    }
    a = prof_event(s);
    b = prof_event(s);
    cudaEventRecord(a, s->stream);
  }
  f();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(s, BDM_ECUDA, "launch of %s failed: %s", name, cudaGetErrorString(e));
  if (s->capturing) s->capture_kernels += 1;
  else bdm_count_launches(1);
  if (stat >= 0) {
    cudaEventRecord(b, s->stream);
    s->pending.push_back(bdm_neurite::Pending{stat, a, b});
  }
  return BDM_OK;
}

#define NRUN(name, body)                               \
  do {                                                 \
    int rc_ = nrun(s, name, [&]() { body; });          \
    if (rc_) return rc_;                               \
  } while (0)

int prof_collect(bdm_neurite* s) {
  NCK(cudaStreamSynchronize(s->stream));
  for (auto& p : s->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    s->stats[p.stat].launches += 1;
    s->stats[p.stat].total_ms += ms;
    s->free_events.push_back(p.a);
    s->free_events.push_back(p.b);
  }
  s->pending.clear();
  return BDM_OK;
}

int enqueue_step(bdm_neurite* s) {
  const unsigned n = (unsigned)s->n;
  cudaStream_t st = s->stream;
  const int c = s->cur, nx = c ^ 1;
  const int bprep = std::max(1, std::min(s->blocks_prep, (int)((n + kNrBlock - 1) / kNrBlock)));
  if (s->mixed)
    NRUN("nr_prepare", (k_nr_prepare<true><<<bprep, kNrBlock, 0, st>>>(
                           n, s->x[c], s->y[c], s->z[c], s->diam, s->inv_rest, s->mother, s->ox,
                           s->oy, s->oz, s->p.spring, s->bx, s->by, s->bz, s->spr, s->spr64,
                           s->axr, s->partials, s->g, s->key, s->rank, s->start,
                           s->p.skin > 0.0 ? s->rec : NrRecords{})));
  else
    NRUN("nr_prepare", (k_nr_prepare<false><<<bprep, kNrBlock, 0, st>>>(
                           n, s->x[c], s->y[c], s->z[c], s->diam, s->inv_rest, s->mother, s->ox,
                           s->oy, s->oz, s->p.spring, s->bx, s->by, s->bz, s->spr, s->spr64,
                           s->axr, s->partials, s->g, s->key, s->rank, s->start, NrRecords{})));
  const bool lists = s->mixed && s->p.skin > 0.0;
  NRUN("nr_finalize", (k_nr_finalize<<<1, kNrBlock, 0, st>>>(s->partials, bprep, n,
                                                              s->p.interaction_radius,
                                                              (unsigned long long)s->box_capacity,
                                                              lists ? s->p.skin : 0.0, s->g)));
  NCK(cudaMemsetAsync(s->tiles, 0, sizeof(unsigned long long) * s->max_tiles, st));
  NRUN("nr_key", (k_nr_key<<<s->blocks_stream, kNrBlock, 0, st>>>(n, s->bx, s->by, s->bz, s->g,
                                                                   s->key, s->rank, s->count)));
  NRUN("nr_scan", launch_scan(st, s->count, s->start, &s->g->nbox1_sort, s->tiles, &s->g->scan_ctr[0],
                              &s->g->err, 1, s->blocks_scan));
  if (s->mixed) {
    NRUN("nr_scatter", (k_nr_scatter<true><<<s->blocks_stream, kNrBlock, 0, st>>>(
                           n, s->key, s->rank, s->start, s->x[c], s->y[c], s->z[c], s->diam,
                           s->mother, s->ox, s->oy, s->oz, s->bx, s->by, s->bz, s->spr, s->axr,
                           s->g, s->rec, lists ? 1 : 0)));
    if (lists)
      NRUN("nr_list_build", (k_nr_list_build<<<s->blocks_force, kNrForceBlock, 0, st>>>(
                                n, s->start, s->key, s->g, s->rec, s->list, s->list_n)));
    if (lists)
      NRUN("nr_force_list", (k_nr_force_list<<<s->blocks_force, kNrForceBlock, 0, st>>>(
                                n, s->start, s->key, s->g, s->rec, s->bx, s->by, s->bz, s->spr,
                                s->p.repulsion, s->p.attraction, s->list, s->list_n, s->out32)));
    else
      NRUN("nr_force", (k_nr_force<true><<<s->blocks_force, kNrForceBlock, 0, st>>>(
                           n, s->start, s->key, s->g, s->rec, s->bx, s->by, s->bz, s->spr,
                           s->spr64, s->p.repulsion, s->p.attraction, s->out32, s->out64)));
    NRUN("nr_update", (k_nr_update<true><<<s->blocks_stream, kNrBlock, 0, st>>>(
                          n, s->x[c], s->y[c], s->z[c], s->x[nx], s->y[nx], s->z[nx], s->out32,
                          s->out64, s->cstart, s->clist, s->nbr, s->g, s->p.dt,
                          s->p.max_displacement, lists ? s->disp : nullptr)));
  } else {
    NRUN("nr_scatter", (k_nr_scatter<false><<<s->blocks_stream, kNrBlock, 0, st>>>(
                           n, s->key, s->rank, s->start, s->x[c], s->y[c], s->z[c], s->diam,
                           s->mother, s->ox, s->oy, s->oz, s->bx, s->by, s->bz, s->spr, s->axr,
                           s->g, s->rec, lists ? 1 : 0)));
    NRUN("nr_force", (k_nr_force<false><<<s->blocks_force, kNrForceBlock, 0, st>>>(
                         n, s->start, s->key, s->g, s->rec, s->bx, s->by, s->bz, s->spr,
                         s->spr64, s->p.repulsion, s->p.attraction, s->out32, s->out64)));
    NRUN("nr_update", (k_nr_update<false><<<s->blocks_stream, kNrBlock, 0, st>>>(
                          n, s->x[c], s->y[c], s->z[c], s->x[nx], s->y[nx], s->z[nx], s->out32,
                          s->out64, s->cstart, s->clist, s->nbr, s->g, s->p.dt,
                          s->p.max_displacement, nullptr)));
  }
  s->cur = nx;
  return BDM_OK;
}

void drop_graphs(bdm_neurite* s) {
  for (auto& gr : s->graph) {
    if (gr) cudaGraphExecDestroy(gr);
    gr = nullptr;
  }
}

int decode(bdm_neurite* s, unsigned e) {
  if (!e) return BDM_OK;
  s->poisoned = true;
  if (e & ERR_GRID_OVERFLOW) return nfail(s, BDM_ENOMEM, "the grid needs more boxes than box_capacity");
  if (e & ERR_TIMEOUT) return nfail(s, BDM_ETIMEOUT, "a bounded scan wait ran out");
  if (e & ERR_RADIUS) return nfail(s, BDM_ESTATE, "non-finite or zero neighbour radius");
  return nfail(s, BDM_ESTATE, "device error bits 0x%x", e);
}

}  // namespace

extern "C" {

int bdm_neurite_create(const bdm_neurite_params* p, bdm_neurite** out) {
  if (!out) return BDM_EINVAL;
  *out = nullptr;
  if (!p || p->struct_size != sizeof(bdm_neurite_params)) return BDM_EINVAL;
  bdm_neurite* s = new bdm_neurite();
  s->p = *p;
  int rc = BDM_OK;
  auto bad = [&](const char* what) { return nfail(s, BDM_EINVAL, "invalid parameter: %s", what); };
  if (p->precision != BDM_FP64 && p->precision != BDM_MIXED) rc = bad("precision");
  else if (!(p->dt > 0.0) || !std::isfinite(p->dt)) rc = bad("dt");
  else if (!(p->max_displacement > 0.0) || !std::isfinite(p->max_displacement)) rc = bad("max_displacement");
  else if (!std::isfinite(p->repulsion) || !std::isfinite(p->attraction) || !std::isfinite(p->spring))
    rc = bad("repulsion / attraction / spring");
  else if (!(p->interaction_radius >= 0.0) || !std::isfinite(p->interaction_radius)) rc = bad("interaction_radius");
  else if (p->capacity == 0 || p->capacity > (1ull << 31)) rc = bad("capacity");
  else if (!(p->skin >= 0.0) || !std::isfinite(p->skin)) rc = bad("skin");
  else if (p->skin > 0.0 && p->precision != BDM_MIXED) rc = bad("skin needs BDM_MIXED");
  if (rc) {
    *out = s;
    return rc;
  }
  s->mixed = p->precision == BDM_MIXED;
  if (s->mixed && p->capacity > (1ull << kNrSlotBits)) {
    *out = s;
    return nfail(s, BDM_EINVAL, "invalid parameter: capacity above 2^27 with BDM_MIXED");
  }
  s->capacity = p->capacity;
  s->box_capacity = p->box_capacity ? p->box_capacity : 2 * p->capacity + 4096;
  if (s->box_capacity > 0xFFFFFFF0ull) s->box_capacity = 0xFFFFFFF0ull;
  *out = s;
  int dev = 0;
  NCK(cudaGetDevice(&dev));
  NCK(cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev));
  if (p->stream) {
    s->stream = (cudaStream_t)p->stream;
  } else {
    NCK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  const size_t C = s->capacity, B = s->box_capacity;
  if ((rc = nalloc(s, &s->g, 1))) return rc;
  NCK(cudaMallocHost((void**)&s->gh, sizeof(NrGrid)));
  for (int k = 0; k < 2; ++k)
    if ((rc = nalloc(s, &s->x[k], C)) || (rc = nalloc(s, &s->y[k], C)) || (rc = nalloc(s, &s->z[k], C)))
      return rc;
  if ((rc = nalloc(s, &s->diam, C)) || (rc = nalloc(s, &s->inv_rest, C)) || (rc = nalloc(s, &s->ox, C)) ||
      (rc = nalloc(s, &s->oy, C)) || (rc = nalloc(s, &s->oz, C)) || (rc = nalloc(s, &s->mother, C)) ||
      (rc = nalloc(s, &s->bx, C)) || (rc = nalloc(s, &s->by, C)) || (rc = nalloc(s, &s->bz, C)) ||
      (rc = nalloc(s, &s->spr, C)) ||
      (rc = nalloc(s, &s->key, C)) || (rc = nalloc(s, &s->rank, C)) || (rc = nalloc(s, &s->nbr, C)) ||
      (rc = nalloc(s, &s->cstart, C + 1)) || (rc = nalloc(s, &s->clist, C)) ||
      (rc = nalloc(s, &s->count, B + 1)) ||
      (rc = nalloc(s, &s->start, B + 1)) || (rc = nalloc(s, &s->partials, kNrMaxPartials * kNrPartialWords)))
    return rc;
  s->max_tiles = (unsigned)((B + 1 + kScanTile - 1) / kScanTile) + 1u;
  if ((rc = nalloc(s, &s->tiles, s->max_tiles))) return rc;
  if (s->mixed) {
    if ((rc = nalloc(s, &s->rec.A32, C)) || (rc = nalloc(s, &s->rec.RB, C))) return rc;
    if ((rc = nalloc(s, &s->out32, C)) || (rc = nalloc(s, &s->axr, C))) return rc;
    if (p->skin > 0.0 &&
        ((rc = nalloc(s, &s->list, (size_t)kNrListCap * ((C + 31) / 32 * 32))) ||
         (rc = nalloc(s, &s->list_n, C)) || (rc = nalloc(s, &s->disp, C))))
      return rc;
  } else {
    if ((rc = nalloc(s, &s->rec.A64, C)) || (rc = nalloc(s, &s->rec.B64, C)) ||
        (rc = nalloc(s, &s->rec.C, C)))
      return rc;
    if ((rc = nalloc(s, &s->out64, C)) || (rc = nalloc(s, &s->spr64, C))) return rc;
  }
  NCK(cudaMemsetAsync(s->count, 0, sizeof(unsigned) * (B + 1), s->stream));
  NCK(cudaMemsetAsync(s->g, 0, sizeof(NrGrid), s->stream));
  // launch shapes: streaming kernels over the SMs, force kernel at its occupancy
  int occ = 0;
  if (s->mixed)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_nr_force<true>, kNrForceBlock, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_nr_force<false>, kNrForceBlock, 0);
  s->blocks_force = s->sms * std::max(1, occ);
  s->blocks_stream = s->sms * 8;
  s->blocks_prep = std::min(kNrMaxPartials, s->sms * 8);
  s->blocks_scan = (int)std::max<size_t>(1, std::min<size_t>(s->max_tiles, (size_t)s->sms * 4));
  NCK(cudaStreamSynchronize(s->stream));
  return BDM_OK;
}

int bdm_neurite_set_agents(bdm_neurite* s, size_t n, const double* x, const double* y,
                           const double* z, const double* diameter, const double* rest,
                           const int32_t* mother, const double* ox, const double* oy,
                           const double* oz) {
  if (!s) return BDM_EINVAL;
  if (s->poisoned) return nfail(s, BDM_ESTATE, "handle is poisoned by an earlier device error");
  if (n > s->capacity) return nfail(s, BDM_ENOMEM, "%zu agents exceed capacity %zu", n, s->capacity);
  if (n && (!x || !y || !z || !diameter || !rest || !mother || !ox || !oy || !oz))
    return nfail(s, BDM_EINVAL, "null input array");
  // topology: CSR of daughters in ascending id (a counting sort over ascending child ids)
  std::vector<unsigned> cstart(n + 1, 0), clist;
  std::vector<double> inv_rest(n, 0.0);
  for (size_t a = 0; a < n; ++a) {
    const int32_t m = mother[a];
    if (!(std::isfinite(x[a]) && std::isfinite(y[a]) && std::isfinite(z[a])))
      return nfail(s, BDM_EINVAL, "agent %zu: non-finite position", a);
    if (!(diameter[a] > 0.0) || !std::isfinite(diameter[a]))
      return nfail(s, BDM_EINVAL, "agent %zu: diameter must be positive", a);
    if (m < -1 || (m >= 0 && (size_t)m >= a))
      return nfail(s, BDM_EINVAL, "agent %zu: mother %d must be -1 or a smaller id", a, (int)m);
    if (m >= 0) {
      if (!(rest[a] > 0.0) || !std::isfinite(rest[a]))
        return nfail(s, BDM_EINVAL, "agent %zu: rest length must be positive", a);
      if (!(std::isfinite(ox[a]) && std::isfinite(oy[a]) && std::isfinite(oz[a])))
        return nfail(s, BDM_EINVAL, "agent %zu: non-finite offset", a);
      cstart[(size_t)m + 1]++;
      inv_rest[a] = 1.0 / rest[a];
    }
  }
  for (size_t a = 0; a < n; ++a) cstart[a + 1] += cstart[a];
  clist.resize(n ? cstart[n] : 0);
  {
    std::vector<unsigned> fill(cstart.begin(), cstart.end() - 1);
    for (size_t a = 0; a < n; ++a)
      if (mother[a] >= 0) clist[fill[(size_t)mother[a]]++] = (unsigned)a;
  }
  NCK(cudaStreamSynchronize(s->stream));
  drop_graphs(s);
  s->cur = 0;
  const size_t b8 = n * sizeof(double);
  if (n) {
    NCK(cudaMemcpyAsync(s->x[0], x, b8, cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemcpyAsync(s->y[0], y, b8, cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemcpyAsync(s->z[0], z, b8, cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemcpyAsync(s->diam, diameter, b8, cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemcpyAsync(s->inv_rest, inv_rest.data(), b8, cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemcpyAsync(s->ox, ox, b8, cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemcpyAsync(s->oy, oy, b8, cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemcpyAsync(s->oz, oz, b8, cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemcpyAsync(s->mother, mother, n * sizeof(int32_t), cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemcpyAsync(s->cstart, cstart.data(), (n + 1) * sizeof(unsigned), cudaMemcpyHostToDevice, s->stream));
    if (!clist.empty())
      NCK(cudaMemcpyAsync(s->clist, clist.data(), clist.size() * sizeof(unsigned), cudaMemcpyHostToDevice, s->stream));
    NCK(cudaMemsetAsync(s->nbr, 0, n * sizeof(unsigned), s->stream));
  }
  NCK(cudaMemsetAsync(s->g, 0, sizeof(NrGrid), s->stream));
  // the pageable-memory copies above are complete when the stream is (host vectors go out of scope)
  NCK(cudaStreamSynchronize(s->stream));
  s->n = n;
  return BDM_OK;
}

int bdm_neurite_step(bdm_neurite* s, int steps) {
  if (!s || steps < 0) return BDM_EINVAL;
  if (s->poisoned) return nfail(s, BDM_ESTATE, "handle is poisoned by an earlier device error");
  if (s->n == 0 || steps == 0) return BDM_OK;
  for (int k = 0; k < steps; ++k) {
    if (s->prof) {
      int rc = enqueue_step(s);
      if (rc) return rc;
      continue;
    }
    const int c = s->cur;
    if (!s->graph[c]) {
      cudaGraph_t graph = nullptr;
      NCK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
      s->capturing = true;
      s->capture_kernels = 0;
      int rc = enqueue_step(s);
      s->capturing = false;
      cudaError_t ce = cudaStreamEndCapture(s->stream, &graph);
      s->cur = c;  // the capture did not run the step
      if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
      }
      if (ce != cudaSuccess) return nfail(s, BDM_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&s->graph[c], graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) return nfail(s, BDM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
      s->graph_kernels = s->capture_kernels;
    }
    NCK(cudaGraphLaunch(s->graph[c], s->stream));
    bdm_count_launches(s->graph_kernels);
    s->cur = c ^ 1;
  }
  return BDM_OK;
}

int bdm_neurite_get_state(bdm_neurite* s, size_t* n_out, double* x, double* y, double* z,
                          uint32_t* neighbour_count, double* L_out) {
  if (!s) return BDM_EINVAL;
  NCK(cudaMemcpyAsync(s->gh, s->g, sizeof(NrGrid), cudaMemcpyDeviceToHost, s->stream));
  NCK(cudaStreamSynchronize(s->stream));
  int rc = decode(s, s->gh->err);
  if (rc) return rc;
  const size_t n = s->n, b8 = n * sizeof(double);
  if (n_out) *n_out = n;
  if (L_out) *L_out = s->gh->L;
  if (n) {
    const int c = s->cur;
    if (x) NCK(cudaMemcpyAsync(x, s->x[c], b8, cudaMemcpyDeviceToHost, s->stream));
    if (y) NCK(cudaMemcpyAsync(y, s->y[c], b8, cudaMemcpyDeviceToHost, s->stream));
    if (z) NCK(cudaMemcpyAsync(z, s->z[c], b8, cudaMemcpyDeviceToHost, s->stream));
    if (neighbour_count)
      NCK(cudaMemcpyAsync(neighbour_count, s->nbr, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s->stream));
  }
  NCK(cudaStreamSynchronize(s->stream));
  return BDM_OK;
}

int bdm_neurite_list_info(bdm_neurite* s, uint64_t* rebuilds, uint64_t* entries) {
  if (!s) return BDM_EINVAL;
  NCK(cudaMemcpyAsync(s->gh, s->g, sizeof(NrGrid), cudaMemcpyDeviceToHost, s->stream));
  NCK(cudaStreamSynchronize(s->stream));
  const bool lists = s->mixed && s->p.skin > 0.0;
  if (rebuilds) *rebuilds = lists ? s->gh->rebuilds : 0;
  if (entries) *entries = lists ? s->gh->list_entries : 0;
  return BDM_OK;
}

int bdm_neurite_profile(bdm_neurite* s, int enable) {
  if (!s) return BDM_EINVAL;
  if (s->prof) {
    int rc = prof_collect(s);
    if (rc) return rc;
  }
  s->prof = enable != 0;
  return BDM_OK;
}

int bdm_neurite_kernel_times(bdm_neurite* s, bdm_kernel_time* out, int max, int* count) {
  if (!s || !count || max < 0 || (max > 0 && !out)) return BDM_EINVAL;
  int rc = prof_collect(s);
  if (rc) return rc;
  *count = (int)s->stats.size();
  for (int k = 0; k < max && k < (int)s->stats.size(); ++k) {
    memset(out[k].name, 0, sizeof(out[k].name));
    strncpy(out[k].name, s->stats[k].name.c_str(), sizeof(out[k].name) - 1);
    out[k].launches = s->stats[k].launches;
    out[k].total_ms = s->stats[k].total_ms;
  }
  return BDM_OK;
}

void bdm_neurite_destroy(bdm_neurite* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  drop_graphs(s);
  for (auto& p : s->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : s->free_events) cudaEventDestroy(e);
  for (void* q : s->allocs) cudaFree(q);
  if (s->gh) cudaFreeHost(s->gh);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

const char* bdm_neurite_last_error(const bdm_neurite* s) { return s ? s->err.c_str() : "null handle"; }

}  // extern "C"
