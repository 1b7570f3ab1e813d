// gridcore.cuh -- the grid of a step from its accumulated bounds (reading R5), shared by the
// single-simulation finalize kernel and the batched mechanics kernels.
#pragma once

#include "common.cuh"

namespace bdm {

// Origin, box length, boxes per axis and the radius-derived constants of a step's grid from the
// bounds accumulated in g (the per-axis min / max of the centres, the largest diameter).  A grid
// with no agents, after an error, or out of range (an error bit is set) has no boxes.
__device__ __forceinline__ void grid_from_bounds(DevGrid* g, const MechConsts& c) {
  if (g->n == 0 || g->err) {
    g->nbox = 0;
    g->nbox1 = 1;
    return;
  }
  double R = c.interaction_radius > 0.0 ? c.interaction_radius
                                        : (double)__uint_as_float(g->acc_maxdiam);
  double L = c.box_length > 0.0 ? c.box_length : R + c.skin;
  bool ok = (R > 0.0) && (L >= R + c.skin) && (L < 2048.0);
  // the mixed path finds contacts among the pairs within R, so R may not be below a diameter
  if (c.mixed && R < (double)__uint_as_float(g->acc_maxdiam)) ok = false;
  long long Lq = (long long)ceil(L * kQScale);
  unsigned long long nbox = 1;
  long long O[3];
  int dims[3];
  for (int a = 0; a < 3 && ok; ++a) {
    double lo = dec_double(g->acc_min[a]), hi = dec_double(g->acc_max[a]);
    ok = fabs(lo) < 1e9 && fabs(hi) < 1e9;  // quantise() needs |v| < 2^40
    if (!ok) break;
    long long Xlo = quantise(lo), Xhi = quantise(hi);
    O[a] = Xlo;
    long long d = (Xhi - Xlo) / Lq + 1;
    ok = d > 0 && d < (1ll << 30);
    dims[a] = (int)d;
    nbox *= (unsigned long long)d;
    if (nbox > 0xFFFFFFF0ull) ok = false;
  }
  if (!ok) {
    atomicOr(&g->err, (unsigned)ERR_RADIUS);
    g->nbox = 0;
    g->nbox1 = 1;
  } else if (nbox > c.box_capacity) {
    atomicOr(&g->err, (unsigned)ERR_GRID_OVERFLOW);
    g->nbox = 0;
    g->nbox1 = 1;
  } else {
    for (int a = 0; a < 3; ++a) {
      g->O[a] = O[a];
      g->dims[a] = dims[a];
    }
    g->Lq = Lq;
    g->nbox = (unsigned)nbox;
    g->nbox1 = (unsigned)nbox + 1;
    g->R = R;
    g->R2 = R * R;
    g->Lf = (float)((double)Lq / kQScale);
    g->R2f = (float)(R * R);
    g->R2lo = g->R2f * (1.0f - 1.0f / 4096.0f);
    g->R2hi = g->R2f * (1.0f + 1.0f / 4096.0f);
    g->invLq = (float)(1.0 / (double)Lq);
    g->list_L2f = (float)((R + c.skin) * (R + c.skin)) * (1.0f + 1.0f / 1024.0f);
  }
}

}  // namespace bdm
