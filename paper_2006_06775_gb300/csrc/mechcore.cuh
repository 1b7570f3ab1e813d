// mechcore.cuh -- per-pair arithmetic of the mixed-precision sphere mechanics (readings R1, R3),
// shared by the single-simulation kernels and the batched mechanics kernels so that both evaluate a
// pair with the same operations in the same order.
#pragma once

#include "common.cuh"

namespace bdm {

// The operations below are explicitly rounded (no contraction left to the compiler), so that every
// kernel that evaluates a pair gets the same bits.

// FP32 squared distance of a pair from its components, (ex ex + ey ey) + ez ez with two FMAs.
__device__ __forceinline__ float pair_d2(float ex, float ey, float ez) {
  return __fmaf_rn(ez, ez, __fmaf_rn(ey, ey, __fmul_rn(ex, ex)));
}

// Contact force of the sphere law (reading R3) in FP32, added to (Fx, Fy, Fz): delta = ri + rj - d,
// F = k delta - gamma sqrt(rho delta), rho = ri rj / (ri + rj), along the centre line (ex, ey, ez).
__device__ __forceinline__ void contact_force(float& Fx, float& Fy, float& Fz, float ex, float ey,
                                              float ez, float ri, float rj, float kf, float gf) {
  const float d2 = pair_d2(ex, ey, ez);
  const float rs = __fadd_rn(ri, rj);
  const float rinv = rsqrtf(d2);
  const float delta = __fsub_rn(rs, __fmul_rn(d2, rinv));
  if (delta > 0.f) {
    const float rd = __fmul_rn(__fdividef(__fmul_rn(ri, rj), rs), delta);  // rho * delta > 0
    const float F = __fsub_rn(__fmul_rn(kf, delta), __fmul_rn(gf, __fmul_rn(rd, rsqrtf(rd))));
    const float sc = __fmul_rn(F, rinv);
    Fx = __fmaf_rn(sc, ex, Fx);
    Fy = __fmaf_rn(sc, ey, Fy);
    Fz = __fmaf_rn(sc, ez, Fz);
  }
}

// Displacement dt F in FP32, scaled to length cap if longer (reading R4).
__device__ __forceinline__ void capped_displacement(float Fx, float Fy, float Fz, float dtf,
                                                    float capf, float& Dx, float& Dy, float& Dz) {
  Dx = __fmul_rn(dtf, Fx);
  Dy = __fmul_rn(dtf, Fy);
  Dz = __fmul_rn(dtf, Fz);
  const float n2 = pair_d2(Dx, Dy, Dz);
  if (n2 > __fmul_rn(capf, capf)) {
    const float f = __fmul_rn(capf, rsqrtf(n2));
    Dx = __fmul_rn(Dx, f);
    Dy = __fmul_rn(Dy, f);
    Dz = __fmul_rn(Dz, f);
  }
}

// The oracle's FP64 neighbour predicate d^2 < R^2 (reading R1), for a candidate inside the FP32 band.
__device__ __forceinline__ unsigned fp64_within(unsigned i, unsigned j, const double* __restrict__ sx,
                                                 const double* __restrict__ sy,
                                                 const double* __restrict__ sz, double R2) {
  const double ax = __dsub_rn(sx[i], sx[j]), ay = __dsub_rn(sy[i], sy[j]), az = __dsub_rn(sz[i], sz[j]);
  const double e2 = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az));
  return e2 < R2 ? 1u : 0u;
}

}  // namespace bdm
