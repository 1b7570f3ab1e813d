// mechanics.cu -- mechanical interaction of spherical agents and the behaviours that change them
// (BioDynaMo, arXiv 2006.06775, Sec. "Simulation concepts": agent operations "calculate mechanical
// forces" and behaviours such as growth, division and secretion; force law and update: readings
// R1-R4, sum order R6, growth/division R7, secretion R8).
#include "common.cuh"

namespace bdm {

// ---------------------------------------------------------------------------------------------
// Force + capped update, one thread per agent in canonical order.  Neighbours are read box by box
// in ascending key -- for each (dz, dy) the up-to-three boxes along x are contiguous in the sorted
// arrays -- which is exactly the oracle's (box, id) summation order.
//
// FP64 variant: every operation is an explicitly rounded FP64 intrinsic in the oracle's order (no
// contraction), so positions can match the FP64 oracle bit for bit.
// MIXED variant: pair geometry and forces in FP32 from box-relative offsets (all |values| < 2 L);
// the neighbour predicate d^2 < R^2 is decided in FP32 outside a +-2^-12 relative band and by the
// FP64 expression of the oracle inside it, so neighbour counts stay exact; the displacement is
// added to the FP64 position.
// The epilogue folds the new centres into the bounds of the next step's grid.
// ---------------------------------------------------------------------------------------------
template <bool MIXED>
__global__ void __launch_bounds__(kBlock, MIXED ? 4 : 1) k_force(
    const double* __restrict__ sx, const double* __restrict__ sy, const double* __restrict__ sz,
    const float* __restrict__ diam, const float4* __restrict__ p4,
    const unsigned* __restrict__ skey, const unsigned* __restrict__ start,
    double* __restrict__ ox, double* __restrict__ oy, double* __restrict__ oz,
    unsigned* __restrict__ nbr, DevGrid* g, MechConsts c) {
  const unsigned n = g->nbox ? g->n : 0u;
  const int d0 = g->dims[0], d1 = g->dims[1], d2 = g->dims[2];
  const double R2 = g->R2;
  const float Lf = g->Lf, R2lo = g->R2lo, R2hi = g->R2hi;
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  unsigned md = 0;
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned b = skey[i];
    const int ix = (int)(b % (unsigned)d0);
    const unsigned t = b / (unsigned)d0;
    const int iy = (int)(t % (unsigned)d1), iz = (int)(t / (unsigned)d1);
    const double xi = sx[i], yi = sy[i], zi = sz[i];
    unsigned cnt = 0;
    double Sx = 0.0, Sy = 0.0, Sz = 0.0;      // FP64 variant
    float Fx = 0.f, Fy = 0.f, Fz = 0.f;       // MIXED variant
    float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
    double ri = 0.0;
    if (MIXED) pi = p4[i];
    else ri = 0.5 * (double)diam[i];
    const int xlo = ix > 0 ? ix - 1 : 0, xhi = ix < d0 - 1 ? ix + 1 : d0 - 1;
    for (int dz = -1; dz <= 1; ++dz) {
      const int jz = iz + dz;
      if (jz < 0 || jz >= d2) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int jy = iy + dy;
        if (jy < 0 || jy >= d1) continue;
        const unsigned row = ((unsigned)jz * (unsigned)d1 + (unsigned)jy) * (unsigned)d0;
        unsigned s0 = start[row + xlo];
        for (int bx = xlo; bx <= xhi; ++bx) {
          const unsigned s1 = start[row + bx + 1];
          if (MIXED) {
            const float shx = (float)(bx - ix) * Lf, shy = (float)dy * Lf, shz = (float)dz * Lf;
            for (unsigned j = s0; j < s1; ++j) {
              if (j == i) continue;
              const float4 q = p4[j];
              const float ex = pi.x - (q.x + shx);
              const float ey = pi.y - (q.y + shy);
              const float ez = pi.z - (q.z + shz);
              const float d2f = ex * ex + ey * ey + ez * ez;
              if (d2f < R2lo) {
                ++cnt;
              } else if (d2f <= R2hi) {
                const double ax = __dsub_rn(xi, sx[j]), ay = __dsub_rn(yi, sy[j]),
                             az = __dsub_rn(zi, sz[j]);
                const double e2 = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)),
                                            __dmul_rn(az, az));
                cnt += e2 < R2 ? 1u : 0u;
              }
              const float rs = pi.w + q.w;
              if (d2f < rs * rs && d2f > 0.f) {
                const float rinv = rsqrtf(d2f);
                const float dd = d2f * rinv;
                const float delta = rs - dd;
                if (delta > 0.f) {
                  const float rd = __fdividef(pi.w * q.w, rs) * delta;  // rho * delta > 0
                  const float F = c.kf * delta - c.gammaf * (rd * rsqrtf(rd));
                  const float s = F * rinv;
                  Fx += s * ex;
                  Fy += s * ey;
                  Fz += s * ez;
                }
              }
            }
          } else {
            for (unsigned j = s0; j < s1; ++j) {
              if (j == i) continue;
              const double ax = __dsub_rn(xi, sx[j]), ay = __dsub_rn(yi, sy[j]),
                           az = __dsub_rn(zi, sz[j]);
              const double e2 = __dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)),
                                          __dmul_rn(az, az));
              if (e2 < R2) ++cnt;
              const double d = __dsqrt_rn(e2);
              const double rj = 0.5 * (double)diam[j];
              const double delta = __dsub_rn(__dadd_rn(ri, rj), d);
              if (delta > 0.0 && d > 0.0) {
                const double rho = __ddiv_rn(__dmul_rn(ri, rj), __dadd_rn(ri, rj));
                const double F = __dsub_rn(__dmul_rn(c.k, delta),
                                           __dmul_rn(c.gamma, __dsqrt_rn(__dmul_rn(rho, delta))));
                const double s = __ddiv_rn(F, d);
                Sx = __dadd_rn(Sx, __dmul_rn(s, ax));
                Sy = __dadd_rn(Sy, __dmul_rn(s, ay));
                Sz = __dadd_rn(Sz, __dmul_rn(s, az));
              }
            }
          }
          s0 = s1;
        }
      }
    }
    double nx, ny, nz;
    if (MIXED) {
      float Dx = c.dtf * Fx, Dy = c.dtf * Fy, Dz = c.dtf * Fz;
      const float n2 = Dx * Dx + Dy * Dy + Dz * Dz;
      if (n2 > c.capf * c.capf) {
        const float f = c.capf * rsqrtf(n2);
        Dx *= f; Dy *= f; Dz *= f;
      }
      nx = __dadd_rn(xi, (double)Dx);
      ny = __dadd_rn(yi, (double)Dy);
      nz = __dadd_rn(zi, (double)Dz);
    } else {
      double Dx = __dmul_rn(c.dt, Sx), Dy = __dmul_rn(c.dt, Sy), Dz = __dmul_rn(c.dt, Sz);
      double nrm = __dadd_rn(__dmul_rn(Dx, Dx), __dmul_rn(Dy, Dy));
      nrm = __dsqrt_rn(__dadd_rn(nrm, __dmul_rn(Dz, Dz)));
      if (nrm > c.cap) {
        const double f = __ddiv_rn(c.cap, nrm);
        Dx = __dmul_rn(Dx, f); Dy = __dmul_rn(Dy, f); Dz = __dmul_rn(Dz, f);
      }
      nx = __dadd_rn(xi, Dx);
      ny = __dadd_rn(yi, Dy);
      nz = __dadd_rn(zi, Dz);
    }
    ox[i] = nx;
    oy[i] = ny;
    oz[i] = nz;
    nbr[i] = cnt;
    const unsigned long long e0 = enc_double(nx), e1 = enc_double(ny), e2 = enc_double(nz);
    mn[0] = e0 < mn[0] ? e0 : mn[0]; mx[0] = e0 > mx[0] ? e0 : mx[0];
    mn[1] = e1 < mn[1] ? e1 : mn[1]; mx[1] = e1 > mx[1] ? e1 : mx[1];
    mn[2] = e2 < mn[2] ? e2 : mn[2]; mx[2] = e2 > mx[2] ? e2 : mx[2];
    const unsigned dbits = MIXED ? __float_as_uint(2.0f * pi.w) : __float_as_uint(diam[i]);
    md = dbits > md ? dbits : md;
  }
  block_commit_bounds(mn, mx, md, g);
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

__global__ void k_step_done(DevGrid* g) {
  if (threadIdx.x == 0 && blockIdx.x == 0) g->step += 1ull;
}

// ---- launch wrappers -------------------------------------------------------------------------
void launch_force(cudaStream_t s, const MechBuffers& b, const AgentArrays& attr, DevGrid* g,
                  MechConsts c, bool mixed, int grid_blocks) {
  if (mixed)
    k_force<true><<<grid_blocks, kBlock, 0, s>>>(b.sorted.x, b.sorted.y, b.sorted.z, attr.diam,
                                                 b.p4, b.skey, b.start, b.pos.x, b.pos.y, b.pos.z,
                                                 b.nbr, g, c);
  else
    k_force<false><<<grid_blocks, kBlock, 0, s>>>(b.sorted.x, b.sorted.y, b.sorted.z, attr.diam,
                                                  b.p4, b.skey, b.start, b.pos.x, b.pos.y,
                                                  b.pos.z, b.nbr, g, c);
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

void launch_step_done(cudaStream_t s, DevGrid* g) { k_step_done<<<1, 32, 0, s>>>(g); }

}  // namespace bdm
