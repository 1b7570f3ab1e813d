// diffusion.cu -- diffusion of an extracellular substance, the standalone operation of the step
// (BioDynaMo, arXiv 2006.06775, Sec. "Simulation concepts").  Reading R9: explicit FTCS 7-point
// update with zero-flux walls and linear decay, FP32 grid, FP64 mass total.
//
// Layout: x fastest.  A block covers 32 x 8 columns and marches 16 planes in z, keeping the z-1, z,
// z+1 values of its column in registers; the x/y neighbours of a plane are read through L1, which
// already holds them from the neighbouring threads' own loads, so DRAM sees ~4 B read + 4 B written
// per voxel.  Mass: each thread adds its 16 outputs in FP32, the block adds the thread sums in FP64
// into one partial per block, and a single block sums the partials in a fixed order.
#include "common.cuh"

namespace bdm {

constexpr int kFX = 32, kFY = 8, kFZ = 16;

__global__ void __launch_bounds__(kFX* kFY) k_ftcs(const float* __restrict__ u,
                                                   float* __restrict__ out, int nx, int ny, int nz,
                                                   float lam, float mu_dt,
                                                   double* __restrict__ partials) {
  const int x = blockIdx.x * kFX + threadIdx.x;
  const int y = blockIdx.y * kFY + threadIdx.y;
  const int z0 = blockIdx.z * kFZ;
  const int z1 = min(z0 + kFZ, nz);
  const size_t plane = (size_t)nx * (size_t)ny;
  float part = 0.f;
  if (x < nx && y < ny) {
    size_t idx = (size_t)x + (size_t)nx * (size_t)y + plane * (size_t)z0;
    float c = u[idx];
    float zm = z0 > 0 ? u[idx - plane] : c;
    for (int z = z0; z < z1; ++z, idx += plane) {
      const float zp = z + 1 < nz ? u[idx + plane] : c;
      const float xm = x > 0 ? u[idx - 1] : c;
      const float xp = x + 1 < nx ? u[idx + 1] : c;
      const float ym = y > 0 ? u[idx - nx] : c;
      const float yp = y + 1 < ny ? u[idx + nx] : c;
      // a missing neighbour equals the cell itself, so its difference is exactly zero
      const float lap = (((((xm - c) + (xp - c)) + (ym - c)) + (yp - c)) + (zm - c)) + (zp - c);
      const float v = (c + lam * lap) - mu_dt * c;
      out[idx] = v;
      part += v;
      zm = c;
      c = zp;
    }
  }
  // block sum of the thread partials in FP64
  __shared__ double s_part[kFX * kFY / 32];
  double dp = (double)part;
  dp = warp_reduce(dp, [](double a, double b) { return a + b; });
  const int t = threadIdx.x + kFX * threadIdx.y;
  if ((t & 31) == 0) s_part[t >> 5] = dp;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < kFX * kFY / 32; ++w) s += s_part[w];
    partials[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
  }
}

// Vector form for x extents that are a multiple of 4 (and 16-byte aligned buffers): each lane updates
// four consecutive voxels of a row with one 16-byte load per neighbour row/plane; the x neighbours
// across its four voxels come from the lanes beside it (shuffles), and only the first and last lane
// of a warp load one scalar from outside.  A block covers 128 x 8 columns and marches 16 planes.  The
// per-voxel arithmetic is the scalar kernel's.  Each thread adds its 64 outputs with compensated
// (Kahan) FP32 summation, so its partial is as accurate as a 16-term plain sum.
constexpr int kVX = 32, kVY = 8, kVZ = 16;

__device__ __forceinline__ float ftcs_voxel(float c, float xm, float xp, float ym, float yp, float zm,
                                            float zp, float lam, float mu_dt) {
  const float lap = (((((xm - c) + (xp - c)) + (ym - c)) + (yp - c)) + (zm - c)) + (zp - c);
  return (c + lam * lap) - mu_dt * c;
}

__global__ void __launch_bounds__(kVX* kVY) k_ftcs4(const float* __restrict__ u,
                                                    float* __restrict__ out, int nx, int ny, int nz,
                                                    float lam, float mu_dt,
                                                    double* __restrict__ partials) {
  const int lane = threadIdx.x;
  const int x0 = (blockIdx.x * kVX + lane) * 4;
  const int y = blockIdx.y * kVY + threadIdx.y;  // one row per warp
  const int z0 = blockIdx.z * kVZ;
  const int z1 = min(z0 + kVZ, nz);
  const size_t plane = (size_t)nx * (size_t)ny;
  const bool act = x0 < nx;
  float sum = 0.f, comp = 0.f;
  if (y < ny) {
    size_t idx = (size_t)(act ? x0 : 0) + (size_t)nx * (size_t)y + plane * (size_t)z0;
    auto ld = [&](size_t k) { return __ldg(reinterpret_cast<const float4*>(u + k)); };
    float4 c = ld(idx);
    float4 zm = z0 > 0 ? ld(idx - plane) : c;
    for (int z = z0; z < z1; ++z, idx += plane) {
      const float4 zp = z + 1 < nz ? ld(idx + plane) : c;
      const float4 ym = y > 0 ? ld(idx - nx) : c;
      const float4 yp = y + 1 < ny ? ld(idx + nx) : c;
      float xl = __shfl_up_sync(0xFFFFFFFFu, c.w, 1);
      float xr = __shfl_down_sync(0xFFFFFFFFu, c.x, 1);
      if (lane == 0 && x0 > 0 && act) xl = __ldg(u + idx - 1);
      if (lane == kVX - 1 && x0 + 4 < nx) xr = __ldg(u + idx + 4);
      if (x0 == 0) xl = c.x;        // wall: the missing neighbour equals the cell itself
      if (x0 + 4 >= nx) xr = c.w;
      float4 v;
      v.x = ftcs_voxel(c.x, xl, c.y, ym.x, yp.x, zm.x, zp.x, lam, mu_dt);
      v.y = ftcs_voxel(c.y, c.x, c.z, ym.y, yp.y, zm.y, zp.y, lam, mu_dt);
      v.z = ftcs_voxel(c.z, c.y, c.w, ym.z, yp.z, zm.z, zp.z, lam, mu_dt);
      v.w = ftcs_voxel(c.w, c.z, xr, ym.w, yp.w, zm.w, zp.w, lam, mu_dt);
      if (act) {
        *reinterpret_cast<float4*>(out + idx) = v;
        const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {  // Kahan
          const float yv = e[k] - comp;
          const float tv = sum + yv;
          comp = (tv - sum) - yv;
          sum = tv;
        }
      }
      zm = c;
      c = zp;
    }
  }
  __shared__ double s_part[kVX * kVY / 32];
  double dp = warp_reduce((double)sum - (double)comp, [](double a, double b) { return a + b; });
  const int t = threadIdx.x + kVX * threadIdx.y;
  if ((t & 31) == 0) s_part[t >> 5] = dp;
  __syncthreads();
  if (t == 0) {
    double acc = 0.0;
    for (int w = 0; w < kVX * kVY / 32; ++w) acc += s_part[w];
    partials[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = acc;
  }
}

// Deterministic FP64 total of the block partials: fixed strided order, fixed tree.
__global__ void __launch_bounds__(1024) k_mass(const double* __restrict__ partials, int count,
                                               DevGrid* g) {
  __shared__ double s[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += 1024) acc += partials[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) g->mass = s[0];
}

// FP64 total of the block partials written to a caller-provided device slot (same order as k_mass).
__global__ void __launch_bounds__(1024) k_mass_to(const double* __restrict__ partials, int count,
                                                  double* __restrict__ out) {
  __shared__ double s[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += 1024) acc += partials[i];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// FP64 total of a grid with the FTCS block layout: FP32 sums of 16 voxels per thread, FP64 per block.
__global__ void __launch_bounds__(kFX* kFY) k_grid_partials(const float* __restrict__ u, int nx,
                                                            int ny, int nz,
                                                            double* __restrict__ partials) {
  const int x = blockIdx.x * kFX + threadIdx.x;
  const int y = blockIdx.y * kFY + threadIdx.y;
  const int z0 = blockIdx.z * kFZ;
  const int z1 = min(z0 + kFZ, nz);
  const size_t plane = (size_t)nx * (size_t)ny;
  float part = 0.f;
  if (x < nx && y < ny)
    for (int z = z0; z < z1; ++z) part += u[(size_t)x + (size_t)nx * (size_t)y + plane * (size_t)z];
  __shared__ double s_part[kFX * kFY / 32];
  double dp = warp_reduce((double)part, [](double a, double b) { return a + b; });
  const int t = threadIdx.x + kFX * threadIdx.y;
  if ((t & 31) == 0) s_part[t >> 5] = dp;
  __syncthreads();
  if (t == 0) {
    double s = 0.0;
    for (int w = 0; w < kFX * kFY / 32; ++w) s += s_part[w];
    partials[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = s;
  }
}

long long ftcs_partials_needed(const int dims[3]) {
  return (long long)((dims[0] + (long long)kFX - 1) / kFX) * ((dims[1] + (long long)kFY - 1) / kFY) *
         ((dims[2] + (long long)kFZ - 1) / kFZ);
}

bool ftcs_launchable(const int dims[3]) {
  // grid.y and grid.z of both FTCS kernels, and the block count the mass kernel takes as an int
  return dims[0] > 0 && dims[1] > 0 && dims[2] > 0 &&
         (dims[1] + (long long)kFY - 1) / kFY <= 65535 &&
         (dims[2] + (long long)kFZ - 1) / kFZ <= 65535 && ftcs_partials_needed(dims) <= INT32_MAX;
}

// One FTCS step into `out` with the block partials of its mass; returns how many partials it wrote
// (the vector kernel when rows are whole 16-byte vectors, else the scalar one).
static int enqueue_ftcs(cudaStream_t s, const float* u, float* out, const int dims[3], float lambda,
                        float mu_dt, double* partials) {
  const bool vec = dims[0] % 4 == 0 && ((uintptr_t)u % 16u) == 0 && ((uintptr_t)out % 16u) == 0;
  if (vec) {
    dim3 grid((dims[0] / 4 + kVX - 1) / kVX, (dims[1] + kVY - 1) / kVY, (dims[2] + kVZ - 1) / kVZ);
    k_ftcs4<<<grid, dim3(kVX, kVY), 0, s>>>(u, out, dims[0], dims[1], dims[2], lambda, mu_dt,
                                            partials);
    return (int)(grid.x * grid.y * grid.z);
  }
  dim3 grid((dims[0] + kFX - 1) / kFX, (dims[1] + kFY - 1) / kFY, (dims[2] + kFZ - 1) / kFZ);
  k_ftcs<<<grid, dim3(kFX, kFY), 0, s>>>(u, out, dims[0], dims[1], dims[2], lambda, mu_dt,
                                         partials);
  return (int)(grid.x * grid.y * grid.z);
}

void launch_ftcs(cudaStream_t s, const float* u, float* out, const int dims[3], float lambda,
                 float mu_dt, double* partials, DevGrid* g) {
  const int count = enqueue_ftcs(s, u, out, dims, lambda, mu_dt, partials);
  k_mass<<<1, 1024, 0, s>>>(partials, count, g);
}

void launch_grid_mass(cudaStream_t s, const float* u, const int dims[3], double* partials, DevGrid* g) {
  dim3 grid((dims[0] + kFX - 1) / kFX, (dims[1] + kFY - 1) / kFY, (dims[2] + kFZ - 1) / kFZ);
  k_grid_partials<<<grid, dim3(kFX, kFY), 0, s>>>(u, dims[0], dims[1], dims[2], partials);
  k_mass<<<1, 1024, 0, s>>>(partials, (int)ftcs_partials_needed(dims), g);
}

void launch_ftcs_mass_to(cudaStream_t s, const float* u, float* out, const int dims[3],
                         float lambda, float mu_dt, double* partials, double* mass) {
  const int count = enqueue_ftcs(s, u, out, dims, lambda, mu_dt, partials);
  if (mass) k_mass_to<<<1, 1024, 0, s>>>(partials, count, mass);
}

}  // namespace bdm
