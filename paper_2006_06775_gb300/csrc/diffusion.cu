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

int ftcs_partials_needed(const int dims[3]) {
  return ((dims[0] + kFX - 1) / kFX) * ((dims[1] + kFY - 1) / kFY) * ((dims[2] + kFZ - 1) / kFZ);
}

void launch_ftcs(cudaStream_t s, const float* u, float* out, const int dims[3], float lambda,
                 float mu_dt, double* partials, DevGrid* g) {
  dim3 grid((dims[0] + kFX - 1) / kFX, (dims[1] + kFY - 1) / kFY, (dims[2] + kFZ - 1) / kFZ);
  k_ftcs<<<grid, dim3(kFX, kFY), 0, s>>>(u, out, dims[0], dims[1], dims[2], lambda, mu_dt,
                                         partials);
  k_mass<<<1, 1024, 0, s>>>(partials, ftcs_partials_needed(dims), g);
}

void launch_grid_mass(cudaStream_t s, const float* u, const int dims[3], double* partials, DevGrid* g) {
  dim3 grid((dims[0] + kFX - 1) / kFX, (dims[1] + kFY - 1) / kFY, (dims[2] + kFZ - 1) / kFZ);
  k_grid_partials<<<grid, dim3(kFX, kFY), 0, s>>>(u, dims[0], dims[1], dims[2], partials);
  k_mass<<<1, 1024, 0, s>>>(partials, ftcs_partials_needed(dims), g);
}

void launch_ftcs_mass_to(cudaStream_t s, const float* u, float* out, const int dims[3],
                         float lambda, float mu_dt, double* partials, double* mass) {
  dim3 grid((dims[0] + kFX - 1) / kFX, (dims[1] + kFY - 1) / kFY, (dims[2] + kFZ - 1) / kFZ);
  k_ftcs<<<grid, dim3(kFX, kFY), 0, s>>>(u, out, dims[0], dims[1], dims[2], lambda, mu_dt,
                                         partials);
  if (mass) k_mass_to<<<1, 1024, 0, s>>>(partials, ftcs_partials_needed(dims), mass);
}

}  // namespace bdm
