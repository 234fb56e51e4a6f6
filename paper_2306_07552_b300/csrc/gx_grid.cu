// Static-scene signed-distance grid.  The paper precomputes its static
// collision structure offline from the scene geometry (appendix "Additional
// Collision-Detection Details"); here the structure is a lattice of signed
// distances to the union of the scene's solid boxes, one thread per node, in
// FP64, rounded once to FP32 for storage.
#include "gx_internal.h"

namespace gx {

namespace {

__global__ void grid_kernel(float* __restrict__ grid, const float* __restrict__ boxes, int n_boxes,
                            float ox, float oy, float oz, float h, int nx, int ny, int nz) {
  extern __shared__ double sb[];  // [n_boxes][6]: centre xyz, half extent xyz
  for (int b = threadIdx.x; b < n_boxes; b += blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      const double lo = boxes[6 * b + a], hi = boxes[6 * b + 3 + a];
      sb[6 * b + a] = 0.5 * (lo + hi);
      sb[6 * b + 3 + a] = 0.5 * (hi - lo);
    }
  }
  __syncthreads();
  const size_t total = (size_t)nx * ny * nz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % nx);
    const int j = (int)((idx / nx) % ny);
    const int k = (int)(idx / ((size_t)nx * ny));
    const double p[3] = {(double)ox + i * (double)h, (double)oy + j * (double)h,
                         (double)oz + k * (double)h};
    double best = 1e300;
    for (int b = 0; b < n_boxes; ++b) {
      double out2 = 0.0, inmax = -1e300;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double q = fabs(p[a] - sb[6 * b + a]) - sb[6 * b + 3 + a];
        out2 += q > 0.0 ? q * q : 0.0;
        inmax = fmax(inmax, q);
      }
      const double d = sqrt(out2) + fmin(inmax, 0.0);
      best = fmin(best, d);
    }
    grid[idx] = (float)best;
  }
}

}  // namespace

void launch_grid_build(float* grid, const float* boxes, int n_boxes, float ox, float oy, float oz,
                       float h, int nx, int ny, int nz, cudaStream_t s) {
  const size_t total = (size_t)nx * ny * nz;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 148 * 64) blocks = 148 * 64;
  const size_t smem = (size_t)n_boxes * 6 * sizeof(double);
  grid_kernel<<<blocks, 256, smem, s>>>(grid, boxes, n_boxes, ox, oy, oz, h, nx, ny, nz);
}

}  // namespace gx
