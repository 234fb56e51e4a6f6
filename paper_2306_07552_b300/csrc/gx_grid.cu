// Static-scene signed-distance grid.  The paper precomputes its static
// collision structure offline from the scene geometry (appendix "Additional
// Collision-Detection Details"); here the structure is a lattice of signed
// distances to the union of the scene's solid boxes, one thread per node, in
// FP64, rounded once to FP32 for storage.
// node values from the dense grid or the box store, per scene at run time
#define GX_STATIC_STORE 2
#include <algorithm>

#include "gx_device.cuh"

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

// Column grid (appendix "Additional Collision-Detection Details"): one
// thread per (radius, column), FP64 like the distance grid: the free spans
// of a sphere centre's height, [ylo, yhi] minus the open interval
// (y0 - e, y1 + e), e = sqrt(R^2 - dxz^2), of every box closer than R in XZ.
// Count pass (offsets == nullptr) then fill pass.
__global__ void column_kernel(const float* __restrict__ boxes, int n_boxes, double ox, double oz,
                              double ylo, double yhi, int ncx, int ncz,
                              const uint32_t* __restrict__ offsets, uint32_t* __restrict__ counts,
                              float2* __restrict__ spans, unsigned* overflow) {
  extern __shared__ double cb[];  // [n_boxes][6]
  for (int b = threadIdx.x; b < n_boxes; b += blockDim.x)
    for (int a = 0; a < 6; ++a) cb[6 * b + a] = boxes[6 * b + a];
  __syncthreads();
  const int total = 3 * ncx * ncz;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int i = idx % ncx, k = (idx / ncx) % ncz, ri = idx / (ncx * ncz);
    const double R = kColumnRadius[ri];
    const double x = ox + i * kColumnSpacing, z = oz + k * kColumnSpacing;
    double lo[kColumnCap], hi[kColumnCap];
    int n = 0;
    for (int b = 0; b < n_boxes; ++b) {
      const double* bx = cb + 6 * b;
      const double dx = fmax(fmax(bx[0] - x, 0.0), x - bx[3]);
      const double dz = fmax(fmax(bx[2] - z, 0.0), z - bx[5]);
      const double d2 = dx * dx + dz * dz;
      if (d2 >= R * R) continue;
      const double e = sqrt(R * R - d2);
      const double l = bx[1] - e, h = bx[4] + e;
      if (h <= ylo || l >= yhi) continue;
      if (n == kColumnCap) {
        atomicOr(overflow, 1u);
        break;
      }
      int m = n++;
      while (m > 0 && lo[m - 1] > l) {
        lo[m] = lo[m - 1];
        hi[m] = hi[m - 1];
        --m;
      }
      lo[m] = l;
      hi[m] = h;
    }
    uint32_t ns = 0;
    const uint32_t o = offsets ? offsets[idx] : 0u;
    double cur = ylo;
    for (int t = 0; t < n; ++t) {
      if (lo[t] > cur) {
        if (offsets) spans[o + ns] = make_float2((float)cur, (float)lo[t]);
        ++ns;
      }
      if (hi[t] > cur) cur = hi[t];
    }
    if (cur <= yhi) {
      if (offsets) spans[o + ns] = make_float2((float)cur, (float)yhi);
      ++ns;
    }
    if (!offsets) counts[idx] = ns;
  }
}

}  // namespace

void launch_column_build(const float* boxes, int n_boxes, double ox, double oz, double ylo,
                         double yhi, int ncx, int ncz, const uint32_t* offsets, uint32_t* counts,
                         float2* spans, unsigned* overflow, cudaStream_t s) {
  const int total = 3 * ncx * ncz;
  int blocks = (total + 127) / 128;
  if (blocks > 148 * 16) blocks = 148 * 16;
  column_kernel<<<blocks, 128, (size_t)n_boxes * 6 * sizeof(double), s>>>(
      boxes, n_boxes, ox, oz, ylo, yhi, ncx, ncz, offsets, counts, spans, overflow);
}

__global__ void static_distance_kernel(const DScene* __restrict__ scenes, int scene,
                                       const float* __restrict__ pts, int n,
                                       float* __restrict__ dist) {
  const DScene& s = scenes[scene];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    float d;
    dist[t] = grid_query(s, pts[3 * t], pts[3 * t + 1], pts[3 * t + 2], d) ? d : CUDART_NAN_F;
  }
}

cudaError_t launch_static_distance(const DScene* scenes, int scene, const float* pts, int n,
                                   float* dist, cudaStream_t s) {
  const int blocks = std::min((n + 255) / 256, 148 * 8);
  static_distance_kernel<<<blocks, 256, 0, s>>>(scenes, scene, pts, n, dist);
  return cudaGetLastError();
}

void launch_grid_build(float* grid, const float* boxes, int n_boxes, float ox, float oy, float oz,
                       float h, int nx, int ny, int nz, cudaStream_t s) {
  const size_t total = (size_t)nx * ny * nz;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 148 * 64) blocks = 148 * 64;
  const size_t smem = (size_t)n_boxes * 6 * sizeof(double);
  grid_kernel<<<blocks, 256, smem, s>>>(grid, boxes, n_boxes, ox, oy, oz, h, nx, ny, nz);
}

}  // namespace gx
