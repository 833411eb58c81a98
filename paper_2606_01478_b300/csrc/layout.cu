// Conversion between the user-facing state rows [n][20] and the five float4
// planes the step kernels read (plane j = state slots 4j..4j+3).  One thread
// per float4: reads of the rows are contiguous across a warp.
#include "internal.h"

namespace cf {

__global__ void rows_to_planes_kernel(const float4* __restrict__ rows, float4* __restrict__ planes,
                                      int n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * 5) return;
  const int64_t i = t / 5, j = t - i * 5;
  planes[j * n + i] = rows[t];
}

__global__ void planes_to_rows_kernel(const float4* __restrict__ planes, float4* __restrict__ rows,
                                      int n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * 5) return;
  const int64_t i = t / 5, j = t - i * 5;
  rows[t] = planes[j * n + i];
}

cudaError_t launch_rows_to_planes(const float4* rows, float4* planes, int n, cudaStream_t st) {
  const int64_t total = (int64_t)n * 5;
  const int tpb = 256;
  rows_to_planes_kernel<<<(unsigned)((total + tpb - 1) / tpb), tpb, 0, st>>>(rows, planes, n);
  return cudaGetLastError();
}

cudaError_t launch_planes_to_rows(const float4* planes, float4* rows, int n, cudaStream_t st) {
  const int64_t total = (int64_t)n * 5;
  const int tpb = 256;
  planes_to_rows_kernel<<<(unsigned)((total + tpb - 1) / tpb), tpb, 0, st>>>(planes, rows, n);
  return cudaGetLastError();
}

}  // namespace cf
