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

// Plain 16-byte copy; with a source in pinned host memory (read through the
// unified address space) it is the host-to-device transfer itself, which SM
// loads move faster than the copy engine on this class of system.
__global__ void copy16_kernel(const float4* __restrict__ src, float4* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

cudaError_t launch_copy16(const float4* src, float4* dst, int64_t n, int max_blocks, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t want = (n + 255) / 256;
  copy16_kernel<<<(unsigned)(want < max_blocks ? want : max_blocks), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
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
