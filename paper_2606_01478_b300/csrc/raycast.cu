// Batched depth rendering by ray casting (the paper's parallel depth images:
// Results, Computation Performance; Materials and Methods, Visualization and
// Collision Checking).  Every drone carries a pinhole depth camera at its
// centre looking along body +x; pixel (row i, column j) casts
//   d_body = normalise(1, -tan(hfov/2) (2 (j + 0.5) / W - 1), -tan(vfov/2) (2 (i + 0.5) / H - 1))
// rotated to the world by R(q).  Depth = distance to the first hit among
// spheres, axis-aligned boxes and the ground plane z = 0, else max_range.
// One thread per ray, one warp per tile of rays; the drone's pose is a
// broadcast load from the state planes; the scene sits in kernel parameter
// space (constant bank).
#include <cmath>

#include "internal.h"
#include "physics.cuh"

namespace cf {
namespace rc {

struct Scene {
  float4 sph[SIM_MAX_SPHERES];  // centre xyz, radius
  float4 lo[SIM_MAX_BOXES];     // box min corner (w unused)
  float4 hi[SIM_MAX_BOXES];     // box max corner
  float4 bsph[SIM_MAX_BOXES];   // each box's bounding sphere (centre, half diagonal)
  int n_sph, n_box;
  int H, W;
  float tan_h, tan_v, max_range;
};

// Tiles of TILE_R x TILE_C pixels, one per warp.  Before its rays are cast, the
// warp drops the primitives that no ray of the tile can reach: the tile's rays
// lie in the pyramid {x (1, y, z) : x >= 0, y in [y_lo, y_hi], z in [z_lo, z_hi]}
// of the camera frame, bounded by four planes through the camera; a sphere
// entirely outside one of them (or behind the camera) is hit by none of these
// rays.  Each lane tests one sphere (boxes by their bounding spheres) with a
// margin of 1e-4 (|c| + r) + 1e-5 against rounding in the per-ray tests, so a
// primitive that a ray's own test could hit is never dropped; the rays then walk
// the surviving set in index order, and every depth is the one the full loop
// gives.  The eight warps of a block render one drone: the primitives' centres
// in its camera frame and their margins are computed once per block.
constexpr int TILE_R = 4, TILE_C = 8;

// c: centre in the camera frame, m: radius plus margin
__device__ __forceinline__ bool outside_tile(float4 c, float ylo, float yhi, float zlo, float zhi,
                                             const float ninv[4]) {
  const float m = c.w;
  return c.x < -m || (ylo * c.x - c.y) * ninv[0] > m || (c.y - yhi * c.x) * ninv[1] > m ||
         (zlo * c.x - c.z) * ninv[2] > m || (c.z - zhi * c.x) * ninv[3] > m;
}

__global__ void __launch_bounds__(256) depth_kernel(const float4* __restrict__ planes, int n, Scene sc,
                                                    float* __restrict__ out) {
  const unsigned FULL = 0xffffffffu;
  const int e = blockIdx.y;
  const float4 a = planes[e], b = planes[(size_t)n + e];
  const float ox = a.x, oy = a.y, oz = a.z;
  float R[9];
  quat_rot(a.w, b.x, b.y, b.z, R);
  auto to_camera = [&](float4 c) {  // (R^T (centre - o), radius + margin)
    const float wx = c.x - ox, wy = c.y - oy, wz = c.z - oz;
    const float x = fmaf(R[0], wx, fmaf(R[3], wy, R[6] * wz));
    const float y = fmaf(R[1], wx, fmaf(R[4], wy, R[7] * wz));
    const float z = fmaf(R[2], wx, fmaf(R[5], wy, R[8] * wz));
    const float m = c.w + fmaf(1e-4f, sqrt_approx(fmaf(x, x, fmaf(y, y, z * z))) + c.w, 1e-5f);
    return make_float4(x, y, z, m);
  };
  // the primitives in this drone's camera frame, once per block, in shared memory
  // (the cull reads one per lane; lanes reading different entries of the
  // constant bank are served one address at a time)
  __shared__ float4 s_sph[SIM_MAX_SPHERES], s_box[SIM_MAX_BOXES];
  for (int k = threadIdx.x; k < sc.n_sph; k += blockDim.x) s_sph[k] = to_camera(sc.sph[k]);
  for (int k = threadIdx.x; k < sc.n_box; k += blockDim.x) s_box[k] = to_camera(sc.bsph[k]);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int tw = (sc.W + TILE_C - 1) / TILE_C, th = (sc.H + TILE_R - 1) / TILE_R;
  const int tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (tile >= tw * th) return;  // the whole warp leaves together (after the block's barrier)
  const int ti = tile / tw, tj = tile - ti * tw;
  const int i = ti * TILE_R + lane / TILE_C, j = tj * TILE_C + lane % TILE_C;
  const bool valid = i < sc.H && j < sc.W;
  const int npx = sc.H * sc.W;
  auto ray_y = [&](int jj) { return -sc.tan_h * fmaf(2.f / sc.W, jj + 0.5f, -1.f); };
  auto ray_z = [&](int ii) { return -sc.tan_v * fmaf(2.f / sc.H, ii + 0.5f, -1.f); };
  // the tile's bounds (ray_y and ray_z fall with the column and the row)
  const int j0 = tj * TILE_C, j1 = min(j0 + TILE_C - 1, sc.W - 1);
  const int i0 = ti * TILE_R, i1 = min(i0 + TILE_R - 1, sc.H - 1);
  const float yhi = ray_y(j0), ylo = ray_y(j1), zhi = ray_z(i0), zlo = ray_z(i1);
  const float ninv[4] = {rsqrtf(fmaf(ylo, ylo, 1.f)), rsqrtf(fmaf(yhi, yhi, 1.f)),
                         rsqrtf(fmaf(zlo, zlo, 1.f)), rsqrtf(fmaf(zhi, zhi, 1.f))};
  unsigned keep_s[2], keep_b;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int s = lane + 32 * h;
    bool keep = false;
    if (s < sc.n_sph) {
      keep = !outside_tile(s_sph[s], ylo, yhi, zlo, zhi, ninv);
    }
    keep_s[h] = __ballot_sync(FULL, keep);
  }
  {
    bool keep = false;
    if (lane < sc.n_box) {
      keep = !outside_tile(s_box[lane], ylo, yhi, zlo, zhi, ninv);
    }
    keep_b = __ballot_sync(FULL, keep);
  }
  const float by = ray_y(j);
  const float bz = ray_z(i);
  const float inv = rsqrtf(fmaf(by, by, fmaf(bz, bz, 1.f)));
  const float ux = inv, uy = by * inv, uz = bz * inv;
  const float dx = fmaf(R[0], ux, fmaf(R[1], uy, R[2] * uz));
  const float dy = fmaf(R[3], ux, fmaf(R[4], uy, R[5] * uz));
  const float dz = fmaf(R[6], ux, fmaf(R[7], uy, R[8] * uz));
  float t = sc.max_range;
  if (dz < 0.f) {
    const float tg = -oz / dz;
    if (tg >= 0.f) t = fminf(t, tg);
  }
  auto sphere = [&](int s) {
    const float4 c = sc.sph[s];
    const float cx = ox - c.x, cy = oy - c.y, cz = oz - c.z;
    const float bb = fmaf(cx, dx, fmaf(cy, dy, cz * dz));
    const float cc = fmaf(cx, cx, fmaf(cy, cy, fmaf(cz, cz, -c.w * c.w)));
    const float disc = fmaf(bb, bb, -cc);
    if (disc >= 0.f) {
      const float q = sqrtf(disc);
      const float t0 = -bb - q, t1 = -bb + q;
      const float th = t0 >= 0.f ? t0 : t1;
      if (th >= 0.f) t = fminf(t, th);
    }
  };
  for (unsigned m = keep_s[0]; m; m &= m - 1u) sphere(__ffs(m) - 1);
  for (unsigned m = keep_s[1]; m; m &= m - 1u) sphere(32 + __ffs(m) - 1);
  if (keep_b) {
    const float ix = 1.f / dx, iy = 1.f / dy, iz = 1.f / dz;  // +-inf on axis-parallel rays
    for (unsigned m = keep_b; m; m &= m - 1u) {
      const int k = __ffs(m) - 1;
      const float4 lo = sc.lo[k], hi = sc.hi[k];
      const float ax = (lo.x - ox) * ix, bx = (hi.x - ox) * ix;
      const float ay = (lo.y - oy) * iy, byy = (hi.y - oy) * iy;
      const float az = (lo.z - oz) * iz, bzz = (hi.z - oz) * iz;
      // fminf/fmaxf drop a NaN operand (0 * inf on a slab plane), as the oracle's nan-min/max
      const float tmin = fmaxf(fmaxf(fminf(ax, bx), fminf(ay, byy)), fminf(az, bzz));
      const float tmax = fminf(fminf(fmaxf(ax, bx), fmaxf(ay, byy)), fmaxf(az, bzz));
      const float te = fmaxf(tmin, 0.f);
      if (tmax >= te) t = fminf(t, te);
    }
  }
  if (valid) out[(size_t)e * npx + i * sc.W + j] = t;
}

}  // namespace rc

cudaError_t launch_depth(const float4* planes, int n, int H, int W, float hfov, float vfov,
                         float max_range, const float* spheres, int n_sph, const float* boxes,
                         int n_box, float* out, cudaStream_t st) {
  rc::Scene sc;
  for (int s = 0; s < SIM_MAX_SPHERES; ++s)
    sc.sph[s] = s < n_sph ? make_float4(spheres[4 * s], spheres[4 * s + 1], spheres[4 * s + 2],
                                        spheres[4 * s + 3])
                          : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = 0; k < SIM_MAX_BOXES; ++k) {
    sc.lo[k] = k < n_box ? make_float4(boxes[6 * k], boxes[6 * k + 1], boxes[6 * k + 2], 0.f)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
    sc.hi[k] = k < n_box ? make_float4(boxes[6 * k + 3], boxes[6 * k + 4], boxes[6 * k + 5], 0.f)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int k = 0; k < SIM_MAX_BOXES; ++k) {
    const float4 lo = sc.lo[k], hi = sc.hi[k];
    const float hx = 0.5f * (hi.x - lo.x), hy = 0.5f * (hi.y - lo.y), hz = 0.5f * (hi.z - lo.z);
    sc.bsph[k] = make_float4(lo.x + hx, lo.y + hy, lo.z + hz,
                             std::sqrt(hx * hx + hy * hy + hz * hz) * 1.0001f + 1e-6f);
  }
  sc.n_sph = n_sph;
  sc.n_box = n_box;
  sc.H = H;
  sc.W = W;
  sc.tan_h = tanf(0.5f * hfov);
  sc.tan_v = tanf(0.5f * vfov);
  sc.max_range = max_range;
  const int tpb = 256;
  const int tiles = ((W + rc::TILE_C - 1) / rc::TILE_C) * ((H + rc::TILE_R - 1) / rc::TILE_R);
  dim3 grid((tiles + tpb / 32 - 1) / (tpb / 32), n);
  rc::depth_kernel<<<grid, tpb, 0, st>>>(planes, n, sc, out);
  return cudaGetLastError();
}

}  // namespace cf
