// Batched depth rendering by ray casting (the paper's parallel depth images:
// Results, Computation Performance; Materials and Methods, Visualization and
// Collision Checking).  Every drone carries a pinhole depth camera at its
// centre looking along body +x; pixel (row i, column j) casts
//   d_body = normalise(1, -tan(hfov/2) (2 (j + 0.5) / W - 1), -tan(vfov/2) (2 (i + 0.5) / H - 1))
// rotated to the world by R(q).  Depth = distance to the first hit among
// spheres, axis-aligned boxes and the ground plane z = 0, else max_range.
// One thread per ray; the drone's pose is a broadcast load from the state
// planes; the scene sits in kernel parameter space (constant bank).
#include "internal.h"
#include "physics.cuh"

namespace cf {
namespace rc {

struct Scene {
  float4 sph[SIM_MAX_SPHERES];  // centre xyz, radius
  float4 lo[SIM_MAX_BOXES];     // box min corner (w unused)
  float4 hi[SIM_MAX_BOXES];     // box max corner
  int n_sph, n_box;
  int H, W;
  float tan_h, tan_v, max_range;
};

__global__ void __launch_bounds__(256) depth_kernel(const float4* __restrict__ planes, int n, Scene sc,
                                                    float* __restrict__ out) {
  const int e = blockIdx.y;
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  const int npx = sc.H * sc.W;
  if (pix >= npx) return;
  const int i = pix / sc.W, j = pix - i * sc.W;
  const float4 a = planes[e], b = planes[(size_t)n + e];
  const float ox = a.x, oy = a.y, oz = a.z;
  float R[9];
  quat_rot(a.w, b.x, b.y, b.z, R);
  const float by = -sc.tan_h * fmaf(2.f / sc.W, j + 0.5f, -1.f);
  const float bz = -sc.tan_v * fmaf(2.f / sc.H, i + 0.5f, -1.f);
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
  for (int s = 0; s < sc.n_sph; ++s) {
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
  }
  if (sc.n_box > 0) {
    const float ix = 1.f / dx, iy = 1.f / dy, iz = 1.f / dz;  // +-inf on axis-parallel rays
    for (int k = 0; k < sc.n_box; ++k) {
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
  out[(size_t)e * npx + pix] = t;
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
  sc.n_sph = n_sph;
  sc.n_box = n_box;
  sc.H = H;
  sc.W = W;
  sc.tan_h = tanf(0.5f * hfov);
  sc.tan_v = tanf(0.5f * vfov);
  sc.max_range = max_range;
  const int tpb = 256;
  dim3 grid((H * W + tpb - 1) / tpb, n);
  rc::depth_kernel<<<grid, tpb, 0, st>>>(planes, n, sc, out);
  return cudaGetLastError();
}

}  // namespace cf
