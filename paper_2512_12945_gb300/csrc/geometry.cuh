// Per-point geometry of the band raycast (Sec. III-A): validity, world
// transform, ray and the Amanatides & Woo traversal of the truncation band.
// Every float operation is one explicitly rounded IEEE-754 op (_rn
// intrinsics, never contracted into an FMA) in a fixed order, so the set of
// voxels and the SDF of each (voxel, point) pair are reproducible bit for
// bit on any IEEE-754 machine that performs the same op sequence.
#pragma once
#include "common.cuh"

namespace slim {

struct Ray {
  float x0, x1, x2;   // world point
  float u0, u1, u2;   // unit ray direction
  float r;            // range from the sensor origin
  float t1;           // band end
  int32_t i0, i1, i2; // current voxel
  int32_t s0, s1, s2; // steps
  float m0, m1, m2;   // tMax
  float e0, e1, e2;   // tDelta
};

// Returns false for an invalid point. On success the ray is positioned on
// the first voxel of the band.
__device__ __forceinline__ bool ray_setup(const ScanGeom& g, float p0, float p1, float p2,
                                          Ray& ry) {
  if (!(isfinite(p0) && isfinite(p1) && isfinite(p2))) return false;
  float qs = __fadd_rn(__fadd_rn(__fmul_rn(p0, p0), __fmul_rn(p1, p1)), __fmul_rn(p2, p2));
  float rs = __fsqrt_rn(qs);
  if (!(rs >= g.rmin && rs <= g.rmax)) return false;
  float x[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float s = __fadd_rn(__fmul_rn(g.R[a * 3 + 0], p0), __fmul_rn(g.R[a * 3 + 1], p1));
    s = __fadd_rn(s, __fmul_rn(g.R[a * 3 + 2], p2));
    x[a] = __fadd_rn(s, g.t[a]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (!(fabsf(x[a]) < g.lim)) return false;
    if (!(fabsf(g.t[a]) < g.lim)) return false;
  }
  float d0 = __fsub_rn(x[0], g.t[0]);
  float d1 = __fsub_rn(x[1], g.t[1]);
  float d2 = __fsub_rn(x[2], g.t[2]);
  float rr = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
  float r = __fsqrt_rn(rr);
  if (!(r > 0.0f) || !isfinite(r)) return false;
  ry.x0 = x[0];
  ry.x1 = x[1];
  ry.x2 = x[2];
  ry.u0 = __fdiv_rn(d0, r);
  ry.u1 = __fdiv_rn(d1, r);
  ry.u2 = __fdiv_rn(d2, r);
  ry.r = r;
  float t0 = __fsub_rn(r, g.tau);
  if (t0 < 0.0f) t0 = 0.0f;
  ry.t1 = __fadd_rn(r, g.tau);
  const float v = g.v;
  const float u[3] = {ry.u0, ry.u1, ry.u2};
  int32_t ii[3], st[3];
  float tm[3], td[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float s = __fadd_rn(g.t[a], __fmul_rn(t0, u[a]));
    ii[a] = (int32_t)floorf(__fdiv_rn(s, v));
    st[a] = u[a] > 0.0f ? 1 : (u[a] < 0.0f ? -1 : 0);
    if (u[a] != 0.0f) {
      td[a] = __fdiv_rn(v, fabsf(u[a]));
      float bnd = __fmul_rn((float)(ii[a] + (st[a] > 0 ? 1 : 0)), v);
      tm[a] = __fadd_rn(t0, __fdiv_rn(__fsub_rn(bnd, s), u[a]));
    } else {
      td[a] = __int_as_float(0x7f800000);
      tm[a] = __int_as_float(0x7f800000);
    }
  }
  ry.i0 = ii[0]; ry.i1 = ii[1]; ry.i2 = ii[2];
  ry.s0 = st[0]; ry.s1 = st[1]; ry.s2 = st[2];
  ry.m0 = tm[0]; ry.m1 = tm[1]; ry.m2 = tm[2];
  ry.e0 = td[0]; ry.e1 = td[1]; ry.e2 = td[2];
  return true;
}

// ray_setup for point j of a scan: read from the AoS array pts, or (depth
// front end) back-projected from pixel (u, v) = (j mod dw, j div dw) of the
// z-depth image as (((u + 0.5) - cx) / fx * z, ((v + 0.5) - cy) / fy * z, z)
// in this FP32 op order; a non-finite or non-positive depth is invalid.
__device__ __forceinline__ bool ray_setup_at(const ScanGeom& g, const float* __restrict__ pts,
                                             int64_t j, Ray& ry) {
  float p0, p1, p2;
  if (g.depth) {
    const float z = __ldg(g.depth + j);
    if (!(z > 0.0f) || !isfinite(z)) return false;
    const int32_t u = (int32_t)(j % g.dw), v = (int32_t)(j / g.dw);
    const float xu = __fdiv_rn(__fsub_rn(__fadd_rn((float)u, 0.5f), g.cx), g.fx);
    const float yv = __fdiv_rn(__fsub_rn(__fadd_rn((float)v, 0.5f), g.cy), g.fy);
    p0 = __fmul_rn(xu, z);
    p1 = __fmul_rn(yv, z);
    p2 = z;
  } else {
    // points are read once per walk: streaming loads, evicted first, so the
    // map's hash and records keep the caches
    p0 = __ldcs(pts + 3 * j);
    p1 = __ldcs(pts + 3 * j + 1);
    p2 = __ldcs(pts + 3 * j + 2);
  }
  return ray_setup(g, p0, p1, p2, ry);
}

// Along-ray SDF of the current voxel's centre: d = (x - c) . u.
__device__ __forceinline__ float ray_sdf(const Ray& ry, float v) {
  float c0 = __fmul_rn(__fadd_rn((float)ry.i0, 0.5f), v);
  float c1 = __fmul_rn(__fadd_rn((float)ry.i1, 0.5f), v);
  float c2 = __fmul_rn(__fadd_rn((float)ry.i2, 0.5f), v);
  float d = __fadd_rn(__fmul_rn(__fsub_rn(ry.x0, c0), ry.u0),
                      __fmul_rn(__fsub_rn(ry.x1, c1), ry.u1));
  return __fadd_rn(d, __fmul_rn(__fsub_rn(ry.x2, c2), ry.u2));
}

// Step to the next voxel (lowest axis on ties). Returns false at band end.
__device__ __forceinline__ bool ray_step(Ray& ry) {
  int a = 0;
  float m = ry.m0;
  if (ry.m1 < m) { a = 1; m = ry.m1; }
  if (ry.m2 < m) { a = 2; m = ry.m2; }
  if (m > ry.t1) return false;
  if (a == 0) {
    ry.i0 += ry.s0;
    ry.m0 = __fadd_rn(ry.m0, ry.e0);
  } else if (a == 1) {
    ry.i1 += ry.s1;
    ry.m1 = __fadd_rn(ry.m1, ry.e1);
  } else {
    ry.i2 += ry.s2;
    ry.m2 = __fadd_rn(ry.m2, ry.e2);
  }
  return true;
}

// ray_step that also reports whether the voxel entered lies in another 8^3
// block than the one left (the stepped index crossed a multiple of 8).
__device__ __forceinline__ bool ray_step_blk(Ray& ry, bool& crossed) {
  int a = 0;
  float m = ry.m0;
  if (ry.m1 < m) { a = 1; m = ry.m1; }
  if (ry.m2 < m) { a = 2; m = ry.m2; }
  if (m > ry.t1) return false;
  int32_t o, nw;
  if (a == 0) {
    o = ry.i0;
    nw = ry.i0 += ry.s0;
    ry.m0 = __fadd_rn(ry.m0, ry.e0);
  } else if (a == 1) {
    o = ry.i1;
    nw = ry.i1 += ry.s1;
    ry.m1 = __fadd_rn(ry.m1, ry.e1);
  } else {
    o = ry.i2;
    nw = ry.i2 += ry.s2;
    ry.m2 = __fadd_rn(ry.m2, ry.e2);
  }
  crossed = ((o ^ nw) >> 3) != 0;
  return true;
}

// As ray_for_each, with f(i0, i1, i2, d, new_block): new_block is true for
// the first kept visit and for every kept visit whose block differs from
// the previous kept visit's (a block change at a skipped visit carries over).
template <class F>
__device__ __forceinline__ void ray_for_each_blk(const ScanGeom& g, Ray& ry, F&& f) {
  bool fresh = true;
  for (int k = 0; k < g.cap; ++k) {
    float d = ray_sdf(ry, g.v);
    if (!(d < -g.tau)) {
      f(ry.i0, ry.i1, ry.i2, d > g.tau ? g.tau : d, fresh);
      fresh = false;
    }
    bool crossed;
    if (!ray_step_blk(ry, crossed)) break;
    fresh |= crossed;
  }
}

// Visit every kept (voxel, point) observation of one point's band in ray
// order: f(i0, i1, i2, d) with d clamped to tau; visits with d < -tau are
// skipped. At most g.cap voxels are entered.
template <class F>
__device__ __forceinline__ void ray_for_each(const ScanGeom& g, Ray& ry, F&& f) {
  for (int k = 0; k < g.cap; ++k) {
    float d = ray_sdf(ry, g.v);
    if (!(d < -g.tau)) f(ry.i0, ry.i1, ry.i2, d > g.tau ? g.tau : d);
    if (!ray_step(ry)) break;
  }
}

}  // namespace slim
