// Line clipping for the node sweeps: the part of a node line (one lattice axis,
// the two other node coordinates fixed) where a particle's signed distance lies
// below a threshold T.
//
// Every shape here is convex in the max-of-planes or Euclidean sense, so along
// a line {phi < T} is one interval: a sphere gives it by its quadratic, a
// cuboid or polytope as the intersection of one half-line per face plane, a
// wall as one half-line.  A node that contributes to any of the sweep's sums
// (volume, moments, the normal's band terms, the deepest node) has both
// distances below w/2 (Sec. 3.3.1's sweep restricted to the nodes where the
// indicator product or one indicator's derivative is non-zero), so a sweep
// clips each line to the two intervals at T = w/2 + kClipMargin and evaluates
// the nodes in between exactly as before: the nodes it skips would have added
// exact zeros.
//
// The bounds are computed in FP32 in the line's node-counter space (the node
// offset along the line relative to the particle's nearest node).  Their
// rounding error is far below the margin: a face value has an absolute error
// below 1e-5 cells, and a bound's relative error of a few ulps moves it by
// less than 1e-5 cells divided by the face's slope along the line, the scale
// at which the margin of 1e-3 cells acts too.  So every node whose FP32
// distances are both below w/2 lies inside the clipped interval.
#pragma once

#include <cuda_runtime.h>

namespace gbc {

constexpr float kClipMargin = 1e-3f;     // cells, added to the threshold of the clip
constexpr float kClipFlat = 1e-20f;      // a face this parallel to the line is constant along it
constexpr float kClipEmpty = 3.0e38f;    // a lower bound that empties the interval

// Three-operand maximum and minimum (one instruction each on this GPU; like
// fmaxf / fminf, a NaN operand gives way to the others).
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// 1 / a for the clip (0 for faces parallel to the line: they take the constant
// branch); the approximate reciprocal's relative error (~2^-22) moves a bound
// by far less than the margin.
__device__ __forceinline__ float clip_inv(float a) { return fabsf(a) > kClipFlat ? __fdividef(1.f, a) : 0.f; }

// |t c + p| < T: c in ((-T - p) / t, (T - p) / t), ordered by the sign of t.
__device__ __forceinline__ void clip_slab(float t, float inv_t, float p, float T, float& lo, float& hi) {
  if (fabsf(t) > kClipFlat) {
    const float a = (-T - p) * inv_t, b = (T - p) * inv_t;
    lo = fmaxf(lo, fminf(a, b));
    hi = fminf(hi, fmaxf(a, b));
  } else if (!(fabsf(p) < T)) {
    lo = kClipEmpty;
  }
}

// m c + p < T: c < (T - p) / m for m > 0, c > (T - p) / m for m < 0.
__device__ __forceinline__ void clip_half(float m, float inv_m, float p, float T, float& lo, float& hi) {
  if (fabsf(m) > kClipFlat) {
    const float b = (T - p) * inv_m;
    if (m > 0.f) hi = fminf(hi, b);
    else lo = fmaxf(lo, b);
  } else if (!(p < T)) {
    lo = kClipEmpty;
  }
}

// sqrt((c - f)^2 + rho2) - r < T: (c - f)^2 < (r + T)^2 - rho2.
__device__ __forceinline__ void clip_ball(float f, float rho2, float r, float T, float& lo, float& hi) {
  const float rt = r + T;
  const float d = fmaf(rt, rt, -rho2);
  if (rt > 0.f && d > 0.f) {
    const float s = sqrtf(d);
    lo = fmaxf(lo, f - s);
    hi = fminf(hi, f + s);
  } else {
    lo = kClipEmpty;
  }
}

// The nodes [first, first + count) of the segment [u0, u0 + len) inside the
// clipped interval [lo, hi] (segment coordinates; lo, hi already intersected
// with the segment's ends, so the conversions stay within int range).
__device__ __forceinline__ int clip_nodes(float lo, float hi, int u0, int len, int* first) {
  lo = fmaxf(lo, static_cast<float>(u0));
  hi = fminf(hi, static_cast<float>(u0 + len - 1));
  *first = u0;
  if (!(lo <= hi)) return 0;
  const int s = static_cast<int>(ceilf(lo)), e = static_cast<int>(floorf(hi));
  *first = s;
  return e >= s ? e - s + 1 : 0;
}

}  // namespace gbc
