// The plane constant of an axis-aligned box (Eq. plic-eq on a cuboid), FP32.
//
// In box coordinates u in [0, 1]^3 the fluid of the plane n.(x - x_c) + C = 0
// is {sum a_i (u_i - 1/2) + C + d >= 0}, a_i = n_i h_i (h the box sides), d
// = n.(box centre - x_c). Mirroring the axes with a_i < 0 and dividing by S
// = sum |a_i| gives {m.u >= 1/2 - (C + d)/S}, m_i = |a_i| / S, sum m_i = 1.
// With V(b) = vol{m.u <= b} the fluid fraction is 1 - V(1/2 - (C + d)/S),
// and V(1 - b) = 1 - V(b), so with g the root of V(g) = min(F, 1 - F) in
// [0, 1/2]: C + d = S (1/2 - g) for F >= 1/2 and S (g - 1/2) below.
//
// For m_1 <= m_2 <= m_3, V(b) is the mean over u_1 of A2(b - m_1 u_1), the
// area of {m_2 y + m_3 z <= t} in the unit square, a piecewise quadratic in
// t with breakpoints 0, m_2, m_3, m_2 + m_3. The mean is integrated exactly,
// piece by piece, in s = b - t in [0, m_1] (so that no width is formed as a
// difference of two numbers of the size of b, which a small m_1 would
// cancel): midpoint value plus the curvature term w^3 A2''/24.
//
// V is convex on [0, 1/2] (its slope is the area of the section {m.u = b}
// of the cube, which grows towards the centre), which bounds the root:
// V(b) <= b (the chord from V(0) = 0 to V(1/2) = 1/2), V(b) <= A2(b) and
// V(b) <= b^3 / (6 m_1 m_2 m_3) (the corner simplex) give lower bounds,
// V(b) >= A2(b - m_1) an upper bound; Newton steps inside that bracket,
// with bisection where a step leaves it, take a few iterations from there.
#pragma once

namespace gvof {

// the sorted slopes and the reciprocals the volume function uses; a slope
// below 1e-20 counts as 0 (it moves V by less than that)
struct BoxSlopes {
  float m1, m2, m3;   // m1 <= m2 <= m3
  float r1, r3, r23;  // 1 / m1, 1 / m3, 1 / (m2 m3); 0 for a zero slope
};

__host__ __device__ inline BoxSlopes box_slopes(float m1, float m2, float m3) {
  if (m1 > m2) { const float t = m1; m1 = m2; m2 = t; }
  if (m2 > m3) { const float t = m2; m2 = m3; m3 = t; }
  if (m1 > m2) { const float t = m1; m1 = m2; m2 = t; }
  if (m1 < 1e-20f) m1 = 0.f;
  if (m2 < 1e-20f) m2 = 0.f;
  BoxSlopes B;
  B.m1 = m1; B.m2 = m2; B.m3 = m3;  // m3 >= 1/3
  B.r1 = m1 > 0.f ? 1.f / m1 : 0.f;
  B.r3 = 1.f / m3;
  B.r23 = m2 > 0.f ? 1.f / (m2 * m3) : 0.f;
  return B;
}

// A2, A2' and A2'' at t (A2'' within a piece)
__host__ __device__ inline float box_area(float t, const BoxSlopes& B, float* d1, float* d2) {
  const float s = B.m2 + B.m3;
  if (t <= 0.f || t >= s) { *d1 = 0.f; *d2 = 0.f; return t <= 0.f ? 0.f : 1.f; }
  if (t < B.m2) { *d1 = t * B.r23; *d2 = B.r23; return 0.5f * t * t * B.r23; }  // triangle
  if (t <= B.m3) { *d1 = B.r3; *d2 = 0.f; return (t - 0.5f * B.m2) * B.r3; }    // band
  const float r = s - t;                                                        // square less
  *d1 = r * B.r23; *d2 = -B.r23;                                                // a triangle
  return 1.f - 0.5f * r * r * B.r23;
}

// V(b) and V'(b) for b in [0, 1/2]
__host__ __device__ inline float box_volume(float b, const BoxSlopes& B, float* slope) {
  float d1, d2;
  if (!(B.m1 > 0.f)) return box_area(b, B, slope, &d2);
  // breakpoints of A2 in s = b - t, increasing: b - m3 <= b - m2 <= b
  const float cut[3] = {b - B.m3, b - B.m2, b};
  float s0 = 0.f, acc = 0.f, dacc = 0.f;
  for (int i = 0; i <= 3; ++i) {
    float s1 = B.m1;
    if (i < 3) {
      if (!(cut[i] > s0 && cut[i] < B.m1)) continue;
      s1 = cut[i];
    }
    const float w = s1 - s0;
    if (w > 0.f) {
      const float a = box_area(b - 0.5f * (s0 + s1), B, &d1, &d2);
      acc += w * a + d2 * w * w * w * (1.f / 24.f);
      dacc += w * d1;  // A2' is linear on the piece: its midpoint value is its mean
    }
    s0 = s1;
  }
  *slope = dacc * B.r1;
  return acc * B.r1;
}

// the root g in [0, 1/2] of V(g) = v, v in [0, 1/2]
__host__ __device__ inline float box_root(float v, const BoxSlopes& B, int* iters = nullptr) {
  // root of A2 = v: A2(m2) = m2 / (2 m3), and A2(m3) = 1 - m2 / (2 m3) >= 1/2
  const float g2 = (B.m2 > 0.f && v <= 0.5f * B.m2 * B.r3) ? sqrtf(2.f * v * B.m2 * B.m3)
                                                           : v * B.m3 + 0.5f * B.m2;
  const float gc = B.m1 > 0.f ? cbrtf(6.f * B.m1 * B.m2 * B.m3 * v) : 0.f;
  float lo = v > g2 ? v : g2;
  if (gc > lo) lo = gc;
  float hi = g2 + B.m1;
  if (hi > 0.5f) hi = 0.5f;
  if (hi < lo) hi = lo;
  float g = lo;
  int it = 0;
  for (; it < 40; ++it) {
    float d;
    const float f = box_volume(g, B, &d) - v;
    if (f == 0.f) break;
    if (f < 0.f) lo = g; else hi = g;
    float gn = 0.5f * (lo + hi);
    if (d > 0.f) {
      const float step = f / d;
      if (fabsf(step) <= 2.5e-7f * g) {  // within ~2 ulp of the root
        g = fminf(fmaxf(g - step, lo), hi);
        break;
      }
      if (g - step > lo && g - step < hi) gn = g - step;
    }
    const bool done = gn == g || !(hi > lo);
    g = gn;
    if (done) break;
  }
  if (iters) *iters = it;
  return g;
}

}  // namespace gvof
