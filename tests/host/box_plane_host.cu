// Host driver of the box plane-constant functions (box_plane.cuh), for the
// CPU tests: reads lines "m1 m2 m3 v" (FP32 values as decimal text) and
// prints the slopes as the functions use them (sorted, tiny ones zeroed),
// the root g of V(g) = v and the number of Newton iterations taken.
#include <cstdio>
#include <cmath>

#include "../../paper_2111_01524_gb300/csrc/box_plane.cuh"

int main() {
  float m1, m2, m3, v;
  while (std::scanf("%f %f %f %f", &m1, &m2, &m3, &v) == 4) {
    const gvof::BoxSlopes B = gvof::box_slopes(m1, m2, m3);
    int it = 0;
    const float g = gvof::box_root(v, B, &it);
    std::printf("%.9g %.9g %.9g %.9g %d\n", B.m1, B.m2, B.m3, g, it);
  }
  return 0;
}
