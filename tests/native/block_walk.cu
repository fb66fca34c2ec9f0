// Host-side check (no GPU) of BlockWalk (csrc/haf_internal.h), the index
// walk of the subset kernel's update pass and gather: for every column
// count L = 1..64, group width G = 1..32 (powers of two) and lane g < G, the
// walk's (i, j) at each element e = g, g + G, ... below 64 * 64 equals
// (e / L, e % L).  Exit status 0 and "block walk ok" on success.
#include <cstdio>

#include "../../paper_1805_12498_gb300/csrc/haf_internal.h"

int main() {
  long bad = 0, checks = 0;
  for (int L = 1; L <= 64; ++L)
    for (int G = 1; G <= 32; G *= 2)
      for (int g = 0; g < G; ++g) {
        hafgb::BlockWalk w(g, G, L);
        for (int e = g; e < 64 * 64; e += G, w.next()) {
          ++checks;
          if (w.i != e / L || w.j != e % L) {
            if (bad++ < 10) std::printf("L=%d G=%d g=%d e=%d: (%d, %d)\n", L, G, g, e, w.i, w.j);
          }
        }
      }
  std::printf("%s (%ld checks, %ld failures)\n", bad ? "block walk FAILED" : "block walk ok", checks, bad);
  return bad ? 1 : 0;
}
