// Host-side check (no GPU) of subset_layout (csrc/haf_internal.h), the
// shared-memory map of one subset that the planner sizes warps by and the
// subset kernel addresses through.  For every element pair the kernels use
// (complex and real, FP64 and FP32-bulk), haf and lhaf, every even N up to
// 56, every h with N <= 2h <= 56 and both leading dimensions, it checks:
//  - the tile (N x ld) and the four series arrays fit before the vectors;
//  - W, P, TV (and VA for lhaf) follow, and La Budde's output and the loop
//    moments either lie past them or, for lhaf with N >= h + 1, sit in W
//    and P, which must then hold h + 1 elements;
//  - in the FP32-bulk mode the FP64 copies lie past the bulk arrays;
//  - every region starts on a 16-byte boundary where the kernel needs it,
//    the pair list fits, and 16 bytes at its start hold the lhaf's beta;
//  - the total is a multiple of 16 and nothing reaches past it.
// Exit status 0 and "layout ok" on success.
#include <cstdio>

#include "../../paper_1805_12498_gb300/csrc/haf_internal.h"

int main() {
  long bad = 0, cases = 0;
  struct Kind {
    int sb, ss;
    bool mixed;
  };
  const Kind kinds[] = {{16, 16, false}, {8, 8, false}, {8, 16, true}, {4, 8, true}};
  auto check = [&](bool ok, const char* what, int N, int ld, int h, const Kind& k, bool loops) {
    if (!ok && bad++ < 20)
      std::printf("%s: N=%d ld=%d h=%d sb=%d ss=%d mixed=%d loops=%d\n", what, N, ld, h, k.sb, k.ss, k.mixed, loops);
  };
  for (const Kind& k : kinds)
    for (int loops = 0; loops < 2; ++loops)
      for (int N = 2; N <= 56; N += 2)
        for (int h = N / 2; h <= 28; ++h)
          for (int ld : {N, N + 1}) {
            ++cases;
            const hafgb::SubsetLayout L = hafgb::subset_layout(N, ld, h, k.sb, k.ss, k.mixed, loops != 0);
            const int vecs = (loops ? 4 : 3) * N * k.sb;
            const int d = (h + 1) * k.sb;
            check(L.vec >= N * ld * k.sb && L.vec >= 4 * (h + 1) * k.ss && L.vec % 16 == 0, "tile/series", N, ld, h,
                  k, loops);
            int bulk_end;
            if (loops && N >= h + 1) {
              check(L.dnb == L.vec && L.ub == L.vec + N * k.sb && h + 1 <= N, "lhaf reuse of W and P", N, ld, h, k,
                    loops);
              bulk_end = L.vec + vecs;
            } else {
              check(L.dnb >= L.vec + vecs, "La Budde output after the vectors", N, ld, h, k, loops);
              if (loops) check(L.ub >= L.dnb + d, "moments after La Budde's output", N, ld, h, k, loops);
              bulk_end = loops ? L.ub + d : L.dnb + d;
            }
            if (k.mixed) {
              check(L.dn >= bulk_end && L.dn % 16 == 0 && L.u == L.dn + (h + 1) * k.ss, "FP64 copies", N, ld, h, k,
                    loops);
              bulk_end = L.u + (loops ? (h + 1) * k.ss : 0);
            } else {
              check(L.dn == L.dnb && L.u == L.ub, "FP64 arrays are the bulk arrays", N, ld, h, k, loops);
            }
            check(L.pos >= bulk_end && L.pos % 16 == 0, "pair list placement", N, ld, h, k, loops);
            check(L.total % 16 == 0 && L.total >= L.pos + 4 * h && L.total - L.pos >= 16, "pair list / beta / total",
                  N, ld, h, k, loops);
            check(hafgb::subset_bytes(N, ld, h, k.sb, k.ss, k.mixed, loops != 0) == L.total, "subset_bytes", N, ld, h,
                  k, loops);
          }
  std::printf("%s (%ld cases, %ld failures)\n", bad ? "layout FAILED" : "layout ok", cases, bad);
  return bad ? 1 : 0;
}
