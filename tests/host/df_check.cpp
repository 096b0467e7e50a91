// Host driver for the double-float helpers of the BSS kernel (csrc/fd_df.cuh): reads commands
// from stdin, one per line, numbers as C99 hex floats, and prints the results the same way.
//   s d               -> hi lo           split of an FP64 value
//   j hi lo           -> d               join of a pair
//   w f               -> d               FP32 -> FP64 on the bit pattern
//   m g4 a4 b4        -> r4              g - a * b for complex pairs (re hi, re lo, im hi, im lo)
//   r g4 c            -> r4              g + c on the real part
//   a r4              -> th tl           |r|^2
//   q th tl           -> yh yl           1 / t
//   g ah al bh bl     -> 0 or 1          a > b
//   c a4 yh yl        -> r4              a * y (complex times real)
// Compile without FP contraction (-ffp-contract=off) so that the FP32 steps round as written.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../paper_2604_02130_gb300/csrc/fd_df.cuh"

using fd::df::c4;

static c4 read4(char** p) {
  c4 r;
  r.x = (float)strtod(*p, p);
  r.y = (float)strtod(*p, p);
  r.z = (float)strtod(*p, p);
  r.w = (float)strtod(*p, p);
  return r;
}

static void print4(c4 r) {
  printf("%a %a %a %a\n", (double)r.x, (double)r.y, (double)r.z, (double)r.w);
}

int main() {
  char line[1024];
  while (fgets(line, sizeof line, stdin)) {
    char* p = line + 1;
    switch (line[0]) {
      case 's': {
        float hi, lo;
        fd::df::split(strtod(p, &p), hi, lo);
        printf("%a %a\n", (double)hi, (double)lo);
        break;
      }
      case 'j': {
        const float hi = (float)strtod(p, &p), lo = (float)strtod(p, &p);
        printf("%a\n", fd::df::join(hi, lo));
        break;
      }
      case 'w': {
        printf("%a\n", fd::df::widen((float)strtod(p, &p)));
        break;
      }
      case 'm': {
        const c4 g = read4(&p), a = read4(&p), b = read4(&p);
        print4(fd::df::cms(g, a, b));
        break;
      }
      case 'r': {
        const c4 g = read4(&p);
        print4(fd::df::add_re(g, (float)strtod(p, &p)));
        break;
      }
      case 'a': {
        float th, tl;
        fd::df::abs2(read4(&p), th, tl);
        printf("%a %a\n", (double)th, (double)tl);
        break;
      }
      case 'q': {
        const float th = (float)strtod(p, &p), tl = (float)strtod(p, &p);
        float yh, yl;
        fd::df::recip(th, tl, yh, yl);
        printf("%a %a\n", (double)yh, (double)yl);
        break;
      }
      case 'g': {
        const float ah = (float)strtod(p, &p), al = (float)strtod(p, &p);
        const float bh = (float)strtod(p, &p), bl = (float)strtod(p, &p);
        printf("%d\n", fd::df::greater(ah, al, bh, bl) ? 1 : 0);
        break;
      }
      case 'c': {
        const c4 a = read4(&p);
        const float yh = (float)strtod(p, &p), yl = (float)strtod(p, &p);
        print4(fd::df::scale(a, yh, yl));
        break;
      }
      default:
        return 2;
    }
  }
  return 0;
}
