// Host-side generation of the stage-ordered twiddle tables of the shared-memory FFT.
//
// For a transform of length L = 2^lgL with radices r_0 .. r_{m-1} (the plan rule of
// fft_plan<T>: radix 16 while at least 4 factors of two remain, except when exactly 5 remain,
// in single precision; radix 8 in double precision; then one radix 4 or 2), stage s has
// p_s = r_0 ... r_{s-1} and needs w^(j k) = exp(-2 pi i j k / (p_s r_s)) for 1 <= j < r_s and
// 0 <= k < p_s.  Entry (j - 1) p_s + k of the stage's block holds it, so the threads of a warp
// (consecutive k) read consecutive entries.  Table A holds the blocks of the plan in order,
// table B those of the reversed plan (used by the inverse half of a fused round trip); B
// follows A.
#pragma once
#include <cmath>

#include "mf_common.cuh"

namespace mf {

inline int plan_lgr(int lgL, bool single, int* lgr) {
  int m = 0, rem = lgL;
  while (rem > 0) {
    int l;
    if (single && VPT >= 16 && rem >= 4 && rem != 5) l = 4;
    else if (rem >= 3) l = 3;
    else l = rem;
    lgr[m++] = l;
    rem -= l;
  }
  return m;
}

// writes (re, im) pairs of tables A then B into out; returns the number of complex entries
template <typename T>
inline int stage_twiddles(int L, T* out) {
  int lgL = 0;
  while ((1 << lgL) < L) ++lgL;
  int lgr[32];
  const int m = plan_lgr(lgL, sizeof(T) == 4, lgr);
  int n = 0;
  for (int pass = 0; pass < 2; ++pass) {
    int lgp = 0;
    for (int s = 0; s < m; ++s) {
      const int l = pass == 0 ? lgr[s] : lgr[m - 1 - s];
      const int R = 1 << l, p = 1 << lgp;
      for (int j = 1; j < R; ++j)
        for (int k = 0; k < p; ++k) {
          const double ang = -2.0 * M_PI * (double)j * (double)k / (double)(p * R);
          out[2 * n] = (T)std::cos(ang);
          out[2 * n + 1] = (T)std::sin(ang);
          ++n;
        }
      lgp += l;
    }
  }
  return n;
}

}  // namespace mf
