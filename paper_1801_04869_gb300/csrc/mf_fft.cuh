// Shared-memory FFT of a batch of lines (Stockham autosort; radix 16 and 8 in single
// precision, radix 8 in double, with one radix-4 or radix-2 stage), the building block of
// every row, column and z pass.
//
// A CTA of NT threads transforms `nlines` lines of length L (a power of two, 2..4096) that
// sit back to back in shared memory (element e at position sp(e)), nlines * L <= BATCH.
// Stages alternate between two shared buffers (each thread keeps one butterfly in registers).
// Twiddles come from a read-only global table in stage order (mf_tables.h), so the lanes of a
// warp read consecutive entries; the inverse uses their conjugates and is unnormalised.
#pragma once
#include "mf_common.cuh"

namespace mf {

// The threads that run one transform together: the whole CTA (the default) or one half of it
// (threads [NT/2 g, NT/2 g + NT/2)) with its own named barrier, so that the two halves work on
// their own lines without waiting for each other.
struct Cta {
  __device__ __forceinline__ int tid() const { return threadIdx.x; }
  static constexpr int nt = NT;
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct HalfCta {
  int g;
  __device__ __forceinline__ int tid() const { return threadIdx.x & (NT / 2 - 1); }
  static constexpr int nt = NT / 2;
  __device__ __forceinline__ void sync() const {
    asm volatile("bar.sync %0, %1;" :: "r"(1 + g), "n"(NT / 2) : "memory");
  }
};

template <typename T> struct Sqrt1_2;
template <> struct Sqrt1_2<float> { static constexpr float v = 0.70710678118654752440f; };
template <> struct Sqrt1_2<double> { static constexpr double v = 0.70710678118654752440; };

template <typename T, int DIR>
__device__ __forceinline__ void dft4(C2<T>& a0, C2<T>& a1, C2<T>& a2, C2<T>& a3) {
  C2<T> t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
  C2<T> t3 = cmul_si(csub(a1, a3), DIR);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

// multiply by (c + DIR i s)
template <typename T, int DIR>
__device__ __forceinline__ C2<T> crot(C2<T> a, T c, T s) {
  const T ss = (T)DIR * s;
  return C2<T>{a.x * c - a.y * ss, a.x * ss + a.y * c};
}

// length-16 DFT as 4 x 4: DFT4 over n1 for each n2, twiddles W16^(n2 k1), DFT4 over n2, and
// the transpose k1 + 4 k2 -> natural order
template <typename T, int DIR>
__device__ __forceinline__ void dft16(C2<T>* v) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, h = Sqrt1_2<T>::v;
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<T, DIR>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);
  // slot 4 k1 + n2 holds y[n2][k1]; multiply by W16^(n2 k1), W16^m = cos(m pi/8) + DIR i sin(m pi/8)
  v[5] = crot<T, DIR>(v[5], c1, s1);                       // n2 = 1, k1 = 1: m = 1
  v[9] = crot<T, DIR>(v[9], h, h);                         // n2 = 1, k1 = 2: m = 2
  v[13] = crot<T, DIR>(v[13], s1, c1);                     // n2 = 1, k1 = 3: m = 3
  v[6] = crot<T, DIR>(v[6], h, h);                         // n2 = 2, k1 = 1: m = 2
  v[10] = cmul_si(v[10], DIR);                             // n2 = 2, k1 = 2: m = 4
  v[14] = crot<T, DIR>(v[14], -h, h);                      // n2 = 2, k1 = 3: m = 6
  v[7] = crot<T, DIR>(v[7], s1, c1);                       // n2 = 3, k1 = 1: m = 3
  v[11] = crot<T, DIR>(v[11], -h, h);                      // n2 = 3, k1 = 2: m = 6
  v[15] = crot<T, DIR>(v[15], -c1, -s1);                   // n2 = 3, k1 = 3: m = 9
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<T, DIR>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  // X[k1 + 4 k2] sits in slot 4 k1 + k2
  C2<T> w[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) w[j] = v[4 * (j & 3) + (j >> 2)];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = w[j];
}

template <typename T, int R, int DIR>
__device__ __forceinline__ void dft(C2<T>* v) {
  if constexpr (R == 16) {
    dft16<T, DIR>(v);
  } else if constexpr (R == 2) {
    C2<T> a = cadd(v[0], v[1]), b = csub(v[0], v[1]);
    v[0] = a; v[1] = b;
  } else if constexpr (R == 4) {
    dft4<T, DIR>(v[0], v[1], v[2], v[3]);
  } else {
    // radix-2 decimation in time over two length-4 transforms
    C2<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C2<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<T, DIR>(e0, e1, e2, e3);
    dft4<T, DIR>(o0, o1, o2, o3);
    const T h = Sqrt1_2<T>::v;
    // W8^1 = (1 + DIR i)/sqrt2, W8^2 = DIR i, W8^3 = (-1 + DIR i)/sqrt2
    C2<T> w1o = {h * (o1.x - (T)DIR * o1.y), h * (o1.y + (T)DIR * o1.x)};
    C2<T> w2o = cmul_si(o2, DIR);
    C2<T> w3o = {h * (-o3.x - (T)DIR * o3.y), h * (-o3.y + (T)DIR * o3.x)};
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1o); v[5] = csub(e1, w1o);
    v[2] = cadd(e2, w2o); v[6] = csub(e2, w2o);
    v[3] = cadd(e3, w3o); v[7] = csub(e3, w3o);
  }
}

// Twiddles w^(j k), 1 <= j < R, of one butterfly, applied in place (v[j] *= w^(j k)): the powers
// j = 1, 2, 4, 8 come from the stage's block of the stage-ordered table (entry (j - 1) p + k;
// twiddle_base loads them, conjugated for the inverse direction), the others are products of
// two of them (w^(3k) = w^(2k) w^k, w^(7k) = w^(4k) w^(3k), ...), at most three roundings from
// the table values.  Each product is formed next to its use, so only the base powers and four
// odd products stay live (register pressure of the radix-16 stage).
template <typename T, int R, int DIR>
__device__ __forceinline__ void twiddle_base(const C2<T>* __restrict__ twk, int p, C2<T>* b) {
#pragma unroll
  for (int j = 1, s = 0; j < R; j <<= 1, ++s) {
    b[s] = ldg_c2(twk + (j - 1) * p);
    if (DIR > 0) b[s].y = -b[s].y;
  }
}
template <typename T, int R>
__device__ __forceinline__ void twiddle_apply(const C2<T>* b, C2<T>* v) {
  v[1] = cmul(v[1], b[0]);
  if constexpr (R > 2) {
    v[2] = cmul(v[2], b[1]);
    const C2<T> w3 = cmul(b[1], b[0]);
    v[3] = cmul(v[3], w3);
    if constexpr (R > 4) {
      v[4] = cmul(v[4], b[2]);
      const C2<T> w5 = cmul(b[2], b[0]), w6 = cmul(b[2], b[1]), w7 = cmul(b[2], w3);
      v[5] = cmul(v[5], w5);
      v[6] = cmul(v[6], w6);
      v[7] = cmul(v[7], w7);
      if constexpr (R > 8) {
        v[8] = cmul(v[8], b[3]);
        v[9] = cmul(v[9], cmul(b[3], b[0]));
        v[10] = cmul(v[10], cmul(b[3], b[1]));
        v[11] = cmul(v[11], cmul(b[3], w3));
        v[12] = cmul(v[12], cmul(b[3], b[2]));
        v[13] = cmul(v[13], cmul(b[3], w5));
        v[14] = cmul(v[14], cmul(b[3], w6));
        v[15] = cmul(v[15], cmul(b[3], w7));
      }
    }
  }
}

// one Stockham stage of radix R from `in` to `out`; p = 2^lgp = product of the radices
// already applied.  Butterfly b of line `line` reads in[i + j L/R] (j < R), multiplies by
// w^(j k) with k = i mod p and w = exp(DIR 2 pi i / (p R)), and writes its length-R DFT to
// out[(i - k) R + k + j p].  `tw` is the stage's block of the stage-ordered table: entry
// (j - 1) p + k holds w^(j k) for the forward direction.
//
// Padded addressing: for a stride s that is a multiple of 16, sp(e + j s) = sp(e) + j (s + s/16),
// so a butterfly's R elements sit at one base plus multiples of a padded stride.  The same
// holds with stride 1 when e is a multiple of R (R divides 16): the R outputs of a p = 1 stage
// share one padding group.  Other strides (short lines) take sp() per element.
template <typename T, int R, int LGR, int DIR, class G = Cta>
__device__ __forceinline__ void fft_stage(const C2<T>* in_p, C2<T>* out_p, int lgL, int lgp, int nlines,
                                          const C2<T>* __restrict__ tw, G grp = G()) {
  C2<T>* const S = dsm<T>();
  const int in = dsm_off(in_p), out = dsm_off(out_p);
  const int lgq = lgL - LGR;          // log2(L / R)
  const int q = 1 << lgq;
  const int p = 1 << lgp;
  const int nb = nlines << lgq;       // butterflies in this stage
  const int qs = q + (q >> 4), ps = p + (p >> 4);
  const bool fast_in = lgq >= 4, fast_out = lgp == 0 || lgp >= 4;
  for (int b = grp.tid(); b < nb; b += G::nt) {
    const int line = b >> lgq, i = b & (q - 1);
    const int k = i & (p - 1);
    const int src = (line << lgL) + i;
    C2<T> v[R];
    if (fast_in) {
      const int a0 = in + sp(src);
#pragma unroll
      for (int j = 0; j < R; ++j) v[j] = S[a0 + j * qs];
    } else {
#pragma unroll
      for (int j = 0; j < R; ++j) v[j] = S[in + sp(src + (j << lgq))];
    }
    if (lgp > 0) {
      C2<T> wb[LGR];
      twiddle_base<T, R, DIR>(tw + k, p, wb);
      twiddle_apply<T, R>(wb, v);
    }
    dft<T, R, DIR>(v);
    const int dst = (line << lgL) + ((i - k) << LGR) + k;
    if (fast_out) {
      const int a0 = out + sp(dst);
#pragma unroll
      for (int j = 0; j < R; ++j) S[a0 + j * ps] = v[j];
    } else {
#pragma unroll
      for (int j = 0; j < R; ++j) S[out + sp(dst + (j << lgp))] = v[j];
    }
  }
  grp.sync();
}

// radix 16 is used in single precision when a thread holds 16 values per stage
template <typename T> constexpr bool kRadix16 = sizeof(T) == 4 && VPT >= 16;

// one stage of radix 2^lgr (the plan's choice) through the matching instantiation
template <typename T, int DIR, class G = Cta>
__device__ __forceinline__ void fft_stage_any(int lgr, const C2<T>* in, C2<T>* out, int lgL, int lgp,
                                              int nlines, const C2<T>* __restrict__ tw, G grp = G()) {
  if constexpr (kRadix16<T>) {
    if (lgr == 4) { fft_stage<T, 16, 4, DIR>(in, out, lgL, lgp, nlines, tw, grp); return; }
  }
  if (lgr == 3) fft_stage<T, 8, 3, DIR>(in, out, lgL, lgp, nlines, tw, grp);
  else if (lgr == 2) fft_stage<T, 4, 2, DIR>(in, out, lgL, lgp, nlines, tw, grp);
  else fft_stage<T, 2, 1, DIR>(in, out, lgL, lgp, nlines, tw, grp);
}

// Stages `first` .. m-1 of the FFT of nlines lines of length 2^lgL held in shared buffer `a`
// (`b` is the second buffer of the autosort); returns the buffer that holds the result.  With
// first = 1 the caller has done stage 0 itself (fft_first_io).  Must be called by all NT
// threads of the CTA (it synchronises).
template <typename T, int DIR, class G = Cta>
__device__ __noinline__ C2<T>* fft_lines_from(C2<T>* a, C2<T>* b, int lgL, int nlines,
                                              const C2<T>* __restrict__ tw, int first, G grp = G()) {
  int lgp = 0;
  int rem = lgL;
  int off = 0;                       // block of the current stage in the stage-ordered table
  C2<T>* in = a;
  C2<T>* out = b;
  for (int stage = 0; rem > 0; ++stage) {
    int l;
    if (kRadix16<T> && rem >= 4 && rem != 5) l = 4;
    else if (rem >= 3) l = 3;
    else l = rem;
    if (stage >= first) {
      fft_stage_any<T, DIR>(l, in, out, lgL, lgp, nlines, tw + off, grp);
      C2<T>* t = in; in = out; out = t;
    }
    off += ((1 << l) - 1) << lgp;
    lgp += l;
    rem -= l;
  }
  return in;
}
// FFT of nlines lines of length 2^lgL held in shared buffer `a`, using `b` as the second
// buffer of the autosort; returns the buffer that holds the result (a or b).  Must be called
// by all NT threads of the CTA (it synchronises).
template <typename T, int DIR, class G = Cta>
__device__ __forceinline__ C2<T>* fft_lines(C2<T>* a, C2<T>* b, int lgL, int nlines,
                                            const C2<T>* __restrict__ tw, G grp = G()) {
  return fft_lines_from<T, DIR>(a, b, lgL, nlines, tw, 0, grp);
}

// ------------------------------------------------------------------------------------------
// Transform with fused global I/O and a fused spectral multiplier.
//
// Forward plan: radices r_0 .. r_{m-1} (the same rule as fft_lines), inverse plan: the reverse
// order.  The forward last stage (p = L / r_{m-1}) leaves every butterfly's outputs at the
// natural positions i + j L/r, which are exactly the inputs of the inverse first stage (p = 1,
// same radix).  So one pass does: forward last stage, multiplier, inverse first stage, all in
// registers.  The first forward stage reads global memory and the last inverse stage writes
// global memory directly (both in natural order, coalesced), so the round trip costs m + 1
// shared-memory exchanges instead of 2m + 3.
// ------------------------------------------------------------------------------------------
// The plan is packed into one integer (4 bits per stage) so that it stays in registers when a
// stage is selected by a run-time index.
struct FftPlan {
  int m;
  unsigned packed;
  __device__ __forceinline__ int lgr(int s) const { return (int)((packed >> (4 * s)) & 15u); }
};
template <typename T>
__device__ __forceinline__ FftPlan fft_plan(int lgL) {
  FftPlan P;
  P.m = 0;
  P.packed = 0;
  int rem = lgL;
  while (rem > 0) {
    int l;
    if (kRadix16<T> && rem >= 4 && rem != 5) l = 4;
    else if (rem >= 3) l = 3;
    else l = rem;
    P.packed |= (unsigned)l << (4 * P.m);
    ++P.m;
    rem -= l;
  }
  return P;
}

// First stage of a transform (p = 1, no twiddles) reading its input through ld(line, pos) (global
// memory) and writing shared buffer `out`.
template <typename T, int R, int LGR, int DIR, class Ld, class G = Cta>
__device__ __forceinline__ void fft_first_io(int lgL, int nlines, Ld ld, C2<T>* out_p, G grp = G()) {
  C2<T>* const S = dsm<T>();
  const int out = dsm_off(out_p);
  const int lgq = lgL - LGR;
  const int q = 1 << lgq;
  const int nb = nlines << lgq;
  for (int b = grp.tid(); b < nb; b += G::nt) {
    const int line = b >> lgq, i = b & (q - 1);
    C2<T> v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = ld(line, i + (j << lgq));
    dft<T, R, DIR>(v);
    const int a0 = out + sp((line << lgL) + (i << LGR));     // a multiple of R: one padding group
#pragma unroll
    for (int j = 0; j < R; ++j) S[a0 + j] = v[j];
  }
  grp.sync();
}
// Last stage of a transform reading shared buffer `in` and writing through st(line, pos, v)
// (global memory).
template <typename T, int R, int LGR, int DIR, class St, class G = Cta>
__device__ __forceinline__ void fft_last_io(const C2<T>* in_p, int lgL, int lgp, int nlines,
                                            const C2<T>* __restrict__ tw, St st, G grp = G()) {
  C2<T>* const S = dsm<T>();
  const int in = dsm_off(in_p);
  const int lgq = lgL - LGR;
  const int q = 1 << lgq;
  const int p = 1 << lgp;
  const int nb = nlines << lgq;
  const int qs = q + (q >> 4);
  for (int b = grp.tid(); b < nb; b += G::nt) {
    const int line = b >> lgq, i = b & (q - 1);
    const int k = i & (p - 1);
    const int src = (line << lgL) + i;
    C2<T> v[R];
    if (lgq >= 4) {
      const int a0 = in + sp(src);
#pragma unroll
      for (int j = 0; j < R; ++j) v[j] = S[a0 + j * qs];
    } else {
#pragma unroll
      for (int j = 0; j < R; ++j) v[j] = S[in + sp(src + (j << lgq))];
    }
    if (lgp > 0) {
      C2<T> wb[LGR];
      twiddle_base<T, R, DIR>(tw + k, p, wb);
      twiddle_apply<T, R>(wb, v);
    }
    dft<T, R, DIR>(v);
    const int dpos = ((i - k) << LGR) + k;
#pragma unroll
    for (int j = 0; j < R; ++j) st(line, dpos + (j << lgp), v[j]);
  }
  grp.sync();
}

template <typename T, int DIR, class Ld, class G = Cta>
__device__ __forceinline__ void fft_first_io_any(int lgr, int lgL, int nlines, Ld ld, C2<T>* out, G grp = G()) {
  if constexpr (kRadix16<T>) {
    if (lgr == 4) { fft_first_io<T, 16, 4, DIR>(lgL, nlines, ld, out, grp); return; }
  }
  if (lgr == 3) fft_first_io<T, 8, 3, DIR>(lgL, nlines, ld, out, grp);
  else if (lgr == 2) fft_first_io<T, 4, 2, DIR>(lgL, nlines, ld, out, grp);
  else fft_first_io<T, 2, 1, DIR>(lgL, nlines, ld, out, grp);
}
template <typename T, int DIR, class St, class G = Cta>
__device__ __forceinline__ void fft_last_io_any(int lgr, const C2<T>* in, int lgL, int lgp, int nlines,
                                                const C2<T>* __restrict__ tw, St st, G grp = G()) {
  if constexpr (kRadix16<T>) {
    if (lgr == 4) { fft_last_io<T, 16, 4, DIR>(in, lgL, lgp, nlines, tw, st, grp); return; }
  }
  if (lgr == 3) fft_last_io<T, 8, 3, DIR>(in, lgL, lgp, nlines, tw, st, grp);
  else if (lgr == 2) fft_last_io<T, 4, 2, DIR>(in, lgL, lgp, nlines, tw, st, grp);
  else fft_last_io<T, 2, 1, DIR>(in, lgL, lgp, nlines, tw, st, grp);
}

// the fused middle pass: forward last stage (radix R) on NFI input fields, mul(l, pos, x[], y[])
// per position, inverse first stage on NFO output fields.  Shared line f * nl + l holds field
// f of line group l.
template <typename T, int R, int LGR, int NFI, int NFO, class Mul, class G = Cta>
__device__ __forceinline__ void fft_middle(const C2<T>* in_p, C2<T>* out_p, int lgL, int nl,
                                           const C2<T>* __restrict__ tw, Mul mul, G grp = G()) {
  C2<T>* const S = dsm<T>();
  const int in = dsm_off(in_p), out = dsm_off(out_p);
  const int lgq = lgL - LGR;
  const int q = 1 << lgq;
  const int nb = nl << lgq;
  const int qs = q + (q >> 4);
  for (int b = grp.tid(); b < nb; b += G::nt) {
    const int l = b >> lgq, i = b & (q - 1);
    C2<T> x[NFI][R];
    // twiddles of the last forward stage (p = q, k = i), from its block of the table
    C2<T> wb[LGR];
    twiddle_base<T, R, -1>(tw + i, q, wb);
#pragma unroll
    for (int f = 0; f < NFI; ++f) {
      const int base = ((f * nl + l) << lgL) + i;
      if (lgq >= 4) {
        const int a0 = in + sp(base);
#pragma unroll
        for (int j = 0; j < R; ++j) x[f][j] = S[a0 + j * qs];
      } else {
#pragma unroll
        for (int j = 0; j < R; ++j) x[f][j] = S[in + sp(base + (j << lgq))];
      }
      twiddle_apply<T, R>(wb, x[f]);
      dft<T, R, -1>(x[f]);
    }
    C2<T> y[NFO][R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      C2<T> xi[NFI], yo[NFO];
#pragma unroll
      for (int f = 0; f < NFI; ++f) xi[f] = x[f][j];
      mul(l, i + (j << lgq), xi, yo);
#pragma unroll
      for (int g = 0; g < NFO; ++g) y[g][j] = yo[g];
    }
#pragma unroll
    for (int g = 0; g < NFO; ++g) {
      dft<T, R, +1>(y[g]);
      const int a0 = out + sp(((g * nl + l) << lgL) + (i << LGR));   // a multiple of R
#pragma unroll
      for (int j = 0; j < R; ++j) S[a0 + j] = y[g][j];
    }
  }
  grp.sync();
}

template <typename T, int NFI, int NFO, class Mul, class G = Cta>
__device__ __forceinline__ void fft_middle_any(int lgr, const C2<T>* in, C2<T>* out, int lgL, int nl,
                                               const C2<T>* __restrict__ tw, Mul mul, G grp = G()) {
  if constexpr (kRadix16<T>) {
    if (lgr == 4) { fft_middle<T, 16, 4, NFI, NFO>(in, out, lgL, nl, tw, mul, grp); return; }
  }
  if (lgr == 3) fft_middle<T, 8, 3, NFI, NFO>(in, out, lgL, nl, tw, mul, grp);
  else if (lgr == 2) fft_middle<T, 4, 2, NFI, NFO>(in, out, lgL, nl, tw, mul, grp);
  else fft_middle<T, 2, 1, NFI, NFO>(in, out, lgL, nl, tw, mul, grp);
}

// Round trip F^-1[M F(.)] of NFI -> NFO fields on nl line groups:
// gsrc(f, l) / gdst(g, l) give the first element of field f / g of group l (contiguous lines,
// global or shared memory); after_first() runs (in every thread) once the first stage has
// consumed the source.  Needs a plan of at least two stages.
template <typename T, int NFI, int NFO, class Src, class Dst, class Mul, class AfterFirst, class G = Cta>
__device__ void fft_round_trip(C2<T>* sa, C2<T>* sb, int lgL, int nl, const C2<T>* __restrict__ tw,
                               Src gsrc, Dst gdst, Mul mul, AfterFirst after_first, G grp = G()) {
  const FftPlan P = fft_plan<T>(lgL);
  const int m = P.m;
  // blocks of the stage-ordered tables: table A (plan order) starts at 0, table B (reversed
  // plan) right after A; both offsets advance as the stages run
  int lenA = 0;
  {
    int lgp = 0;
    for (int s = 0; s < m; ++s) { lenA += ((1 << P.lgr(s)) - 1) << lgp; lgp += P.lgr(s); }
  }
  int offA = 0;
  int lgp = 0;
  // forward stage 0: source -> sa
  const int l0 = P.lgr(0);
  fft_first_io_any<T, -1>(l0, lgL, NFI * nl,
      [=](int line, int pos) { const int f = line / nl; return lds_c2(gsrc(f, line - f * nl) + pos); }, sa, grp);
  after_first();                     // the source of the first stage is no longer needed
  offA += ((1 << l0) - 1) << lgp;
  lgp += l0;
  C2<T>* cur = sa;
  C2<T>* oth = sb;
  for (int s = 1; s < m - 1; ++s) {
    const int lgr = P.lgr(s);
    fft_stage_any<T, -1>(lgr, cur, oth, lgL, lgp, NFI * nl, tw + offA, grp);
    offA += ((1 << lgr) - 1) << lgp;
    lgp += lgr;
    C2<T>* tt = cur; cur = oth; oth = tt;
  }
  // forward last stage + multiplier + inverse first stage (p = 1: no twiddles)
  const int lm = P.lgr(m - 1);
  fft_middle_any<T, NFI, NFO>(lm, cur, oth, lgL, nl, tw + offA, mul, grp);
  { C2<T>* tt = cur; cur = oth; oth = tt; }
  int offB = lenA + ((1 << lm) - 1);  // table B block of the inverse stage after the fused one
  int lgpi = lm;
  for (int s = m - 2; s >= 1; --s) {
    const int lgr = P.lgr(s);
    fft_stage_any<T, +1>(lgr, cur, oth, lgL, lgpi, NFO * nl, tw + offB, grp);
    offB += ((1 << lgr) - 1) << lgpi;
    lgpi += lgr;
    C2<T>* tt = cur; cur = oth; oth = tt;
  }
  // inverse last stage: shared -> destination
  fft_last_io_any<T, +1>(l0, cur, lgL, lgpi, NFO * nl, tw + offB,
      [=](int line, int pos, C2<T> v) { const int g = line / nl; gdst(g, line - g * nl)[pos] = v; }, grp);
}

}  // namespace mf
