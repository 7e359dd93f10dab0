// Thin-film (2D) right-hand side and BS23 integrator: the device code of the persistent kernels.
//
// Method: Section 2 of Prigozhin & Sokolovsky (arXiv:1801.04869).  One right-hand side
// f(t, g) runs, as phases separated by grid barriers:
//   P1  x pass of the stage input g_s = y + h sum a_j k_j           -> Sa
//   P2  y pass: smoothed gradient  i k_{x,y} G                         (Section 2.2)
//   P3  x pass: j = (g_y, -g_x) (Eq. 2), e = rho(|j|) j (Eq. 3), forward x pass of e -> Sb
//   P4  y pass: -curl e = -i G (k_x e_y - k_y e_x)                     (Eq. 4 / Eq. 9)
//   P5  x pass: h_dot_in on the conductor, warm h_dot on free space, sum for A (Eq. 10)
//   loop (Eqs. 11-12):
//   P6  y pass: 2/|k|
//   P7  x pass: g_dot = raw - A q1 - C, residual sum over free space of |g_dot| (the stop
//       test of Section 2.3), forward of mask_out g_dot
//   P9  y pass: lambda (|k|/2) G (only when the stop test did not end the loop)
//   P10 x pass: h_dot_out <- h_dot_out - A - w, sums for the next A and C, forward
//   end: g_dot on the conductor, 0 on free space (FP64)
// The shift A (Eq. 10) is applied lazily through q1 = F^-1[K1 F(out)] (exact by linearity).
// The centring constant C (Eq. 11), the mean over free space of raw - A q1, is known before
// the x pass that forms g_dot: K1 is real and even, so sum_out F^-1[K1 F h] = <q1, h>, and
// C = (<q1, h> - A sum_out q1) / n_out with <q1, h> summed where h is written (P5, P10).
#pragma once
#include "mf_rhs_common.cuh"

namespace mf {

enum Op2 { OP_GRAD = 0, OP_CURLNEG = 1, OP_K1 = 2, OP_K2 = 3, OP_KH = 4, OP_ID = 5 };

// raw pointers and sizes the x-pass epilogues need, held by value (registers)
template <typename T>
struct FilmPtrs {
  const uint8_t* mask;
  const T* jcmap;
  T* hd;
  T* u;
  const T* q1;
  const T* q2;
  int nx;
};

template <typename T>
struct Film {
  const Desc& d;
  C2<T>* sm;         // shared buffer A (BATCH values)
  C2<T>* sm2;        // shared buffer B
  Shared& sh;
  int nx, ny, lgx, lgy, half, nkx;
  long long nspec, ncell;
  C2<T>* Sa;
  C2<T>* Sb;
  T* hd;
  T* u;
  const T* q1;
  const T* q2;
  const uint8_t* mask;
  const T* jcmap;
  const C2<T>* twx;
  const C2<T>* twy;
  const T* ktab;     // kx values (half entries), then ky values (ny entries)
  const T* gtab;     // Gaussian factors, same layout
  int rb1, rb2;      // rows per item for one- and two-field row passes
  int vb;            // this CTA's index among the CTAs that run this film
  unsigned nblocks;  // how many CTAs run this film

  __device__ Film(const Desc& dd, C2<T>* s, Shared& shr, int vblock, unsigned nblk)
      : d(dd), sm(s), sm2(s + BATCH_PAD), sh(shr) {
    nx = d.nx; ny = d.ny; lgx = d.lgx; lgy = d.lgy; half = nx / 2; nkx = half + 1;
    nspec = (long long)nkx * ny;
    ncell = (long long)nx * ny;
    Sa = (C2<T>*)d.Sa; Sb = (C2<T>*)d.Sb;
    hd = (T*)d.hd; u = (T*)d.u; q1 = (const T*)d.q1; q2 = (const T*)d.q2;
    mask = d.mask; jcmap = (const T*)d.jcmap;
    twx = (const C2<T>*)d.tw_x;                 // stage-ordered twiddle tables (read-only)
    twy = (const C2<T>*)d.tw_y;
    ktab = (const T*)d.ktab;
    gtab = (const T*)d.gtab;
    rb1 = d.rows_per_item;
    rb2 = d.zs_per_item;
    vb = vblock;
    nblocks = nblk;
  }

  __device__ bool sync(int where) { return grid_sync(d.gb, nblocks, where, &sh.bar_passed, d.barrier_ns); }

  __device__ FilmPtrs<T> ptrs() const { return FilmPtrs<T>{mask, jcmap, hd, u, q1, q2, nx}; }

  // ---- y pass: forward, multiplier, inverse on nl consecutive x-wavenumber lines ----
  // shared line f * nl + l holds field f of line kx0 + l
  __device__ __noinline__ void col_item(int kx0, int nl, const C2<T>* Sin, int nin, C2<T>* Sout, int nout, int op) {
    if (fft_plan<T>(lgy).m >= 2) {
      // fused round trip: global -> first stage, multiplier between the forward last and the
      // inverse first stage, last stage -> global.  Everything the lambdas use is a copy held
      // in registers.
      const long long nspec = this->nspec;
      const int ny = this->ny, nkx = this->nkx, half = this->half;
      const T* const ktab = this->ktab;
      const T* const gtab = this->gtab;
      const T lam = (T)d.lam;
      auto src = [=](int f, int l) { return Sin + f * nspec + (long long)(kx0 + l) * ny; };
      auto dst = [=](int g, int l) { return Sout + g * nspec + (long long)(kx0 + l) * ny; };
      const T s = (T)1 / (T)ncell;
      // single precision: k_y = pi m / L_y (m in FFT order) and its Gaussian factor are
      // computed from the index (a few ulp from the tables); double precision reads the tables
      const T ky_scale = (T)(PI_D / d.Ly), g_half = (T)(0.5 * d.sigma * d.sigma);
      auto coef = [=](int l, int ky, T& kxo, T& kyo, T& k2, T& G) {
        const int kx = kx0 + l;
        const T kxv = ldg_tab(&ktab[kx]);
        T kyv, gy;
        if constexpr (sizeof(T) == 4) {
          kyv = (T)(ky < ny / 2 ? ky : ky - ny) * ky_scale;
          gy = __expf(-kyv * kyv * g_half);
        } else {
          kyv = ldg_tab(&ktab[nkx + ky]);
          gy = ldg_tab(&gtab[nkx + ky]);
        }
        kxo = (kx == half) ? (T)0 : kxv;
        kyo = (ky == ny / 2) ? (T)0 : kyv;
        k2 = kxv * kxv + kyv * kyv;
        G = ldg_tab(&gtab[kx]) * gy;
      };
      if (op == OP_GRAD) {
        fft_round_trip<T, 1, 2>(sm, sm2, lgy, nl, twy, src, dst,
            [=](int l, int ky, const C2<T>* x, C2<T>* y) {
              T kxo, kyo, k2, G; coef(l, ky, kxo, kyo, k2, G);
              y[0] = cmul_si(cscale(x[0], kxo * G * s), 1);
              y[1] = cmul_si(cscale(x[0], kyo * G * s), 1);
            }, [] {});
      } else if (op == OP_CURLNEG) {
        fft_round_trip<T, 2, 1>(sm, sm2, lgy, nl, twy, src, dst,
            [=](int l, int ky, const C2<T>* x, C2<T>* y) {
              T kxo, kyo, k2, G; coef(l, ky, kxo, kyo, k2, G);
              // -(i kx G e_y - i ky G e_x) = i G (ky e_x - kx e_y)
              const C2<T> c = {kyo * x[0].x - kxo * x[1].x, kyo * x[0].y - kxo * x[1].y};
              y[0] = cmul_si(cscale(c, G * s), 1);
            }, [] {});
      } else {
        fft_round_trip<T, 1, 1>(sm, sm2, lgy, nl, twy, src, dst,
            [=](int l, int ky, const C2<T>* x, C2<T>* y) {
              T kxo, kyo, k2, G; coef(l, ky, kxo, kyo, k2, G);
              // |k| and 1/|k| from one reciprocal square root in single precision (a few ulp,
              // far below the FP32 transform error); correctly rounded sqrt and divide in double
              T kabs, kinv;
              if constexpr (sizeof(T) == 4) {
                kinv = k2 > (T)0 ? rsqrtf(k2) : (T)0;
                kabs = k2 * kinv;
              } else {
                kabs = sqrt(k2);
                kinv = k2 > (T)0 ? (T)1 / kabs : (T)0;
              }
              T m;
              if (op == OP_K1) m = (T)2 * kinv;
              else if (op == OP_K2) m = lam * kabs * (T)0.5 * G;
              else if (op == OP_KH) m = kabs * (T)0.5;
              else m = (T)1;
              y[0] = cscale(x[0], m * s);
            }, [] {});
      }
      return;
    }
    gather_batched<T, 4>(sm, Sin, (nin * nl) << lgy,
        [=](int e) {
          const int j = e >> lgy, f = j / nl, l = j - f * nl;
          return f * nspec + (long long)(kx0 + l) * ny + (e & (ny - 1));
        },
        [](int e) { return e; });
    C2<T>* X = fft_lines<T, -1>(sm, sm2, lgy, nin * nl, twy);
    C2<T>* Y = X == sm ? sm2 : sm;
    const T s = (T)1 / (T)ncell;
    for (int e = threadIdx.x; e < (nl << lgy); e += NT) {
      const int l = e >> lgy, ky = e & (ny - 1);
      const int kx = kx0 + l;
      const T kxv = ldg_tab(&ktab[kx]), gx = ldg_tab(&gtab[kx]);
      const T kxo = (kx == half) ? (T)0 : kxv;
      const T kyv = ldg_tab(&ktab[nkx + ky]), G = gx * ldg_tab(&gtab[nkx + ky]);
      const T kyo = (ky == ny / 2) ? (T)0 : kyv;
      const T k2 = kxv * kxv + kyv * kyv;
      const int i0 = (0 * nl + l) * ny + ky, i1 = (1 * nl + l) * ny + ky;
      C2<T> a = X[sp(i0)];
      if (op == OP_GRAD) {
        const T fx = kxo * G * s, fy = kyo * G * s;
        X[sp(i0)] = cmul_si(cscale(a, fx), 1);
        X[sp(i1)] = cmul_si(cscale(a, fy), 1);
      } else if (op == OP_CURLNEG) {
        const C2<T> b = X[sp(i1)];
        // -(i kx G e_y - i ky G e_x) = i G (ky e_x - kx e_y)
        C2<T> c = {kyo * a.x - kxo * b.x, kyo * a.y - kxo * b.y};
        X[sp(i0)] = cmul_si(cscale(c, G * s), 1);
      } else {
        T m;
        const T kabs = sqrt(k2);
        if (op == OP_K1) m = (k2 > (T)0) ? (T)2 / kabs : (T)0;
        else if (op == OP_K2) m = (T)d.lam * kabs * (T)0.5 * G;
        else if (op == OP_KH) m = kabs * (T)0.5;
        else m = (T)1;
        X[sp(i0)] = cscale(a, m * s);
      }
    }
    __syncthreads();
    const C2<T>* Z = fft_lines<T, +1>(X, Y, lgy, nout * nl, twy);
    for (int e = threadIdx.x; e < ((nout * nl) << lgy); e += NT) {
      const int j = e >> lgy, f = j / nl, l = j - f * nl;
      Sout[f * nspec + (long long)(kx0 + l) * ny + (e & (ny - 1))] = Z[sp(e)];
    }
    __syncthreads();
  }

  // ---- y pass of one line kx with a one-field multiplier, by half of the CTA (group g, its
  // own line region of both shared buffers and its own named barrier) ----
  __device__ __noinline__ void col_line_half(int kx, const C2<T>* Sin, C2<T>* Sout, int op, int g) {
    const int ny = this->ny, half = this->half;
    const T* const ktab = this->ktab;
    const T* const gtab = this->gtab;
    const T lam = (T)d.lam;
    const C2<T>* const src0 = Sin + (long long)kx * ny;
    C2<T>* const dst0 = Sout + (long long)kx * ny;
    auto src = [=](int, int) { return src0; };
    auto dst = [=](int, int) { return dst0; };
    const T s = (T)1 / (T)ncell;
    const T ky_scale = (T)(PI_D / d.Ly), g_half = (T)(0.5 * d.sigma * d.sigma);
    const T kxv = ldg_tab(&ktab[kx]), gx = ldg_tab(&gtab[kx]);
    const int nkx = this->nkx;
    (void)half;
    fft_round_trip<T, 1, 1>(sm + sp(g << lgy), sm2 + sp(g << lgy), lgy, 1, twy, src, dst,
        [=](int, int ky, const C2<T>* x, C2<T>* y) {
          T kyv, gy;
          if constexpr (sizeof(T) == 4) {
            kyv = (T)(ky < ny / 2 ? ky : ky - ny) * ky_scale;
            gy = __expf(-kyv * kyv * g_half);
          } else {
            kyv = ldg_tab(&ktab[nkx + ky]);
            gy = ldg_tab(&gtab[nkx + ky]);
          }
          const T k2 = kxv * kxv + kyv * kyv;
          T kabs, kinv;
          if constexpr (sizeof(T) == 4) {
            kinv = k2 > (T)0 ? rsqrtf(k2) : (T)0;
            kabs = k2 * kinv;
          } else {
            kabs = sqrt(k2);
            kinv = k2 > (T)0 ? (T)1 / kabs : (T)0;
          }
          T m;
          if (op == OP_K1) m = (T)2 * kinv;
          else if (op == OP_K2) m = lam * kabs * (T)0.5 * (gx * gy);
          else if (op == OP_KH) m = kabs * (T)0.5;
          else m = (T)1;
          y[0] = cscale(x[0], m * s);
        }, [] {}, HalfCta{g});
  }

  // lines per column item: fill the shared batch (two lines for single-field operators)
  __device__ int col_lines(int nf) const {
    int nl = BATCH / (nf * ny);
    return nl < 1 ? 1 : (nl > 2 ? 2 : nl);
  }

  __device__ void cols(const C2<T>* Sin, int nin, C2<T>* Sout, int nout, int op) {
    const int nl = col_lines(nin > nout ? nin : nout);
    const int nitems = (nkx + nl - 1) / nl;
    if (nin == 1 && nout == 1 && nl == 2 && fft_plan<T>(lgy).m >= 2) {
      // one line per half of the CTA: the halves run their transforms independently
      const int g = (int)threadIdx.x / (NT / 2);
      for (int it = vb; it < nitems; it += (int)nblocks) {
        const int kx = it * 2 + g;
        if (kx < nkx) col_line_half(kx, Sin, Sout, op, g);
      }
      return;
    }
    for (int it = vb; it < nitems; it += (int)nblocks) {
      const int kx0 = it * nl;
      col_item(kx0, kx0 + nl <= nkx ? nl : nkx - kx0, Sin, nin, Sout, nout, op);
    }
  }

  // ---- x pass over rows [y0, y0 + rb): inverse of NIN fields, epilogue, forward of NOUT ----
  // epi(row, x, in[], out[]) is called for every cell of the item.
  template <int NIN, int NOUT, class Epi>
  __device__ __forceinline__ void row_item(int y0, int rb, const C2<T>* Sin, C2<T>* Sout, Epi& epi_io) {
    // inlined into the pass loop (a call per item cost a save and restore of the caller's live
    // registers); works on register copies of the epilogue and of the members used in the loops
    Epi epi = epi_io;
    C2<T>* const smA = sm;
    C2<T>* const smB = sm2;
    const int nx = this->nx, lgx = this->lgx, ny = this->ny;
    const long long nspec = this->nspec;
    const C2<T>* const twx = this->twx;
    const int npair = rb / 2;
    C2<T>* X = smA;
    const int lgpair = __ffs(npair) - 1;
    if constexpr (NIN > 0) X = rows_gather_inverse<T, NIN>(smA, smB, Sin + y0, nspec, ny, npair, lgpair, lgx, twx);
    C2<T>* Y = X == smA ? smB : smA;
    C2<T>* const S = dsm<T>();
    const int ix = dsm_off(X);
    // four consecutive cells of both rows of a pair per step; the epilogue issues its global
    // loads for the four cells together (x0 is a multiple of 4: one padding group)
    const int lgq = lgx - 2;
#pragma unroll 4
    for (int e = threadIdx.x; e < (npair << lgq); e += NT) {
      const int pr = e >> lgq, x0 = (e & ((1 << lgq) - 1)) << 2;
      V4<T> ina[NIN > 0 ? NIN : 1], inb[NIN > 0 ? NIN : 1], oa[NOUT > 0 ? NOUT : 1], ob[NOUT > 0 ? NOUT : 1];
#pragma unroll
      for (int f = 0; f < NIN; ++f) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const C2<T> z = S[ix + sp(((f * npair + pr) << lgx) + x0) + j];
          ina[f].v[j] = z.x; inb[f].v[j] = z.y;
        }
      }
      const long long i0 = (long long)(y0 + 2 * pr) * nx + x0;
      if constexpr (Epi::kPair) {
        epi.pair(i0, i0 + nx, ina, inb, oa, ob);
      } else {
        epi(i0, ina, oa);
        epi(i0 + nx, inb, ob);
      }
#pragma unroll
      for (int f = 0; f < NOUT; ++f) {
#pragma unroll
        for (int j = 0; j < 4; ++j) S[ix + sp(((f * npair + pr) << lgx) + x0) + j] = C2<T>{oa[f].v[j], ob[f].v[j]};
      }
    }
    __syncthreads();
    if constexpr (NOUT > 0) rows_forward_scatter<T, NOUT>(X, Y, Sout + y0, nspec, ny, npair, lgpair, lgx, twx);
    epi_io.acc = epi.acc;
    epi_io.accmax = epi.accmax;
    epi_io.acc2 = epi.acc2;
  }

  // rows pass with optional per-item reductions into partials slots `slot` (acc or accmax)
  // and `slot2` (acc2)
  template <int NIN, int NOUT, class Epi>
  __device__ void rows(int rb, const C2<T>* Sin, C2<T>* Sout, Epi& epi, int slot, int slot2 = -1) {
    const int nitems = ny / rb;
    for (int it = vb; it < nitems; it += (int)nblocks) {
      epi.acc = 0.0;
      epi.accmax = 0.0;
      epi.acc2 = 0.0;
      row_item<NIN, NOUT>(it * rb, rb, Sin, Sout, epi);
      if (slot >= 0) {
        const double v = epi.is_max ? block_max(epi.accmax, sh.red) : block_sum(epi.acc, sh.red);
        if (threadIdx.x == 0) d.partials[(size_t)slot * d.max_items + it] = v;
      }
      if (slot2 >= 0) {
        const double v = block_sum(epi.acc2, sh.red);
        if (threadIdx.x == 0) d.partials[(size_t)slot2 * d.max_items + it] = v;
      }
    }
  }
  __device__ double total(int slot, int rb, bool is_max = false) {
    return reduce_partials(d.partials, d.max_items, slot, ny / rb, is_max, sh.red);
  }
  // Eq. 10 and Eq. 11 constants from the sums of h (slot 0) and q1 h (slot 5) of the pass that
  // wrote h: A = (sum h - N h_e_dot) / n_out, C = (<q1, h> - A sum_out q1) / n_out; computed once
  // by thread 0 and broadcast (the double-precision division runs at a low rate on this part)
  __device__ void shifts(int rb, double N, double hed, double nout, double& A, double& C) {
    reduce_partials2(d.partials, d.max_items, 0, 5, ny / rb, sh.red);
    __syncthreads();
    if (threadIdx.x == 0) {
      const double a = (sh.red[0] - N * hed) / nout;
      sh.red[2] = a;
      sh.red[3] = (sh.red[1] - a * sh.q11) / nout;
    }
    __syncthreads();
    A = sh.red[2];
    C = sh.red[3];
    __syncthreads();
  }
  // mean over free space of the residual sum in slot 2 (broadcast like shifts)
  __device__ double mean_out(int slot, int rb, double nout) {
    const double s = reduce_partials(d.partials, d.max_items, slot, ny / rb, false, sh.red);
    if (threadIdx.x == 0) sh.red[2] = s / nout;
    __syncthreads();
    const double r = sh.red[2];
    __syncthreads();
    return r;
  }
};

// ------------------------------------------------------------------------------------------
// epilogues
// ------------------------------------------------------------------------------------------
// Epilogues of the x pass: called with the index i of the first of four consecutive cells of
// one row, the inverse-transformed inputs in[f].v[0..3] and outputs out[f].v[0..3].

// P1 / readouts: field from the FP64 stage input
template <typename T>
struct EpiStage : EpiBase<T> {
  FilmPtrs<T> P;
  StageIn in;
  __device__ void operator()(long long i, const V4<T>*, V4<T>* out) {
    V4<double> v = ld4(in.y + i);
    for (int j = 0; j < in.nk; ++j) {
      const V4<double> k = ld4(in.k[j] + i);
#pragma unroll
      for (int q = 0; q < 4; ++q) v.v[q] += in.c[j] * k.v[q];
    }
    if (in.ynew) st4(in.ynew + i, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[0].v[q] = (T)v.v[q];
  }
};

// mask indicator of free space (set-up of q1, q2)
template <typename T>
struct EpiOut : EpiBase<T> {
  FilmPtrs<T> P;
  __device__ void operator()(long long i, const V4<T>*, V4<T>* out) {
    const uchar4 m = ldmask4(P.mask + i);
#pragma unroll
    for (int q = 0; q < 4; ++q) out[0].v[q] = mask_at(m, q) == 0 ? (T)1 : (T)0;
  }
};

// store a real field (set-up); sum of it over free space
template <typename T>
struct EpiStoreT : EpiBase<T> {
  FilmPtrs<T> P;
  T* dst;
  __device__ void operator()(long long i, const V4<T>* in, V4<T>*) {
    st4(dst + i, in[0]);
    const uchar4 m = ldmask4(P.mask + i);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (mask_at(m, q) == 0) this->acc += (double)in[0].v[q];
  }
};
// h_z readout (FP64)
template <typename T>
struct EpiStoreHz : EpiBase<T> {
  FilmPtrs<T> P;
  double* dst;
  double he;
  __device__ void operator()(long long i, const V4<T>* in, V4<T>*) {
    V4<double> o;
#pragma unroll
    for (int q = 0; q < 4; ++q) o.v[q] = he + (double)in[0].v[q];
    st4(dst + i, o);
  }
};

// P3: power law.  ig2 = 1/gamma^2 of the elliptic law e = rho(j_eff) (j_x, j_y/gamma^2),
// j_eff^2 = j_x^2 + j_y^2/gamma^2 in the superconductor (Eq. 3 at gamma = 1, where the extra
// products by 1 are exact)
template <typename T>
struct EpiPower : EpiBase<T> {
  FilmPtrs<T> P;
  T n, e0, jc, rho_out, ig2;
  __device__ void operator()(long long i, const V4<T>* in, V4<T>* out) {
    const uchar4 m = ldmask4(P.mask + i);
    V4<T> jcl;
    if (P.jcmap) jcl = ldg4(P.jcmap + i);
    else jcl = V4<T>{{jc, jc, jc, jc}};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T gx = in[0].v[q], gy = in[1].v[q];
      const T jx = gy, jy = -gx;                              // Eq. 2
      const int mq = mask_at(m, q);
      const T a = mq == 1 ? ig2 : (T)1;
      const T rho = resistivity<T>(jx * jx + jy * jy * a, jcl.v[q], mq, n, e0, rho_out);
      out[0].v[q] = rho * jx;                                 // Eq. 3
      out[1].v[q] = rho * jy * a;
    }
  }
};

// P5: initial h_dot (warm start), sum over D
template <typename T>
struct EpiInit : EpiBase<T, T> {
  FilmPtrs<T> P;
  bool warm;
  const T* wsrc;          // warm start (the previous time step's or the most recent iterate)
  T A_prev, hed;
  struct Ld { uchar4 m; V4<T> w, q1; };
  __device__ __forceinline__ Ld load(long long i) const {
    Ld l;
    l.m = ldmask4(P.mask + i);
    if (warm) l.w = ld4(wsrc + i);
    l.q1 = ldg4(P.q1 + i);
    return l;
  }
  __device__ __forceinline__ V4<T> apply(const Ld& l, const V4<T>* in) {
    V4<T> h;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (mask_at(l.m, q) != 0) h.v[q] = in[0].v[q];           // h_dot_in on the conductor
      else h.v[q] = warm ? l.w.v[q] - A_prev : hed;           // warm start (Section 2.2)
      this->acc += h.v[q];
      this->acc2 += l.q1.v[q] * h.v[q];                       // <q1, h> for C
    }
    return h;
  }
  __device__ void operator()(long long i, const V4<T>* in, V4<T>* out) {
    const V4<T> h = apply(load(i), in);
    st4(P.hd + i, h);
    out[0] = h;
  }
  static constexpr bool kPair = true;
  __device__ __forceinline__ void pair(long long ia, long long ib, const V4<T>* ina, const V4<T>* inb,
                                       V4<T>* oa, V4<T>* ob) {
    const Ld la = load(ia), lb = load(ib);
    oa[0] = apply(la, ina);
    ob[0] = apply(lb, inb);
    st4(P.hd + ia, oa[0]);
    st4(P.hd + ib, ob[0]);
  }
};

// P7: g_dot = raw - A q1 - C (Eq. 11), stored; residual sum over free space of |g_dot|
// (Section 2.3); forward of mask_out g_dot (the input of Eq. 12)
template <typename T>
struct EpiU : EpiBase<T, T> {
  FilmPtrs<T> P;
  T A, C;
  __device__ void operator()(long long i, const V4<T>* in, V4<T>* out) {
    const uchar4 m = ldmask4(P.mask + i);
    const V4<T> q1 = ldg4(P.q1 + i);
    V4<T> v;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v.v[q] = (in[0].v[q] - A * q1.v[q]) - C;
      const bool o = mask_at(m, q) == 0;
      if (o) this->acc += fabs(v.v[q]);
      out[0].v[q] = o ? v.v[q] : (T)0;
    }
    st4(P.u + i, v);
  }
};

// P10: h_dot update on free space (Eq. 12: w is the transform of mask_out g_dot), sums over D
// of h (for A) and of q1 h (for C), forward
template <typename T>
struct EpiUpdate : EpiBase<T, T> {
  FilmPtrs<T> P;
  T A;
  struct Ld { uchar4 m; V4<T> h, q1; };
  __device__ __forceinline__ Ld load(long long i) const {
    return Ld{ldmask4(P.mask + i), ld4(P.hd + i), ldg4(P.q1 + i)};
  }
  __device__ __forceinline__ V4<T> apply(Ld l, const V4<T>* in) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (mask_at(l.m, q) == 0) l.h.v[q] = (l.h.v[q] - A) - in[0].v[q];
      this->acc += l.h.v[q];
      this->acc2 += l.q1.v[q] * l.h.v[q];
    }
    return l.h;
  }
  __device__ void operator()(long long i, const V4<T>* in, V4<T>* out) {
    const V4<T> h = apply(load(i), in);
    st4(P.hd + i, h);
    out[0] = h;
  }
  static constexpr bool kPair = true;
  __device__ __forceinline__ void pair(long long ia, long long ib, const V4<T>* ina, const V4<T>* inb,
                                       V4<T>* oa, V4<T>* ob) {
    const Ld la = load(ia), lb = load(ib);
    oa[0] = apply(la, ina);
    ob[0] = apply(lb, inb);
    st4(P.hd + ia, oa[0]);
    st4(P.hd + ib, ob[0]);
  }
};

// finalize: g_dot (stored by P7) on the conductor; optional BS23 error contribution
template <typename T>
struct EpiFinal : EpiBase<T> {
  FilmPtrs<T> P;
  double* kout;
  // error estimate (stage 4 of a step): E = h (e1 k1 + e2 k2 + e3 k3 + e4 k4)
  bool err;
  double h, rtol, atol;
  const double* k1; const double* k2; const double* k3; const double* y; const double* ynew;
  __device__ void operator()(long long i, const V4<T>*, V4<T>*) {
    const uchar4 m = ldmask4(P.mask + i);
    const V4<T> u = ld4(P.u + i);
    V4<double> g;
#pragma unroll
    for (int q = 0; q < 4; ++q) g.v[q] = mask_at(m, q) != 0 ? (double)u.v[q] : 0.0;
    if (err) {
      // the loads before the store (a store could alias a later load as far as the compiler
      // knows, which would put the loads behind it)
      const V4<double> a1 = ld4(k1 + i), a2 = ld4(k2 + i), a3 = ld4(k3 + i), yy = ld4(y + i), yn = ld4(ynew + i);
      st4(kout + i, g);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double E = h * (-5.0 / 72.0 * a1.v[q] + 1.0 / 12.0 * a2.v[q] + 1.0 / 9.0 * a3.v[q] - 0.125 * g.v[q]);
        const double sc = atol + rtol * fmax(fabs(yy.v[q]), fabs(yn.v[q]));
        // E and its scale in FP64; their ratio, which only feeds the accept test and the step
        // size factor, in the transform precision (FP64 division runs at a small fraction of the
        // FP32 rate on this part)
        double r;
        if constexpr (sizeof(T) == 4) r = (double)__fdiv_rn((float)fabs(E), (float)sc);
        else r = fabs(E) / sc;
        if (!(r == r) || isinf(r)) r = 1e300;                // non-finite -> rejected step
        this->accmax = fmax(this->accmax, r);
      }
    } else {
      st4(kout + i, g);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (!isfinite(g.v[q])) this->accmax = 1.0;
    }
  }
};

// e readout (FP64, 2 fields): e = rho(|j|) j with j = (g_y, -g_x) (Eq. 2, Eq. 3), Ohm law
// rho_out j on free space and filled holes
template <typename T>
struct EpiStoreE : EpiBase<T> {
  FilmPtrs<T> P;
  T n, e0, jc, rho_out, ig2;
  double* dst;
  long long ncell;
  __device__ void operator()(long long i, const V4<T>* in, V4<T>*) {
    const uchar4 m = ldmask4(P.mask + i);
    V4<T> jcl;
    if (P.jcmap) jcl = ldg4(P.jcmap + i);
    else jcl = V4<T>{{jc, jc, jc, jc}};
    V4<double> ex, ey;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T jx = in[1].v[q], jy = -in[0].v[q];
      const int mq = mask_at(m, q);
      const T a = mq == 1 ? ig2 : (T)1;                       // elliptic law, as in EpiPower
      const T rho = resistivity<T>(jx * jx + jy * jy * a, jcl.v[q], mq, n, e0, rho_out);
      ex.v[q] = (double)(rho * jx);
      ey.v[q] = (double)(rho * jy * a);
    }
    st4(dst + i, ex);
    st4(dst + ncell + i, ey);
  }
};

// magnetization: sum over D of g (times dx dy on the host side)
template <typename T>
struct EpiMoment : EpiBase<T> {
  FilmPtrs<T> P;
  const double* g;
  __device__ void operator()(long long i, const V4<T>*, V4<T>*) {
    const V4<double> v = ld4(g + i);
    this->acc += (v.v[0] + v.v[1]) + (v.v[2] + v.v[3]);
  }
};

// ------------------------------------------------------------------------------------------
// one right-hand side.  Returns ST_OK / ST_NOCONV / ST_BARRIER (same in every CTA).
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ RhsOut film_rhs(Film<T>& F, double t, int seg, const StageIn& sin, double* kout,
                           int force_iters, bool want_err, double h_err, const double* e_k1,
                           const double* e_k2, const double* e_k3, const double* e_y,
                           const double* e_ynew) {
  const Desc& d = F.d;
  RhsOut res{ST_OK, 0, 0.0, 0.0, 0};
  const double hed = he_dot(d, t, seg);
  const double N = (double)F.ncell;
  const double nout = (double)d.nout;
  const bool first = F.sh.attempt_first != 0;   // read by every thread before it is cleared
  // h_dot buffers: this call writes hdw; hdc holds the committed (accepted-step) h_dot
  T* const hdw = (T*)(F.sh.hd_sel ? d.hd2 : d.hd);
  const T* const hdc = (const T*)(F.sh.hd_sel ? d.hd : d.hd2);

  // P1
  {
    EpiStage<T> e; e.P = F.ptrs(); e.in = sin;
    F.rows<0, 1>(F.rb1, nullptr, F.Sa, e, -1);
  }
  if (!F.sync(1)) { res.status = ST_BARRIER; return res; }
  F.cols(F.Sa, 1, F.Sa, 2, OP_GRAD);                                    // P2
  if (!F.sync(2)) { res.status = ST_BARRIER; return res; }
  {
    EpiPower<T> e; e.P = F.ptrs();
    e.n = (T)d.n; e.e0 = (T)d.e0; e.jc = (T)d.jc; e.rho_out = (T)d.rho_out;
    e.ig2 = (T)(1.0 / (d.gamma * d.gamma));
    F.rows<2, 2>(F.rb2, F.Sa, F.Sb, e, -1);                             // P3
  }
  if (!F.sync(3)) { res.status = ST_BARRIER; return res; }
  F.cols(F.Sb, 2, F.Sb, 1, OP_CURLNEG);                                 // P4
  if (!F.sync(4)) { res.status = ST_BARRIER; return res; }

  const bool have_out = d.nout > 0;
  {
    // initial approximation "from the previous time step" (Section 2.2): the first evaluation
    // of a step attempt starts from the accepted step's h_dot, later stages (and calls outside
    // the integrator) from the most recent call's iterate; the very first call from h_e_dot
    EpiInit<T> e; e.P = F.ptrs(); e.P.hd = hdw;
    const bool com = first && F.sh.com_valid != 0;
    e.warm = com || F.sh.warm_valid != 0;
    e.wsrc = com ? hdc : hdw;
    e.A_prev = (T)(com ? F.sh.A_com : F.sh.A_prev); e.hed = (T)hed;
    F.rows<1, 1>(F.rb1, F.Sb, F.Sa, e, 0, 5);                           // P5
  }
  if (!F.sync(5)) { res.status = ST_BARRIER; return res; }
  // Eq. 10: A; Eq. 11: C = (<q1, h> - A sum_out q1) / n_out (K1 is real and even)
  double A = 0.0, C = 0.0;
  if (have_out) F.shifts(F.rb1, N, hed, nout, A, C);
  double r = 0.0;
  const bool forced = force_iters > 0;
  const bool fixed = d.iter_tol <= 0.0;
  int itmax = forced ? force_iters : d.iter_max;
  if (!have_out) itmax = 1;
  int i = 0;
  for (; i < itmax; ++i) {
    F.cols(F.Sa, 1, F.Sa, 1, OP_K1);                                    // P6
    if (!F.sync(6)) { res.status = ST_BARRIER; return res; }
    {
      EpiU<T> e; e.P = F.ptrs(); e.A = (T)A; e.C = (T)C;
      F.rows<1, 1>(F.rb1, F.Sa, F.Sb, e, 2);                            // P7
    }
    if (!F.sync(7)) { res.status = ST_BARRIER; return res; }
    if (!have_out) { r = 0.0; break; }
    r = F.mean_out(2, F.rb1, nout);                                     // Section 2.3
    const bool last = (i == itmax - 1);
    const bool stop = (forced || fixed) ? last : (r < d.iter_tol || last);
    if (stop) break;
    F.cols(F.Sb, 1, F.Sb, 1, OP_K2);                                    // P9 (Eq. 12)
    if (!F.sync(8)) { res.status = ST_BARRIER; return res; }
    {
      EpiUpdate<T> e; e.P = F.ptrs(); e.P.hd = hdw; e.A = (T)A;
      F.rows<1, 1>(F.rb1, F.Sb, F.Sa, e, 0, 5);                         // P10
    }
    if (!F.sync(10)) { res.status = ST_BARRIER; return res; }
    F.shifts(F.rb1, N, hed, nout, A, C);                                // Eq. 10, Eq. 11
  }
  res.iters = i + 1;
  res.r = r;
  res.status = (!have_out || fixed || r < d.iter_tol) ? ST_OK : ST_NOCONV;
  // warm start for the next call: h_dot stored, A still to subtract on free space.  A call that
  // failed with a residual above 1e3 tol (or not finite) diverged: the next call starts cold.
  const bool diverged = res.status == ST_NOCONV && !(r < 1e3 * d.iter_tol);
  F.sh.warm_valid = diverged ? 0 : 1;
  F.sh.A_prev = A;
  F.sh.attempt_first = 0;

  // finalize
  {
    EpiFinal<T> e; e.P = F.ptrs(); e.kout = kout; e.is_max = true;
    e.err = want_err; e.h = h_err; e.rtol = d.rtol; e.atol = d.atol;
    e.k1 = e_k1; e.k2 = e_k2; e.k3 = e_k3; e.y = e_y; e.ynew = e_ynew;
    F.rows<0, 0>(F.rb1, nullptr, nullptr, e, 3);
  }
  if (!F.sync(11)) { res.status = ST_BARRIER; return res; }
  const double q = F.total(3, F.rb1, true);
  if (want_err) res.err = q;
  else res.nonfinite = q > 0.0;
  return res;
}

// adapter used by the shared BS23 integrator loop
template <typename T>
struct FilmRhs {
  Film<T>& F;
  __device__ RhsOut operator()(double t, int seg, const StageIn& in, double* kout, int force,
                               bool want_err, double h, const double* k1, const double* k2,
                               const double* k3, const double* y, const double* yn) {
    return film_rhs<T>(F, t, seg, in, kout, force, want_err, h, k1, k2, k3, y, yn);
  }
  // the integrator accepted a step: the last call's h_dot (written to hd_sel) becomes the
  // committed initial approximation, and later calls write the other buffer
  __device__ void on_attempt() {
    __syncthreads();
    if (threadIdx.x == 0) F.sh.attempt_first = 1;
    __syncthreads();
  }
  __device__ void on_accept() {
    __syncthreads();
    const int sel = F.sh.hd_sel;
    const double A = F.sh.A_prev;
    __syncthreads();
    if (threadIdx.x == 0) { F.sh.com_valid = 1; F.sh.A_com = A; F.sh.hd_sel = sel ^ 1; }
    __syncthreads();
  }
};

// ------------------------------------------------------------------------------------------
// the persistent kernel
// ------------------------------------------------------------------------------------------
// The body of a launch for one film, run by CTAs vb = 0 .. vn - 1 of that film.
template <typename T>
__device__ __forceinline__ void film_main(const Desc& d, const KernelArgs& a, int vb, unsigned vn) {
  C2<T>* sm = dsm<T>();
  __shared__ Shared sh;
  // one copy of the pass object per CTA, in shared memory: its members are read as broadcasts
  // instead of per-thread local-memory copies
  __shared__ __align__(16) unsigned char objraw[sizeof(Film<T>)];
  SolverState* st = d.st;
  if (threadIdx.x == 0) {
    sh.warm_valid = st->warm_valid;
    sh.bar_passed = 0;
    sh.A_prev = st->A_prev;
    sh.com_valid = st->com_valid;
    sh.hd_sel = st->hd_sel;
    sh.A_com = st->A_com;
    sh.attempt_first = 0;
    sh.q11 = st->q11;
  }
  if (threadIdx.x == 0) new (objraw) Film<T>(d, sm, sh, vb, vn);
  __syncthreads();
  Film<T>& F = *reinterpret_cast<Film<T>*>(objraw);
  const bool leader = vb == 0 && threadIdx.x == 0;
  int status = ST_OK;

  if (a.mode == MODE_SETUP) {
    // q1 = F^-1[K1 F(out)], q2 = F^-1[K2 F(out)]
    for (int pass = 0; pass < 2; ++pass) {
      EpiOut<T> eo; eo.P = F.ptrs();
      F.rows<0, 1>(F.rb1, nullptr, F.Sa, eo, -1);
      if (!F.sync(20)) { status = ST_BARRIER; break; }
      F.cols(F.Sa, 1, F.Sa, 1, pass == 0 ? OP_K1 : OP_K2);
      if (!F.sync(21)) { status = ST_BARRIER; break; }
      EpiStoreT<T> es; es.P = F.ptrs(); es.dst = (T*)(pass == 0 ? d.q1 : d.q2);
      F.rows<1, 0>(F.rb1, F.Sa, nullptr, es, 4);
      if (!F.sync(22)) { status = ST_BARRIER; break; }
      if (pass == 0) {
        const double q11 = F.total(4, F.rb1);          // sum over free space of q1
        if (leader) st->q11 = q11;
      }
    }
  } else if (a.mode == MODE_HZ) {
    EpiStage<T> e; e.P = F.ptrs(); e.in = StageIn{a.y_in, 0, {0, 0, 0}, {nullptr, nullptr, nullptr}, nullptr};
    F.rows<0, 1>(F.rb1, nullptr, F.Sa, e, -1);
    if (F.sync(30)) {
      F.cols(F.Sa, 1, F.Sa, 1, OP_KH);
      if (F.sync(31)) {
        EpiStoreHz<T> es; es.P = F.ptrs(); es.dst = a.out; es.he = he_value(d, a.t);
        F.rows<1, 0>(F.rb1, F.Sa, nullptr, es, -1);
      } else status = ST_BARRIER;
    } else status = ST_BARRIER;
  } else if (a.mode == MODE_E) {
    EpiStage<T> e; e.P = F.ptrs(); e.in = StageIn{a.y_in, 0, {0, 0, 0}, {nullptr, nullptr, nullptr}, nullptr};
    F.rows<0, 1>(F.rb1, nullptr, F.Sa, e, -1);
    if (F.sync(50)) {
      F.cols(F.Sa, 1, F.Sa, 2, OP_GRAD);
      if (F.sync(51)) {
        EpiStoreE<T> es; es.P = F.ptrs(); es.dst = a.out; es.ncell = F.ncell;
        es.n = (T)d.n; es.e0 = (T)d.e0; es.jc = (T)d.jc; es.rho_out = (T)d.rho_out;
        es.ig2 = (T)(1.0 / (d.gamma * d.gamma));
        F.rows<2, 0>(F.rb2, F.Sa, nullptr, es, -1);
      } else status = ST_BARRIER;
    } else status = ST_BARRIER;
  } else if (a.mode == MODE_MOMENT) {
    EpiMoment<T> e; e.P = F.ptrs(); e.g = a.y_in;
    F.rows<0, 0>(F.rb1, nullptr, nullptr, e, 4);
    if (F.sync(40)) {
      const double s = F.total(4, F.rb1);
      if (leader) a.out[0] = s * d.dx * d.dy;
    } else status = ST_BARRIER;
  } else if (a.mode == MODE_RHS) {
    StageIn in{a.y_in, 0, {0, 0, 0}, {nullptr, nullptr, nullptr}, nullptr};
    RhsOut r = film_rhs<T>(F, a.t, a.seg, in, a.out, a.force_iters, false, 0.0, nullptr, nullptr,
                           nullptr, nullptr, nullptr);
    status = r.status == ST_OK && r.nonfinite ? ST_NONFINITE : r.status;
    if (leader) { st->last_iters = r.iters; st->last_r = r.r; st->n_rhs += 1; st->n_iters += r.iters; }
  } else if (a.mode == MODE_ADVANCE) {
    FilmRhs<T> R{F};
    status = bs23_advance(R, d, st, a, leader);
  }
  if (leader) {
    st->warm_valid = sh.warm_valid;
    st->A_prev = sh.A_prev;
    st->com_valid = sh.com_valid;
    st->hd_sel = sh.hd_sel;
    st->A_com = sh.A_com;
    st->status = status;
  }
}

// the two FFT buffers (twiddles stay in global memory, read through L1)
inline size_t film_smem_bytes(int precision) {
  return 2 * (size_t)BATCH_PAD * (precision ? sizeof(C2<float>) : sizeof(C2<double>));
}

}  // namespace mf
