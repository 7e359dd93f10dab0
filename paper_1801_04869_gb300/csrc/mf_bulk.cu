// Bulk (3D) right-hand side in the magnetic-field formulation and its BS23 integrator, as one
// persistent cooperative kernel.
//
// Method: Section 3.1 of Prigozhin & Sokolovsky (arXiv:1801.04869).  The state h has three
// components (component-major).  A vector "round trip" F^-1[M F(v)] runs as five passes
// separated by grid barriers:
//   X   x pass: rows of the real field, R2C along x           -> S1[c][z][kx][y]
//   Yf  y pass: forward along y                                -> S2[c][kx][ky][z]
//   Z   z pass: forward along z, the 3x3 multiplier M, inverse along z (in place in S2)
//   Yi  y pass: inverse along y                                -> S1
//   X   x pass: C2R along x, epilogue on all three components, and the forward x pass of the
//       next round trip's input
// Multipliers: the Gaussian-smoothed curl i G k x (Section 3.1, last paragraph) and the
// Biot-Savart operator Phi = (i/|k|^2) k x (Eq. 17, 1/|k|^2 -> 0 at k = 0).
// One right-hand side (Eqs. 13-14 and the iteration of Eq. 18):
//   j = curl h;  e = rho(|j|) j (Eq. 13) or rho_out j;  h_dot_in = -curl e on the conductor
//   repeat: j_dot = curl h_dot, kept on the conductor;  h_dot_out = h_e_dot + Phi[j_dot] on
//   free space;  stop when mean_out |h_dot^{i+1} - h_dot^i| < delta_it max(|h_e_dot|, 1).
#include "mf_rhs_common.cuh"

namespace mf {

enum Op3 { OP3_CURL = 0, OP3_CURLNEG = 1, OP3_PHI = 2 };

// y and z lines of at least 2^TMA_MIN_LG points are staged by bulk copies (tensor memory
// accelerator); shorter ones by per-thread cp.async into a rotating third buffer, which issues
// the next item's gather earlier (measured faster for the 128-point lines of a 128^3 grid)
constexpr int TMA_MIN_LG = 8;

// raw pointers and sizes the x-pass epilogues need, held by value (registers)
template <typename T>
struct BulkPtrs {
  const uint8_t* mask;
  const T* jcmap;
  T* hd;
  long long ncell;
  int nx, ny;
  double Lx, Ly, Lz, dx, dy, dz;
};

template <typename T>
struct Bulk {
  const Desc& d;
  C2<T>* sm;
  C2<T>* sm2;
  C2<T>* sm3;        // third buffer: the next item's gather in the y and z passes
  Shared& sh;
  int nx, ny, nz, lgx, lgy, lgz, half, nkx;
  long long nspec, ncell;
  C2<T>* S1;
  C2<T>* S2;
  T* hd;
  const uint8_t* mask;
  const T* jcmap;
  const C2<T>* twx; const C2<T>* twy; const C2<T>* twz;
  const T* ktab; const T* gtab;     // kx (nkx), ky (ny), kz (nz)
  int rb, zs, P;
  unsigned nblocks;

  __device__ Bulk(const Desc& dd, C2<T>* s, Shared& shr)
      : d(dd), sm(s), sm2(s + BATCH_PAD), sm3(s + 2 * BATCH_PAD), sh(shr) {
    nx = d.nx; ny = d.ny; nz = d.nz; lgx = d.lgx; lgy = d.lgy; lgz = d.lgz;
    half = nx / 2; nkx = half + 1;
    nspec = (long long)nkx * ny * nz;
    ncell = (long long)nx * ny * nz;
    S1 = (C2<T>*)d.Sa; S2 = (C2<T>*)d.Sb;
    hd = (T*)d.hd;
    mask = d.mask; jcmap = (const T*)d.jcmap;
    twx = (const C2<T>*)d.tw_x;
    twy = (const C2<T>*)d.tw_y;
    twz = (const C2<T>*)d.tw_z;
    ktab = (const T*)d.ktab; gtab = (const T*)d.gtab;
    rb = d.rows_per_item;
    zs = d.zs_per_item;
    P = BATCH / (3 * nz);
    if (P > ny) P = ny;
    int p2 = 1;
    while (p2 * 2 <= P) p2 *= 2;
    P = p2;
    nblocks = gridDim.x;
  }

  __device__ bool sync(int where) { return grid_sync(d.gb, nblocks, where, &sh.bar_passed, d.barrier_ns); }

  __device__ BulkPtrs<T> ptrs() const {
    return BulkPtrs<T>{mask, jcmap, hd, ncell, nx, ny, d.Lx, d.Ly, d.Lz, d.dx, d.dy, d.dz};
  }

  // ---- x pass over rows (z, y0 .. y0 + rb): inverse of NIN = 0|3 fields, epilogue, forward ----
  // With inputs, the item's half spectra arrive staged in the third buffer (cp.async); once the
  // first inverse stage has read them, the next item's (x pass item `next`, -1: none) are
  // issued into the same buffer and load while this item finishes.
  __device__ __forceinline__ void xstage(int it, int nin) {
    const int per_z = ny / rb;
    const long long off = (long long)(it / per_z) * nkx * ny + (it % per_z) * rb;
    if (nin == 3) stage_rows_async<T, 3>(sm3, S1 + off, nspec, ny, rb, lgx);
  }
  template <int NIN, int NOUT, class Epi>
  __device__ __forceinline__ void xitem(int z, int y0, int next, Epi& epi_io) {
    Epi epi = epi_io;                   // register copy of the epilogue
    const int nx = this->nx, ny = this->ny, lgx = this->lgx, nkx = this->nkx, rb = this->rb;
    const long long nspec = this->nspec;
    C2<T>* const sm = this->sm;
    C2<T>* const sm2 = this->sm2;
    C2<T>* const S1 = this->S1;
    const C2<T>* const twx = this->twx;
    const int npair = rb / 2;
    const long long off = (long long)z * nkx * ny + y0;
    C2<T>* X = sm;
    const int lgpair = __ffs(npair) - 1;
    (void)off;
    if constexpr (NIN > 0) {
      cp_async_wait<0>();
      __syncthreads();
      X = rows_inverse_staged<T, NIN>(sm3, sm, sm2, npair, lgpair, lgx, twx, [&] {
        if (next >= 0) xstage(next, NIN);
      });
    }
    C2<T>* Y = X == sm ? sm2 : sm;
    // not unrolled: a second cell in flight spilled the epilogues' live values (26% slower
    // per outside iteration on the 128^3 grid)
#pragma unroll 1
    for (int e = threadIdx.x; e < (npair << lgx); e += NT) {
      const int pr = e >> lgx, x = e & (nx - 1);
      T ina[3], inb[3], oa[3], ob[3];
#pragma unroll
      for (int f = 0; f < NIN; ++f) {
        const C2<T> v = X[sp(((f * npair + pr) << lgx) + x)];
        ina[f] = v.x; inb[f] = v.y;
      }
      const long long i0 = ((long long)z * ny + y0 + 2 * pr) * nx + x;
      if constexpr (Epi::kPair) {
        epi.pair(i0, i0 + nx, ina, inb, oa, ob);
      } else {
        epi(i0, ina, oa);
        epi(i0 + nx, inb, ob);
      }
#pragma unroll
      for (int f = 0; f < NOUT; ++f) X[sp(((f * npair + pr) << lgx) + x)] = C2<T>{oa[f], ob[f]};
    }
    __syncthreads();
    if constexpr (NOUT > 0) rows_forward_scatter<T, NOUT>(X, Y, S1 + off, nspec, ny, npair, lgpair, lgx, twx);
    epi_io.acc = epi.acc;
    epi_io.accmax = epi.accmax;
  }
  template <int NIN, int NOUT, class Epi>
  __device__ void xpass(Epi& epi, int slot) {
    const int per_z = ny / rb;
    const int nitems = per_z * nz;
    if (NIN > 0 && (int)blockIdx.x < nitems) xstage((int)blockIdx.x, NIN);
    for (int it = (int)blockIdx.x; it < nitems; it += (int)gridDim.x) {
      epi.acc = 0.0;
      epi.accmax = 0.0;
      const int next = it + (int)gridDim.x < nitems ? it + (int)gridDim.x : -1;
      xitem<NIN, NOUT>(it / per_z, (it % per_z) * rb, next, epi);
      if (slot >= 0) {
        const double v = epi.is_max ? block_max(epi.accmax, sh.red) : block_sum(epi.acc, sh.red);
        if (threadIdx.x == 0) d.partials[(size_t)slot * d.max_items + it] = v;
      }
    }
  }
  __device__ double total(int slot, bool is_max = false) {
    return reduce_partials(d.partials, d.max_items, slot, (ny / rb) * nz, is_max, sh.red);
  }

  // ---- the y and z passes: items it = blockIdx.x, + gridDim.x, ... with the gather of the next
  // item in flight (cp.async into the third shared buffer) while the current one transforms in
  // the other two.  issue(it, buf) starts item it's gather into buf; work(it, a, b) transforms
  // the item gathered in a (b is its second buffer), writes its result and ends with a CTA
  // barrier.  The buffers rotate: the next input is the prefetch buffer, the next prefetch goes
  // to the buffer the finished item used last. ----
  template <class Issue, class Work>
  __device__ __forceinline__ void pipelined(int nitems, Issue issue, Work work) {
    C2<T>* a = sm;
    C2<T>* b = sm2;
    C2<T>* c = sm3;
    int it = (int)blockIdx.x;
    if (it < nitems) issue(it, a);
    for (; it < nitems; it += (int)gridDim.x) {
      const int nxt = it + (int)gridDim.x;
      if (nxt < nitems) {
        issue(nxt, c);
        cp_async_wait<1>();                 // this item's group; the next one stays in flight
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      work(it, a, b);
      C2<T>* const t = a;
      a = c;
      c = b;
      b = t;
    }
  }

  // ---- passes whose items are contiguous lines: item it's `nl` lines of length 2^lg (line l
  // at src(it, l)) are copied by the tensor memory accelerator (cp.async.bulk) into the third
  // buffer, line l at l (2^lg + 2) (the two spare values per line shift successive lines by
  // four banks), completion counted on the CTA's mbarrier.  work(it, after_first) runs the item
  // and calls after_first() once its first transform stage has read the staging buffer; that
  // issues the next item's copies, which then land while this item finishes. ----
  template <class Src, class Work>
  __device__ __forceinline__ void tma_lines(int nitems, int nl, int lg, Src src, Work work) {
    unsigned long long* const bar = &sh.tma_bar;
    const int stride = (1 << lg) + 2;
    const unsigned bytes = (unsigned)sizeof(C2<T>) << lg;
    C2<T>* const stg = sm3;
    auto issue = [&](int it) {
      if (threadIdx.x == 0) {
        fence_proxy_async();
        mbar_expect_tx(bar, bytes * (unsigned)nl);
        for (int l = 0; l < nl; ++l) bulk_g2s(stg + l * stride, src(it, l), bytes, bar);
      }
    };
    unsigned parity = sh.tma_parity;
    int it = (int)blockIdx.x;
    if (it < nitems) issue(it);
    for (; it < nitems; it += (int)gridDim.x) {
      mbar_wait(bar, parity, d.gb, d.barrier_ns);
      parity ^= 1u;
      const int nxt = it + (int)gridDim.x;
      work(it, [&] { if (nxt < nitems) issue(nxt); });
    }
    __syncthreads();
    if (threadIdx.x == 0) sh.tma_parity = parity;
    __syncthreads();
  }
  // first (inverse or forward) transform stage of nl staged lines into `out`, then after_first()
  template <int DIR, class AfterFirst>
  __device__ __forceinline__ void first_from_stage(int lg, int nl, C2<T>* out, AfterFirst after_first) {
    C2<T>* const S = dsm<T>();
    const int st = dsm_off(sm3);
    const int stride = (1 << lg) + 2;
    const FftPlan P = fft_plan<T>(lg);
    fft_first_io_any<T, DIR>(P.lgr(0), lg, nl, [=](int line, int pos) { return S[st + line * stride + pos]; }, out);
    after_first();
  }

  // ---- y pass, forward: S1[c][z][kx][:] -> S2[c][kx][:][z] for z in [z0, z0 + zs) ----
  __device__ __noinline__ void yfwd() {
    const int ny = this->ny, nz = this->nz, lgy = this->lgy, nkx = this->nkx, zs = this->zs;
    const long long nspec = this->nspec;
    C2<T>* const S1 = this->S1;
    C2<T>* const S2 = this->S2;
    const C2<T>* const twy = this->twy;
    const int per_kx = nz / zs;
    const int nl = 3 * zs;
    // transposed write of the item's transformed lines (X: line c zs + dz, wavenumber ky)
    auto scatter = [=](const C2<T>* X, int kx, int z0) {
      for (int e = threadIdx.x; e < (nl << lgy); e += NT) {
        const int dz = e % zs, rest = e / zs;
        const int ky = rest & (ny - 1), c = rest >> lgy;
        S2[c * nspec + ((long long)kx * ny + ky) * nz + z0 + dz] = X[sp(((c * zs + dz) << lgy) + ky)];
      }
      __syncthreads();
    };
    if (lgy >= TMA_MIN_LG) {
      tma_lines(nkx * per_kx, nl, lgy,
          [=](int it, int l) {
            const int kx = it / per_kx, z0 = (it % per_kx) * zs;
            const int c = l / zs, dz = l - c * zs;
            return (const C2<T>*)(S1 + c * nspec + ((long long)(z0 + dz) * nkx + kx) * ny);
          },
          [&](int it, auto after_first) {
            first_from_stage<-1>(lgy, nl, sm, after_first);
            scatter(fft_lines_from<T, -1>(sm, sm2, lgy, nl, twy, 1), it / per_kx, (it % per_kx) * zs);
          });
      return;
    }
    pipelined(nkx * per_kx,
        [=](int it, C2<T>* buf) {
          const int kx = it / per_kx, z0 = (it % per_kx) * zs;
          gather_async<T>(buf, S1, nl << lgy,
              [=](int e) {
                const int l = e >> lgy, y = e & (ny - 1);
                const int c = l / zs, dz = l - c * zs;
                return c * nspec + ((long long)(z0 + dz) * nkx + kx) * ny + y;
              },
              [](int e) { return e; });
        },
        [=](int it, C2<T>* a, C2<T>* b) {
          scatter(fft_lines<T, -1>(a, b, lgy, nl, twy), it / per_kx, (it % per_kx) * zs);
        });
  }
  // ---- y pass, inverse: S2 -> S1 ----
  __device__ __noinline__ void yinv() {
    const int ny = this->ny, nz = this->nz, lgy = this->lgy, nkx = this->nkx, zs = this->zs;
    const long long nspec = this->nspec;
    C2<T>* const S1 = this->S1;
    C2<T>* const S2 = this->S2;
    const C2<T>* const twy = this->twy;
    const int per_kx = nz / zs;
    const int nl = 3 * zs;
    pipelined(nkx * per_kx,
        [=](int it, C2<T>* buf) {
          const int kx = it / per_kx, z0 = (it % per_kx) * zs;
          gather_async<T>(buf, S2, nl << lgy,
              [=](int e) {
                const int dz = e % zs, rest = e / zs;
                const int ky = rest & (ny - 1), c = rest >> lgy;
                return c * nspec + ((long long)kx * ny + ky) * nz + z0 + dz;
              },
              [=](int e) {
                const int dz = e % zs, rest = e / zs;
                const int ky = rest & (ny - 1), c = rest >> lgy;
                return ((c * zs + dz) << lgy) + ky;
              });
        },
        [=](int it, C2<T>* a, C2<T>* b) {
          const int kx = it / per_kx, z0 = (it % per_kx) * zs;
          const C2<T>* X = fft_lines<T, +1>(a, b, lgy, nl, twy);
          for (int e = threadIdx.x; e < (nl << lgy); e += NT) {
            const int l = e >> lgy, y = e & (ny - 1);
            const int c = l / zs, dz = l - c * zs;
            S1[c * nspec + ((long long)(z0 + dz) * nkx + kx) * ny + y] = X[sp(e)];
          }
          __syncthreads();
        });
  }
  // ---- z pass: forward, 3x3 multiplier, inverse on lines (kx, ky0 .. ky0 + P) ----
  __device__ __noinline__ void zpass(int op) {
    const int ny = this->ny, nz = this->nz, lgz = this->lgz, nkx = this->nkx, half = this->half, P = this->P;
    const long long nspec = this->nspec, ncell = this->ncell;
    C2<T>* const S2 = this->S2;
    const C2<T>* const twz = this->twz;
    const T* const ktab = this->ktab;
    const T* const gtab = this->gtab;
    const int per_kx = ny / P;
    const T s = (T)1 / (T)ncell;
    const int pl = P << lgz;                         // values per component
    // multiplier, inverse transform and write of an item whose forward transform is in X (Y:
    // the other buffer)
    auto finish = [=](C2<T>* X, C2<T>* Y, int kx, int ky0) {
      const long long base = ((long long)kx * ny + ky0) * nz;
      const T kxv = ldg_tab(&ktab[kx]), gx = ldg_tab(&gtab[kx]);
      const T kxo = kx == half ? (T)0 : kxv;
      for (int e = threadIdx.x; e < pl; e += NT) {
        const int p = e >> lgz, kz = e & (nz - 1);
        const int ky = ky0 + p;
        const T kyv = ldg_tab(&ktab[nkx + ky]), kzv = ldg_tab(&ktab[nkx + ny + kz]);
        const T kyo = ky == ny / 2 ? (T)0 : kyv;
        const T kzo = kz == nz / 2 ? (T)0 : kzv;
        const C2<T> va = X[sp(e)], vb = X[sp(pl + e)], vc = X[sp(2 * pl + e)];
        // cross product k x v with the odd (Nyquist-free) wavenumbers
        C2<T> cx = {kyo * vc.x - kzo * vb.x, kyo * vc.y - kzo * vb.y};
        C2<T> cy = {kzo * va.x - kxo * vc.x, kzo * va.y - kxo * vc.y};
        C2<T> cz = {kxo * vb.x - kyo * va.x, kxo * vb.y - kyo * va.y};
        T f;
        if (op == OP3_PHI) {
          const T k2 = kxv * kxv + kyv * kyv + kzv * kzv;
          f = k2 > (T)0 ? s / k2 : (T)0;                   // Eq. 17
        } else {
          const T G = gx * ldg_tab(&gtab[nkx + ky]) * ldg_tab(&gtab[nkx + ny + kz]);
          f = (op == OP3_CURL ? G : -G) * s;               // smoothed curl
        }
        X[sp(e)] = cmul_si(cscale(cx, f), 1);
        X[sp(pl + e)] = cmul_si(cscale(cy, f), 1);
        X[sp(2 * pl + e)] = cmul_si(cscale(cz, f), 1);
      }
      __syncthreads();
      const C2<T>* Z = fft_lines<T, +1>(X, Y, lgz, 3 * P, twz);
      for (int e = threadIdx.x; e < 3 * pl; e += NT) {
        const int c = e / pl, r = e - c * pl;
        S2[c * nspec + base + r] = Z[sp(e)];
      }
      __syncthreads();
    };
    if (lgz >= TMA_MIN_LG) {
      tma_lines(nkx * per_kx, 3 * P, lgz,
          [=](int it, int l) {
            const int kx = it / per_kx, ky0 = (it % per_kx) * P;
            const int c = l / P, p = l - c * P;
            return (const C2<T>*)(S2 + c * nspec + ((long long)kx * ny + ky0 + p) * nz);
          },
          [&](int it, auto after_first) {
            first_from_stage<-1>(lgz, 3 * P, sm, after_first);
            C2<T>* X = fft_lines_from<T, -1>(sm, sm2, lgz, 3 * P, twz, 1);
            finish(X, X == sm ? sm2 : sm, it / per_kx, (it % per_kx) * P);
          });
      return;
    }
    pipelined(nkx * per_kx,
        [=](int it, C2<T>* buf) {
          const long long base = ((long long)(it / per_kx) * ny + (it % per_kx) * P) * nz;
          gather_async<T>(buf, S2, 3 * pl,
              [=](int e) { const int c = e / pl; return c * nspec + base + (e - c * pl); },
              [](int e) { return e; });
        },
        [=](int it, C2<T>* a, C2<T>* b) {
          C2<T>* X = fft_lines<T, -1>(a, b, lgz, 3 * P, twz);
          finish(X, X == a ? b : a, it / per_kx, (it % per_kx) * P);
        });
  }

  // Yf, Z(op), Yi with barriers; the x passes before and after are separate
  __device__ bool yzy(int op, int where) {
    yfwd();
    if (!sync(where)) return false;
    zpass(op);
    if (!sync(where + 1)) return false;
    yinv();
    return sync(where + 2);
  }
};

// ------------------------------------------------------------------------------------------
// epilogues of the x pass (cell index i, three components in / out)
// ------------------------------------------------------------------------------------------
// Stage state y + sum c_j k_j.  With a field-dependent critical current (kim) the stage
// field's magnitude |h| is kept, in the transform precision, in the first component of the
// h_dot iterate at superconductor cells: those entries are rewritten by BInit before anything
// reads them as an iterate, and the warm start lives on free space only.
template <typename T>
struct BStage : EpiBase<T> {
  BulkPtrs<T> P;
  StageIn in;
  bool kim;
  __device__ void operator()(long long i, const T*, T* out) {
    // every load of the cell before its first store (a store could alias a later load as far
    // as the compiler knows, which would put each load behind the previous store)
    double v[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) v[c] = in.y[c * P.ncell + i];
    for (int j = 0; j < in.nk; ++j) {
#pragma unroll
      for (int c = 0; c < 3; ++c) v[c] += in.c[j] * in.k[j][c * P.ncell + i];
    }
    double h2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (in.ynew) in.ynew[c * P.ncell + i] = v[c];
      out[c] = (T)v[c];
      h2 += v[c] * v[c];
    }
    if (kim && __ldg(&P.mask[i]) == 1) P.hd[i] = (T)sqrt(h2);
  }
};

// local law of the superconductor: critical current (Kim-type jc / (1 + |h|/b0) when ib0 > 0,
// |h| left by BStage) and the elliptic weight a = 1/gamma^2 of j_z
template <typename T>
__device__ __forceinline__ T bulk_jc(const BulkPtrs<T>& P, long long i, int m, T jc, T ib0) {
  T jcl = P.jcmap ? __ldg(&P.jcmap[i]) : jc;
  if (ib0 > (T)0 && m == 1) jcl = jcl / ((T)1 + P.hd[i] * ib0);
  return jcl;
}

template <typename T>
struct BPower : EpiBase<T> {               // j -> e (Eq. 13 / Ohm law; elliptic and Kim laws)
  BulkPtrs<T> P;
  T n, e0, jc, rho_out, ig2, ib0;
  __device__ void operator()(long long i, const T* in, T* out) {
    const int m = __ldg(&P.mask[i]);
    const T jcl = bulk_jc(P, i, m, jc, ib0);
    const T a = m == 1 ? ig2 : (T)1;
    const T rho = resistivity<T>(in[0] * in[0] + in[1] * in[1] + in[2] * in[2] * a, jcl, m, n, e0, rho_out);
    out[0] = rho * in[0]; out[1] = rho * in[1]; out[2] = rho * in[2] * a;
  }
};

template <typename T>
struct BInit : EpiBase<T> {                // h_dot^0: h_dot_in on the conductor, warm or h_e_dot outside
  BulkPtrs<T> P;
  bool warm;
  T hed[3];
  static constexpr bool kPair = true;
  __device__ __forceinline__ void pair(long long ia, long long ib, const T* ina, const T* inb, T* oa, T* ob) {
    const bool ca = __ldg(&P.mask[ia]) != 0, cb = __ldg(&P.mask[ib]) != 0;
    T wa[3], wb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      wa[c] = (!ca && warm) ? P.hd[c * P.ncell + ia] : hed[c];
      wb[c] = (!cb && warm) ? P.hd[c * P.ncell + ib] : hed[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      oa[c] = ca ? ina[c] : wa[c];                         // -curl e (Eq. 14) on the conductor
      ob[c] = cb ? inb[c] : wb[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      P.hd[c * P.ncell + ia] = oa[c];
      P.hd[c * P.ncell + ib] = ob[c];
    }
  }
};

template <typename T>
struct BMaskCond : EpiBase<T> {            // j_dot_in: keep on the conductor only
  BulkPtrs<T> P;
  __device__ void operator()(long long i, const T* in, T* out) {
    const bool cond = __ldg(&P.mask[i]) != 0;
    out[0] = cond ? in[0] : (T)0; out[1] = cond ? in[1] : (T)0; out[2] = cond ? in[2] : (T)0;
  }
};

template <typename T>
struct BUpdate : EpiBase<T, T> {           // Eq. 18 on free space, residual, forward
  BulkPtrs<T> P;
  T hed[3];
  static constexpr bool kPair = true;
  __device__ __forceinline__ void pair(long long ia, long long ib, const T* ina, const T* inb, T* oa, T* ob) {
    const bool fa = __ldg(&P.mask[ia]) == 0, fb = __ldg(&P.mask[ib]) == 0;
    T ha[3], hb[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ha[c] = P.hd[c * P.ncell + ia];
      hb[c] = P.hd[c * P.ncell + ib];
    }
    T sa = 0, sb = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T na = hed[c] + ina[c], nb = hed[c] + inb[c];
      sa += (na - ha[c]) * (na - ha[c]);
      sb += (nb - hb[c]) * (nb - hb[c]);
      oa[c] = fa ? na : ha[c];
      ob[c] = fb ? nb : hb[c];
    }
    if (fa) this->acc += sqrt(sa);
    if (fb) this->acc += sqrt(sb);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (fa) P.hd[c * P.ncell + ia] = oa[c];
      if (fb) P.hd[c * P.ncell + ib] = ob[c];
    }
  }
};

template <typename T>
struct BFinal : EpiBase<T> {               // h_dot out (FP64); optional BS23 error contribution
  BulkPtrs<T> P;
  double* kout;
  bool err;
  double h, rtol, atol;
  const double* k1; const double* k2; const double* k3; const double* y; const double* ynew;
  __device__ void operator()(long long i, const T*, T*) {
    double g[3];                                             // loads before the stores (see BStage)
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] = (double)P.hd[c * P.ncell + i];
#pragma unroll
    for (int c = 0; c < 3; ++c) kout[c * P.ncell + i] = g[c];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const long long k = c * P.ncell + i;
      if (err) {
        const double E = h * (-5.0 / 72.0 * k1[k] + 1.0 / 12.0 * k2[k] + 1.0 / 9.0 * k3[k] - 0.125 * g[c]);
        const double sc = atol + rtol * fmax(fabs(y[k]), fabs(ynew[k]));
        double q;                                            // the ratio in the transform precision
        if constexpr (sizeof(T) == 4) q = (double)__fdiv_rn((float)fabs(E), (float)sc);
        else q = fabs(E) / sc;
        if (!(q == q) || isinf(q)) q = 1e300;
        this->accmax = fmax(this->accmax, q);
      } else if (!isfinite(g[c])) {
        this->accmax = 1.0;
      }
    }
  }
};

template <typename T>
struct BStoreJ : EpiBase<T> {              // readout of j = curl h (FP64)
  BulkPtrs<T> P;
  double* out;
  __device__ void operator()(long long i, const T* in, T*) {
    out[i] = in[0]; out[P.ncell + i] = in[1]; out[2 * P.ncell + i] = in[2];
  }
};

template <typename T>
struct BStoreE : EpiBase<T> {              // readout of e, the law of BPower (FP64)
  BulkPtrs<T> P;
  T n, e0, jc, rho_out, ig2, ib0;
  double* out;
  __device__ void operator()(long long i, const T* in, T*) {
    const int m = __ldg(&P.mask[i]);
    const T jcl = bulk_jc(P, i, m, jc, ib0);
    const T a = m == 1 ? ig2 : (T)1;
    const T rho = resistivity<T>(in[0] * in[0] + in[1] * in[1] + in[2] * in[2] * a, jcl, m, n, e0, rho_out);
    out[i] = rho * in[0]; out[P.ncell + i] = rho * in[1]; out[2 * P.ncell + i] = rho * in[2] * a;
  }
};

template <typename T>
struct BMoment : EpiBase<T> {              // m = 1/2 sum dV r x j over the conductor, component `comp`
  BulkPtrs<T> P;
  int comp;
  __device__ void operator()(long long i, const T* in, T*) {
    if (__ldg(&P.mask[i]) == 0) return;
    const int x = (int)(i % P.nx), y = (int)((i / P.nx) % P.ny), z = (int)(i / ((long long)P.nx * P.ny));
    const double rx = -P.Lx + (x + 0.5) * P.dx;
    const double ry = -P.Ly + (y + 0.5) * P.dy;
    const double rz = -P.Lz + (z + 0.5) * P.dz;
    double v;
    if (comp == 0) v = ry * in[2] - rz * in[1];
    else if (comp == 1) v = rz * in[0] - rx * in[2];
    else v = rx * in[1] - ry * in[0];
    this->acc += v;
  }
};

// ------------------------------------------------------------------------------------------
// one bulk right-hand side
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ RhsOut bulk_rhs(Bulk<T>& B, double t, int seg, const StageIn& sin, double* kout,
                                        int force_iters, bool want_err, double h_err, const double* e_k1,
                                        const double* e_k2, const double* e_k3, const double* e_y,
                                        const double* e_ynew) {
  const Desc& d = B.d;
  RhsOut res{ST_OK, 0, 0.0, 0.0, 0};
  const double hs = he_dot(d, t, seg);
  const double hed[3] = {hs * d.he_dir[0], hs * d.he_dir[1], hs * d.he_dir[2]};
  const double hed_norm = sqrt(hed[0] * hed[0] + hed[1] * hed[1] + hed[2] * hed[2]);
#define BSYNC(w) if (!B.sync(w)) { res.status = ST_BARRIER; return res; }
#define BYZY(op, w) if (!B.yzy(op, w)) { res.status = ST_BARRIER; return res; }
  { BStage<T> e; e.P = B.ptrs(); e.in = sin; e.kim = d.b0 > 0.0; B.xpass<0, 3>(e, -1); }
  BSYNC(101);
  BYZY(OP3_CURL, 102);                                                   // j = curl h
  {
    BPower<T> e; e.P = B.ptrs(); e.n = (T)d.n; e.e0 = (T)d.e0; e.jc = (T)d.jc; e.rho_out = (T)d.rho_out;
    e.ig2 = (T)(1.0 / (d.gamma * d.gamma)); e.ib0 = d.b0 > 0.0 ? (T)(1.0 / d.b0) : (T)0;
    B.xpass<3, 3>(e, -1);                                                // e = rho j
  }
  BSYNC(105);
  BYZY(OP3_CURLNEG, 106);                                                // -curl e
  {
    BInit<T> e; e.P = B.ptrs(); e.warm = B.sh.warm_valid != 0;
    for (int c = 0; c < 3; ++c) e.hed[c] = (T)hed[c];
    B.xpass<3, 3>(e, -1);                                                // h_dot^0
  }
  BSYNC(109);
  const bool have_out = d.nout > 0;
  const double thresh = d.iter_tol * fmax(hed_norm, 1.0);
  const bool forced = force_iters > 0;
  const bool fixed = d.iter_tol <= 0.0;
  const int itmax = forced ? force_iters : d.iter_max;
  double r = 0.0;
  int i = 0;
  if (have_out) {
    for (; i < itmax; ++i) {
      BYZY(OP3_CURL, 110);                                               // j_dot = curl h_dot
      { BMaskCond<T> e; e.P = B.ptrs(); B.xpass<3, 3>(e, -1); }                // j_dot_in
      BSYNC(113);
      BYZY(OP3_PHI, 114);                                                // Phi[j_dot_in]
      {
        BUpdate<T> e; e.P = B.ptrs();
        for (int c = 0; c < 3; ++c) e.hed[c] = (T)hed[c];
        B.xpass<3, 3>(e, 0);                                             // Eq. 18
      }
      BSYNC(117);
      r = B.total(0) / (double)d.nout;
      if (!(forced || fixed) && r < thresh) { ++i; break; }
    }
    if (i > itmax) i = itmax;
  }
  res.iters = i;
  res.r = r;
  res.status = (!have_out || fixed || r < thresh) ? ST_OK : ST_NOCONV;
  // a call that failed with a residual above 1e3 times the threshold (or not finite) diverged:
  // the next call starts cold
  B.sh.warm_valid = (res.status == ST_NOCONV && !(r < 1e3 * thresh)) ? 0 : 1;
  {
    BFinal<T> e; e.P = B.ptrs(); e.kout = kout; e.is_max = true;
    e.err = want_err; e.h = h_err; e.rtol = d.rtol; e.atol = d.atol;
    e.k1 = e_k1; e.k2 = e_k2; e.k3 = e_k3; e.y = e_y; e.ynew = e_ynew;
    B.xpass<0, 0>(e, 3);
  }
  BSYNC(120);
  const double q = B.total(3, true);
  if (want_err) res.err = q;
  else res.nonfinite = q > 0.0;
#undef BSYNC
#undef BYZY
  return res;
}

template <typename T>
struct BulkRhs {
  Bulk<T>& B;
  __device__ RhsOut operator()(double t, int seg, const StageIn& in, double* kout, int force,
                               bool want_err, double h, const double* k1, const double* k2,
                               const double* k3, const double* y, const double* yn) {
    return bulk_rhs<T>(B, t, seg, in, kout, force, want_err, h, k1, k2, k3, y, yn);
  }
  __device__ void on_accept() {}     // 3D: every call starts from the most recent iterate
  __device__ void on_attempt() {}
};

template <typename T>
__global__ void __launch_bounds__(NT, 2) bulk_kernel(const Desc* __restrict__ dg, KernelArgs a) {
  C2<T>* sm = dsm<T>();
  __shared__ Shared sh;
  // one copy of the pass object per CTA, in shared memory: its members are read as broadcasts
  // instead of per-thread local-memory copies
  __shared__ __align__(16) unsigned char objraw[sizeof(Bulk<T>)];
  const Desc& d = *dg;
  SolverState* st = d.st;
  if (threadIdx.x == 0) {
    sh.warm_valid = st->warm_valid;
    sh.bar_passed = 0;
    sh.A_prev = 0.0;
    sh.tma_parity = 0;
    mbar_init(&sh.tma_bar);
  }
  if (threadIdx.x == 0) new (objraw) Bulk<T>(d, sm, sh);
  __syncthreads();
  Bulk<T>& B = *reinterpret_cast<Bulk<T>*>(objraw);
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  int status = ST_OK;

  if (a.mode == MODE_RHS) {
    StageIn in{a.y_in, 0, {0, 0, 0}, {nullptr, nullptr, nullptr}, nullptr};
    RhsOut r = bulk_rhs<T>(B, a.t, a.seg, in, a.out, a.force_iters, false, 0.0, nullptr, nullptr,
                           nullptr, nullptr, nullptr);
    status = r.status == ST_OK && r.nonfinite ? ST_NONFINITE : r.status;
    if (leader) { st->last_iters = r.iters; st->last_r = r.r; st->n_rhs += 1; st->n_iters += r.iters; }
  } else if (a.mode == MODE_J || a.mode == MODE_E || a.mode == MODE_MOMENT) {
    StageIn in{a.y_in, 0, {0, 0, 0}, {nullptr, nullptr, nullptr}, nullptr};
    { BStage<T> e; e.P = B.ptrs(); e.in = in; e.kim = a.mode == MODE_E && d.b0 > 0.0; B.xpass<0, 3>(e, -1); }
    bool ok = B.sync(201) && B.yzy(OP3_CURL, 202);
    if (ok) {
      if (a.mode == MODE_J) {
        BStoreJ<T> e; e.P = B.ptrs(); e.out = a.out;
        B.xpass<3, 0>(e, -1);
      } else if (a.mode == MODE_E) {
        BStoreE<T> e; e.P = B.ptrs(); e.out = a.out;
        e.n = (T)d.n; e.e0 = (T)d.e0; e.jc = (T)d.jc; e.rho_out = (T)d.rho_out;
        e.ig2 = (T)(1.0 / (d.gamma * d.gamma)); e.ib0 = d.b0 > 0.0 ? (T)(1.0 / d.b0) : (T)0;
        B.xpass<3, 0>(e, -1);
      } else {
        for (int c = 0; c < 3 && ok; ++c) {
          BMoment<T> e; e.P = B.ptrs(); e.comp = c;
          B.xpass<3, 0>(e, 4 + c);      // reads S1 only
          ok = B.sync(205 + c);
        }
        if (ok) {
          for (int c = 0; c < 3; ++c) {
            const double s = B.total(4 + c);
            if (leader) a.out[c] = 0.5 * s * d.dx * d.dy * d.dz;
          }
        }
      }
    }
    if (!ok) status = ST_BARRIER;
  } else if (a.mode == MODE_ADVANCE) {
    BulkRhs<T> R{B};
    status = bs23_advance(R, d, st, a, leader);
  }
  if (leader) {
    st->warm_valid = sh.warm_valid;
    st->status = status;
  }
}

int bulk_max_blocks(int precision, size_t smem) {
  int nb = 0;
  if (precision) {
    cudaFuncSetAttribute(bulk_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bulk_kernel<float>, NT, smem);
  } else {
    cudaFuncSetAttribute(bulk_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bulk_kernel<double>, NT, smem);
  }
  return nb;
}

cudaError_t bulk_launch(int precision, const Desc& d, const KernelArgs& a, cudaStream_t s) {
  const Desc* dg = d.dev;
  KernelArgs aa = a;
  void* args[] = {&dg, &aa};
  const size_t smem = kernel_smem_bytes(d);
  const void* fn = precision ? (const void*)bulk_kernel<float> : (const void*)bulk_kernel<double>;
  return cudaLaunchCooperativeKernel(fn, dim3(d.grid), dim3(NT), args, smem, s);
}

}  // namespace mf
