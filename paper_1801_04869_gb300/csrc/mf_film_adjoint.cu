// Transpose of a film's outside iteration (Eqs. 10-12), the linear core of the right-hand
// side's vector-Jacobian product.  The adjoint has no counterpart in the paper.
//
// With a cold start and a fixed count I, the iteration maps (h_dot_in, h_e_dot) linearly to
// g_dot (the conductor's output):
//   h_0 = shift(h_dot_in on the conductor, h_e_dot on free space)        shift: Eq. 10
//   u_i = K1 h_i,  g_i = u_i - C(u_i)                                     Eq. 11 (K1 = 2/|k|)
//   h_{i+1} = shift(h_i - out K2 (out g_i))                               Eq. 12 (K2 = lambda |k|/2 G)
//   g_dot = conductor * g_{I-1}
// Its transpose runs the loop backwards.  K1 and K2 are real and even, so they are their own
// transposes; the centring (-C) and the shift (-A) are rank-one corrections whose transposes
// need one grid sum each, applied after the transform through the precomputed responses
// q1 = K1 out and q2 = K2 out (by linearity), so each backward iteration is two round trips,
// as forward:
//   V3  hbar_i = zbar_i + K1 gbar_i - (S_i / n_out) q1      (zbar_{I-1} = 0), tot_i = sum_out hbar_i
//   V5  gbar_{i-1} = out (K2(-out hbar_i) + (tot_i / n_out) q2),  zbar_{i-1} = hbar_i - tot_i / n_out,
//       S_{i-1} = sum gbar_{i-1};   sbar += (N / n_out) tot_i
//   end hbar_in = conductor * (hbar_0 - tot_0 / n_out),  sbar += (N / n_out) tot_0
// The h_dot buffers of the warm start hold hbar and zbar, so the warm start is cleared.
//
// Warm-started calls (the integrator's: each call starts from the previous call's last iterate
// instead of h_e_dot) add one input and one output to the linear map: the warm start on free
// space and the last iterate h_{I-1}.  The cotangent of the last iterate (wbar_out, free space)
// enters hbar_{I-1}; the cotangent of the warm start is out * (hbar_0 - tot_0 / n_out), written
// beside hbar_in (wbar_in).  (Its sum over free space is zero, so a cold start, whose warm start
// is h_e_dot on free space, adds nothing to sbar.)
//
// The full vector-Jacobian product of f(g; jc, h_e_dot) adds the nonlinear ends around it:
//   j = (d_y g, -d_x g) is recomputed from g (Eq. 2; gradient column pass at the start, stored
//   as two real fields), r = -conductor * hbar_in, ebar = (d_y r, -d_x r) (the transposed
//   -curl of Eq. 4 is the smoothed gradient column pass), the linearised power law
//   jbar = rho (ebar + (n - 1) j^ (j^ . ebar)) in the film and rho_out ebar elsewhere, with
//   jcbar = -(n / jc) ebar . e in the film (Eq. 3), and gbar = d_x jbar_y - d_y jbar_x, which is
//   minus the -curl column pass of jbar.
#include "mf_film.cuh"

namespace mf {

struct AdjArgs {
  const double* v;      // cotangent of g_dot (FP64, ncell)
  double* hin_bar;      // cotangent of h_dot_in (FP64, ncell; 0 on free space); outside only
  double* sbar;         // cotangent of h_e_dot (FP64 scalar)
  int iters;
  const double* g;      // full product: the state g (FP64, ncell); null: the outside iteration only
  double* gbar;         // full product: cotangent of g (FP64, ncell)
  double* jcbar;        // full product: cotangent of the jc map (FP64, ncell; 0 outside the film)
  const double* wbar_out;  // cotangent of the last iterate (FP64, ncell, free space) or null
  double* wbar_in;      // cotangent of the warm start (FP64, ncell, 0 on the conductor) or null
};

// full product, V1: gbar_{I-1} = conductor * v (with its sum) and g, forward of both
template <typename T>
struct EpiPT0g : EpiBase<T, T> {
  FilmPtrs<T> P;
  const double* v;
  const double* g;
  __device__ void operator()(long long i, const V4<T>*, V4<T>* out) {
    const uchar4 m = ldmask4(P.mask + i);
    const V4<double> x = ld4(v + i);
    const V4<double> y = ld4(g + i);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T gb = mask_at(m, q) != 0 ? (T)x.v[q] : (T)0;
      this->acc += gb;
      out[0].v[q] = gb;
      out[1].v[q] = (T)y.v[q];
    }
  }
};

// full product: j = (d_y g, -d_x g) stored as two real fields
template <typename T>
struct EpiStoreJ : EpiBase<T, T> {
  FilmPtrs<T> P;
  T* jx;
  T* jy;
  __device__ void operator()(long long i, const V4<T>* in, V4<T>*) {
    V4<T> a, b;
#pragma unroll
    for (int q = 0; q < 4; ++q) { a.v[q] = in[1].v[q]; b.v[q] = -in[0].v[q]; }
    st4(jx + i, a);
    st4(jy + i, b);
  }
};

// full product: r = -conductor * hbar_in = -conductor * (hbar_0 - tot_0/n_out), forward
template <typename T>
struct EpiRbar : EpiBase<T, T> {
  FilmPtrs<T> P;
  T t_q;
  double* wdst;         // cotangent of the warm start (free space) or null
  __device__ void operator()(long long i, const V4<T>*, V4<T>* out) {
    const uchar4 m = ldmask4(P.mask + i);
    const V4<T> h = ld4(P.hd + i);
    V4<double> w;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      out[0].v[q] = mask_at(m, q) != 0 ? -(h.v[q] - t_q) : (T)0;
      w.v[q] = mask_at(m, q) == 0 ? (double)(h.v[q] - t_q) : 0.0;
    }
    if (wdst) st4(wdst + i, w);
  }
};

// full product: ebar = (d_y r, -d_x r); linearised power law -> jbar (forward), jcbar.
// Elliptic law e = rho(s) A j, s^2 = j^T A j, A = diag(1, a), a = 1/gamma^2 in the
// superconductor: jbar = rho A ebar + (n-1) rho (A j)(A j . ebar) / s^2 and
// jcbar = -(n/jc) rho (A j . ebar) (rho scales as jc^-n at fixed j)
template <typename T>
struct EpiPowVJP : EpiBase<T, T> {
  FilmPtrs<T> P;
  const T* jx;
  const T* jy;
  double* jcbar;
  T n, e0, jc, rho_out, ig2;
  __device__ void operator()(long long i, const V4<T>* in, V4<T>* out) {
    const uchar4 m = ldmask4(P.mask + i);
    V4<T> jcl;
    if (P.jcmap) jcl = ldg4(P.jcmap + i);
    else jcl = V4<T>{{jc, jc, jc, jc}};
    const V4<T> ax = ld4(jx + i), ay = ld4(jy + i);
    V4<double> cb;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T ex = in[1].v[q], ey = -in[0].v[q];                 // transposed -curl
      const T x = ax.v[q], y = ay.v[q];
      const int mq = mask_at(m, q);
      const T a = mq == 1 ? ig2 : (T)1;
      const T Ay = y * a;                                          // (A j)_y
      const T j2 = x * x + y * Ay;
      const T rho = resistivity<T>(j2, jcl.v[q], mq, n, e0, rho_out);
      T bx = rho * ex, by = rho * ey * a;
      double c = 0.0;
      if (mq == 1) {
        if (j2 > (T)0) {
          const T inv = (T)1 / sqrt(j2);
          const T ux = x * inv, uy = Ay * inv;
          const T pr = (n - (T)1) * rho * (ux * ex + uy * ey);
          bx += pr * ux;
          by += pr * uy;
        }
        c = -(double)(n / jcl.v[q]) * (double)(rho * (ex * x + ey * Ay));
      }
      out[0].v[q] = bx;
      out[1].v[q] = by;
      cb.v[q] = c;
    }
    st4(jcbar + i, cb);
  }
};

// full product: gbar = -(the -curl pass of jbar)
template <typename T>
struct EpiGbar : EpiBase<T, T> {
  FilmPtrs<T> P;
  double* dst;
  __device__ void operator()(long long i, const V4<T>* in, V4<T>*) {
    V4<double> r;
#pragma unroll
    for (int q = 0; q < 4; ++q) r.v[q] = -(double)in[0].v[q];
    st4(dst + i, r);
  }
};

// V1: gbar_{I-1} = conductor * v, and its sum
template <typename T>
struct EpiPT0 : EpiBase<T, T> {
  FilmPtrs<T> P;
  const double* v;
  __device__ void operator()(long long i, const V4<T>*, V4<T>* out) {
    const uchar4 m = ldmask4(P.mask + i);
    const V4<double> x = ld4(v + i);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T g = mask_at(m, q) != 0 ? (T)x.v[q] : (T)0;
      this->acc += g;
      out[0].v[q] = g;
    }
  }
};

// V3: hbar = zbar + K1 gbar - (S/n_out) q1 -> hd; sum over free space; forward of -out hbar
template <typename T>
struct EpiPTh : EpiBase<T, T> {
  FilmPtrs<T> P;
  const T* zbar;        // null on the first backward iteration
  const double* om;     // first backward iteration: cotangent of the last iterate, or null
  T s_q1;               // S / n_out
  __device__ void operator()(long long i, const V4<T>* in, V4<T>* out) {
    const uchar4 m = ldmask4(P.mask + i);
    const V4<T> q1 = ldg4(P.q1 + i);
    V4<T> z;
    if (zbar) z = ld4(zbar + i);
    else if (om) {
      const V4<double> w = ld4(om + i);
#pragma unroll
      for (int q = 0; q < 4; ++q) z.v[q] = mask_at(m, q) == 0 ? (T)w.v[q] : (T)0;
    }
    V4<T> h;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      h.v[q] = ((zbar || om) ? z.v[q] : (T)0) + in[0].v[q] - s_q1 * q1.v[q];
      const bool o = mask_at(m, q) == 0;
      if (o) this->acc += h.v[q];
      out[0].v[q] = o ? -h.v[q] : (T)0;
    }
    st4(P.hd + i, h);
  }
};

// V5: gbar = out (K2(-out hbar) + (tot/n_out) q2), sum; zbar = hbar - tot/n_out -> zbuf
template <typename T>
struct EpiPTg : EpiBase<T, T> {
  FilmPtrs<T> P;
  T* zbuf;
  T t_q;                // tot / n_out
  __device__ void operator()(long long i, const V4<T>* in, V4<T>* out) {
    const uchar4 m = ldmask4(P.mask + i);
    const V4<T> q2 = ldg4(P.q2 + i);
    const V4<T> h = ld4(P.hd + i);
    V4<T> z;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T g = mask_at(m, q) == 0 ? in[0].v[q] + t_q * q2.v[q] : (T)0;
      this->acc += g;
      out[0].v[q] = g;
      z.v[q] = h.v[q] - t_q;
    }
    st4(zbuf + i, z);
  }
};

// end: hbar_in = conductor * (hbar_0 - tot_0/n_out)
template <typename T>
struct EpiPTout : EpiBase<T, T> {
  FilmPtrs<T> P;
  double* dst;
  double* wdst;         // cotangent of the warm start (free space) or null
  T t_q;
  __device__ void operator()(long long i, const V4<T>*, V4<T>*) {
    const uchar4 m = ldmask4(P.mask + i);
    const V4<T> h = ld4(P.hd + i);
    V4<double> r, w;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      r.v[q] = mask_at(m, q) != 0 ? (double)(h.v[q] - t_q) : 0.0;
      w.v[q] = mask_at(m, q) == 0 ? (double)(h.v[q] - t_q) : 0.0;
    }
    st4(dst + i, r);
    if (wdst) st4(wdst + i, w);
  }
};

template <typename T>
__global__ void __launch_bounds__(NT, 2) film_adjoint_kernel(const Desc* __restrict__ dg, AdjArgs a) {
  C2<T>* sm = dsm<T>();
  __shared__ Shared sh;
  __shared__ __align__(16) unsigned char objraw[sizeof(Film<T>)];
  const Desc& d = *dg;
  SolverState* st = d.st;
  if (threadIdx.x == 0) {
    sh.bar_passed = 0;
    new (objraw) Film<T>(d, sm, sh, (int)blockIdx.x, gridDim.x);
  }
  __syncthreads();
  Film<T>& F = *reinterpret_cast<Film<T>*>(objraw);
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const double nout = (double)d.nout, N = (double)F.ncell;
  T* const zbuf = (T*)d.hd2;
  int status = ST_OK;
  double sbar = 0.0;
  const bool full = a.g != nullptr;
  T* const jx = (T*)d.u;                         // j for the full product: the raw g_dot buffer
  T* const jy = (T*)(F.Sb + 2 * F.nspec);        // and the third field of Sb, as real storage
  do {
    double S;
    if (full) {
      EpiPT0g<T> e; e.P = F.ptrs(); e.v = a.v; e.g = a.g;
      F.rows<0, 2>(F.rb2, nullptr, F.Sa, e, 0);                         // V1 (+ g)
      if (!F.sync(60)) { status = ST_BARRIER; break; }
      S = F.total(0, F.rb2);
    } else {
      EpiPT0<T> e; e.P = F.ptrs(); e.v = a.v;
      F.rows<0, 1>(F.rb1, nullptr, F.Sa, e, 0);                         // V1
      if (!F.sync(50)) { status = ST_BARRIER; break; }
      S = F.total(0, F.rb1);
    }
    F.cols(F.Sa, 1, F.Sa, 1, OP_K1);                                    // V2
    if (full) F.cols(F.Sa + F.nspec, 1, F.Sa + F.nspec, 2, OP_GRAD);    // grad g -> Sa 1, 2
    if (!F.sync(51)) { status = ST_BARRIER; break; }
    if (full) {
      EpiStoreJ<T> e; e.P = F.ptrs(); e.jx = jx; e.jy = jy;
      F.rows<2, 0>(F.rb2, F.Sa + F.nspec, nullptr, e, -1);              // j (Eq. 2)
      if (!F.sync(61)) { status = ST_BARRIER; break; }
    }
    for (int i = a.iters - 1; i >= 0; --i) {
      const bool first = i == a.iters - 1;
      {
        EpiPTh<T> e; e.P = F.ptrs(); e.zbar = first ? nullptr : zbuf; e.s_q1 = (T)(S / nout);
        e.om = first ? a.wbar_out : nullptr;
        if (i > 0) F.rows<1, 1>(F.rb1, F.Sa, F.Sb, e, 1);               // V3
        else F.rows<1, 0>(F.rb1, F.Sa, nullptr, e, 1);
      }
      if (!F.sync(52)) { status = ST_BARRIER; break; }
      const double tot = F.total(1, F.rb1);
      sbar += N / nout * tot;
      if (i == 0) {
        if (!full) {
          EpiPTout<T> e; e.P = F.ptrs(); e.dst = a.hin_bar; e.wdst = a.wbar_in; e.t_q = (T)(tot / nout);
          F.rows<0, 0>(F.rb1, nullptr, nullptr, e, -1);
          break;
        }
        {
          EpiRbar<T> e; e.P = F.ptrs(); e.t_q = (T)(tot / nout); e.wdst = a.wbar_in;
          F.rows<0, 1>(F.rb1, nullptr, F.Sb, e, -1);                    // r
        }
        if (!F.sync(62)) { status = ST_BARRIER; break; }
        F.cols(F.Sb, 1, F.Sb, 2, OP_GRAD);                              // grad r -> Sb 0, 1
        if (!F.sync(63)) { status = ST_BARRIER; break; }
        {
          EpiPowVJP<T> e; e.P = F.ptrs(); e.jx = jx; e.jy = jy; e.jcbar = a.jcbar;
          e.n = (T)d.n; e.e0 = (T)d.e0; e.jc = (T)d.jc; e.rho_out = (T)d.rho_out;
          e.ig2 = (T)(1.0 / (d.gamma * d.gamma));
          F.rows<2, 2>(F.rb2, F.Sb, F.Sa, e, -1);                       // jbar, jcbar (Eq. 3)
        }
        if (!F.sync(64)) { status = ST_BARRIER; break; }
        F.cols(F.Sa, 2, F.Sa, 1, OP_CURLNEG);                           // -curl jbar
        if (!F.sync(65)) { status = ST_BARRIER; break; }
        {
          EpiGbar<T> e; e.P = F.ptrs(); e.dst = a.gbar;
          F.rows<1, 0>(F.rb1, F.Sa, nullptr, e, -1);                    // gbar
        }
        break;
      }
      F.cols(F.Sb, 1, F.Sb, 1, OP_K2);                                  // V4
      if (!F.sync(53)) { status = ST_BARRIER; break; }
      {
        EpiPTg<T> e; e.P = F.ptrs(); e.zbuf = zbuf; e.t_q = (T)(tot / nout);
        F.rows<1, 1>(F.rb1, F.Sb, F.Sa, e, 0);                          // V5
      }
      if (!F.sync(54)) { status = ST_BARRIER; break; }
      S = F.total(0, F.rb1);
      F.cols(F.Sa, 1, F.Sa, 1, OP_K1);                                  // V6
      if (!F.sync(55)) { status = ST_BARRIER; break; }
    }
  } while (false);
  if (leader) {
    *a.sbar = sbar;
    st->warm_valid = 0; st->com_valid = 0; st->hd_sel = 0; st->A_prev = 0.0; st->A_com = 0.0;
    st->status = status;
  }
}

// ---- elementwise helpers of the frozen-step adjoint solve (FP64 state vectors) ----
// out = c0 x0 + c1 x1 + c2 x2 + c3 x3 + b over the first nt terms; out may be x0 (in place)
__global__ void lincomb_kernel(long long n, double* out, int nt, const double* x0, double c0,
                               const double* x1, double c1, const double* x2, double c2,
                               const double* x3, double c3, double b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double s = b;
    if (nt > 0) s += c0 * x0[i];
    if (nt > 1) s += c1 * x1[i];
    if (nt > 2) s += c2 * x2[i];
    if (nt > 3) s += c3 * x3[i];
    out[i] = s;
  }
}

// out[0] = sum x, out[1] = sum x^2, in a fixed order (one block)
__global__ void __launch_bounds__(1024) sums_kernel(long long n, const double* x, double* out) {
  __shared__ double s1[1024], s2[1024];
  double a = 0.0, b = 0.0;
  for (long long i = threadIdx.x; i < n; i += 1024) {
    const double v = x[i];
    a += v;
    b += v * v;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = s1[0]; out[1] = s2[0]; }
}

// FP64 -> transform precision copy (a jc map set after creation)
__global__ void to_float_kernel(long long n, const double* x, float* y) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

cudaError_t adj_to_float(long long n, const double* x, float* y, cudaStream_t s) {
  to_float_kernel<<<304, 256, 0, s>>>(n, x, y);
  return cudaGetLastError();
}

cudaError_t adj_lincomb(long long n, double* out, int nt, const double* const* x, const double* c,
                        double b, cudaStream_t s) {
  const double* z = nullptr;
  // grid-stride: 304 blocks (two per SM of a GB300) cover any length
  lincomb_kernel<<<304, 256, 0, s>>>(n, out, nt, nt > 0 ? x[0] : z, nt > 0 ? c[0] : 0.0,
                                     nt > 1 ? x[1] : z, nt > 1 ? c[1] : 0.0, nt > 2 ? x[2] : z,
                                     nt > 2 ? c[2] : 0.0, nt > 3 ? x[3] : z, nt > 3 ? c[3] : 0.0, b);
  return cudaGetLastError();
}

cudaError_t adj_sums(long long n, const double* x, double* out, cudaStream_t s) {
  sums_kernel<<<1, 1024, 0, s>>>(n, x, out);
  return cudaGetLastError();
}

// the warm start of a film right-hand side: dst = h_dot - A on free space, 0 elsewhere (FP64) for
// save; h_dot = src on free space for load (the caller sets A = 0)
template <typename T>
__global__ void warm_io_kernel(long long n, int load, const uint8_t* mask, T* hd, double A,
                               double* dst, const double* src) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const bool o = mask[i] == 0;
    if (load) hd[i] = o ? (T)src[i] : (T)0;
    else dst[i] = o ? (double)hd[i] - A : 0.0;
  }
}

cudaError_t adj_warm_io(int precision, long long n, int load, const uint8_t* mask, void* hd,
                        double A, double* dst, const double* src, cudaStream_t s) {
  if (precision) warm_io_kernel<float><<<304, 256, 0, s>>>(n, load, mask, (float*)hd, A, dst, src);
  else warm_io_kernel<double><<<304, 256, 0, s>>>(n, load, mask, (double*)hd, A, dst, src);
  return cudaGetLastError();
}

cudaError_t film_adjoint_launch(int precision, const Desc& d, const double* v, double* hin_bar,
                                double* sbar, int iters, const double* g, double* gbar,
                                double* jcbar, const double* wbar_out, double* wbar_in,
                                cudaStream_t s) {
  const Desc* dg = d.dev;
  AdjArgs a{v, hin_bar, sbar, iters, g, gbar, jcbar, wbar_out, wbar_in};
  void* args[] = {&dg, &a};
  const size_t smem = film_smem_bytes(precision);
  const void* fn = precision ? (const void*)film_adjoint_kernel<float> : (const void*)film_adjoint_kernel<double>;
  cudaError_t e = precision
      ? cudaFuncSetAttribute(film_adjoint_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
      : cudaFuncSetAttribute(film_adjoint_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(fn, dim3(d.grid), dim3(NT), args, smem, s);
}

}  // namespace mf
