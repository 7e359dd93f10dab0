// Row (x) and line passes shared by the film (2D) and bulk (3D) kernels.
//
// Spectrum layouts (complex, transform precision T, "half" = nx/2 + 1 x-wavenumbers):
//   2D  S[f][kx][y]          after the x pass; the y pass works on contiguous lines
//   3D  S1[f][z][kx][y]      after the x pass (y lines contiguous)
//       S2[f][kx][ky][z]     after the y pass (z lines contiguous)
// A real row pass handles `rb` consecutive rows that share every other index; rows are
// transformed in pairs as one complex line (a + i b) and split or packed with the Hermitian
// symmetry of real data.
#pragma once
#include "mf_common.cuh"
#include "mf_fft.cuh"

namespace mf {

// Two adjacent complex values (one pair of rows at one x-wavenumber) moved as one vector.
template <typename T> struct alignas(2 * sizeof(C2<T>)) CPair { C2<T> a, b; };

// Two adjacent complex values from global memory, not kept in L1 (streamed once per pass).
__device__ __forceinline__ CPair<float> ld_pair_stream(const C2<float>* p) {
  CPair<float> v;
  asm volatile("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.a.x), "=f"(v.a.y), "=f"(v.b.x), "=f"(v.b.y) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ CPair<double> ld_pair_stream(const C2<double>* p) {
  CPair<double> v;
  v.a = lds_c2(p);
  v.b = lds_c2(p + 1);
  return v;
}

// Bulk copies global -> shared by the tensor memory accelerator (cp.async.bulk, the 1-D form):
// one thread arms the CTA's mbarrier with the transaction bytes and issues the copies; every
// thread then waits on the barrier's phase, which completes when all bytes have landed.
// Addresses 16-byte aligned, sizes multiples of 16 bytes.  A wait that exceeds the time limit
// raises the grid barrier's abort flag, so the launch stops at its next grid barrier, and then
// keeps waiting (up to the default barrier limit) so that no copy is still landing in shared
// memory when the CTA leaves.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
               " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// generic-proxy accesses (earlier stores to global by any CTA, earlier reads of the staging
// buffer) ordered before the async-proxy copies issued after it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async;" ::: "memory"); }
__device__ __forceinline__ void mbar_wait(unsigned long long* bar, unsigned parity, GridBarrier* gb,
                                          unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return;
  const unsigned long long lim = limit_ns ? limit_ns : BARRIER_LIMIT_NS;
  const unsigned long long t0 = globaltimer_ns();
  bool raised = false;
  while (!mbar_try_wait(bar, parity)) {
    const unsigned long long el = globaltimer_ns() - t0;
    if (!raised && el > lim) {
      atomicOr(&gb->count, BARRIER_ABORT);
      raised = true;
    }
    if (el > lim + BARRIER_LIMIT_NS) return;       // the copies never landed: give up
  }
}

// Asynchronous copies global -> shared (cp.async): issued without a register round trip,
// complete at cp_async_wait (this thread's groups; a CTA barrier after it makes every thread's
// copies visible).  gather_async issues value e from src[goff(e)] to sm[sp(soff(e))] for
// e < total as one group.
__device__ __forceinline__ void cp_async_c2(C2<float>* s, const C2<float>* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
               :: "r"((unsigned)__cvta_generic_to_shared(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_c2(C2<double>* s, const C2<double>* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
               :: "r"((unsigned)__cvta_generic_to_shared(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }
// Inverse-transform along x the half spectra of rows [2 pr, 2 pr + 1] of NIN fields, packed
// as complex lines a + i b (Hermitian symmetry of real rows): returns the shared buffer (sm or
// sm2) holding the rows, row 2pr in .x and row 2pr+1 in .y.  Global element (f, kx, row r)
// lives at src + f * fstride + kx * kstride + r.  The first transform stage reads its inputs
// straight from global memory, all of a butterfly's loads in flight together: position m of
// a packed line is A[m] + i B[m] for m <= nx/2 and conj(A[nx-m]) + i conj(B[nx-m]) above,
// with the imaginary parts of the real DC and Nyquist terms dropped.
template <typename T, int NIN, class G = Cta>
__device__ __forceinline__ C2<T>* rows_gather_inverse(C2<T>* sm, C2<T>* sm2, const C2<T>* src,
                                                      long long fstride, long long kstride,
                                                      int npair, int lgpair, int lgx,
                                                      const C2<T>* __restrict__ twx, G grp = G()) {
  const int nx = 1 << lgx, half = nx >> 1;
  auto ld = [=](int line, int m) -> C2<T> {
    const int f = line >> lgpair, pr = line & (npair - 1);
    const int k = m <= half ? m : nx - m;
    const CPair<T> v = ld_pair_stream(src + f * fstride + (long long)k * kstride + 2 * pr);
    const C2<T> A = v.a, B = v.b;
    if (k == 0 || k == half) return C2<T>{A.x, B.x};
    if (m < half) return C2<T>{A.x - B.y, A.y + B.x};          // A + i B
    return C2<T>{A.x + B.y, B.x - A.y};                         // conj(A) + i conj(B)
  };
  const FftPlan P = fft_plan<T>(lgx);
  const int l0 = P.lgr(0);
  fft_first_io_any<T, +1>(l0, lgx, NIN * npair, ld, sm, grp);
  return fft_lines_from<T, +1>(sm, sm2, lgx, NIN * npair, twx, 1, grp);
}

// The same inverse transform from a staged copy of the half spectra in shared memory (element
// (f, kx, row r) at position sp((f (nx/2 + 1) + kx) rb + r), rb = 2 npair), written by
// stage_rows_async; the staging buffer is free again when this returns.
// after_first() runs (in every thread) once the first stage has read the staging buffer.
template <typename T, int NIN, class AfterFirst>
__device__ __forceinline__ C2<T>* rows_inverse_staged(const C2<T>* stg, C2<T>* sm, C2<T>* sm2, int npair,
                                                      int lgpair, int lgx, const C2<T>* __restrict__ twx,
                                                      AfterFirst after_first) {
  const int nx = 1 << lgx, half = nx >> 1, rb = 2 * npair;
  C2<T>* const S = dsm<T>();
  const int st = dsm_off(stg);
  auto ld = [=](int line, int m) -> C2<T> {
    const int f = line >> lgpair, pr = line & (npair - 1);
    const int k = m <= half ? m : nx - m;
    const int e = (f * (half + 1) + k) * rb + 2 * pr;      // even: the pair shares a padding group
    const C2<T> A = S[st + sp(e)], B = S[st + sp(e) + 1];
    if (k == 0 || k == half) return C2<T>{A.x, B.x};
    if (m < half) return C2<T>{A.x - B.y, A.y + B.x};          // A + i B
    return C2<T>{A.x + B.y, B.x - A.y};                         // conj(A) + i conj(B)
  };
  const FftPlan P = fft_plan<T>(lgx);
  fft_first_io_any<T, +1>(P.lgr(0), lgx, NIN * npair, ld, sm);
  after_first();
  return fft_lines_from<T, +1>(sm, sm2, lgx, NIN * npair, twx, 1);
}
// Issue (cp.async, one group) the copy of the half spectra rows [0, rb) of NIN fields, global
// element (f, kx, r) at src + f fstride + kx kstride + r, into the staging layout above.
template <typename T, int NIN>
__device__ __forceinline__ void stage_rows_async(C2<T>* stg, const C2<T>* src, long long fstride,
                                                 long long kstride, int rb, int lgx) {
  const int nk = (1 << (lgx - 1)) + 1;
  const int per_f = nk * rb;
  for (int e = threadIdx.x; e < NIN * per_f; e += NT) {
    const int f = e / per_f, rest = e - f * per_f;
    const int k = rest / rb, r = rest - k * rb;
    cp_async_c2(stg + sp(e), src + f * fstride + (long long)k * kstride + r);
  }
  cp_async_commit();
}

// Forward-transform NOUT fields of packed row pairs (in `sm_in`, second buffer `sm2`) along x
// and scatter their half spectra.
template <typename T, int NOUT, class G = Cta>
__device__ __forceinline__ void rows_forward_scatter(C2<T>* sm_in, C2<T>* sm2, C2<T>* dst,
                                                     long long fstride, long long kstride,
                                                     int npair, int lgpair, int lgx,
                                                     const C2<T>* __restrict__ twx, G grp = G()) {
  const int nx = 1 << lgx, half = nx >> 1;
  const C2<T>* sm = fft_lines<T, -1>(sm_in, sm2, lgx, NOUT * npair, twx, grp);
  C2<T>* const S = dsm<T>();
  const int io = dsm_off(sm);
  const int per_f = npair * (half + 1);
  for (int e = grp.tid(); e < NOUT * per_f; e += G::nt) {
    const int f = e >= per_f ? (e >= 2 * per_f ? 2 : 1) : 0;
    const int rest = e - f * per_f;
    const int k = rest >> lgpair, pr = rest & (npair - 1);
    const int z0 = (f * npair + pr) << lgx;
    const C2<T> zk = S[io + sp(z0 + k)], zm = S[io + sp(z0 + ((nx - k) & (nx - 1)))];
    const T hh = (T)0.5;
    CPair<T> o;
    o.a = C2<T>{hh * (zk.x + zm.x), hh * (zk.y - zm.y)};
    o.b = C2<T>{hh * (zk.y + zm.y), hh * (zm.x - zk.x)};   // -i (zk - conj(zm)) / 2
    *(CPair<T>*)(dst + f * fstride + (long long)k * kstride + 2 * pr) = o;
  }
  grp.sync();
}

// Load `n` contiguous lines of length L (line j at src + j * stride) into shared memory,
// U loads in flight per thread.
template <typename T>
__device__ __forceinline__ void lines_load(C2<T>* sm, const C2<T>* src, long long stride, int n, int lgL) {
  constexpr int U = 4;
  const int L = 1 << lgL;
  const int total = n << lgL;
  for (int e0 = threadIdx.x; e0 < total; e0 += NT * U) {
    C2<T> v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * NT;
      if (e < total) v[u] = src[(e >> lgL) * stride + (e & (L - 1))];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * NT;
      if (e < total) sm[sp(e)] = v[u];
    }
  }
  __syncthreads();
}
template <typename T>
__device__ __forceinline__ void lines_store(const C2<T>* sm, C2<T>* dst, long long stride, int n, int lgL) {
  const int L = 1 << lgL;
  for (int e = threadIdx.x; e < (n << lgL); e += NT) {
    const int j = e >> lgL, i = e & (L - 1);
    dst[j * stride + i] = sm[sp(e)];
  }
  __syncthreads();
}

template <typename T, class GOff, class SOff>
__device__ __forceinline__ void gather_async(C2<T>* sm, const C2<T>* src, int total, GOff goff, SOff soff) {
  for (int e = threadIdx.x; e < total; e += NT) cp_async_c2(sm + sp(soff(e)), src + goff(e));
  cp_async_commit();
}

// Gather `total` complex values into shared memory, value e from src[goff(e)] to
// sm[sp(soff(e))], with U loads in flight per thread; synchronises at the end.
template <typename T, int U, class GOff, class SOff>
__device__ __forceinline__ void gather_batched(C2<T>* sm, const C2<T>* src, int total, GOff goff, SOff soff) {
  for (int e0 = threadIdx.x; e0 < total; e0 += NT * U) {
    C2<T> v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * NT;
      if (e < total) v[u] = lds_c2(src + goff(e));
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * NT;
      if (e < total) sm[sp(soff(e))] = v[u];
    }
  }
  __syncthreads();
}


// ------------------------------------------------------------------------------------------
// four consecutive cells: vector loads and stores (index a multiple of 4, 16-byte aligned)
// ------------------------------------------------------------------------------------------
template <typename T> struct V4 { T v[4]; };
// field loads of the epilogues stream through once per pass: not kept in L1
__device__ __forceinline__ V4<float> ld4(const float* p) {
  V4<float> r;
  asm volatile("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "l"(p) : "memory");
  return r;
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  V4<double> r;
  asm volatile("ld.global.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(r.v[0]), "=d"(r.v[1]) : "l"(p) : "memory");
  asm volatile("ld.global.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(r.v[2]), "=d"(r.v[3]) : "l"(p + 2) : "memory");
  return r;
}
// read-only for the whole launch (non-coherent path)
__device__ __forceinline__ V4<float> ldg4(const float* p) {
  V4<float> r;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]) : "l"(p));
  return r;
}
__device__ __forceinline__ V4<double> ldg4(const double* p) {
  V4<double> r;
  asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(r.v[0]), "=d"(r.v[1]) : "l"(p));
  asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(r.v[2]), "=d"(r.v[3]) : "l"(p + 2));
  return r;
}
__device__ __forceinline__ void st4(float* p, const V4<float>& v) {
  *(float4*)p = make_float4(v.v[0], v.v[1], v.v[2], v.v[3]);
}
__device__ __forceinline__ void st4(double* p, const V4<double>& v) {
  ((double2*)p)[0] = make_double2(v.v[0], v.v[1]);
  ((double2*)p)[1] = make_double2(v.v[2], v.v[3]);
}
__device__ __forceinline__ uchar4 ldmask4(const uint8_t* p) {
  unsigned int w;
  asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(w) : "l"(p));
  return make_uchar4(w & 255u, (w >> 8) & 255u, (w >> 16) & 255u, w >> 24);
}
__device__ __forceinline__ int mask_at(const uchar4& m, int j) {
  return j == 0 ? m.x : (j == 1 ? m.y : (j == 2 ? m.z : m.w));
}

__device__ __forceinline__ float powt(float a, float b) { return powf(a, b); }
__device__ __forceinline__ double powt(double a, double b) { return pow(a, b); }

// power law of Eq. 3 / Eq. 13:  rho = (e0/jc) (|j|/jc)^(n-1) in the superconductor (mask 1),
// rho_out elsewhere.  Takes |j|^2.
template <typename T>
__device__ __forceinline__ T resistivity(T j2, T jc, int m, T n, T e0, T rho_out) {
  if (m != 1) return rho_out;
  const T x2 = j2 / (jc * jc);
  // (|j|/jc)^(n-1) = (|j|^2/jc^2)^((n-1)/2); exactly 1 for n = 1 (including j = 0)
  T pw;
  if (n == (T)1) pw = (T)1;
  else if (x2 <= (T)0) pw = (T)0;
  else pw = powt(x2, (n - (T)1) * (T)0.5);
  return e0 / jc * pw;
}

}  // namespace mf
