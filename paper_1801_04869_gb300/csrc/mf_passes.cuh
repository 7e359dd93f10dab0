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

// Gather the half spectra of rows [2 pr, 2 pr + 1] of `nin` fields from global memory into
// packed complex lines of length nx in shared buffer `sm`, then inverse-transform them along
// x (second buffer `sm2`).  Returns the buffer holding the rows (row 2pr in .x, 2pr+1 in .y).
// Global element (f, kx, row r) lives at src + f * fstride + kx * kstride + r.
template <typename T>
__device__ __forceinline__ C2<T>* rows_gather_inverse(C2<T>* sm, C2<T>* sm2, const C2<T>* src, long long fstride,
                                                    long long kstride, int nin, int npair,
                                                    int lgx, const C2<T>* __restrict__ twx) {
  const int nx = 1 << lgx, half = nx >> 1;
  const int per_f = npair * (half + 1);
  for (int e = threadIdx.x; e < nin * per_f; e += NT) {
    const int f = e / per_f;
    const int rest = e - f * per_f;
    const int k = rest / npair;
    const int pr = rest - k * npair;
    const C2<T>* p = src + f * fstride + (long long)k * kstride + 2 * pr;
    const C2<T> A = p[0], B = p[1];
    const int z0 = (f * npair + pr) << lgx;
    if (k == 0 || k == half) {
      sm[sp(z0 + k)] = C2<T>{A.x, B.x};
    } else {
      sm[sp(z0 + k)] = C2<T>{A.x - B.y, A.y + B.x};          // A + i B
      sm[sp(z0 + nx - k)] = C2<T>{A.x + B.y, B.x - A.y};     // conj(A) + i conj(B)
    }
  }
  __syncthreads();
  return fft_lines<T, +1>(sm, sm2, lgx, nin * npair, twx);
}

// Forward-transform `nout` fields of packed row pairs (in `sm`, second buffer `sm2`) along x
// and scatter their half spectra.
template <typename T>
__device__ __forceinline__ void rows_forward_scatter(C2<T>* sm_in, C2<T>* sm2, C2<T>* dst, long long fstride,
                                                     long long kstride, int nout, int npair,
                                                     int lgx, const C2<T>* __restrict__ twx) {
  const int nx = 1 << lgx, half = nx >> 1;
  const C2<T>* sm = fft_lines<T, -1>(sm_in, sm2, lgx, nout * npair, twx);
  const int per_f = npair * (half + 1);
  for (int e = threadIdx.x; e < nout * per_f; e += NT) {
    const int f = e / per_f;
    const int rest = e - f * per_f;
    const int k = rest / npair;
    const int pr = rest - k * npair;
    const int z0 = (f * npair + pr) << lgx;
    const C2<T> zk = sm[sp(z0 + k)], zm = sm[sp(z0 + ((nx - k) & (nx - 1)))];
    const T hh = (T)0.5;
    C2<T> A = {hh * (zk.x + zm.x), hh * (zk.y - zm.y)};
    C2<T> B = {hh * (zk.y + zm.y), hh * (zm.x - zk.x)};   // -i (zk - conj(zm)) / 2
    C2<T>* p = dst + f * fstride + (long long)k * kstride + 2 * pr;
    p[0] = A;
    p[1] = B;
  }
  __syncthreads();
}

// Load `n` contiguous lines of length L (line j at src + j * stride) into shared memory.
template <typename T>
__device__ __forceinline__ void lines_load(C2<T>* sm, const C2<T>* src, long long stride, int n, int lgL) {
  const int L = 1 << lgL;
  for (int e = threadIdx.x; e < (n << lgL); e += NT) {
    const int j = e >> lgL, i = e & (L - 1);
    sm[sp(e)] = src[j * stride + i];
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
