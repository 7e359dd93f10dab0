// Thin-film right-hand side for callers that cannot allocate device memory.
//
// The regular interface (mf_create + mf_rhs) runs in a workspace that the caller allocates.
// Some callers cannot do that: a host application that owns every device byte through its
// own pool and forbids cudaMalloc (which synchronises the device and fragments the pool), or
// a latency-critical loop where an allocation's implicit synchronisation is not acceptable.
// mf_film_rhs_noalloc serves them: it evaluates one film right-hand side with the same
// persistent kernel, but every intermediate buffer (spectra, h_dot iterate, free-space
// responses q1 and q2, tables, reductions, solver state and grid barrier) lives in one
// file-scope device array of fixed size, NOALLOC_BYTES, that every GPU loading this library
// holds until the process exits.  Nothing is allocated, on the device or the host.
//
// Rules of use (also stated in include/mf.h):
//   * the first call on a device looks up the array's device address (cudaGetSymbolAddress)
//     with that device current;
//   * every call copies the tables, mask, jc map, state and descriptor into the array and
//     synchronises `stream` several times (host-side staging and the status read-back), so a
//     call can never be part of a stream capture;
//   * all calls share the array and it keeps the last call's contents, so calls whose GPU
//     work overlaps (two streams, two host threads, two devices sharing nothing is fine) race;
//   * each call starts the outside iteration cold (no warm start is kept between calls).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/mf.h"
#include "mf_common.cuh"
#include "mf_tables.h"

using namespace mf;

namespace {

constexpr size_t NOALLOC_BYTES = 8u << 20;       // 8 MiB: films up to 256 x 256 cells
constexpr int NOALLOC_MAX_N = 256;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_scratch[NOALLOC_BYTES];

std::mutex g_mutex;
void* g_scratch_ptr[MAX_DEVICES] = {nullptr};

void set_err(char* err, size_t len, const char* msg) {
  if (err && len) std::snprintf(err, len, "%s", msg);
}

size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" mf_status mf_film_rhs_noalloc(const mf_params* p, double t, const double* d_y,
                                         double* d_ydot, int force_iters, void* stream,
                                         int* iters_out, char* err, size_t err_len) {
  set_err(err, err_len, "");
  if (!p || !d_y || !d_ydot) { set_err(err, err_len, "null argument"); return MF_ERR_ARG; }
  if (mf_workspace_bytes(p) == 0) { set_err(err, err_len, "invalid parameters"); return MF_ERR_ARG; }
  if (p->dim != 2) { set_err(err, err_len, "only thin films (dim 2) are supported"); return MF_ERR_ARG; }
  if (p->nx > NOALLOC_MAX_N || p->ny > NOALLOC_MAX_N) {
    char m[160];
    std::snprintf(m, sizeof(m), "grid %dx%d exceeds the static scratch limit of %dx%d cells (%zu bytes)",
                  p->nx, p->ny, NOALLOC_MAX_N, NOALLOC_MAX_N, NOALLOC_BYTES);
    set_err(err, err_len, m);
    return MF_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    set_err(err, err_len, "no current CUDA device");
    return MF_ERR_CUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
      if (e != cudaSuccess || !ptr) {
        set_err(err, err_len, cudaGetErrorString(e));
        return MF_ERR_CUDA;
      }
      g_scratch_ptr[dev] = ptr;
    }
    base = g_scratch_ptr[dev];
  }

  // layout inside the static array (only what one right-hand side needs)
  const int nx = p->nx, ny = p->ny;
  const int precision = p->precision;
  const size_t ts = precision ? 4 : 8;
  const long long ncell = (long long)nx * ny;
  const long long nspec = (long long)(nx / 2 + 1) * ny;
  const int nk = nx / 2 + 1 + ny + 1;
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = up256(o + bytes); return at; };
  const size_t oSa = take(2 * nspec * 2 * ts), oSb = take(2 * nspec * 2 * ts);
  const size_t ohd = take(ncell * ts), ou = take(ncell * ts), oq1 = take(ncell * ts), oq2 = take(ncell * ts);
  const size_t ojc = take(p->jc_map ? ncell * ts : 0), omask = take(ncell);
  const size_t otwx = take(2 * nx * 2 * ts), otwy = take(2 * ny * 2 * ts), otwz = take(2 * ts);
  const size_t okt = take(nk * ts), ogt = take(nk * ts);
  const size_t opart = take((size_t)8 * ny * 8), ost = take(sizeof(SolverState)), ogb = take(sizeof(GridBarrier));
  const size_t oknots = take(2 * (size_t)(p->he_knots > 0 ? p->he_knots : 1) * 8);
  const size_t odesc = take(sizeof(Desc));
  if (o > NOALLOC_BYTES) {
    set_err(err, err_len, "static scratch too small for these parameters");
    return MF_ERR_WORKSPACE;
  }
  char* w = (char*)base;

  Desc d;
  std::memset(&d, 0, sizeof(d));
  d.dim = 2; d.nx = nx; d.ny = ny; d.nz = 1; d.precision = precision;
  d.barrier_ns = BARRIER_LIMIT_NS;
  int l = 0; while ((1 << l) < nx) ++l; d.lgx = l;
  l = 0; while ((1 << l) < ny) ++l; d.lgy = l;
  d.Lx = p->Lx; d.Ly = p->Ly;
  d.dx = 2 * p->Lx / nx; d.dy = 2 * p->Ly / ny;
  d.sigma = p->sigma > 0 ? p->sigma : std::sqrt(d.dx * d.dx + d.dy * d.dy);
  d.n = p->n; d.e0 = p->e0; d.jc = p->jc; d.rho_out = p->rho_out; d.lam = p->lambda;
  d.gamma = p->gamma; d.b0 = p->b0;
  d.iter_tol = p->iter_tol; d.iter_max = p->iter_max;
  d.rtol = p->rtol; d.atol = p->atol; d.h_min = p->h_min;
  d.he_knots = p->he_knots; d.he_sin_amp = p->he_sin_amp; d.he_sin_period = p->he_sin_period;
  d.ncell = ncell; d.nspec = nspec;
  long long nout = 0;
  for (long long i = 0; i < ncell; ++i) {
    if (p->mask[i] > 2) { set_err(err, err_len, "mask values must be 0, 1 or 2"); return MF_ERR_ARG; }
    nout += p->mask[i] == 0;
  }
  d.nout = nout;
  d.Sa = w + oSa; d.Sb = w + oSb; d.hd = w + ohd; d.hd2 = d.hd; d.u = w + ou; d.q1 = w + oq1; d.q2 = w + oq2;
  d.jcmap = p->jc_map ? (const void*)(w + ojc) : nullptr;
  d.mask = (const uint8_t*)(w + omask);
  d.tw_x = w + otwx; d.tw_y = w + otwy; d.tw_z = w + otwz;
  d.ktab = w + okt; d.gtab = w + ogt;
  d.partials = (double*)(w + opart); d.max_items = ny;
  d.st = (SolverState*)(w + ost); d.gb = (GridBarrier*)(w + ogb);
  d.he_t = (const double*)(w + oknots);
  d.he_v = d.he_t + (p->he_knots > 0 ? p->he_knots : 1);
  d.dev = (const Desc*)(w + odesc);

  d.nz = 1;
  const size_t smem = kernel_smem_bytes(d);
  const int per_sm = film_max_blocks(precision, smem);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (per_sm < 1 || nsm < 1) { set_err(err, err_len, "kernel does not fit on this device"); return MF_ERR_CUDA; }
  {
    const int coresident = per_sm * nsm;
    int rb1 = std::min(ny, 2 * BATCH / nx), rb2 = std::min(ny, BATCH / nx);
    const int want = nx / 2 + 1;
    const int grid = std::min(coresident, want);
    while (rb1 > 2 && ny / rb1 < grid) rb1 /= 2;
    while (rb2 > 2 && ny / rb2 < grid) rb2 /= 2;
    d.rows_per_item = rb1;
    d.zs_per_item = rb2;
    d.grid = std::max(1, std::min(coresident, std::max(want, ny / rb1)));
  }

  // inputs and tables, staged through fixed-size stack buffers (synchronous copies)
  cudaError_t e = cudaSuccess;
  auto copy_sync = [&](void* dst, const void* src, size_t n) {
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  };
  copy_sync(w + omask, p->mask, (size_t)ncell);
  {
    double tw[4 * NOALLOC_MAX_N], kt[NOALLOC_MAX_N / 2 + 1 + NOALLOC_MAX_N + 1],
        gt[NOALLOC_MAX_N / 2 + 1 + NOALLOC_MAX_N + 1];
    float twf[4 * NOALLOC_MAX_N], ktf[NOALLOC_MAX_N / 2 + 1 + NOALLOC_MAX_N + 1],
        gtf[NOALLOC_MAX_N / 2 + 1 + NOALLOC_MAX_N + 1];
    const int ns[2] = {nx, ny};
    const size_t to[2] = {otwx, otwy};
    for (int a = 0; a < 2; ++a) {
      // stage-ordered twiddle tables (A then B), as mf_create writes them
      if (precision) {
        const int n = stage_twiddles<float>(ns[a], twf);
        copy_sync(w + to[a], twf, (size_t)n * 2 * 4);
      } else {
        const int n = stage_twiddles<double>(ns[a], tw);
        copy_sync(w + to[a], tw, (size_t)n * 2 * 8);
      }
    }
    int c = 0;
    const double Ls[2] = {p->Lx, p->Ly};
    for (int a = 0; a < 2; ++a) {
      const int n = ns[a], cnt = a == 0 ? n / 2 + 1 : n;
      for (int i = 0; i < cnt; ++i) {
        int m = i < n / 2 ? i : i - n;
        if (a == 0 && i == n / 2) m = -n / 2;
        const double kv = M_PI * (double)m / Ls[a];
        kt[c] = kv; gt[c] = std::exp(-kv * kv * d.sigma * d.sigma / 2.0);
        ktf[c] = (float)kt[c]; gtf[c] = (float)gt[c];
        ++c;
      }
    }
    if (precision) { copy_sync(w + okt, ktf, c * 4); copy_sync(w + ogt, gtf, c * 4); }
    else { copy_sync(w + okt, kt, c * 8); copy_sync(w + ogt, gt, c * 8); }
    double kn[64];
    const int K = p->he_knots;
    if (K > 0 && K <= 32) {
      for (int i = 0; i < K; ++i) { kn[i] = p->he_t[i]; kn[K + i] = p->he_v[i]; }
      copy_sync(w + oknots, kn, (size_t)2 * K * 8);
    } else if (K > 32) {
      copy_sync(w + oknots, p->he_t, (size_t)K * 8);
      copy_sync(w + oknots + (size_t)K * 8, p->he_v, (size_t)K * 8);
    }
  }
  if (p->jc_map) {
    if (!precision) {
      copy_sync(w + ojc, p->jc_map, (size_t)ncell * 8);
    } else {
      float chunk[1024];
      for (long long i0 = 0; i0 < ncell && e == cudaSuccess; i0 += 1024) {
        const long long n = std::min<long long>(1024, ncell - i0);
        for (long long i = 0; i < n; ++i) chunk[i] = (float)p->jc_map[i0 + i];
        copy_sync(w + ojc + i0 * 4, chunk, (size_t)n * 4);
      }
    }
  }
  // state that must start at zero: solver state (cold start), barrier
  SolverState s0;
  std::memset(&s0, 0, sizeof(s0));
  copy_sync(w + ost, &s0, sizeof(s0));
  copy_sync(w + odesc, &d, sizeof(Desc));   // the kernel reads the descriptor from here
  if (e != cudaSuccess) { set_err(err, err_len, cudaGetErrorString(e)); return MF_ERR_CUDA; }

  KernelArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int pass = 0; pass < 2; ++pass) {
    a.mode = pass == 0 ? MODE_SETUP : MODE_RHS;
    a.t = t; a.y_in = d_y; a.out = d_ydot; a.force_iters = force_iters; a.seg = -2;
    e = cudaMemsetAsync(d.gb, 0, sizeof(GridBarrier), st);
    if (e == cudaSuccess) e = film_launch(precision, d, a, st);
    SolverState s;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s, d.st, sizeof(s), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_err(err, err_len, cudaGetErrorString(e)); return MF_ERR_CUDA; }
    if (s.status != ST_OK && !(pass == 1 && s.status == ST_NOCONV)) {
      set_err(err, err_len, s.status == ST_BARRIER ? "grid barrier timed out" : "kernel reported an error");
      return (mf_status)s.status;
    }
    if (pass == 1) {
      if (iters_out) *iters_out = s.last_iters;
      if (s.status == ST_NOCONV) set_err(err, err_len, "outside iteration did not converge");
      return (mf_status)s.status;
    }
  }
  return MF_OK;
}
