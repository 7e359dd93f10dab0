// Host side of the C interface declared in include/mf.h: parameter checks, the workspace
// layout, transform tables, and the launches of the persistent kernels.
#include <algorithm>
#include <array>
#include <cmath>
#include <initializer_list>
#include <cstdio>
#include <cstring>
#include <string>
#include <queue>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mf.h"
#include "mf_common.cuh"
#include "mf_tables.h"

using namespace mf;

struct mf_problem {
  mf_params p;
  Desc d;
  cudaStream_t stream;
  int device;
  char* ws;
  size_t ws_bytes;
  size_t used;
  double* scratch_m;            // device scalar(s) for moment readouts (in the workspace)
  std::string err;
  bool have_knots;
  double batch_work = 0.0;      // field passes per step attempt in the last mf_advance_batch
};

namespace mf {
// transposed outside iteration of a film (csrc/mf_film_adjoint.cu)
cudaError_t film_adjoint_launch(int precision, const Desc& d, const double* v, double* hin_bar,
                                double* sbar, int iters, const double* g, double* gbar,
                                double* jcbar, const double* wbar_out, double* wbar_in,
                                cudaStream_t s);
cudaError_t adj_warm_io(int precision, long long n, int load, const uint8_t* mask, void* hd,
                        double A, double* dst, const double* src, cudaStream_t s);
cudaError_t adj_lincomb(long long n, double* out, int nt, const double* const* x, const double* c,
                        double b, cudaStream_t s);
cudaError_t adj_sums(long long n, const double* x, double* out, cudaStream_t s);
cudaError_t adj_to_float(long long n, const double* x, float* y, cudaStream_t s);
}  // namespace mf

namespace {

// NVTX range over one host call (shown by nsys / ncu timelines; free when no tool is attached)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

constexpr long long LOG_CAP = 1 << 16;
constexpr int NSLOTS = 8;

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(int v) { int l = 0; while ((1 << l) < v) ++l; return l; }
size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Layout {
  size_t Sa, Sb, hd, hd2, u, q1, q2, jc, mask, twx, twy, twz, ktab, gtab, fbuf[6], partials, st, gb,
      log, knots, mscr, desc, total;
  long long ncell, nspec, nstate;
  int max_items;
};

mf_status check_params(const mf_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return MF_ERR_ARG; }
  if (p->dim != 2 && p->dim != 3) { why = "dim must be 2 or 3"; return MF_ERR_ARG; }
  const int nz = p->dim == 2 ? 1 : p->nz;
  if (!is_pow2(p->nx) || !is_pow2(p->ny) || !is_pow2(nz)) { why = "grid extents must be powers of two"; return MF_ERR_ARG; }
  if (p->dim == 2) {
    if (p->nx < 8 || p->ny < 8 || p->nx > 2048 || p->ny > 2048) { why = "film grid must be 8..2048 per axis"; return MF_ERR_ARG; }
    if (p->nz != 1) { why = "film needs nz = 1"; return MF_ERR_ARG; }
  } else {
    if (p->nx < 8 || p->ny < 8 || nz < 8 || p->nx > 512 || p->ny > 512 || nz > 512) { why = "bulk grid must be 8..512 per axis"; return MF_ERR_ARG; }
  }
  if (!(p->Lx > 0) || !(p->Ly > 0) || (p->dim == 3 && !(p->Lz > 0))) { why = "half extents must be positive"; return MF_ERR_ARG; }
  if (!p->mask) { why = "mask is NULL"; return MF_ERR_ARG; }
  if (!(p->n >= 1) || !(p->jc > 0) || !(p->e0 > 0) || !(p->rho_out >= 0)) { why = "need n >= 1, jc > 0, e0 > 0, rho_out >= 0"; return MF_ERR_ARG; }
  if (p->iter_max < 1) { why = "iter_max must be >= 1"; return MF_ERR_ARG; }
  if (p->precision != 0 && p->precision != 1) { why = "precision must be 0 or 1"; return MF_ERR_ARG; }
  if (p->he_knots < 0 || (p->he_knots > 0 && (!p->he_t || !p->he_v))) { why = "bad h_e knots"; return MF_ERR_ARG; }
  for (int i = 1; i < p->he_knots; ++i)
    if (!(p->he_t[i] > p->he_t[i - 1])) { why = "h_e knot times must increase"; return MF_ERR_ARG; }
  if (p->he_knots == 0 && !(p->he_sin_period > 0)) { why = "sinusoid period must be positive"; return MF_ERR_ARG; }
  if (!(p->rtol >= 0) || !(p->atol > 0)) { why = "need rtol >= 0 and atol > 0"; return MF_ERR_ARG; }
  if (!(p->gamma > 0) || !std::isfinite(p->gamma)) { why = "gamma must be positive and finite"; return MF_ERR_ARG; }
  if (!(p->b0 >= 0) || !std::isfinite(p->b0)) { why = "b0 must be >= 0 and finite"; return MF_ERR_ARG; }
  if (p->dim == 2 && p->b0 > 0) { why = "the field-dependent jc (b0 > 0) is a bulk law"; return MF_ERR_ARG; }
  return MF_OK;
}

Layout layout(const mf_params* p) {
  Layout L{};
  const int nz = p->dim == 2 ? 1 : p->nz;
  const size_t ts = p->precision ? 4 : 8;
  const int ncomp = p->dim == 2 ? 1 : 3;
  L.ncell = (long long)p->nx * p->ny * nz;
  L.nspec = (long long)(p->nx / 2 + 1) * p->ny * nz;
  L.nstate = L.ncell * ncomp;
  L.max_items = (int)(p->dim == 2 ? p->ny : (long long)p->ny * nz);
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
  L.Sa = take(3 * L.nspec * 2 * ts);
  L.Sb = take(3 * L.nspec * 2 * ts);
  L.hd = take(ncomp * L.ncell * ts);
  L.hd2 = take(p->dim == 2 ? L.ncell * ts : 0);
  L.u = take(p->dim == 2 ? L.ncell * ts : 0);
  L.q1 = take(p->dim == 2 ? L.ncell * ts : 0);
  L.q2 = take(p->dim == 2 ? L.ncell * ts : 0);
  L.jc = take(p->jc_map ? L.ncell * ts : 0);
  L.mask = take(L.ncell);
  L.twx = take(2 * p->nx * 2 * ts);             // stage-ordered tables A and B (< 2 L entries)
  L.twy = take(2 * p->ny * 2 * ts);
  L.twz = take(2 * nz * 2 * ts);
  const int nk = p->nx / 2 + 1 + p->ny + nz;
  L.ktab = take(nk * ts);
  L.gtab = take(nk * ts);
  for (int i = 0; i < 6; ++i) L.fbuf[i] = take(L.nstate * 8);
  L.partials = take((size_t)NSLOTS * L.max_items * 8);
  L.st = take(sizeof(SolverState));
  L.gb = take(sizeof(GridBarrier));
  L.log = take(LOG_CAP * sizeof(StepLog));
  L.knots = take(2 * (size_t)(p->he_knots > 0 ? p->he_knots : 1) * 8);
  L.mscr = take(8 * 8);
  L.desc = take(sizeof(Desc));
  L.total = o;
  return L;
}

template <typename T>
void fill_tables(const mf_params* p, double sigma, std::vector<char>& tw, std::vector<char>& kt,
                 std::vector<char>& gt) {
  const int nz = p->dim == 2 ? 1 : p->nz;
  const int ns[3] = {p->nx, p->ny, nz};
  // per axis: stage-ordered twiddle tables, each block padded to 2 L complex entries
  std::vector<T> t;
  for (int a = 0; a < 3; ++a) {
    std::vector<T> blk(4 * (size_t)ns[a], (T)0);
    stage_twiddles<T>(ns[a], blk.data());
    t.insert(t.end(), blk.begin(), blk.end());
  }
  tw.assign((const char*)t.data(), (const char*)(t.data() + t.size()));
  std::vector<T> k, g;
  const double Ls[3] = {p->Lx, p->Ly, p->dim == 2 ? 1.0 : p->Lz};
  for (int a = 0; a < 3; ++a) {
    const int n = ns[a];
    const int cnt = a == 0 ? n / 2 + 1 : n;
    for (int i = 0; i < cnt; ++i) {
      int m = i < n / 2 ? i : i - n;     // FFT order; index n/2 is the Nyquist m = -n/2
      if (a == 0 && i == n / 2) m = -n / 2;
      const double kv = M_PI * (double)m / Ls[a];
      k.push_back((T)kv);
      g.push_back((T)std::exp(-kv * kv * sigma * sigma / 2.0));
    }
  }
  kt.assign((const char*)k.data(), (const char*)(k.data() + k.size()));
  gt.assign((const char*)g.data(), (const char*)(g.data() + g.size()));
}

mf_status cuda_fail(mf_problem* pb, cudaError_t e, const char* what) {
  if (pb) pb->err = std::string(what) + ": " + cudaGetErrorString(e);
  return MF_ERR_CUDA;
}

#define MF_CUDA(pb, call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(pb, e_, #call); \
  } while (0)

#define MF_TRY_STATUS(x)             \
  do {                               \
    mf_status r_ = (x);              \
    if (r_ != MF_OK) return r_;      \
  } while (0)

mf_status read_state(mf_problem* pb, SolverState* s) {
  MF_CUDA(pb, cudaMemcpyAsync(s, pb->d.st, sizeof(SolverState), cudaMemcpyDeviceToHost, pb->stream));
  MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  return MF_OK;
}
mf_status write_state(mf_problem* pb, const SolverState* s) {
  MF_CUDA(pb, cudaMemcpyAsync(pb->d.st, s, sizeof(SolverState), cudaMemcpyHostToDevice, pb->stream));
  MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  return MF_OK;
}

// enqueue one persistent launch on the problem's stream (no wait)
mf_status launch_enqueue(mf_problem* pb, const KernelArgs& a) {
  MF_CUDA(pb, cudaSetDevice(pb->device));
  MF_CUDA(pb, cudaMemsetAsync(pb->d.gb, 0, sizeof(GridBarrier), pb->stream));
  cudaError_t e = pb->d.dim == 2 ? film_launch(pb->d.precision, pb->d, a, pb->stream)
                                 : bulk_launch(pb->d.precision, pb->d, a, pb->stream);
  if (e != cudaSuccess) return cuda_fail(pb, e, "persistent kernel launch");
  return MF_OK;
}
// wait for the problem's stream and turn the kernel's sticky status into the return value
mf_status launch_finish(mf_problem* pb) {
  SolverState s;
  mf_status r = read_state(pb, &s);
  if (r != MF_OK) return r;
  if (s.status != ST_OK) {
    static const char* names[] = {"ok", "argument", "cuda", "outside iteration did not converge",
                                  "non-finite derivative", "step size underflow", "workspace",
                                  "grid barrier timed out"};
    pb->err = names[s.status >= 0 && s.status <= 7 ? s.status : 0];
    return (mf_status)s.status;
  }
  return MF_OK;
}

mf_status launch(mf_problem* pb, const KernelArgs& a) {
  mf_status r = launch_enqueue(pb, a);
  return r != MF_OK ? r : launch_finish(pb);
}

}  // namespace

extern "C" {

void mf_default_params(mf_params* p) {
  std::memset(p, 0, sizeof(*p));
  p->dim = 2;
  p->nz = 1;
  p->jc = 1.0; p->n = 19.0; p->e0 = 1.0; p->rho_out = 1.0; p->sigma = 0.0;
  p->lambda = 0.7; p->iter_tol = 2e-4; p->iter_max = 1000;
  p->precision = 0;
  p->rtol = 1e-6; p->atol = 1e-6; p->h0 = 0.0; p->h_min = 1e-12;
  p->he_sin_amp = 0.0; p->he_sin_period = 1.0;
  p->he_dir[0] = 0.0; p->he_dir[1] = 0.0; p->he_dir[2] = 1.0;
  p->gamma = 1.0; p->b0 = 0.0;
}

size_t mf_workspace_bytes(const mf_params* p) {
  std::string why;
  if (check_params(p, why) != MF_OK) return 0;
  return layout(p).total;
}

mf_status mf_create(const mf_params* p, void* d_workspace, size_t bytes, void* stream,
                    mf_problem** out) {
  if (!out) return MF_ERR_ARG;
  *out = nullptr;
  std::string why;
  mf_status cs = check_params(p, why);
  if (cs != MF_OK) return cs;
  const Layout L = layout(p);
  if (!d_workspace || bytes < L.total || ((uintptr_t)d_workspace & 255)) return MF_ERR_WORKSPACE;

  mf_problem* pb = new mf_problem();
  pb->p = *p;
  pb->stream = (cudaStream_t)stream;
  pb->ws = (char*)d_workspace;
  pb->ws_bytes = bytes;
  pb->used = L.total;
  if (cudaGetDevice(&pb->device) != cudaSuccess) { delete pb; return MF_ERR_CUDA; }

  const int nz = p->dim == 2 ? 1 : p->nz;
  Desc& d = pb->d;
  std::memset(&d, 0, sizeof(d));
  d.dim = p->dim; d.nx = p->nx; d.ny = p->ny; d.nz = nz; d.precision = p->precision;
  d.lgx = ilog2(p->nx); d.lgy = ilog2(p->ny); d.lgz = ilog2(nz);
  d.Lx = p->Lx; d.Ly = p->Ly; d.Lz = p->dim == 2 ? 0.0 : p->Lz;
  d.dx = 2 * p->Lx / p->nx; d.dy = 2 * p->Ly / p->ny; d.dz = p->dim == 2 ? 0.0 : 2 * p->Lz / nz;
  const double s2 = d.dx * d.dx + d.dy * d.dy + d.dz * d.dz;
  d.sigma = p->sigma > 0 ? p->sigma : std::sqrt(s2);   // Section 2.2 / Section 3.2 choice
  d.n = p->n; d.e0 = p->e0; d.jc = p->jc; d.rho_out = p->rho_out; d.lam = p->lambda;
  d.gamma = p->gamma; d.b0 = p->b0;
  d.iter_tol = p->iter_tol; d.iter_max = p->iter_max;
  d.barrier_ns = BARRIER_LIMIT_NS;
  d.rtol = p->rtol; d.atol = p->atol; d.h_min = p->h_min;
  d.he_knots = p->he_knots; d.he_sin_amp = p->he_sin_amp; d.he_sin_period = p->he_sin_period;
  for (int i = 0; i < 3; ++i) d.he_dir[i] = p->he_dir[i];
  d.ncell = L.ncell; d.nspec = L.nspec;
  long long nout = 0;
  for (long long i = 0; i < L.ncell; ++i) nout += p->mask[i] == 0;
  for (long long i = 0; i < L.ncell; ++i)
    if (p->mask[i] > 2) { delete pb; return MF_ERR_ARG; }
  d.nout = nout;
  char* w = pb->ws;
  d.Sa = w + L.Sa; d.Sb = w + L.Sb; d.hd = w + L.hd; d.hd2 = p->dim == 2 ? (void*)(w + L.hd2) : d.hd; d.u = w + L.u; d.q1 = w + L.q1; d.q2 = w + L.q2;
  d.jcmap = p->jc_map ? (const void*)(w + L.jc) : nullptr;
  d.mask = (const uint8_t*)(w + L.mask);
  d.tw_x = w + L.twx; d.tw_y = w + L.twy; d.tw_z = w + L.twz;
  d.ktab = w + L.ktab; d.gtab = w + L.gtab;
  for (int i = 0; i < 6; ++i) d.fbuf[i] = (double*)(w + L.fbuf[i]);
  d.partials = (double*)(w + L.partials);
  d.max_items = L.max_items;
  d.st = (SolverState*)(w + L.st);
  d.gb = (GridBarrier*)(w + L.gb);
  d.log = (StepLog*)(w + L.log);
  d.log_cap = LOG_CAP;
  d.he_t = (const double*)(w + L.knots);
  d.he_v = d.he_t + (p->he_knots > 0 ? p->he_knots : 1);
  pb->scratch_m = (double*)(w + L.mscr);
  d.dev = (const Desc*)(w + L.desc);

  // launch configuration: all CTAs co-resident, no more than the widest pass can use
  const size_t smem = kernel_smem_bytes(d);
  int per_sm = p->dim == 2 ? film_max_blocks(p->precision, smem) : bulk_max_blocks(p->precision, smem);
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pb->device);
  cudaError_t le = cudaGetLastError();
  if (per_sm < 1 || nsm < 1 || le != cudaSuccess) {
    pb->err = "kernel does not fit on this device";
    delete pb;
    return MF_ERR_CUDA;
  }
  const int coresident = per_sm * nsm;
  if (p->dim == 2) {
    int rb1 = std::min(p->ny, 2 * BATCH / p->nx);
    int rb2 = std::min(p->ny, BATCH / p->nx);
    const int want = std::max(p->nx / 2 + 1, 1);
    const int grid = std::min(coresident, want);
    while (rb1 > 2 && p->ny / rb1 < grid) rb1 /= 2;
    while (rb2 > 2 && p->ny / rb2 < grid) rb2 /= 2;
    d.rows_per_item = rb1;
    d.zs_per_item = rb2;
    d.grid = std::max(1, std::min(coresident, std::max(want, p->ny / rb1)));
  } else {
    // x pass: rb rows of 3 fields; y pass: zs z-lines of 3 fields
    int rb = std::min(p->ny, 2 * BATCH / (3 * p->nx));
    rb = std::max(2, rb & ~1);
    while (rb & (rb - 1)) rb &= rb - 1;
    int zs = std::min(nz, BATCH / (3 * p->ny));
    zs = std::max(1, zs);
    while (zs & (zs - 1)) zs &= zs - 1;
    const long long xitems = (long long)p->ny * nz / rb;
    const long long zlines = (long long)(p->nx / 2 + 1) * p->ny;
    const int grid = (int)std::min<long long>(coresident, std::max(xitems, zlines));
    while (rb > 2 && (long long)p->ny * nz / rb < grid) rb /= 2;
    while (zs > 1 && (long long)(p->nx / 2 + 1) * nz / zs < grid) zs /= 2;
    d.rows_per_item = rb;
    d.zs_per_item = zs;
    d.grid = std::max(1, grid);
    if (3 * p->nx * (rb / 2) > BATCH || 3 * p->ny * zs > BATCH || 3 * nz > BATCH) {
      pb->err = "grid too large for the shared-memory batch";
      delete pb;
      return MF_ERR_ARG;
    }
  }

  // tables and inputs
  std::vector<char> tw, kt, gt;
  if (p->precision) fill_tables<float>(p, d.sigma, tw, kt, gt);
  else fill_tables<double>(p, d.sigma, tw, kt, gt);
  const size_t ts = p->precision ? 4 : 8;
  std::vector<char> jcbuf;
  if (p->jc_map) {
    jcbuf.resize(L.ncell * ts);
    for (long long i = 0; i < L.ncell; ++i) {
      if (p->precision) ((float*)jcbuf.data())[i] = (float)p->jc_map[i];
      else ((double*)jcbuf.data())[i] = p->jc_map[i];
    }
  }
  std::vector<double> knots(2 * (p->he_knots > 0 ? p->he_knots : 1), 0.0);
  for (int i = 0; i < p->he_knots; ++i) { knots[i] = p->he_t[i]; knots[p->he_knots + i] = p->he_v[i]; }
  SolverState s0;
  std::memset(&s0, 0, sizeof(s0));
  s0.t = 0.0;
  s0.h = p->h0;
  s0.ybuf = 0; s0.ynewbuf = 1; s0.k1buf = 2; s0.k4buf = 5;
  cudaStream_t st = pb->stream;
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t n) {
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st);
  };
  cp(w + L.mask, p->mask, L.ncell);
  if (p->jc_map) cp(w + L.jc, jcbuf.data(), jcbuf.size());
  const size_t twx = 2 * p->nx * 2 * ts, twy = 2 * p->ny * 2 * ts, twz = 2 * nz * 2 * ts;
  cp(w + L.twx, tw.data(), twx);
  cp(w + L.twy, tw.data() + twx, twy);
  cp(w + L.twz, tw.data() + twx + twy, twz);
  cp(w + L.ktab, kt.data(), kt.size());
  cp(w + L.gtab, gt.data(), gt.size());
  cp(w + L.knots, knots.data(), knots.size() * 8);
  cp(w + L.st, &s0, sizeof(s0));
  cp(w + L.desc, &d, sizeof(Desc));     // the kernels read the descriptor from here
  if (e == cudaSuccess) e = cudaMemsetAsync(w + L.fbuf[0], 0, L.nstate * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w + L.hd, 0, (p->dim == 2 ? 1 : 3) * L.ncell * ts, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // host staging buffers die below
  if (e != cudaSuccess) {
    cuda_fail(pb, e, "mf_create copies");
    delete pb;
    return MF_ERR_CUDA;
  }
  if (p->dim == 2) {
    KernelArgs a{};
    a.mode = MODE_SETUP;
    mf_status r = launch(pb, a);
    if (r != MF_OK) { delete pb; return r; }
  }
  *out = pb;
  return MF_OK;
}

mf_status mf_rhs_ex(mf_problem* pb, double t, int seg, const double* d_y, double* d_ydot,
                    int force_iters, int* iters_out) {
  Range range_("mf_rhs");
  if (!pb || !d_y || !d_ydot) return MF_ERR_ARG;
  KernelArgs a{};
  a.mode = MODE_RHS; a.t = t; a.y_in = d_y; a.out = d_ydot; a.force_iters = force_iters; a.seg = seg;
  mf_status r = launch(pb, a);
  if (iters_out) {
    SolverState s;
    if (read_state(pb, &s) == MF_OK) *iters_out = s.last_iters;
  }
  return r;
}

mf_status mf_rhs(mf_problem* pb, double t, const double* d_y, double* d_ydot, int* iters_out) {
  return mf_rhs_ex(pb, t, -2, d_y, d_ydot, 0, iters_out);
}

mf_status mf_set_barrier_timeout(mf_problem* pb, double seconds) {
  if (!pb || !(seconds == seconds) || seconds > 3600.0) return MF_ERR_ARG;
  pb->d.barrier_ns = seconds <= 0.0 ? BARRIER_LIMIT_NS
                                    : std::max(1ull, (unsigned long long)(seconds * 1e9));
  MF_CUDA(pb, cudaMemcpyAsync((void*)pb->d.dev, &pb->d, sizeof(Desc), cudaMemcpyHostToDevice, pb->stream));
  MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  return MF_OK;
}

mf_status mf_reset_warm(mf_problem* pb) {
  if (!pb) return MF_ERR_ARG;
  SolverState s;
  mf_status r = read_state(pb, &s);
  if (r != MF_OK) return r;
  s.warm_valid = 0;
  s.A_prev = 0.0;
  s.com_valid = 0;
  s.hd_sel = 0;
  s.A_com = 0.0;
  return write_state(pb, &s);
}

mf_status mf_set_state(mf_problem* pb, double t, double h, const double* d_y) {
  if (!pb) return MF_ERR_ARG;
  SolverState s;
  mf_status r = read_state(pb, &s);
  if (r != MF_OK) return r;
  s.t = t;
  s.h = h;
  s.k1_valid = 0;
  s.failed = 0;
  s.log_count = 0;
  s.status = ST_OK;
  if (d_y) MF_CUDA(pb, cudaMemcpyAsync(pb->d.fbuf[s.ybuf], d_y, pb->d.ncell * (pb->d.dim == 2 ? 1 : 3) * 8,
                                       cudaMemcpyDeviceToDevice, pb->stream));
  return write_state(pb, &s);
}

mf_status mf_get_state(mf_problem* pb, double* t, double* h, double* d_y) {
  if (!pb) return MF_ERR_ARG;
  SolverState s;
  mf_status r = read_state(pb, &s);
  if (r != MF_OK) return r;
  if (t) *t = s.t;
  if (h) *h = s.h;
  if (d_y) {
    MF_CUDA(pb, cudaMemcpyAsync(d_y, pb->d.fbuf[s.ybuf], pb->d.ncell * (pb->d.dim == 2 ? 1 : 3) * 8,
                                cudaMemcpyDeviceToDevice, pb->stream));
    MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  }
  return MF_OK;
}

static mf_status ensure_h(mf_problem* pb, double t_target) {
  SolverState s;
  mf_status r = read_state(pb, &s);
  if (r != MF_OK) return r;
  if (!(s.h > 0)) {
    s.h = std::min(1e-3, 0.01 * (t_target - s.t));
    if (!(s.h > 0)) s.h = 1e-3;
    return write_state(pb, &s);
  }
  return MF_OK;
}

// transform work of one pass over a film: cells x log2 cells
static double film_cost(int nx, int ny) {
  const double c = (double)nx * (double)ny;
  return c * std::log2(c);
}

// CTAs per film of a shared launch: one each, then one at a time to the film with the most
// work per CTA until the grid is full or every film has the CTAs its own launch would use
// (this minimises the largest work per CTA, which sets how long the launch lasts)
static void split_ctas(const double* cost, const int* own, const int* films, int n, int total,
                       int* ctas) {
  std::priority_queue<std::pair<double, int>> q;
  for (int k = 0; k < n; ++k) {
    const int i = films[k];
    ctas[i] = 1;
    if (ctas[i] < own[i]) q.push({cost[i], k});
  }
  for (int used = n; used < total && !q.empty(); ++used) {
    const int k = q.top().second;
    const int i = films[k];
    q.pop();
    ++ctas[i];
    if (ctas[i] < own[i]) q.push({cost[i] / ctas[i], k});
  }
}

// field passes (19 per right-hand side, 14 per outside iteration) per step attempt
static double passes_per_attempt(long long rhs, long long iters, long long attempts) {
  return (19.0 * (double)rhs + 14.0 * (double)iters) / (double)std::max(attempts, 1LL);
}

// Advance the films pbs[idx[k]] (one device, one precision) as mf_batch_plan arranges them;
// statuses go to st[idx[k]].  Shared launches go on the first shared film's stream, one after
// the other; films with a launch of their own go on their own streams.
static void advance_films_together(mf_problem* const* pbs, const std::vector<int>& idx,
                                   const double* t_targets, long long max_attempts,
                                   std::vector<mf_status>& st) {
  mf_problem* p0 = pbs[idx[0]];
  cudaError_t e = cudaSetDevice(p0->device);
  if (e != cudaSuccess) {
    for (int i : idx) st[i] = cuda_fail(pbs[i], e, "cudaSetDevice");
    return;
  }
  const int prec = p0->d.precision;
  const int per_sm = film_batch_max_blocks(prec, kernel_smem_bytes(p0->d));
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p0->device);
  e = cudaGetLastError();
  if (e != cudaSuccess || per_sm < 1 || nsm < 1) {
    if (e == cudaSuccess) e = cudaErrorInvalidConfiguration;
    for (int i : idx) st[i] = cuda_fail(pbs[i], e, "shared launch configuration");
    return;
  }
  // work already queued on the films' own streams comes first
  std::vector<int> live;
  for (int i : idx) {
    e = cudaStreamSynchronize(pbs[i]->stream);
    if (e != cudaSuccess) st[i] = cuda_fail(pbs[i], e, "cudaStreamSynchronize");
    else live.push_back(i);
  }
  const int n = (int)live.size();
  if (n == 0) return;
  // each film's work per attempt: what it took in the previous batch call, else its average
  // so far, else 3.5 right-hand sides of 5 outside iterations; times cells x log2 cells
  std::vector<int> nx(n), ny(n), own(n), order(n), launch(n), ctas(n);
  std::vector<double> work(n);
  std::vector<SolverState> before(n);
  for (int k = 0; k < n; ++k) {
    mf_problem* f = pbs[live[k]];
    nx[k] = f->d.nx; ny[k] = f->d.ny; own[k] = f->d.grid;
    if (read_state(f, &before[k]) != MF_OK) std::memset(&before[k], 0, sizeof(SolverState));
    const SolverState& b0 = before[k];
    double w = f->batch_work;
    if (!(w > 0.0)) w = b0.n_attempts > 0 ? passes_per_attempt(b0.n_rhs, b0.n_iters, b0.n_attempts)
                                          : passes_per_attempt(7, 35, 2);
    const double c = (double)nx[k] * (double)ny[k];
    work[k] = w * c * std::log2(c);
  }
  const int nlaunch = mf_batch_plan(n, nx.data(), ny.data(), own.data(), work.data(), per_sm * nsm,
                                    order.data(), launch.data(), ctas.data());
  std::vector<int> alone, shared;
  for (int k : order) {
    const int i = live[k];
    if (launch[k] >= 0) continue;
    KernelArgs a{};
    a.mode = MODE_ADVANCE; a.t_target = t_targets[i]; a.max_attempts = max_attempts;
    st[i] = launch_enqueue(pbs[i], a);
    if (st[i] == MF_OK) alone.push_back(i);
  }
  cudaStream_t s = p0->stream;
  for (int k : order)
    if (launch[k] >= 0) { s = pbs[live[k]]->stream; break; }
  BatchTable tab;           // 8 KB, copied into each launch's parameters
  for (int j = 0; j < nlaunch; ++j) {
    std::vector<int> members;
    tab.n = 0;
    int b = 0;
    e = cudaSuccess;
    for (int k : order) {
      if (launch[k] != j) continue;
      mf_problem* f = pbs[live[k]];
      if (e == cudaSuccess) e = cudaMemsetAsync(f->d.gb, 0, sizeof(GridBarrier), s);
      tab.job[tab.n++] = BatchJob{f->d.dev, t_targets[live[k]], max_attempts, b, ctas[k]};
      b += ctas[k];
      members.push_back(live[k]);
    }
    if (e == cudaSuccess) e = film_batch_launch(prec, tab, b, s);
    for (int i : members) {
      if (e == cudaSuccess) shared.push_back(i);
      else st[i] = cuda_fail(pbs[i], e, "shared persistent launch");
    }
  }
  e = shared.empty() ? cudaSuccess : cudaStreamSynchronize(s);
  for (int i : shared) st[i] = e == cudaSuccess ? launch_finish(pbs[i]) : cuda_fail(pbs[i], e, "shared persistent launch");
  for (int i : alone) st[i] = launch_finish(pbs[i]);
  // remember what each film's attempts cost in this call for the next arrangement
  for (int k = 0; k < n; ++k) {
    SolverState a1;
    mf_problem* f = pbs[live[k]];
    if (read_state(f, &a1) != MF_OK) continue;
    const long long att = a1.n_attempts - before[k].n_attempts;
    if (att > 0)
      f->batch_work = passes_per_attempt(a1.n_rhs - before[k].n_rhs, a1.n_iters - before[k].n_iters, att);
  }
}

int mf_batch_plan(int n, const int* nx, const int* ny, const int* own_grid, const double* work,
                  int coresident, int* order, int* launch, int* ctas) {
  if (n < 0 || (n > 0 && (!nx || !ny || !own_grid || !order || !launch || !ctas)) || coresident < 1)
    return -1;
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i) {
    if (nx[i] < 1 || ny[i] < 1 || own_grid[i] < 1) return -1;
    cost[i] = work ? work[i] : film_cost(nx[i], ny[i]);
    if (!(cost[i] > 0.0) || !std::isfinite(cost[i])) return -1;
  }
  for (int i = 0; i < n; ++i) order[i] = i;
  // most work first (stable: equal films keep their order)
  std::stable_sort(order, order + n, [&](int a, int b) { return cost[a] > cost[b]; });
  // films whose own launch fills the GPU keep it
  std::vector<int> sh;
  for (int k = 0; k < n; ++k) {
    const int i = order[k];
    if (own_grid[i] >= coresident) { launch[i] = -1; ctas[i] = coresident; }
    else sh.push_back(i);
  }
  // the others fill shared launches, most work first; a launch is closed before a film whose
  // share of the grid in proportion to its work would be below one CTA
  const size_t cap = (size_t)std::min(MAX_BATCH, coresident);
  int nl = 0;
  for (size_t k0 = 0; k0 < sh.size(); ++nl) {
    double sum = cost[sh[k0]];
    size_t k1 = k0 + 1;
    for (; k1 < sh.size() && k1 - k0 < cap; ++k1) {
      const double c = cost[sh[k1]];
      if (sum + c > (double)coresident * c) break;
      sum += c;
    }
    for (size_t k = k0; k < k1; ++k) launch[sh[k]] = nl;
    split_ctas(cost.data(), own_grid, sh.data() + k0, (int)(k1 - k0), coresident, ctas);
    k0 = k1;
  }
  return nl;
}

mf_status mf_advance(mf_problem* pb, double t_target, long long max_attempts) {
  Range range_("mf_advance");
  if (!pb) return MF_ERR_ARG;
  mf_status r = ensure_h(pb, t_target);
  if (r != MF_OK) return r;
  KernelArgs a{};
  a.mode = MODE_ADVANCE; a.t_target = t_target; a.max_attempts = max_attempts;
  return launch(pb, a);
}

mf_status mf_advance_batch(mf_problem* const* pbs, int n, const double* t_targets,
                           long long max_attempts, mf_status* statuses) {
  Range range_("mf_advance_batch");
  if (!pbs || !t_targets || n < 0) return MF_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!pbs[i]) return MF_ERR_ARG;
  {
    // a repeated problem would run twice at once on one workspace and grid barrier
    std::vector<mf_problem*> seen(pbs, pbs + n);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return MF_ERR_ARG;
  }
  std::vector<mf_status> st(n, MF_OK);
  for (int i = 0; i < n; ++i) st[i] = ensure_h(pbs[i], t_targets[i]);
  // films of one device and precision share persistent launches; bulk bodies get one launch
  // each, all enqueued on their own streams before any is waited for
  std::vector<char> grouped(n, 0);
  for (int i = 0; i < n; ++i) {
    if (grouped[i] || st[i] != MF_OK || pbs[i]->d.dim != 2) continue;
    std::vector<int> idx;
    for (int j = i; j < n; ++j)
      if (!grouped[j] && st[j] == MF_OK && pbs[j]->d.dim == 2 && pbs[j]->device == pbs[i]->device &&
          pbs[j]->d.precision == pbs[i]->d.precision) {
        idx.push_back(j);
        grouped[j] = 1;
      }
    advance_films_together(pbs, idx, t_targets, max_attempts, st);
  }
  std::vector<char> launched(n, 0);
  for (int i = 0; i < n; ++i) {
    if (grouped[i] || st[i] != MF_OK) continue;
    KernelArgs a{};
    a.mode = MODE_ADVANCE; a.t_target = t_targets[i]; a.max_attempts = max_attempts;
    st[i] = launch_enqueue(pbs[i], a);
    launched[i] = st[i] == MF_OK;
  }
  mf_status first = MF_OK;
  for (int i = 0; i < n; ++i) {
    if (launched[i]) st[i] = launch_finish(pbs[i]);
    if (statuses) statuses[i] = st[i];
    if (first == MF_OK) first = st[i];
  }
  return first;
}

mf_status mf_step(mf_problem* pb, double t_max, int* accepted) {
  Range range_("mf_step");
  if (!pb) return MF_ERR_ARG;
  SolverState s0;
  mf_status r = read_state(pb, &s0);
  if (r != MF_OK) return r;
  r = mf_advance(pb, t_max, 1);
  if (accepted) {
    SolverState s1;
    if (read_state(pb, &s1) == MF_OK) *accepted = s1.n_accepted > s0.n_accepted;
  }
  return r;
}

mf_status mf_readout_of(mf_problem* pb, int what, double t, const double* d_y, double* out) {
  if (!pb || !d_y || !out) return MF_ERR_ARG;
  KernelArgs a{};
  a.t = t; a.y_in = d_y;
  if (what == MF_READ_MOMENT) {
    a.mode = MODE_MOMENT; a.out = pb->scratch_m;
    mf_status r = launch(pb, a);
    if (r != MF_OK) return r;
    const int nm = pb->d.dim == 2 ? 1 : 3;
    MF_CUDA(pb, cudaMemcpyAsync(out, pb->scratch_m, nm * 8, cudaMemcpyDeviceToHost, pb->stream));
    MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
    return MF_OK;
  }
  if (what == MF_READ_HZ && pb->d.dim == 2) { a.mode = MODE_HZ; a.out = out; return launch(pb, a); }
  if (what == MF_READ_J && pb->d.dim == 3) { a.mode = MODE_J; a.out = out; return launch(pb, a); }
  if (what == MF_READ_E) { a.mode = MODE_E; a.out = out; return launch(pb, a); }
  pb->err = "readout not available for this dimension";
  return MF_ERR_ARG;
}

mf_status mf_readout(mf_problem* pb, int what, double* out) {
  if (!pb) return MF_ERR_ARG;
  SolverState s;
  mf_status r = read_state(pb, &s);
  if (r != MF_OK) return r;
  return mf_readout_of(pb, what, s.t, pb->d.fbuf[s.ybuf], out);
}

mf_status mf_run_ramp(mf_problem* pb, int n_out, const double* t_out, double* h_m_out,
                      double* d_hz_out) {
  Range range_("mf_run_ramp");
  if (!pb || n_out < 0 || (n_out > 0 && !t_out)) return MF_ERR_ARG;
  const int nm = pb->d.dim == 2 ? 1 : 3;
  const long long per = pb->d.dim == 2 ? pb->d.ncell : 3 * pb->d.ncell;
  if (n_out > 0) {
    // an unset first step is chosen for the whole ramp [t, last output time], as for one
    // advance to its end (an integrator given all output times at once sees the whole span)
    mf_status r = ensure_h(pb, t_out[n_out - 1]);
    if (r != MF_OK) return r;
  }
  for (int k = 0; k < n_out; ++k) {
    mf_status r = mf_advance(pb, t_out[k], 1LL << 40);
    if (r != MF_OK) return r;
    if (h_m_out) {
      r = mf_readout(pb, MF_READ_MOMENT, h_m_out + (size_t)k * nm);
      if (r != MF_OK) return r;
    }
    if (d_hz_out) {
      r = mf_readout(pb, pb->d.dim == 2 ? MF_READ_HZ : MF_READ_J, d_hz_out + (size_t)k * per);
      if (r != MF_OK) return r;
    }
  }
  return MF_OK;
}

// work-item shapes and launch widths the persistent kernels accept for this problem
static std::vector<std::array<int, 3>> tuning_candidates(const mf_problem* pb, int coresident) {
  const Desc& d = pb->d;
  std::vector<std::array<int, 3>> c;
  std::vector<int> grids = {d.grid, coresident, coresident / 2};
  std::sort(grids.begin(), grids.end());
  grids.erase(std::unique(grids.begin(), grids.end()), grids.end());
  auto add = [&](int rb, int zs) {
    for (int g : grids)
      if (g >= 1 && g <= coresident) c.push_back({rb, zs, g});
  };
  if (d.dim == 2) {
    // row passes: rb one-field rows (and min(rb, BATCH / nx) two-field rows) per item
    const int rb_max = std::min(d.ny, 2 * BATCH / d.nx);
    for (int rb = 2; rb <= rb_max; rb *= 2) add(rb, std::max(2, std::min(rb, BATCH / d.nx)));
  } else {
    // x pass: rb rows of 3 fields; y pass: zs z-lines of 3 fields
    for (int rb = 2; rb <= d.ny && 3 * d.nx * (rb / 2) <= BATCH; rb *= 2)
      for (int zs = 1; zs <= d.nz && 3 * d.ny * zs <= BATCH; zs *= 2) add(rb, zs);
  }
  return c;
}

mf_status mf_autotune(mf_problem* pb, int reps, int force_iters, mf_tuning* out) {
  Range range_("mf_autotune");
  if (!pb || reps < 1 || force_iters < 1) return MF_ERR_ARG;
  MF_CUDA(pb, cudaSetDevice(pb->device));
  SolverState s0;
  mf_status r = read_state(pb, &s0);
  if (r != MF_OK) return r;
  const int per_sm = pb->d.dim == 2 ? film_max_blocks(pb->d.precision, kernel_smem_bytes(pb->d))
                                    : bulk_max_blocks(pb->d.precision, kernel_smem_bytes(pb->d));
  int nsm = 0;
  MF_CUDA(pb, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, pb->device));
  if (per_sm < 1 || nsm < 1) { pb->err = "kernel does not fit on this device"; return MF_ERR_CUDA; }
  const Desc base = pb->d;
  const std::vector<std::array<int, 3>> cand = tuning_candidates(pb, per_sm * nsm);
  // right-hand sides of the current state into a buffer the state does not use
  KernelArgs a{};
  a.mode = MODE_RHS; a.t = s0.t; a.seg = -2; a.force_iters = force_iters;
  a.y_in = base.fbuf[s0.ybuf];
  a.out = base.fbuf[(s0.ybuf + 1) % 6];
  cudaEvent_t e0, e1;
  MF_CUDA(pb, cudaEventCreate(&e0));
  MF_CUDA(pb, cudaEventCreate(&e1));
  auto upload = [&](const Desc& d) {
    cudaError_t e = cudaMemcpyAsync((void*)d.dev, &d, sizeof(Desc), cudaMemcpyHostToDevice, pb->stream);
    return e == cudaSuccess ? cudaStreamSynchronize(pb->stream) : e;   // the host copy is a local
  };
  double best = 0.0, dflt = 0.0;
  size_t ibest = cand.size();
  for (size_t i = 0; i < cand.size() && r == MF_OK; ++i) {
    pb->d = base;
    pb->d.rows_per_item = cand[i][0];
    pb->d.zs_per_item = cand[i][1];
    pb->d.grid = cand[i][2];
    cudaError_t e = upload(pb->d);
    if (e != cudaSuccess) { r = cuda_fail(pb, e, "descriptor upload"); break; }
    // forced iterations may end above the tolerance (MF_ERR_NOCONV): the timing is what counts
    r = launch(pb, a);                                   // warm-up
    if (r == MF_ERR_NOCONV) r = MF_OK;
    for (int k = 0; k <= reps && r == MF_OK; ++k) {
      if (k == 0) e = cudaEventRecord(e0, pb->stream);
      else r = launch_enqueue(pb, a);
      if (k == reps && r == MF_OK) e = cudaEventRecord(e1, pb->stream);
      if (e != cudaSuccess) r = cuda_fail(pb, e, "cudaEventRecord");
    }
    if (r == MF_OK) r = launch_finish(pb);
    if (r == MF_ERR_NOCONV) r = MF_OK;
    float ms = 0.f;
    if (r == MF_OK) {
      e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) r = cuda_fail(pb, e, "cudaEventElapsedTime");
    }
    if (r != MF_OK) break;
    const double per = (double)ms / reps;
    const bool is_default = cand[i][0] == base.rows_per_item && cand[i][1] == base.zs_per_item &&
                            cand[i][2] == base.grid;
    if (is_default) dflt = per;
    if (ibest == cand.size() || per < best) { best = per; ibest = i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pb->d = base;
  if (r == MF_OK && ibest < cand.size()) {
    pb->d.rows_per_item = cand[ibest][0];
    pb->d.zs_per_item = cand[ibest][1];
    pb->d.grid = cand[ibest][2];
  }
  cudaError_t e = upload(pb->d);
  if (e != cudaSuccess && r == MF_OK) r = cuda_fail(pb, e, "descriptor upload");
  // the state, step size and counters as they were; the tuning runs overwrote the outside
  // iteration's warm start and a derivative buffer
  SolverState s1 = s0;
  s1.k1_valid = 0;
  s1.warm_valid = 0; s1.A_prev = 0.0; s1.com_valid = 0; s1.hd_sel = 0; s1.A_com = 0.0;
  const mf_status w = write_state(pb, &s1);
  if (r == MF_OK) r = w;
  if (r == MF_OK && out) {
    out->rows_per_item = pb->d.rows_per_item;
    out->zs_per_item = pb->d.zs_per_item;
    out->grid = pb->d.grid;
    out->candidates = (int)cand.size();
    out->ms_per_rhs = best;
    out->ms_per_rhs_default = dflt;
  }
  return r;
}

// ---- checkpoints: everything a continuation reads, in one caller-owned blob ----
namespace {
constexpr unsigned long long CKPT_MAGIC = 0x314b43504f46464dull;   // "MFFOPCK1"
struct CkptHeader {
  unsigned long long magic, bytes;
  int dim, nx, ny, nz, precision, rows_per_item, zs_per_item, grid;
};
// (device pointer, bytes) of every saved region, in blob order after the header
std::vector<std::pair<void*, size_t>> ckpt_regions(const mf_problem* pb) {
  const Desc& d = pb->d;
  const size_t ts = d.precision ? 4 : 8;
  const size_t ncomp = d.dim == 2 ? 1 : 3;
  const size_t nstate = (size_t)d.ncell * ncomp;
  std::vector<std::pair<void*, size_t>> r;
  r.push_back({(void*)d.st, sizeof(SolverState)});
  for (int i = 0; i < 6; ++i) r.push_back({(void*)d.fbuf[i], nstate * 8});
  r.push_back({d.hd, ncomp * (size_t)d.ncell * ts});
  if (d.dim == 2) r.push_back({d.hd2, (size_t)d.ncell * ts});
  r.push_back({(void*)d.log, (size_t)d.log_cap * sizeof(StepLog)});
  return r;
}
size_t ckpt_bytes(const mf_problem* pb) {
  size_t b = sizeof(CkptHeader);
  for (const auto& x : ckpt_regions(pb)) b += x.second;
  return b;
}
}  // namespace

size_t mf_checkpoint_bytes(const mf_problem* pb) { return pb ? ckpt_bytes(pb) : 0; }

mf_status mf_checkpoint_save(mf_problem* pb, void* dst) {
  Range range_("mf_checkpoint_save");
  if (!pb || !dst) return MF_ERR_ARG;
  MF_CUDA(pb, cudaSetDevice(pb->device));
  CkptHeader h{CKPT_MAGIC, ckpt_bytes(pb), pb->d.dim, pb->d.nx, pb->d.ny, pb->d.nz, pb->d.precision,
               pb->d.rows_per_item, pb->d.zs_per_item, pb->d.grid};
  char* o = (char*)dst;
  MF_CUDA(pb, cudaMemcpyAsync(o, &h, sizeof(h), cudaMemcpyDefault, pb->stream));
  o += sizeof(h);
  for (const auto& x : ckpt_regions(pb)) {
    MF_CUDA(pb, cudaMemcpyAsync(o, x.first, x.second, cudaMemcpyDefault, pb->stream));
    o += x.second;
  }
  MF_CUDA(pb, cudaStreamSynchronize(pb->stream));   // the header is a host local
  return MF_OK;
}

mf_status mf_checkpoint_restore(mf_problem* pb, const void* src) {
  Range range_("mf_checkpoint_restore");
  if (!pb || !src) return MF_ERR_ARG;
  MF_CUDA(pb, cudaSetDevice(pb->device));
  CkptHeader h;
  MF_CUDA(pb, cudaMemcpyAsync(&h, src, sizeof(h), cudaMemcpyDefault, pb->stream));
  MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  if (h.magic != CKPT_MAGIC || h.bytes != ckpt_bytes(pb) || h.dim != pb->d.dim || h.nx != pb->d.nx ||
      h.ny != pb->d.ny || h.nz != pb->d.nz || h.precision != pb->d.precision) {
    pb->err = "checkpoint does not match this problem (grid, dimension or precision)";
    return MF_ERR_ARG;
  }
  const char* i = (const char*)src + sizeof(h);
  for (const auto& x : ckpt_regions(pb)) {
    MF_CUDA(pb, cudaMemcpyAsync(x.first, i, x.second, cudaMemcpyDefault, pb->stream));
    i += x.second;
  }
  // the work-item shape (it sets the order of the sums) and launch width it was saved with
  pb->d.rows_per_item = h.rows_per_item;
  pb->d.zs_per_item = h.zs_per_item;
  pb->d.grid = h.grid;
  MF_CUDA(pb, cudaMemcpyAsync((void*)pb->d.dev, &pb->d, sizeof(Desc), cudaMemcpyHostToDevice, pb->stream));
  MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  return MF_OK;
}

// one launch of the film's adjoint kernel: the outside iteration alone (g null) or the whole
// right-hand side's vector-Jacobian product
static mf_status film_adjoint(mf_problem* pb, int iters, const double* d_v, double* d_hin_bar,
                              const double* d_g, double* d_gbar, double* d_jcbar,
                              const double* d_wbar_out, double* d_wbar_in, double* sbar) {
  if (pb->d.dim != 2 || pb->d.nout <= 0) {
    pb->err = "the film adjoint needs a film with free space";
    return MF_ERR_ARG;
  }
  MF_CUDA(pb, cudaSetDevice(pb->device));
  MF_CUDA(pb, cudaMemsetAsync(pb->d.gb, 0, sizeof(GridBarrier), pb->stream));
  cudaError_t e = film_adjoint_launch(pb->d.precision, pb->d, d_v, d_hin_bar, pb->scratch_m, iters,
                                      d_g, d_gbar, d_jcbar, d_wbar_out, d_wbar_in, pb->stream);
  if (e != cudaSuccess) return cuda_fail(pb, e, "adjoint kernel launch");
  mf_status r = launch_finish(pb);
  if (r == MF_OK && sbar) {
    MF_CUDA(pb, cudaMemcpyAsync(sbar, pb->scratch_m, sizeof(double), cudaMemcpyDeviceToHost, pb->stream));
    MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  }
  return r;
}

mf_status mf_film_outside_vjp(mf_problem* pb, int iters, const double* d_v, double* d_hin_bar,
                              double* sbar) {
  Range range_("mf_film_outside_vjp");
  if (!pb || !d_v || !d_hin_bar || iters < 1) return MF_ERR_ARG;
  return film_adjoint(pb, iters, d_v, d_hin_bar, nullptr, nullptr, nullptr, nullptr, nullptr, sbar);
}

mf_status mf_film_rhs_vjp(mf_problem* pb, int iters, const double* d_g, const double* d_v,
                          double* d_gbar, double* d_jcbar, double* sbar) {
  Range range_("mf_film_rhs_vjp");
  if (!pb || !d_g || !d_v || !d_gbar || !d_jcbar || iters < 1) return MF_ERR_ARG;
  return film_adjoint(pb, iters, d_v, nullptr, d_g, d_gbar, d_jcbar, nullptr, nullptr, sbar);
}

mf_status mf_film_rhs_vjp_warm(mf_problem* pb, int iters, const double* d_g, const double* d_v,
                               const double* d_wbar_out, double* d_gbar, double* d_jcbar,
                               double* d_wbar_in, double* sbar) {
  Range range_("mf_film_rhs_vjp_warm");
  if (!pb || !d_g || !d_v || !d_gbar || !d_jcbar || iters < 1) return MF_ERR_ARG;
  return film_adjoint(pb, iters, d_v, nullptr, d_g, d_gbar, d_jcbar, d_wbar_out, d_wbar_in, sbar);
}

// the warm start of the next film right-hand side (the most recent call's iterate, its shift
// applied) as an FP64 free-space field, or a given field made the warm start
static mf_status warm_save(mf_problem* pb, double* dst) {
  SolverState s;
  MF_TRY_STATUS(read_state(pb, &s));
  void* hd = s.hd_sel ? pb->d.hd2 : pb->d.hd;
  cudaError_t e = adj_warm_io(pb->d.precision, pb->d.ncell, 0, pb->d.mask, hd, s.A_prev, dst, nullptr,
                              pb->stream);
  return e == cudaSuccess ? MF_OK : cuda_fail(pb, e, "warm start save");
}
static mf_status warm_load(mf_problem* pb, const double* src) {
  SolverState s;
  MF_TRY_STATUS(read_state(pb, &s));
  s.hd_sel = 0; s.warm_valid = 1; s.A_prev = 0.0; s.com_valid = 0; s.A_com = 0.0;
  cudaError_t e = adj_warm_io(pb->d.precision, pb->d.ncell, 1, pb->d.mask, pb->d.hd, 0.0, nullptr, src,
                              pb->stream);
  if (e != cudaSuccess) return cuda_fail(pb, e, "warm start load");
  return write_state(pb, &s);
}

size_t mf_film_solve_gradient_work_bytes(const mf_problem* pb, int n_steps, int ckpt_every) {
  if (!pb || n_steps < 1 || ckpt_every < 1 || pb->d.dim != 2) return 0;
  const size_t C = (size_t)std::min(ckpt_every, n_steps);
  const size_t S = ((size_t)n_steps + C - 1) / C;
  // 2 fields per checkpoint (state, warm start), 3 stage inputs per step of a segment, 12 more
  return (2 * S + 3 * C + 12) * (size_t)pb->d.ncell * sizeof(double) + 64;
}

mf_status mf_film_solve_gradient(mf_problem* pb, int n_steps, const double* t_steps,
                                 const double* h_steps, const int* iters, int ckpt_every,
                                 const double* d_g0, const double* d_warm0, const double* d_target,
                                 void* d_work, size_t work_bytes, double* d_jcbar, double* knots_bar,
                                 int n_knots, double* d_warm0_bar, double* d_hz_T, double* loss) {
  Range range_("mf_film_solve_gradient");
  if (!pb || n_steps < 1 || ckpt_every < 1 || !t_steps || !h_steps || !iters || !d_g0 ||
      !d_target || !d_work || !loss)
    return MF_ERR_ARG;
  if (pb->d.dim != 2 || pb->d.nout <= 0 || pb->p.he_knots < 2) {
    pb->err = "the solve gradient needs a film with free space and a piecewise-linear h_e";
    return MF_ERR_ARG;
  }
  const bool want_grad = d_jcbar != nullptr || knots_bar != nullptr || d_warm0_bar != nullptr;
  if (want_grad && (!d_jcbar || !knots_bar || (d_warm0_bar && !d_warm0))) {
    pb->err = "a gradient needs d_jcbar and knots_bar (and d_warm0 for d_warm0_bar)";
    return MF_ERR_ARG;
  }
  const int K = pb->p.he_knots;
  if (knots_bar && n_knots != K) {
    pb->err = "n_knots differs from the problem's number of h_e knots";
    return MF_ERR_ARG;
  }
  for (int i = 0; i < 3 * n_steps; ++i)
    if (iters[i] < 1) { pb->err = "every call needs at least one outside iteration"; return MF_ERR_ARG; }
  if (work_bytes < mf_film_solve_gradient_work_bytes(pb, n_steps, ckpt_every)) {
    pb->err = "work buffer smaller than mf_film_solve_gradient_work_bytes";
    return MF_ERR_WORKSPACE;
  }
  MF_CUDA(pb, cudaSetDevice(pb->device));
  std::vector<double> kn(2 * K);
  MF_CUDA(pb, cudaMemcpyAsync(kn.data(), pb->d.he_t, 2 * K * sizeof(double), cudaMemcpyDeviceToHost, pb->stream));
  MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  const double* kt = kn.data();
  const double* kv = kn.data() + K;
  // each step inside one waveform segment
  std::vector<int> seg(n_steps);
  for (int i = 0; i < n_steps; ++i) {
    const double t = t_steps[i], h = h_steps[i];
    int k = (int)(std::upper_bound(kt, kt + K, t) - kt) - 1;
    if (!(h > 0.0) || k < 0 || k >= K - 1 || t + h > kt[k + 1] * (1.0 + 1e-15) + 1e-300) {
      pb->err = "every step must lie inside one segment of the h_e knots";
      return MF_ERR_ARG;
    }
    seg[i] = k;
  }
  const long long n = pb->d.ncell;
  const cudaStream_t st = pb->stream;
  const int C = std::min(ckpt_every, n_steps);
  const int S = (n_steps + C - 1) / C;
  double* CKY = (double*)d_work;                // S checkpointed states
  double* CKW = CKY + (size_t)S * n;            // S checkpointed warm starts
  double* GS = CKW + (size_t)S * n;             // 3 C stage inputs of one segment
  double* Y = GS + (size_t)3 * C * n;
  double* K1 = Y + n;
  double* K2 = K1 + n;
  double* K3 = K2 + n;
  double* LAM = K3 + n;
  double* V = LAM + n;
  double* G = V + n;
  double* JT = G + n;
  double* TMP = JT + n;
  double* OM0 = TMP + n;                        // cotangents of the warm start, in turn
  double* OM1 = OM0 + n;
  double* SC = OM1 + n;                         // 2 device scalars
  const double b1 = 2.0 / 9.0, b2 = 1.0 / 3.0, b3 = 4.0 / 9.0;
  auto lin = [&](double* out, std::initializer_list<std::pair<const double*, double>> terms,
                 double c = 0.0) -> mf_status {
    const double* x[4];
    double co[4];
    int m = 0;
    for (const auto& tc : terms) { x[m] = tc.first; co[m] = tc.second; ++m; }
    cudaError_t e = adj_lincomb(n, out, m, x, co, c, st);
    return e == cudaSuccess ? MF_OK : cuda_fail(pb, e, "lincomb");
  };
  // a call as the integrator makes it, with its frozen count; the stop tolerance is set to 0
  // for the duration so that a count that ends above it neither fails nor drops the warm start
  const double tol_saved = pb->d.iter_tol;
  auto set_tol = [&](double tol) -> mf_status {
    pb->d.iter_tol = tol;
    MF_CUDA(pb, cudaMemcpyAsync((void*)pb->d.dev, &pb->d, sizeof(Desc), cudaMemcpyHostToDevice, st));
    return MF_OK;
  };
  auto f = [&](const double* y, double* out, int step, int call) -> mf_status {
    return mf_rhs_ex(pb, t_steps[step], seg[step], y, out, iters[call], nullptr);
  };
  auto start_warm = [&](int s) -> mf_status {        // the warm start of segment s's first call
    if (s == 0 && !d_warm0) return mf_reset_warm(pb);
    return warm_load(pb, s == 0 ? d_warm0 : CKW + (size_t)s * n);
  };
  // one step from Y (kept stage inputs in gs when non-null)
  auto step_fwd = [&](int i, double* gs) -> mf_status {
    const double h = h_steps[i];
    if (gs) MF_CUDA(pb, cudaMemcpyAsync(gs, Y, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    MF_TRY_STATUS(f(Y, K1, i, 3 * i));
    double* y2 = gs ? gs + n : TMP;
    MF_TRY_STATUS(lin(y2, {{Y, 1.0}, {K1, 0.5 * h}}));
    MF_TRY_STATUS(f(y2, K2, i, 3 * i + 1));
    double* y3 = gs ? gs + 2 * n : TMP;
    MF_TRY_STATUS(lin(y3, {{Y, 1.0}, {K2, 0.75 * h}}));
    MF_TRY_STATUS(f(y3, K3, i, 3 * i + 2));
    return lin(Y, {{Y, 1.0}, {K1, h * b1}, {K2, h * b2}, {K3, h * b3}});
  };
  mf_status r = set_tol(0.0);
  auto body = [&]() -> mf_status {
    // forward over the frozen steps, a checkpoint (state and warm start) every C steps
    MF_CUDA(pb, cudaMemcpyAsync(Y, d_g0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    MF_TRY_STATUS(start_warm(0));
    for (int i = 0; i < n_steps; ++i) {
      if (i % C == 0) {
        MF_CUDA(pb, cudaMemcpyAsync(CKY + (size_t)(i / C) * n, Y, n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
        if (i > 0) MF_TRY_STATUS(warm_save(pb, CKW + (size_t)(i / C) * n));
      }
      MF_TRY_STATUS(step_fwd(i, nullptr));
    }
    // loss: res = h_z(T) - target
    const double T = t_steps[n_steps - 1] + h_steps[n_steps - 1];
    int kT = (int)(std::upper_bound(kt, kt + K, T) - kt) - 1;
    kT = std::min(std::max(kT, 0), K - 2);
    const double wT = (T - kt[kT]) / (kt[kT + 1] - kt[kT]);
    const double heT = kv[kT] + wT * (kv[kT + 1] - kv[kT]);
    const double dA = pb->d.dx * pb->d.dy;
    MF_TRY_STATUS(mf_readout_of(pb, MF_READ_HZ, T, Y, TMP));
    if (d_hz_T) MF_CUDA(pb, cudaMemcpyAsync(d_hz_T, TMP, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    MF_TRY_STATUS(lin(TMP, {{TMP, 1.0}, {d_target, -1.0}}));
    double sums[2];
    {
      cudaError_t e = adj_sums(n, TMP, SC, st);
      if (e != cudaSuccess) return cuda_fail(pb, e, "sums");
    }
    MF_CUDA(pb, cudaMemcpyAsync(sums, SC, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MF_CUDA(pb, cudaStreamSynchronize(st));
    *loss = 0.5 * dA * sums[1];
    if (!want_grad) return MF_OK;
    for (int k = 0; k < K; ++k) knots_bar[k] = 0.0;
    knots_bar[kT] += (1.0 - wT) * dA * sums[0];
    knots_bar[kT + 1] += wT * dA * sums[0];
    // cotangent of the final state: lambda = dA K_h res (h_z readout of res, minus its h_e)
    MF_TRY_STATUS(mf_readout_of(pb, MF_READ_HZ, T, TMP, V));
    MF_TRY_STATUS(lin(LAM, {{V, dA}}, -dA * heT));
    MF_CUDA(pb, cudaMemsetAsync(d_jcbar, 0, n * sizeof(double), st));
    const double* om = nullptr;                  // cotangent of the last call's iterate
    double* om_next = OM0;
    // reverse sweep, segment by segment: recompute the segment's stage inputs from its
    // checkpoint, then the three products per step with the warm-start cotangent carried
    for (int s = S - 1; s >= 0; --s) {
      const int i0 = s * C, i1 = std::min(n_steps, i0 + C);
      MF_CUDA(pb, cudaMemcpyAsync(Y, CKY + (size_t)s * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      MF_TRY_STATUS(start_warm(s));
      for (int i = i0; i < i1; ++i) MF_TRY_STATUS(step_fwd(i, GS + (size_t)3 * (i - i0) * n));
      for (int i = i1 - 1; i >= i0; --i) {
        const double h = h_steps[i];
        const double* g1 = GS + (size_t)3 * (i - i0) * n;
        double sb[3];
        auto vjp = [&](const double* g, int call, double* gbar, double* sbo) -> mf_status {
          MF_TRY_STATUS(mf_film_rhs_vjp_warm(pb, iters[call], g, V, om, gbar, JT, om_next, sbo));
          om = om_next;
          om_next = om_next == OM0 ? OM1 : OM0;
          return lin(d_jcbar, {{d_jcbar, 1.0}, {JT, 1.0}});
        };
        MF_TRY_STATUS(lin(V, {{LAM, h * b3}}));
        MF_TRY_STATUS(vjp(g1 + 2 * n, 3 * i + 2, K3, &sb[2]));               // k3 = f(y + 3h/4 k2)
        MF_TRY_STATUS(lin(V, {{LAM, h * b2}, {K3, 0.75 * h}}));
        MF_TRY_STATUS(vjp(g1 + n, 3 * i + 1, K2, &sb[1]));                    // k2 = f(y + h/2 k1)
        MF_TRY_STATUS(lin(V, {{LAM, h * b1}, {K2, 0.5 * h}}));
        MF_TRY_STATUS(vjp(g1, 3 * i, K1, &sb[0]));                            // k1 = f(y)
        MF_TRY_STATUS(lin(LAM, {{LAM, 1.0}, {K3, 1.0}, {K2, 1.0}, {K1, 1.0}}));
        const int k = seg[i];
        const double dt = kt[k + 1] - kt[k];
        const double sbar = sb[0] + sb[1] + sb[2];                           // h_e_dot = slope of k
        knots_bar[k + 1] += sbar / dt;
        knots_bar[k] -= sbar / dt;
      }
    }
    // a cold first call starts from h_e_dot on free space, whose cotangent sums to zero; a given
    // first warm start gets its cotangent
    if (d_warm0_bar)
      MF_CUDA(pb, cudaMemcpyAsync(d_warm0_bar, om, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    return MF_OK;
  };
  if (r == MF_OK) r = body();
  const std::string err = pb->err;
  const mf_status r2 = set_tol(tol_saved);
  mf_reset_warm(pb);                            // the calls used the warm start's buffers
  MF_CUDA(pb, cudaStreamSynchronize(st));
  pb->err = err;
  return r != MF_OK ? r : r2;
}

mf_status mf_set_jc_map(mf_problem* pb, const double* d_jc) {
  if (!pb || !d_jc) return MF_ERR_ARG;
  if (!pb->d.jcmap) {
    pb->err = "the problem was created without a jc map";
    return MF_ERR_ARG;
  }
  MF_CUDA(pb, cudaSetDevice(pb->device));
  const long long n = pb->d.ncell;
  if (pb->d.precision) {
    cudaError_t e = adj_to_float(n, d_jc, (float*)pb->d.jcmap, pb->stream);
    if (e != cudaSuccess) return cuda_fail(pb, e, "jc map conversion");
  } else {
    MF_CUDA(pb, cudaMemcpyAsync((void*)pb->d.jcmap, d_jc, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                pb->stream));
  }
  MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  return MF_OK;
}

mf_status mf_set_knot_values(mf_problem* pb, const double* h_values, int n_values) {
  if (!pb || !h_values) return MF_ERR_ARG;
  if (pb->p.he_knots < 1) {
    pb->err = "the problem's h_e is not piecewise linear";
    return MF_ERR_ARG;
  }
  if (n_values != pb->p.he_knots) {
    pb->err = "n_values differs from the problem's number of h_e knots";
    return MF_ERR_ARG;
  }
  MF_CUDA(pb, cudaSetDevice(pb->device));
  MF_CUDA(pb, cudaMemcpyAsync((void*)pb->d.he_v, h_values, pb->p.he_knots * sizeof(double),
                              cudaMemcpyHostToDevice, pb->stream));
  MF_CUDA(pb, cudaStreamSynchronize(pb->stream));      // the values are a host buffer
  return MF_OK;
}

mf_status mf_get_info(mf_problem* pb, mf_info* out) {
  if (!pb || !out) return MF_ERR_ARG;
  SolverState s;
  mf_status r = read_state(pb, &s);
  if (r != MF_OK) return r;
  std::memset(out, 0, sizeof(*out));
  out->t = s.t; out->h = s.h;
  out->n_attempts = s.n_attempts; out->n_accepted = s.n_accepted; out->n_rejected = s.n_rejected;
  out->n_rhs = s.n_rhs; out->n_iters = s.n_iters; out->n_noconv = s.n_noconv;
  out->log_count = s.log_count; out->last_iters = s.last_iters;
  out->last_r = s.last_r; out->last_err = s.last_err;
  out->grid = pb->d.grid; out->threads = NT;
  out->smem_bytes = (int)kernel_smem_bytes(pb->d);
  out->rows_per_item = pb->d.rows_per_item;
  out->workspace_used = (long long)pb->used;
  return MF_OK;
}

mf_status mf_get_log(mf_problem* pb, mf_step_log* out, long long cap, long long* count) {
  if (!pb) return MF_ERR_ARG;
  SolverState s;
  mf_status r = read_state(pb, &s);
  if (r != MF_OK) return r;
  const long long n = std::min(std::min(s.log_count, (long long)LOG_CAP), cap);
  if (count) *count = s.log_count;
  static_assert(sizeof(mf_step_log) == sizeof(StepLog), "log layout");
  if (n > 0 && out) {
    MF_CUDA(pb, cudaMemcpyAsync(out, pb->d.log, n * sizeof(StepLog), cudaMemcpyDeviceToHost, pb->stream));
    MF_CUDA(pb, cudaStreamSynchronize(pb->stream));
  }
  return MF_OK;
}

const char* mf_last_error(const mf_problem* pb) { return pb ? pb->err.c_str() : "null handle"; }

void mf_destroy(mf_problem* pb) { delete pb; }

}  // extern "C"
