// Common device-side types for the FFT method-of-lines kernels (sm_103a).
//
// Complex arithmetic, the problem descriptor shared by all phases, the device-resident
// integrator state, a bounded grid-wide barrier for the persistent cooperative kernels and
// deterministic block reductions.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mf {

constexpr int NT = 256;           // threads per CTA of the persistent kernels
constexpr int VPT = 16;           // complex values each thread holds per FFT stage
constexpr int BATCH = NT * VPT;   // complex points one CTA transforms at once (4096)
// shared-memory position of FFT element e: one padding slot every 16 complex values keeps the
// strided butterfly writes of the early Stockham stages to at most 2-way bank conflicts
__host__ __device__ __forceinline__ constexpr int sp(int e) { return e + (e >> 4); }
constexpr int BATCH_PAD = BATCH + BATCH / 16;

// The dynamic shared memory of the persistent kernels: two FFT buffers of BATCH_PAD complex
// values each.  Passes address it by element offset from this base, so that every access is a
// shared-memory access with 32-bit index arithmetic.
extern __shared__ __align__(16) unsigned char mf_dsmem[];

// ------------------------------------------------------------------------------------------
// complex numbers
// ------------------------------------------------------------------------------------------
// 8-byte (float) or 16-byte (double) alignment so that a complex value moves as one vector access
template <typename T> struct alignas(2 * sizeof(T)) C2 { T x, y; };
template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ C2<T> cconj(C2<T> a) { return {a.x, -a.y}; }
template <typename T> __device__ __forceinline__ C2<T> cscale(C2<T> a, T s) { return {a.x * s, a.y * s}; }
// a * (s i) for s = +-1
template <typename T> __device__ __forceinline__ C2<T> cmul_si(C2<T> a, int s) {
  return s > 0 ? C2<T>{-a.y, a.x} : C2<T>{a.y, -a.x};
}

template <typename T> __device__ __forceinline__ C2<T>* dsm() { return reinterpret_cast<C2<T>*>(mf_dsmem); }
// element offset of a pointer into the dynamic shared memory
template <typename T> __device__ __forceinline__ int dsm_off(const C2<T>* p) { return (int)(p - dsm<T>()); }

// Loads with L1 placement hints.  Tables (twiddles, wavenumbers) are read over and over and
// should stay in L1 (evict_last); field data streams through once per pass and should not
// displace them (no_allocate).  ldg_* use the read-only path and are only for data that no
// thread writes during the launch (plain asm: the compiler may move and batch them); lds_* are
// coherent loads for data written by earlier phases (volatile, ordered with the barriers).
__device__ __forceinline__ C2<float> ldg_c2(const C2<float>* p) {
  float2 v;
  asm("ld.global.nc.L1::evict_last.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return {v.x, v.y};
}
__device__ __forceinline__ C2<double> ldg_c2(const C2<double>* p) {
  double2 v;
  asm("ld.global.nc.L1::evict_last.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return {v.x, v.y};
}
__device__ __forceinline__ float ldg_tab(const float* p) {
  float v;
  asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ldg_tab(const double* p) {
  double v;
  asm("ld.global.nc.L1::evict_last.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ C2<float> lds_c2(const C2<float>* p) {
  float2 v;
  asm volatile("ld.global.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p) : "memory");
  return {v.x, v.y};
}
__device__ __forceinline__ C2<double> lds_c2(const C2<double>* p) {
  double2 v;
  asm volatile("ld.global.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p) : "memory");
  return {v.x, v.y};
}

// ------------------------------------------------------------------------------------------
// status codes (mirrors mf_status of the C interface)
// ------------------------------------------------------------------------------------------
enum : int { ST_OK = 0, ST_ARG = 1, ST_CUDA = 2, ST_NOCONV = 3, ST_NONFINITE = 4,
             ST_UNDERFLOW = 5, ST_WORKSPACE = 6, ST_BARRIER = 7 };

// ------------------------------------------------------------------------------------------
// device-resident solver state (one per problem, in the workspace)
// ------------------------------------------------------------------------------------------
struct StepLog {                 // one attempted BS23 step
  double t, h, t_new, err;
  int outcome;                   // 0 reject (error), 1 accept, 2 reject (iteration failed)
  int iters[4];                  // outside iterations of k1..k4, -1 when not evaluated
  int pad;
};

struct SolverState {
  double t, h;
  double A_prev;                 // shift still to subtract on free space from the warm h_dot (2D)
  int warm_valid;                // the most recent call's h_dot iterate is a usable start
  int com_valid;                 // (2D) an accepted step's h_dot is the initial approximation
  int hd_sel;                    // (2D) h_dot buffer the next call writes; the other one is committed
  double A_com;                  // (2D) shift still to subtract from the committed h_dot
  int k1_valid;                  // first-same-as-last derivative available
  int failed;                    // the previous attempt was rejected
  int ybuf, ynewbuf, k1buf, k4buf;   // rotation of the FP64 state buffers
  int status;                    // sticky error status of the last launch
  int last_iters;                // iterations of the last right-hand side
  long long n_attempts, n_accepted, n_rejected, n_rhs, n_iters, n_noconv;
  long long log_count;
  double last_r;                 // last convergence residual
  double last_err;
  double q11;                    // (2D) sum over free space of q1 = F^-1[K1 F(out)] (set-up)
  double pad[2];
};

// Barrier state of one launch (zeroed before every launch).  `count` is a monotonic arrival
// counter: the k-th barrier of the launch is passed once it reaches k * grid.  Bit 63 is the
// abort flag, so one polled word carries both.
constexpr unsigned long long BARRIER_ABORT = 1ull << 63;
struct alignas(128) GridBarrier {
  unsigned long long count;
  int where;                     // site number of the barrier whose wait timed out
  unsigned int pad0[29];
};


// ------------------------------------------------------------------------------------------
// problem descriptor (kernel argument, plain data)
// ------------------------------------------------------------------------------------------
struct Desc {
  int dim, nx, ny, nz;
  int precision;                 // 0 FP64 transforms, 1 FP32 transforms
  int lgx, lgy, lgz;
  double Lx, Ly, Lz, dx, dy, dz;
  double n, e0, jc, rho_out, sigma, lam, iter_tol;
  double gamma, b0;              // elliptic anisotropy (1: isotropic); Kim field scale (0: none)
  int iter_max;
  double rtol, atol, h_min;
  // applied field
  int he_knots;
  const double* he_t;
  const double* he_v;
  double he_sin_amp, he_sin_period;
  double he_dir[3];
  // counts
  long long ncell;               // nx ny nz
  long long nout;                // free-space cells
  long long nspec;               // complex values of one half spectrum ((nx/2+1) ny nz)
  // device buffers (transform precision T unless noted)
  void* Sa;                      // spectra, 3 fields
  void* Sb;                      // spectra, 3 fields (3D: second buffer of the transpose chain)
  void* hd;                      // h_dot iterate (1 or 3 fields)
  void* hd2;                     // second h_dot buffer (2D: the previous time step's h_dot)
  void* u;                       // raw g_dot (2D)
  void* q1;                      // F^-1[K1 F(out)] (2D)
  void* q2;                      // F^-1[K2 F(out)] (2D)
  const void* jcmap;             // per-cell jc or null
  const uint8_t* mask;
  const void* tw_x; const void* tw_y; const void* tw_z;   // twiddle tables exp(-2 pi i j / n)
  const void* ktab;              // wavenumbers: kx (nx/2+1 values), ky (ny), kz (nz)
  const void* gtab;              // Gaussian factors exp(-k^2 sigma^2 / 2), same layout
  double* fbuf[6];               // FP64 state buffers (y, y_new, k1..k4 under rotation)
  double* partials;              // per-work-item partial reductions
  int max_items;
  SolverState* st;
  GridBarrier* gb;
  StepLog* log;
  long long log_cap;
  int rows_per_item;             // 2D row pass / 3D x pass rows per work item (even)
  int zs_per_item;               // 3D y pass z-lines per work item
  int grid;                      // CTAs of the persistent launch
  unsigned long long barrier_ns; // time limit of one grid-barrier wait (ns)
  const struct Desc* dev;        // device copy of this descriptor (what the kernels read)
};

// ------------------------------------------------------------------------------------------
// bounded grid barrier for cooperative launches.  Every CTA is co-resident (cooperative
// launch), so the wait ends unless a CTA has already left; a wait that exceeds the time
// limit raises the abort flag, which every waiter polls, so all CTAs leave promptly.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

constexpr unsigned long long BARRIER_LIMIT_NS = 4000000000ull;   // default: 4 s per barrier

// Returns false when the launch must stop (abort raised).  `passed` counts the barriers this
// CTA has passed in the launch (shared memory, written by thread 0 only, zero at launch).
// Arrival is a fire-and-forget release add after the CTA barrier; the wait polls the same word
// with acquire loads.  A wait longer than `limit_ns` raises the abort flag.
__device__ __forceinline__ bool grid_sync(GridBarrier* gb, unsigned int nblocks, int where,
                                          unsigned long long* passed,
                                          unsigned long long limit_ns = BARRIER_LIMIT_NS) {
  __shared__ int s_ok;
  const unsigned long long lim = limit_ns ? limit_ns : BARRIER_LIMIT_NS;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long target = (*passed + 1) * nblocks;
    *passed += 1;
    red_release_add_u64(&gb->count, 1ull);
    unsigned long long v = ld_acquire_u64(&gb->count);
    if ((v & ~BARRIER_ABORT) < target && !(v & BARRIER_ABORT)) {
      const unsigned long long t0 = globaltimer_ns();
      unsigned int nap = 32;
      do {
        __nanosleep(nap);
        if (nap < 128) nap <<= 1;
        if (globaltimer_ns() - t0 > lim) {
          atomicOr(&gb->count, BARRIER_ABORT);
          atomicExch(&gb->where, where);
          v |= BARRIER_ABORT;
          break;
        }
        v = ld_acquire_u64(&gb->count);
      } while ((v & ~BARRIER_ABORT) < target && !(v & BARRIER_ABORT));
    }
    s_ok = (v & BARRIER_ABORT) ? 0 : 1;
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------------------------------------
// deterministic block reductions (fixed tree) of NT values
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// sum over the CTA of single-precision partials (warp level in FP32, across warps in FP64);
// result valid in all threads
__device__ __forceinline__ double block_sum(float v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = (double)v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < NT / 32) ? red[l] : 0.0;
    s = warp_sum(s);
    if (l == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}
// sum over the CTA; result valid in all threads.  `red` holds NT/32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < NT / 32) ? red[l] : 0.0;
    s = warp_sum(s);
    if (l == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}
__device__ __forceinline__ double block_max(double v, double* red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (l < NT / 32) ? red[l] : 0.0;
    s = warp_max(s);
    if (l == 0) red[0] = s;
  }
  __syncthreads();
  s = red[0];
  __syncthreads();
  return s;
}

// Sum (or max) of partials[slot * max_items + i] over i < n, in a fixed order, computed
// identically by every CTA.
// The first warp does it alone (loads through L2 only: the partials were written by other CTAs
// in this launch), so the CTA synchronises once instead of four times.
__device__ __forceinline__ double reduce_partials(const double* partials, int max_items, int slot,
                                                  int n, bool is_max, double* red) {
  const double* p = partials + (size_t)slot * max_items;
  if (threadIdx.x < 32) {
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) {
      const double x = __ldcg(p + i);
      v = is_max ? fmax(v, x) : v + x;
    }
    v = is_max ? warp_max(v) : warp_sum(v);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double s = red[0];
  __syncthreads();
  return s;
}

// Sums of two slots over i < n (fixed order, as reduce_partials), read in one pass by the first
// warp; red[0], red[1] receive them.  The caller combines them in thread 0 and broadcasts.
__device__ __forceinline__ void reduce_partials2(const double* partials, int max_items, int slot_a,
                                                 int slot_b, int n, double* red) {
  if (threadIdx.x < 32) {
    const double* pa = partials + (size_t)slot_a * max_items;
    const double* pb = partials + (size_t)slot_b * max_items;
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) {
      a += __ldcg(pa + i);
      b += __ldcg(pb + i);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    if (threadIdx.x == 0) { red[0] = a; red[1] = b; }
  }
}

// ------------------------------------------------------------------------------------------
// launch arguments of the persistent kernels
// ------------------------------------------------------------------------------------------
enum Mode { MODE_RHS = 0, MODE_ADVANCE = 1, MODE_HZ = 2, MODE_SETUP = 3, MODE_MOMENT = 4,
            MODE_J = 5, MODE_E = 6 };

struct KernelArgs {
  int mode;
  double t;                   // MODE_RHS / MODE_HZ / MODE_J / MODE_E: time
  double t_target;            // MODE_ADVANCE
  long long max_attempts;     // MODE_ADVANCE
  const double* y_in;         // MODE_RHS / MODE_HZ / MODE_MOMENT / MODE_J input (FP64)
  double* out;                // MODE_RHS: derivative; MODE_HZ: h_z; MODE_J: j; MODE_E: e; MODE_MOMENT
  int force_iters;            // > 0: run exactly this many outside iterations
  int seg;                    // waveform segment for MODE_RHS (-2: from t)
};

// One film of a shared launch (film_batch_kernel): CTAs [b0, b0 + nb) of the launch advance
// it, with the film's own grid barrier, items and partials; nothing is shared between films.
struct BatchJob {
  const Desc* desc;           // the film's descriptor (device memory)
  double t_target;
  long long max_attempts;
  int b0, nb;
};
constexpr int MAX_BATCH = 256;
// passed by value as the kernel parameter (8 KB, under the 32 KB parameter limit)
struct BatchTable {
  int n;
  BatchJob job[MAX_BATCH];
};

// launch helpers implemented next to each kernel
cudaError_t film_launch(int precision, const Desc& d, const KernelArgs& a, cudaStream_t s);
cudaError_t film_batch_launch(int precision, const BatchTable& tab, int grid, cudaStream_t s);
int film_batch_max_blocks(int precision, size_t smem);
cudaError_t bulk_launch(int precision, const Desc& d, const KernelArgs& a, cudaStream_t s);
int film_max_blocks(int precision, size_t smem);
int bulk_max_blocks(int precision, size_t smem);
size_t kernel_smem_bytes(const Desc& d);

}  // namespace mf
