// Pieces shared by the film (2D) and bulk (3D) right-hand sides: the applied field h_e(t),
// the stage input of the integrator, per-CTA scalars and epilogue/result records.
#pragma once
#include <new>

#include "mf_passes.cuh"

namespace mf {

constexpr double PI_D = 3.14159265358979323846;

// stage input y + sum c_j k_j (FP64), optionally written to ynew
struct StageIn {
  const double* y;
  int nk;
  double c[3];
  const double* k[3];
  double* ynew;
};

// per-CTA copy of the scalars every CTA agrees on
struct Shared {
  double red[NT / 32];
  double A, C, r, hed;
  int warm_valid;
  double A_prev;
  int com_valid, hd_sel;         // (2D) accepted-step initial approximation, see SolverState
  double A_com;
  double q11;                    // (2D) sum over free space of q1 (from the solver state)
  int attempt_first;             // (2D) the next right-hand side is the first of a step attempt
  unsigned long long bar_passed;  // grid barriers passed in this launch (thread 0)
  unsigned long long tma_bar;     // (3D) mbarrier of the bulk copies into the staging buffer
  unsigned tma_parity;            // (3D) phase parity the next wait on tma_bar expects
};

// ------------------------------------------------------------------------------------------
// applied field
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ int he_segment(const Desc& d, double t) {
  if (d.he_knots <= 0) return 0;
  int k = -1;
  for (int i = 0; i < d.he_knots; ++i)
    if (d.he_t[i] <= t) k = i;
  return k;
}
__device__ __forceinline__ double he_value(const Desc& d, double t) {
  if (d.he_knots <= 0) return d.he_sin_amp * sin(2.0 * PI_D * t / d.he_sin_period);
  const int k = he_segment(d, t);
  if (k < 0) return d.he_v[0];
  if (k >= d.he_knots - 1) return d.he_v[d.he_knots - 1];
  const double s = (t - d.he_t[k]) / (d.he_t[k + 1] - d.he_t[k]);
  return d.he_v[k] + s * (d.he_v[k + 1] - d.he_v[k]);
}
__device__ __forceinline__ double he_dot(const Desc& d, double t, int seg) {
  if (d.he_knots <= 0) {
    const double w = 2.0 * PI_D / d.he_sin_period;
    return d.he_sin_amp * w * cos(w * t);
  }
  const int k = (seg == -2) ? he_segment(d, t) : seg;
  if (k < 0 || k >= d.he_knots - 1) return 0.0;
  return (d.he_v[k + 1] - d.he_v[k]) / (d.he_t[k + 1] - d.he_t[k]);
}
__device__ __forceinline__ double he_next_knot(const Desc& d, double t) {
  for (int i = 0; i < d.he_knots; ++i)
    if (d.he_t[i] > t) return d.he_t[i];
  return INFINITY;
}

// Acc is the type of the per-thread partial sums: the transform precision T in the epilogues of
// the outside iteration (FP64 arithmetic runs at a small fraction of the FP32 rate on this part),
// double where a sum feeds the integrator's error norm or a readout.  The partials of a CTA
// are combined in double.
template <typename T, typename Acc = double>
struct EpiBase {
  Acc acc = 0, accmax = 0;
  Acc acc2 = 0;                 // a second sum (rows() with a second slot)
  bool is_max = false;
  // kPair: the epilogue also has pair(ia, ib, ...) for the two rows of a cell pair, which issues
  // every load of both before any store (a store may alias a later load as far as the compiler
  // knows, so two separate calls would wait for the first call's loads before the second's)
  static constexpr bool kPair = false;
};

struct RhsOut {
  int status, iters;
  double r;
  double err;          // BS23 error norm when requested
  int nonfinite;
};


// ------------------------------------------------------------------------------------------
// BS23 integrator loop shared by the film and bulk kernels: adaptive steps until t_target or
// max_attempts, first same as last, every decision taken identically by every CTA.
// R(t, seg, stage_in, k_out, force_iters, want_err, h, k1, k2, k3, y, ynew) evaluates one
// right-hand side.  Returns the launch status.
// ------------------------------------------------------------------------------------------
template <class Rhs>
__device__ int bs23_advance(Rhs& R, const Desc& d, SolverState* st, const KernelArgs& a, bool leader) {
  int status = ST_OK;
    // BS23 with first-same-as-last, all decisions on the device
    double t = st->t, h = st->h;
    int failed = st->failed, k1_valid = st->k1_valid;
    int iy = st->ybuf, iyn = st->ynewbuf, ik1 = st->k1buf, ik4 = st->k4buf;
    // k2, k3 live in the two remaining buffers
    int others[2], no = 0;
    for (int b = 0; b < 6 && no < 2; ++b)
      if (b != iy && b != iyn && b != ik1 && b != ik4) others[no++] = b;
    const int ik2 = others[0], ik3 = others[1];
    long long att = 0, n_rhs = 0, n_it = 0, n_acc = 0, n_rej = 0, n_nc = 0;
    double last_r = 0.0, last_err = 0.0;
    while (t < a.t_target && att < a.max_attempts) {
      const double t_lim = fmin(a.t_target, he_next_knot(d, t));
      const double h_prop = h;         // the controller's proposal before clipping
      const bool clipped = t + 1.1 * h >= t_lim;
      if (clipped) h = t_lim - t;
      R.on_attempt();                  // the attempt's first evaluation starts from the accepted step
      const int seg = he_segment(d, t);
      int it[4] = {-1, -1, -1, -1};
      double* y = d.fbuf[iy];
      double* yn = d.fbuf[iyn];
      double* k1 = d.fbuf[ik1];
      double* k2 = d.fbuf[ik2];
      double* k3 = d.fbuf[ik3];
      double* k4 = d.fbuf[ik4];
      RhsOut r;
      r.status = ST_OK;
      r.r = 0.0;
      if (!k1_valid) {
        // a k1 whose outside iteration did not converge rejects the attempt like any other
        // stage; the warm start keeps the progress, so the next attempt continues from it
        StageIn in{y, 0, {0, 0, 0}, {nullptr, nullptr, nullptr}, nullptr};
        r = R(t, seg, in, k1, 0, false, 0, nullptr, nullptr, nullptr, nullptr, nullptr);
        ++n_rhs; n_it += r.iters; it[0] = r.iters;
        if (r.status == ST_BARRIER) { status = ST_BARRIER; break; }
        if (r.status == ST_OK && r.nonfinite) { status = ST_NONFINITE; break; }
        if (r.status == ST_OK) k1_valid = 1;
      }
      int outcome = 1;
      double err = INFINITY;
      if (r.status == ST_OK) {
        StageIn s2{y, 1, {0.5 * h, 0, 0}, {k1, nullptr, nullptr}, nullptr};
        r = R(t + 0.5 * h, seg, s2, k2, 0, false, 0, nullptr, nullptr, nullptr, nullptr, nullptr);
        ++n_rhs; n_it += r.iters; it[1] = r.iters;
        if (r.status == ST_BARRIER) { status = ST_BARRIER; break; }
      }
      if (r.status == ST_OK) {
        StageIn s3{y, 1, {0.75 * h, 0, 0}, {k2, nullptr, nullptr}, nullptr};
        r = R(t + 0.75 * h, seg, s3, k3, 0, false, 0, nullptr, nullptr, nullptr, nullptr, nullptr);
        ++n_rhs; n_it += r.iters; it[2] = r.iters;
        if (r.status == ST_BARRIER) { status = ST_BARRIER; break; }
      }
      const double t_new = clipped ? t_lim : t + h;
      if (r.status == ST_OK) {
        StageIn s4{y, 3, {h * (2.0 / 9.0), h * (1.0 / 3.0), h * (4.0 / 9.0)}, {k1, k2, k3}, yn};
        r = R(t_new, seg, s4, k4, 0, true, h, k1, k2, k3, y, yn);
        ++n_rhs; n_it += r.iters; it[3] = r.iters;
        if (r.status == ST_BARRIER) { status = ST_BARRIER; break; }
        if (r.status == ST_OK) err = r.err;
      }
      last_r = r.r;
      if (r.status != ST_OK) { outcome = 2; ++n_nc; }
      else outcome = err <= 1.0 ? 1 : 0;
      if (leader && st->log_count < d.log_cap) {
        StepLog L; L.t = t; L.h = h; L.t_new = outcome == 1 ? t_new : t; L.err = err;
        L.outcome = outcome; for (int q = 0; q < 4; ++q) L.iters[q] = it[q]; L.pad = 0;
        d.log[st->log_count] = L;
      }
      if (leader) st->log_count += 1;
      ++att;
      if (outcome == 1) {
        R.on_accept();                 // the last evaluation's iterate starts later calls
        const bool knot_hit = clipped && t_lim == he_next_knot(d, t);
        t = t_new;
        int tmp = iy; iy = iyn; iyn = tmp;
        tmp = ik1; ik1 = ik4; ik4 = tmp;
        k1_valid = knot_hit ? 0 : 1;
        double fac = err == 0.0 ? 5.0 : fmin(5.0, fmax(0.2, 0.9 * pow(err, -1.0 / 3.0)));
        if (failed) fac = fmin(fac, 1.0);
        // a step shortened to end on a knot or output time says nothing about longer steps:
        // the next one starts from the proposal it replaced (never above it)
        h = (clipped && h < h_prop) ? h_prop * fmin(fac, 1.0) : h * fac;
        failed = 0;
        ++n_acc;
        last_err = err;
      } else if (outcome == 0) {
        h = h * fmax(0.2, 0.9 * pow(err, -1.0 / 3.0));
        failed = 1;
        ++n_rej;
      } else {
        h = 0.5 * h;
        failed = 1;
        ++n_rej;
      }
      if (h < d.h_min) { status = ST_UNDERFLOW; break; }
    }
    if (leader) {
      st->t = t; st->h = h; st->failed = failed; st->k1_valid = k1_valid;
      st->ybuf = iy; st->ynewbuf = iyn; st->k1buf = ik1; st->k4buf = ik4;
      st->n_attempts += att; st->n_rhs += n_rhs; st->n_iters += n_it; st->n_accepted += n_acc;
      st->n_rejected += n_rej; st->n_noconv += n_nc; st->last_r = last_r; st->last_err = last_err;
    }
    return status;
}

}  // namespace mf
