// scan_ops.cuh -- the parallel filter / smoother algebra of Corenflos, Zhao,
// Sarkka, "Temporal Gaussian Process Regression in Logarithmic Time", as
// per-thread register code.
//
// Coordinates: everything on the device is in the balanced basis z = D^{-1} x
// of Sec. 4.2 scaled so that the measurement row is H = e_0^T; then
// S = P_00 + R and K = P[:,0] / S need no multiplication by H.
#pragma once
#include "linalg.cuh"

namespace pssgp {

constexpr int NT = 16;          // Taylor coefficients per entry (pssgp.h: PSSGP_NTAYLOR)

template <int D> struct Sym { static constexpr int N = D * (D + 1) / 2; };
template <int D>
__host__ __device__ constexpr int pidx(int i, int j) {   // packed upper index, i <= j
  return i * D - i * (i - 1) / 2 + (j - i);
}

// Model constants for the kernels (passed by value: constant bank, uniform
// across the warp).  F_e(h) = sum_m fc[e][m] h^m; Q_e(h) = h sum_m qc[e][m] h^m
// for packed upper entries e; K terms suffice for h <= hthr_*[K]; steps longer
// than hmax are halved and doubled back.
template <int D>
struct DevModel {
  double Pinf[Sym<D>::N];
  double Dsc[D];                // x = Dsc .* z
  double fc[D * D][NT];
  double qc[Sym<D>::N][NT];
  double rsup[D][D];            // companion row recursion (see pssgp.h)
  double rlast[D][D];
  double wg[D];                 // W[d-1][d-1] / G[i][i+1] (companion Q rows)
  int qrows;                    // companion drift and W = w e_{d-1} e_{d-1}^T
  float hthr_f[NT + 1];
  float hthr_q[NT + 1];
  float hmax;
  int companion;
  // mixed precision: the terms from the split point on (table hthr_*32) are
  // summed in FP32 with these coefficients
  float fc32[D * D][NT];
  float qc32[Sym<D>::N][NT];
  float hthr_f32[NT + 1];
  float hthr_q32[NT + 1];
};

// ---------------------------------------------------------------------------
// Discretisation (supplement Eq. (ss-gp-formation)): F = exp(hG),
// Q = int_0^h e^{sG} W e^{sG}^T ds, by the Taylor series of both in h with
// host-precomputed coefficients.  The term counts are chosen per warp from the
// warp's longest step against bounds built from the exact norms ||G^m||, ||W_m||
// (float arithmetic, off the FP64 pipe).  For a companion-form drift only row 0
// of F is summed; row i+1 is row i times G scaled (2 FP64 ops per entry); with
// a rank-one diffusion on the last state also only row 0 of Q is summed and
// the other rows follow from the Lyapunov identity (companion_q_rows).
// Steps longer than hmax are halved s times and doubled back with
// F(2h) = F(h)^2, Q(2h) = F(h) Q(h) F(h)^T + Q(h).
// first = true gives the prior at a series' first time: F = 0, Q = P_inf.
// Must be called by all 32 lanes of a warp (warp reductions inside).
// ---------------------------------------------------------------------------
// s doublings F <- F F, Q <- F Q F^T + Q
template <int D>
__device__ __forceinline__ void double_steps_body(Mat<D>& F, Mat<D>& Q, int s, int smax) {
#pragma unroll 1
  for (int r = 0; r < smax; ++r) {
    if (r < s) {
      Mat<D> T, Q2, F2;
      mul<D>(F, Q, T);
      mul_Bt_sym_add<D>(T, F, Q, Q2);
      mul<D>(F, F, F2);
      copy<D>(Q2, Q);
      copy<D>(F2, F);
    }
  }
}
// out of line (rare path) for kernels whose registers are needed elsewhere;
// the call keeps F and Q in a stack frame.  Kernels that only discretise
// take the inline body (INL below) and need no frame.
template <int D>
__device__ __noinline__ void double_steps(Mat<D>& F, Mat<D>& Q, int s, int smax) {
  double_steps_body<D>(F, Q, s, smax);
}

// Rows 1..d-1 of Q from its row 0 and the last column f of F, for a
// companion drift (rows 0..d-2 of G hold only g_i = G[i][i+1]) and a rank-one
// diffusion W = w e_{d-1} e_{d-1}^T.  Differentiating
// Q(h) = int_0^h e^{sG} W e^{sG}^T ds gives G Q + Q G^T = F W F^T - W, whose
// entries (i, j), i < d-1, read
//   g_i Q[i+1][j] + g_j Q[i][j+1]               = w f_i f_j    (j < d-1)
//   g_i Q[i+1][d-1] + sum_k G[d-1][k] Q[i][k]   = w f_i f_{d-1}
// so row i+1 follows from row i in O(d) operations per entry instead of a
// Taylor sum.  For steps short against the model's scale the two sides of
// each line are of the same order in h and every entry keeps its relative
// accuracy; for long steps the error is small against sqrt(Q_ii Q_jj).
// qscale multiplies w (Q is linear in W).  Row 0 must be complete on entry.
template <int D>
__device__ __forceinline__ void companion_q_rows(const DevModel<D>& m, const Mat<D>& F, Mat<D>& Q,
                                                 double qscale) {
#pragma unroll
  for (int j = 1; j < D; ++j) Q[j][0] = Q[0][j];
#pragma unroll
  for (int i = 0; i + 1 < D; ++i) {
    const double wf = (qscale * m.wg[i]) * F[i][D - 1];
#pragma unroll
    for (int j = i + 1; j + 1 < D; ++j) Q[i + 1][j] = fma(wf, F[j][D - 1], -m.rsup[i][j + 1] * Q[i][j + 1]);
    double s = wf * F[D - 1][D - 1];
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(-m.rlast[i][k], Q[i][k], s);
    Q[i + 1][D - 1] = s;
#pragma unroll
    for (int j = i + 2; j < D; ++j) Q[j][i + 1] = Q[i + 1][j];
  }
}

// uscale, qscale: for a kernel with a lengthscale and a variance, the model
// at (l, s2) in l-scaled coordinates has F(h) = F1(h / l), Q(h) = s2 Q1(h / l),
// P_inf = s2 P_inf1, with (F1, Q1, P_inf1) the model at l = 1, s2 = 1; so one
// unit model serves a batch of series with uscale = 1/l and qscale = s2 each
// (both 1 for a model built at its own hyperparameters).
// all_terms: sum every stored Taylor term (entrywise accuracy of the small
// entries of Q for short steps, which the per-warp normwise term count does
// not give; needed where Q is factorised, as in the prior simulation).
template <int D, bool INL = false>
__device__ __forceinline__ void discretize_fp64(const DevModel<D>& m, double h, bool first, bool active,
                                           Mat<D>& F, Mat<D>& Q, double uscale = 1.0, double qscale = 1.0,
                                           bool all_terms = false) {
  h *= uscale;
  float hf = (float)h;
  int s = 0;
  if (active && !first && hf > m.hmax) {
    s = (int)ceilf(log2f(hf / m.hmax));
    if (s < 0) s = 0;
    if (s > 60) s = 60;
    hf = ldexpf(hf, -s);
    if (hf > m.hmax) { ++s; hf *= 0.5f; }
  }
  if (!active || first || !(hf > 0.0f)) hf = 0.0f;
  const float hw = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(hf)));
  int kf = NT, kq = NT;
#pragma unroll 1
  for (int k = 1; k <= NT; ++k) if (hw <= m.hthr_f[k]) { kf = k; break; }
#pragma unroll 1
  for (int k = 1; k <= NT; ++k) if (hw <= m.hthr_q[k]) { kq = k; break; }
  if (all_terms) { kf = NT; kq = NT; }
  const int smax = (int)__reduce_max_sync(0xffffffffu, (unsigned)s);
  double hs = (s > 0) ? h * __longlong_as_double((long long)(1023 - s) << 52) : h;
  if (first || !active) hs = 0.0;
  if (m.companion) {
    // row 0 by Horner, the other rows by the companion recursion
#pragma unroll
    for (int j = 0; j < D; ++j) F[0][j] = m.fc[j][kf - 1];
#pragma unroll 1
    for (int t = kf - 2; t >= 0; --t) {
#pragma unroll
      for (int j = 0; j < D; ++j) F[0][j] = fma(F[0][j], hs, m.fc[j][t]);
    }
#pragma unroll
    for (int i = 0; i + 1 < D; ++i) {
      F[i + 1][0] = F[i][D - 1] * m.rlast[i][0];
#pragma unroll
      for (int j = 1; j < D; ++j) F[i + 1][j] = fma(F[i][j - 1], m.rsup[i][j], F[i][D - 1] * m.rlast[i][j]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) F[i][j] = m.fc[i * D + j][kf - 1];
#pragma unroll 1
    for (int t = kf - 2; t >= 0; --t) {
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) F[i][j] = fma(F[i][j], hs, m.fc[i * D + j][t]);
    }
  }
  const double hq = hs * qscale;
  if (m.qrows && !all_terms) {
    // row 0 by Horner, the other rows from the Lyapunov identity
#pragma unroll
    for (int j = 0; j < D; ++j) Q[0][j] = m.qc[j][kq - 1];
#pragma unroll 1
    for (int t = kq - 2; t >= 0; --t) {
#pragma unroll
      for (int j = 0; j < D; ++j) Q[0][j] = fma(Q[0][j], hs, m.qc[j][t]);
    }
#pragma unroll
    for (int j = 0; j < D; ++j) Q[0][j] *= hq;
    companion_q_rows<D>(m, F, Q, qscale);
  } else {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) Q[i][j] = m.qc[pidx<D>(i, j)][kq - 1];
#pragma unroll 1
    for (int t = kq - 2; t >= 0; --t) {
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) Q[i][j] = fma(Q[i][j], hs, m.qc[pidx<D>(i, j)][t]);
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) { Q[i][j] *= hq; Q[j][i] = Q[i][j]; }
  }
  // doubling for long steps (rare; each lane applies its own count)
  if (smax > 0) {
    if constexpr (INL) double_steps_body<D>(F, Q, s, smax);
    else double_steps<D>(F, Q, s, smax);
  }
  if (first) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        F[i][j] = 0.0;
        Q[i][j] = qscale * m.Pinf[i <= j ? pidx<D>(i, j) : pidx<D>(j, i)];
      }
  }
}

template <int D, bool INL = false>
__device__ __forceinline__ void discretize_split(const DevModel<D>& m, double h, bool first, bool active,
                                           Mat<D>& F, Mat<D>& Q, double uscale = 1.0, double qscale = 1.0,
                                           bool all_terms = false) {
  h *= uscale;
  float hf = (float)h;
  int s = 0;
  if (active && !first && hf > m.hmax) {
    s = (int)ceilf(log2f(hf / m.hmax));
    if (s < 0) s = 0;
    if (s > 60) s = 60;
    hf = ldexpf(hf, -s);
    if (hf > m.hmax) { ++s; hf *= 0.5f; }
  }
  if (!active || first || !(hf > 0.0f)) hf = 0.0f;
  const float hw = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(hf)));
  // term counts: the first K with hw <= thr[K] (thresholds non-decreasing in
  // K), i.e. 1 + the number of thresholds below hw, by independent compares
  int kf = 1, kq = 1, mf = 1, mq = 1;
#pragma unroll
  for (int k = 1; k < NT; ++k) {
    kf += (hw > m.hthr_f[k]) ? 1 : 0;
    kq += (hw > m.hthr_q[k]) ? 1 : 0;
    mf += (hw > m.hthr_f32[k]) ? 1 : 0;
    mq += (hw > m.hthr_q32[k]) ? 1 : 0;
  }
  // split points: terms from mf / mq on are summed in FP32 (below 2^-36 of
  // the series, so their FP32 rounding stays below 2^-55); used only when the
  // split moves at least 3 terms (the FP32 -> FP64 conversion of each entry
  // costs about one FP64 operation), never with all_terms
  if (all_terms) { kf = NT; kq = NT; }
  if (all_terms || kf - mf < 3) mf = kf;
  if (all_terms || kq - mq < 3) mq = kq;
  const int smax = (int)__reduce_max_sync(0xffffffffu, (unsigned)s);
  double hs = (s > 0) ? h * __longlong_as_double((long long)(1023 - s) << 52) : h;
  if (first || !active) hs = 0.0;
  const float h32 = (float)hs;
  if (m.companion) {
    // row 0 by Horner (FP32 tail, FP64 head), the other rows by the
    // companion recursion
    int t0 = kf - 2;
    if (mf < kf) {
      float a[D];
#pragma unroll
      for (int j = 0; j < D; ++j) a[j] = m.fc32[j][kf - 1];
#pragma unroll 1
      for (int t = kf - 2; t >= mf; --t) {
#pragma unroll
        for (int j = 0; j < D; ++j) a[j] = fmaf(a[j], h32, m.fc32[j][t]);
      }
#pragma unroll
      for (int j = 0; j < D; ++j) F[0][j] = (double)a[j];
      t0 = mf - 1;
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) F[0][j] = m.fc[j][kf - 1];
    }
#pragma unroll 1
    for (int t = t0; t >= 0; --t) {
#pragma unroll
      for (int j = 0; j < D; ++j) F[0][j] = fma(F[0][j], hs, m.fc[j][t]);
    }
#pragma unroll
    for (int i = 0; i + 1 < D; ++i) {
      F[i + 1][0] = F[i][D - 1] * m.rlast[i][0];
#pragma unroll
      for (int j = 1; j < D; ++j) F[i + 1][j] = fma(F[i][j - 1], m.rsup[i][j], F[i][D - 1] * m.rlast[i][j]);
    }
  } else {
    int t0 = kf - 2;
    if (mf < kf) {
      float a[D * D];
#pragma unroll
      for (int e = 0; e < D * D; ++e) a[e] = m.fc32[e][kf - 1];
#pragma unroll 1
      for (int t = kf - 2; t >= mf; --t) {
#pragma unroll
        for (int e = 0; e < D * D; ++e) a[e] = fmaf(a[e], h32, m.fc32[e][t]);
      }
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) F[i][j] = (double)a[i * D + j];
      t0 = mf - 1;
    } else {
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) F[i][j] = m.fc[i * D + j][kf - 1];
    }
#pragma unroll 1
    for (int t = t0; t >= 0; --t) {
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) F[i][j] = fma(F[i][j], hs, m.fc[i * D + j][t]);
    }
  }
  const double hq = hs * qscale;
  if (m.qrows && !all_terms) {
    // row 0 by Horner (FP32 tail, FP64 head), the other rows from the
    // Lyapunov identity
    int t0 = kq - 2;
    if (mq < kq) {
      float a[D];
#pragma unroll
      for (int j = 0; j < D; ++j) a[j] = m.qc32[j][kq - 1];
#pragma unroll 1
      for (int t = kq - 2; t >= mq; --t) {
#pragma unroll
        for (int j = 0; j < D; ++j) a[j] = fmaf(a[j], h32, m.qc32[j][t]);
      }
#pragma unroll
      for (int j = 0; j < D; ++j) Q[0][j] = (double)a[j];
      t0 = mq - 1;
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) Q[0][j] = m.qc[j][kq - 1];
    }
#pragma unroll 1
    for (int t = t0; t >= 0; --t) {
#pragma unroll
      for (int j = 0; j < D; ++j) Q[0][j] = fma(Q[0][j], hs, m.qc[j][t]);
    }
#pragma unroll
    for (int j = 0; j < D; ++j) Q[0][j] *= hq;
    companion_q_rows<D>(m, F, Q, qscale);
  } else {
    int t0 = kq - 2;
    if (mq < kq) {
      float a[Sym<D>::N];
#pragma unroll
      for (int e = 0; e < Sym<D>::N; ++e) a[e] = m.qc32[e][kq - 1];
#pragma unroll 1
      for (int t = kq - 2; t >= mq; --t) {
#pragma unroll
        for (int e = 0; e < Sym<D>::N; ++e) a[e] = fmaf(a[e], h32, m.qc32[e][t]);
      }
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) Q[i][j] = (double)a[pidx<D>(i, j)];
      t0 = mq - 1;
    } else {
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) Q[i][j] = m.qc[pidx<D>(i, j)][kq - 1];
    }
#pragma unroll 1
    for (int t = t0; t >= 0; --t) {
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) Q[i][j] = fma(Q[i][j], hs, m.qc[pidx<D>(i, j)][t]);
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) { Q[i][j] *= hq; Q[j][i] = Q[i][j]; }
  }
  // doubling for long steps (rare; each lane applies its own count)
  if (smax > 0) {
    if constexpr (INL) double_steps_body<D>(F, Q, s, smax);
    else double_steps<D>(F, Q, s, smax);
  }
  if (first) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) {
        F[i][j] = 0.0;
        Q[i][j] = qscale * m.Pinf[i <= j ? pidx<D>(i, j) : pidx<D>(j, i)];
      }
  }
}

// SPLIT = true: mixed precision (the terms below 2^-36 of the series summed in
// FP32), for kernels where steps are long relative to the model's scale (the
// batched path); SPLIT = false keeps every term in FP64 and the term counts
// warp-uniform through the uniform datapath.  INL = true inlines the doubling
// of long steps (kernels that do nothing but discretise).
template <int D, bool SPLIT = false, bool INL = false>
__device__ __forceinline__ void discretize(const DevModel<D>& m, double h, bool first, bool active,
                                           Mat<D>& F, Mat<D>& Q, double uscale = 1.0, double qscale = 1.0,
                                           bool all_terms = false) {
  if constexpr (SPLIT) discretize_split<D, INL>(m, h, first, active, F, Q, uscale, qscale, all_terms);
  else discretize_fp64<D, INL>(m, h, first, active, F, Q, uscale, qscale, all_terms);
}

// ---------------------------------------------------------------------------
// Filtering elements and operator (Sec. 3).
// ---------------------------------------------------------------------------
template <int D>
struct FAgg {
  Mat<D> A;
  Vec<D> b;
  Mat<D> C;     // symmetric
  Vec<D> eta;
  Mat<D> J;     // symmetric
};
template <int D> struct FAggSize { static constexpr int N = D * D + 2 * D + 2 * Sym<D>::N; };

// Aggregate of a run of consecutive elements, folded one raw element at a
// time.  The tuple (A, b, C, eta, J) of elements s+1..k encodes the affine
// conditional p(x_k | x_s, y_{s+1:k}) = N(A x_s + b, C) and the likelihood
// p(y_{s+1:k} | x_s) = N_I(eta, J).  Applying the operator with the element
// of step k+1 (Sec. 3) reduces -- as in the proof of Prop. 1, where the
// operator with an element is shown to be a Kalman step -- to a prediction
// through (F, Q) followed by a scalar update whose innovation is affine in
// x_s:  v = r - w^T x_s, with w = row 0 of F A and r = y - (F b)_0, which adds
// w w^T / S to J and w r / S to eta.  An unobserved step keeps only the
// prediction (the missing-element case of Sec. 3).  A series' first step has
// F = 0, Q = P_inf, giving A = 0, eta = 0, J = 0 as for the k = 1 elements.
// The chunk aggregate is split between registers (b, C) and shared memory
// (A double-buffered, J and eta; element e of a thread's matrix at
// ptr[e * SST], so a warp's accesses hit 32 consecutive banks).
// P^- = F C F^T + Q is built one row of F C at a time, and A' = F A row by
// row.  Returns the step's S = H P^- H^T + R, 1/S and innovation r = y - H F b
// (1/S = r = 0 on a missing step): the terms of the chunk's log-likelihood
// given the state 0 before it.
template <int D, int SST>
__device__ __forceinline__ void fagg_fold_step_smem(Vec<D>& b, Mat<D>& C, const double* __restrict__ Ain,
                                                    double* __restrict__ Aout, double* __restrict__ J,
                                                    double* __restrict__ eta, const Mat<D>& F, const Mat<D>& Q,
                                                    bool observed, double y, double R, bool& bad, double& S_out,
                                                    double& Si_out, double& r_out) {
  Mat<D> Pm;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double t[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      double s = F[i][0] * C[0][k];
#pragma unroll
      for (int l = 1; l < D; ++l) s = fma(F[i][l], C[l][k], s);
      t[k] = s;
    }
#pragma unroll
    for (int j = i; j < D; ++j) {
      double s = Q[i][j];
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(t[k], F[j][k], s);
      Pm[i][j] = s;
      Pm[j][i] = s;
    }
  }
  Vec<D> bm, w;
  mulv<D>(F, b, bm);
  // w = row 0 of F A
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double s = F[0][0] * Ain[(0 * D + j) * SST];
#pragma unroll
    for (int k = 1; k < D; ++k) s = fma(F[0][k], Ain[(k * D + j) * SST], s);
    w[j] = s;
  }
  // the update without a branch: on a missing step 1/S and the innovation
  // are 0, so every line below reduces exactly to the prediction (keeps the
  // step one basic block for the scheduler)
  const double S = Pm[0][0] + R;
  if (observed && bad_pos(S)) bad = true;
  const double Si = observed ? __drcp_rn(S) : 0.0;
  const double r = observed ? y - bm[0] : 0.0;
  S_out = S;
  Si_out = Si;
  r_out = r;
  Vec<D> K;
#pragma unroll
  for (int i = 0; i < D; ++i) K[i] = Pm[i][0] * Si;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const double wsi = w[i] * Si;
#pragma unroll
    for (int j = i; j < D; ++j) J[pidx<D>(i, j) * SST] = fma(wsi, w[j], J[pidx<D>(i, j) * SST]);
    eta[i * SST] = fma(wsi, r, eta[i * SST]);
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    b[i] = fma(K[i], r, bm[i]);
#pragma unroll
    for (int j = i; j < D; ++j) { C[i][j] = fma(-K[i], Pm[0][j], Pm[i][j]); C[j][i] = C[i][j]; }
  }
  // A' = (F A) - K w, row by row (row 0 of F A is w)
#pragma unroll
  for (int j = 0; j < D; ++j) Aout[(0 * D + j) * SST] = fma(-K[0], w[j], w[j]);
#pragma unroll
  for (int i = 1; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = F[i][0] * Ain[(0 * D + j) * SST];
#pragma unroll
      for (int k = 1; k < D; ++k) s = fma(F[i][k], Ain[(k * D + j) * SST], s);
      Aout[(i * D + j) * SST] = fma(-K[i], w[j], s);
    }
}

// General filtering operator of Sec. 3, o = a (earlier) x b (later):
//   M = I + C_a J_b,  X_A = M^{-1} A_a,  x_b = M^{-1}(b_a + C_a eta_b),
//   X_C = M^{-1} C_a,  v = eta_b - J_b b_a,  x_v = M^{-1} C_a v,
//   A = A_b X_A,  b = A_b x_b + b_b,  C = A_b X_C A_b^T + C_b,
//   eta = A_a^T (v - J_b x_v) + eta_a     [(I + J C)^{-1} = I - J M^{-1} C],
//   J = A_a^T (J_b X_A) + J_a             [(I + J C)^{-1} J = J M^{-1}],
// one LU factorisation with partial pivoting of M for all right-hand sides.
template <int D>
__device__ __noinline__ bool fagg_combine(const FAgg<D>& a, const FAgg<D>& b, FAgg<D>& o) {
  Mat<D> M;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(a.C[i][k], b.J[k][j], s);
      M[i][j] = s;
    }
  Vec<D> v;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = b.eta[i];
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(-b.J[i][k], a.b[k], s);
    v[i] = s;
  }
  constexpr int NR = 2 * D + 2;
  double X[D][NR];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double sb = a.b[i], sv = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) { sb = fma(a.C[i][k], b.eta[k], sb); sv = fma(a.C[i][k], v[k], sv); }
#pragma unroll
    for (int j = 0; j < D; ++j) { X[i][j] = a.A[i][j]; X[i][D + 1 + j] = a.C[i][j]; }
    X[i][D] = sb;
    X[i][2 * D + 1] = sv;
  }
  int perm[D];
  double invd[D];
  const bool ok = lu_factor<D>(M, perm, invd);
  lu_solve<D, NR>(M, perm, invd, X);
  Mat<D> T;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = 0.0, t = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) { s = fma(b.A[i][k], X[k][j], s); t = fma(b.A[i][k], X[k][D + 1 + j], t); }
      o.A[i][j] = s;
      T[i][j] = t;
    }
    double sb = b.b[i];
#pragma unroll
    for (int k = 0; k < D; ++k) sb = fma(b.A[i][k], X[k][D], sb);
    o.b[i] = sb;
  }
  mul_Bt_sym_add<D>(T, b.A, b.C, o.C);
  Mat<D> U;
  Vec<D> w;
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(b.J[i][k], X[k][j], s);
      U[i][j] = s;
    }
    double sw = v[i];
#pragma unroll
    for (int k = 0; k < D; ++k) sw = fma(-b.J[i][k], X[k][2 * D + 1], sw);
    w[i] = sw;
  }
  mul_At_sym_add<D>(a.A, U, a.J, o.J);
  mulTv_add<D>(a.A, w, a.eta, o.eta);
  return ok;
}

// fagg_combine with the operands and the result in shared memory, in the
// packed layout of store_fagg (entry e of this thread's aggregate at
// ptr[e * SST]), and the right-hand sides of the LU solve taken one column
// at a time: only M's factors and a few vectors live in registers, so the
// combine needs no local memory.  The same operations in the same order as
// fagg_combine (bit-identical results).  o must not alias a or b; o's A
// block holds the product A_b M^{-1} C_a while the C block is formed.
template <int D, int SST>
__device__ __forceinline__ bool fagg_combine_smem(const double* __restrict__ a, const double* __restrict__ b,
                                                  double* __restrict__ o) {
  constexpr int S = Sym<D>::N;
  constexpr int OA = 0, OB = D * D, OC = D * D + D, OE = D * D + D + S, OJ = D * D + 2 * D + S;
  auto A_ = [](const double* p, int i, int j) { return p[(OA + i * D + j) * SST]; };
  auto b_ = [](const double* p, int i) { return p[(OB + i) * SST]; };
  auto C_ = [](const double* p, int i, int j) { return p[(OC + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))) * SST]; };
  auto e_ = [](const double* p, int i) { return p[(OE + i) * SST]; };
  auto J_ = [](const double* p, int i, int j) { return p[(OJ + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))) * SST]; };
  Mat<D> M;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(C_(a, i, k), J_(b, k, j), s);
      M[i][j] = s;
    }
  Vec<D> v;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = e_(b, i);
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(-J_(b, i, k), b_(a, k), s);
    v[i] = s;
  }
  double X2[D][2];   // [x_b | x_v] right-hand sides
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double sb = b_(a, i), sv = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) { sb = fma(C_(a, i, k), e_(b, k), sb); sv = fma(C_(a, i, k), v[k], sv); }
    X2[i][0] = sb;
    X2[i][1] = sv;
  }
  int perm[D];
  double invd[D];
  const bool ok = lu_factor<D>(M, perm, invd);
  lu_solve<D, 2>(M, perm, invd, X2);
  // b = A_b x_b + b_b ; eta = A_a^T (v - J_b x_v) + eta_a
  Vec<D> w;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double sb = b_(b, i);
#pragma unroll
    for (int k = 0; k < D; ++k) sb = fma(A_(b, i, k), X2[k][0], sb);
    o[(OB + i) * SST] = sb;
    double sw = v[i];
#pragma unroll
    for (int k = 0; k < D; ++k) sw = fma(-J_(b, i, k), X2[k][1], sw);
    w[i] = sw;
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = e_(a, i);
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(A_(a, k, i), w[k], s);
    o[(OE + i) * SST] = s;
  }
  // T = A_b M^{-1} C_a, column by column into o's A block; C = T A_b^T + C_b
#pragma unroll 1
  for (int j = 0; j < D; ++j) {
    double x[D][1];
#pragma unroll
    for (int i = 0; i < D; ++i) x[i][0] = C_(a, i, j);
    lu_solve<D, 1>(M, perm, invd, x);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) t = fma(A_(b, i, k), x[k][0], t);
      o[(OA + i * D + j) * SST] = t;
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      double s = C_(b, i, j);
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(A_(o, i, k), A_(b, j, k), s);
      o[(OC + pidx<D>(i, j)) * SST] = s;
    }
  // A = A_b M^{-1} A_a and U = J_b M^{-1} A_a, column by column;
  // J = A_a^T U + J_a (upper triangle: column j gives the rows i <= j)
#pragma unroll 1
  for (int j = 0; j < D; ++j) {
    double x[D][1];
#pragma unroll
    for (int i = 0; i < D; ++i) x[i][0] = A_(a, i, j);
    lu_solve<D, 1>(M, perm, invd, x);
    Vec<D> u;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double s = 0.0, q = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) { s = fma(A_(b, i, k), x[k][0], s); q = fma(J_(b, i, k), x[k][0], q); }
      o[(OA + i * D + j) * SST] = s;
      u[i] = q;
    }
#pragma unroll
    for (int i = 0; i <= j; ++i) {
      double s = J_(a, i, j);
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(A_(a, k, i), u[k], s);
      o[(OJ + pidx<D>(i, j)) * SST] = s;
    }
  }
  return ok;
}

// T x b for the transition element of one step, T = (F, 0, Q, 0, 0), read
// from the step's F/Q record (F row-major, then Q packed upper), b and o as
// in fagg_combine_smem.  With b_a = 0, eta_a = 0 and J_a = 0 the operator
// reduces to (v = eta_b, x_v = x_b):
//   M = I + Q J_b,  x_b = M^{-1} Q eta_b,  b = A_b x_b + b_b,
//   eta = F^T (eta_b - J_b x_b),  C = A_b M^{-1} Q A_b^T + C_b,
//   A = A_b M^{-1} F,  J = F^T J_b M^{-1} F.
template <int D, int SST>
__device__ __noinline__ bool fagg_transition_combine_smem(const double* __restrict__ rec,
                                                             const double* __restrict__ b,
                                                             double* __restrict__ o) {
  constexpr int S = Sym<D>::N;
  constexpr int OA = 0, OB = D * D, OC = D * D + D, OE = D * D + D + S, OJ = D * D + 2 * D + S;
  auto F_ = [&](int i, int j) { return rec[i * D + j]; };
  auto Q_ = [&](int i, int j) { return rec[D * D + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))]; };
  auto A_ = [](const double* p, int i, int j) { return p[(OA + i * D + j) * SST]; };
  auto b_ = [](const double* p, int i) { return p[(OB + i) * SST]; };
  auto C_ = [](const double* p, int i, int j) { return p[(OC + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))) * SST]; };
  auto e_ = [](const double* p, int i) { return p[(OE + i) * SST]; };
  auto J_ = [](const double* p, int i, int j) { return p[(OJ + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))) * SST]; };
  Mat<D> M;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(Q_(i, k), J_(b, k, j), s);
      M[i][j] = s;
    }
  double x[D][1];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(Q_(i, k), e_(b, k), s);
    x[i][0] = s;
  }
  int perm[D];
  double invd[D];
  const bool ok = lu_factor<D>(M, perm, invd);
  lu_solve<D, 1>(M, perm, invd, x);
  Vec<D> w;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double sb = b_(b, i);
#pragma unroll
    for (int k = 0; k < D; ++k) sb = fma(A_(b, i, k), x[k][0], sb);
    o[(OB + i) * SST] = sb;
    double sw = e_(b, i);
#pragma unroll
    for (int k = 0; k < D; ++k) sw = fma(-J_(b, i, k), x[k][0], sw);
    w[i] = sw;
  }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(F_(k, i), w[k], s);
    o[(OE + i) * SST] = s;
  }
  // A_b M^{-1} Q column by column into o's A block; C = that A_b^T + C_b
#pragma unroll 1
  for (int j = 0; j < D; ++j) {
    double y[D][1];
#pragma unroll
    for (int i = 0; i < D; ++i) y[i][0] = Q_(i, j);
    lu_solve<D, 1>(M, perm, invd, y);
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) t = fma(A_(b, i, k), y[k][0], t);
      o[(OA + i * D + j) * SST] = t;
    }
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      double s = C_(b, i, j);
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(A_(o, i, k), A_(b, j, k), s);
      o[(OC + pidx<D>(i, j)) * SST] = s;
    }
  // A = A_b M^{-1} F and U = J_b M^{-1} F column by column; J = F^T U
#pragma unroll 1
  for (int j = 0; j < D; ++j) {
    double y[D][1];
#pragma unroll
    for (int i = 0; i < D; ++i) y[i][0] = F_(i, j);
    lu_solve<D, 1>(M, perm, invd, y);
    Vec<D> u;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double s = 0.0, q = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) { s = fma(A_(b, i, k), y[k][0], s); q = fma(J_(b, i, k), y[k][0], q); }
      o[(OA + i * D + j) * SST] = s;
      u[i] = q;
    }
#pragma unroll
    for (int i = 0; i <= j; ++i) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(F_(k, i), u[k], s);
      o[(OJ + pidx<D>(i, j)) * SST] = s;
    }
  }
  return ok;
}

// A filter state (x, P) -- a prefix aggregate, which has A = 0, eta = 0, J = 0
// because it contains the first step -- combined with an aggregate b:
//   M = I + P J_b,  x' = A_b M^{-1} (x + P eta_b) + b_b,
//   P' = A_b M^{-1} P A_b^T + C_b.
// The aggregate b is read in place from a packed array (entry e at p[e * st],
// the layout of store_fagg), so that no copy of it is made.
template <int D>
__device__ __noinline__ bool fstate_combine(const Vec<D>& x, const Mat<D>& P, const double* __restrict__ p,
                                               int64_t st, Vec<D>& xo, Mat<D>& Po) {
  constexpr int S = Sym<D>::N;
  auto A_ = [&](int i, int j) { return p[(int64_t)(i * D + j) * st]; };
  auto C_ = [&](int i, int j) { return p[(int64_t)(D * D + D + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))) * st]; };
  auto J_ = [&](int i, int j) {
    return p[(int64_t)(D * D + 2 * D + S + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))) * st];
  };
  Mat<D> M;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(P[i][k], J_(k, j), s);
      M[i][j] = s;
    }
  constexpr int NR = D + 1;
  double X[D][NR];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = x[i];
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(P[i][k], p[(int64_t)(D * D + D + S + k) * st], s);
    X[i][0] = s;
#pragma unroll
    for (int j = 0; j < D; ++j) X[i][1 + j] = P[i][j];
  }
  int perm[D];
  double invd[D];
  const bool ok = lu_factor<D>(M, perm, invd);
  lu_solve<D, NR>(M, perm, invd, X);
  Mat<D> T, Ab;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) Ab[i][j] = A_(i, j);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double sx = p[(int64_t)(D * D + i) * st];
#pragma unroll
    for (int k = 0; k < D; ++k) sx = fma(Ab[i][k], X[k][0], sx);
    xo[i] = sx;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) t = fma(Ab[i][k], X[k][1 + j], t);
      T[i][j] = t;
    }
  }
  Mat<D> Cb;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) Cb[i][j] = C_(i, j);
  mul_Bt_sym_add<D>(T, Ab, Cb, Po);
  return ok;
}

// ---------------------------------------------------------------------------
// Smoothing elements and operator (supplement, Prop. 2).
// ---------------------------------------------------------------------------
template <int D>
struct SAgg {
  Mat<D> E;
  Vec<D> g;
  Mat<D> L;     // symmetric
};
template <int D> struct SAggSize { static constexpr int N = D * D + D + Sym<D>::N; };

template <int D>
__device__ __forceinline__ void sagg_identity(SAgg<D>& a) {
  set_eye<D>(a.E);
  set_zero<D>(a.L);
#pragma unroll
  for (int i = 0; i < D; ++i) a.g[i] = 0.0;
}

// (E_a, g_a, L_a) x (E_b, g_b, L_b) = (E_a E_b, E_a g_b + g_a, E_a L_b E_a^T + L_a),
// a earlier.  Used for the in-chunk fold and for the scan levels.
template <int D>
__device__ __forceinline__ void sagg_combine(const SAgg<D>& a, const SAgg<D>& b, SAgg<D>& o) {
  Mat<D> T;
  mul<D>(a.E, b.E, o.E);
  mulv_add<D>(a.E, b.g, a.g, o.g);
  mul<D>(a.E, b.L, T);
  mul_Bt_sym_add<D>(T, a.E, a.L, o.L);
}

// Smoother element of step k from the filter state (x_k, P_k) and the
// transition into step k+1, given T = F P_k, x^- = F x_k and
// P^- = F P_k F^T + Q (the Kalman prediction of step k+1):
//   E = P_k F^T (P^-)^{-1}, g = x_k - E x^-, L = P_k - E F P_k,
// with P^- = Lu diag(d) Lu^T (square-root free), W = Lu^{-1} T,
// V = diag(1/d) W, L = P_k - W^T V, E^T = Lu^{-T} V.
template <int D>
__device__ __forceinline__ bool smoother_element(const Vec<D>& x, const Mat<D>& P, const Mat<D>& T,
                                                 const Vec<D>& xm, const Mat<D>& Pm, SAgg<D>& e) {
  Mat<D> Lu, V;
  double rd[D];
  const bool ok = ldlt<D>(Pm, Lu, rd);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = T[i][j];
#pragma unroll
      for (int k = 0; k < i; ++k) s = fma(-Lu[i][k], V[k][j], s);
      V[i][j] = s;
    }
  // L = P - sum_k W_k^T V_k over the rows k; row k of W becomes V_k once used
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) e.L[i][j] = P[i][j];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    double vk[D];
#pragma unroll
    for (int j = 0; j < D; ++j) vk[j] = V[k][j] * rd[k];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) e.L[i][j] = fma(-V[k][i], vk[j], e.L[i][j]);
#pragma unroll
    for (int j = 0; j < D; ++j) V[k][j] = vk[j];
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < i; ++j) e.L[i][j] = e.L[j][i];
#pragma unroll
  for (int i = D - 1; i >= 0; --i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = V[i][j];
#pragma unroll
      for (int k = i + 1; k < D; ++k) s = fma(-Lu[k][i], e.E[j][k], s);
      e.E[j][i] = s;
    }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = x[i];
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(-e.E[i][k], xm[k], s);
    e.g[i] = s;
  }
  return ok;
}

// Chunk aggregate of the smoothing operator from the joint of its first and
// last states.  The product of the smoothing elements of steps s..e-1 is the
// conditional p(x_s | x_e, y_{1:e-1}) = N(E x_e + g, L) (each element is
// p(x_k | x_{k+1}, y_{1:k}), supplement Prop. 2, and the chain is Markov).
// Given mu = E[x_s | y_{1:e-1}], V = Cov(x_s | y_{1:e-1}) and
// Sig = Cov(x_s, x_{e-1} | y_{1:e-1}) (k_filter_propagate forms them in closed
// form from the filter aggregate of steps s+1..e-1), the prediction
// (x^-, P^-) of step e closes it:
//   E = Sig F_e^T (P^-)^{-1}, g = mu - E x^-, L = V - E (Sig F_e^T)^T.
template <int D>
struct FixedPoint {
  Vec<D> mu;
  Mat<D> V;     // symmetric
  Mat<D> Sig;
};

// chunk end: aggregate (E, g, L) from (mu, V, Sig) and the prediction
// (xm, Pm) of the step after the chunk, Pm = Lc Lc^T given.
template <int D>
__device__ __forceinline__ void fixed_point_finish(const FixedPoint<D>& f, const Mat<D>& F, const Vec<D>& xm,
                                                   const Mat<D>& Lc, const double (&invd)[D], SAgg<D>& a) {
  // Z = (Sig F^T)^T = F Sig^T ; W = Lc^{-1} Z ; E^T = Lc^{-T} W ; L = V - W^T W
  Mat<D> Wm;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double z = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) z = fma(F[i][k], f.Sig[j][k], z);
      Wm[i][j] = z;
    }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = Wm[i][j];
#pragma unroll
      for (int k = 0; k < i; ++k) s = fma(-Lc[i][k], Wm[k][j], s);
      Wm[i][j] = s * invd[i];
    }
#pragma unroll
  for (int i = D - 1; i >= 0; --i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = Wm[i][j];
#pragma unroll
      for (int k = i + 1; k < D; ++k) s = fma(-Lc[k][i], a.E[j][k], s);
      a.E[j][i] = s * invd[i];
    }
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = f.mu[i];
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(-a.E[i][k], xm[k], s);
    a.g[i] = s;
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      double s = f.V[i][j];
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(-Wm[k][i], Wm[k][j], s);
      a.L[i][j] = s;
      a.L[j][i] = s;
    }
}

// ---------------------------------------------------------------------------
// (De)serialisation of aggregates: entry-major with a stride, so that the
// lanes of a warp touch consecutive addresses.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void store_fagg(double* p, int64_t st, const FAgg<D>& a) {
  int e = 0;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) p[(e++) * st] = a.A[i][j];
#pragma unroll
  for (int i = 0; i < D; ++i) p[(e++) * st] = a.b[i];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) p[(e++) * st] = a.C[i][j];
#pragma unroll
  for (int i = 0; i < D; ++i) p[(e++) * st] = a.eta[i];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) p[(e++) * st] = a.J[i][j];
}
template <int D>
__device__ __forceinline__ void load_fagg(const double* p, int64_t st, FAgg<D>& a) {
  int e = 0;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) a.A[i][j] = p[(e++) * st];
#pragma unroll
  for (int i = 0; i < D; ++i) a.b[i] = p[(e++) * st];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) { a.C[i][j] = p[(e++) * st]; a.C[j][i] = a.C[i][j]; }
#pragma unroll
  for (int i = 0; i < D; ++i) a.eta[i] = p[(e++) * st];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) { a.J[i][j] = p[(e++) * st]; a.J[j][i] = a.J[i][j]; }
}
template <int D>
__device__ __forceinline__ void store_sagg(double* p, int64_t st, const SAgg<D>& a) {
  int e = 0;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) p[(e++) * st] = a.E[i][j];
#pragma unroll
  for (int i = 0; i < D; ++i) p[(e++) * st] = a.g[i];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) p[(e++) * st] = a.L[i][j];
}
template <int D>
__device__ __forceinline__ void load_sagg(const double* p, int64_t st, SAgg<D>& a) {
  int e = 0;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) a.E[i][j] = p[(e++) * st];
#pragma unroll
  for (int i = 0; i < D; ++i) a.g[i] = p[(e++) * st];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) { a.L[i][j] = p[(e++) * st]; a.L[j][i] = a.L[i][j]; }
}

template <int D>
__device__ __forceinline__ void shfl_up_fagg(FAgg<D>& a, int off) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) a.A[i][j] = __shfl_up_sync(0xffffffffu, a.A[i][j], off);
    a.b[i] = __shfl_up_sync(0xffffffffu, a.b[i], off);
    a.eta[i] = __shfl_up_sync(0xffffffffu, a.eta[i], off);
#pragma unroll
    for (int j = i; j < D; ++j) {
      a.C[i][j] = __shfl_up_sync(0xffffffffu, a.C[i][j], off); a.C[j][i] = a.C[i][j];
      a.J[i][j] = __shfl_up_sync(0xffffffffu, a.J[i][j], off); a.J[j][i] = a.J[i][j];
    }
  }
}
template <int D>
__device__ __forceinline__ void shfl_down_sagg(SAgg<D>& a, int off) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
#pragma unroll
    for (int j = 0; j < D; ++j) a.E[i][j] = __shfl_down_sync(0xffffffffu, a.E[i][j], off);
    a.g[i] = __shfl_down_sync(0xffffffffu, a.g[i], off);
#pragma unroll
    for (int j = i; j < D; ++j) { a.L[i][j] = __shfl_down_sync(0xffffffffu, a.L[i][j], off); a.L[j][i] = a.L[i][j]; }
  }
}

}  // namespace pssgp
