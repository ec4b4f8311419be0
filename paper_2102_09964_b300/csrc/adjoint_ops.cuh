// adjoint_ops.cuh -- device algebra of the reverse-mode (adjoint) gradient of
// the log marginal likelihood (Sec. 2, parameter estimation) with respect to
// theta = (log lengthscale, log variance, log noise variance).
//
// With H = e0^T (balanced coordinates) the filter step k is
//   m_k = F_k x_{k-1},  M_k = F_k P_{k-1} F_k^T + Q_k               (predict)
//   S = M_k[0][0] + R,  v = y_k - m_k[0],  K = M_k[:,0] / S
//   x_k = m_k + K v,    P_k = M_k - K S K^T                         (update)
//   l_k = -1/2 [log 2 pi S + v^2 / S]
// and a missing step keeps (x_k, P_k) = (m_k, M_k), l_k = 0.  Differentiating
// backwards, the adjoints of the predicted moments obey, with A_k = I - e0 K^T,
// Si = 1/S, c_k = -1/2 (Si - v^2 Si^2) (all zero on missing steps):
//   xb_k  = F_{k+1}^T mb_{k+1}                  (adjoint of x_k)
//   Pb_k  = F_{k+1}^T Mb_{k+1} F_{k+1}          (adjoint of P_k)
//   mb_k  = A_k xb_k + e0 v Si
//   Mb_k  = A_k Pb_k A_k^T + (v Si / 2)(xb_k e0^T + e0 xb_k^T)
//           + (c_k - v Si K^T xb_k) e0 e0^T
//   dl/dR_k = K^T Pb_k K - v Si K^T xb_k + c_k
// with mb_n = 0, Mb_n = 0 (F_n := 0).  Both are backward recursions of the
// smoothing operator's form (supplement Prop. 2): mb_k = E_k mb_{k+1} + g_k and
// Mb_k = E_k Mb_{k+1} E_k^T + B_k with E_k = A_k F_{k+1}^T, g_k = e0 v Si;
// B_k depends on mb_{k+1}, so the mean adjoint is scanned first.
//
// The model is the kernel family rescaled in time and amplitude:
// F_k = F1(tau_k), Q_k = q Q1(tau_k), tau_k = h_k l0 / l, q = s2 / s20, with
// (G, W) the drift and diffusion of the model built at (l0, s20).  Hence
//   dF_k / dlog l = -tau_k G F_k,  dQ_k / dlog l = -tau_k (G Q_k + Q_k G^T + q W)
//   dQ_k / dlog s2 = Q_k (also at a series' first step, Q = q P_inf)
// and, with the adjoints F_bar = mb m_prev^T + 2 Mb F P_prev, Q_bar = Mb,
//   dl/dlog l  += -tau_k [mb_k^T G m_k + 2 tr(Mb_k G M_k) + q tr(Mb_k W)]
//   dl/dlog s2 += tr(Mb_k Q_k)
//   dl/dlog R  += (dl/dR_k) R_k.
#pragma once
#include "scan_ops.cuh"

namespace pssgp {

// per-step record of the forward pass: predicted mean m_k, predicted
// covariance M_k (packed), innovation v and 1/S (0 on missing steps)
template <int D> __host__ __device__ constexpr int adjs_of() { return (D + Sym<D>::N + 2 + 1) / 2 * 2; }

template <int D>
__device__ __forceinline__ void store_adj(double* rec, int64_t k, const Vec<D>& xm, const Mat<D>& Pm, double v,
                                          double Si) {
  double* p = rec + k * adjs_of<D>();
#pragma unroll
  for (int i = 0; i < D; ++i) p[i] = xm[i];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) p[D + pidx<D>(i, j)] = Pm[i][j];
  p[D + Sym<D>::N] = v;
  p[D + Sym<D>::N + 1] = Si;
}

// predicted mean and column 0 of the predicted covariance only
template <int D>
__device__ __forceinline__ void load_adj_col0(const double* rec, int64_t k, Vec<D>& xm, Vec<D>& c0, double& v,
                                              double& Si) {
  const double* p = rec + k * adjs_of<D>();
#pragma unroll
  for (int i = 0; i < D; ++i) xm[i] = p[i];
#pragma unroll
  for (int i = 0; i < D; ++i) c0[i] = p[D + pidx<D>(0, i)];
  v = p[D + Sym<D>::N];
  Si = p[D + Sym<D>::N + 1];
}

template <int D>
__device__ __forceinline__ double load_adj_M(const double* rec, int64_t k, int i, int j) {
  return rec[k * adjs_of<D>() + D + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))];
}

template <int D>
__device__ __forceinline__ void load_F(const double* rec, int64_t k, int fqs, Mat<D>& F) {
  const double* p = rec + k * fqs;
  // 16-byte loads (every record starts on a 16-byte boundary), a scalar tail for odd d * d
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int e = 0; e + 1 < D * D; e += 2) {
    const double2 v = q[e / 2];
    F[e / D][e % D] = v.x;
    F[(e + 1) / D][(e + 1) % D] = v.y;
  }
  if constexpr ((D * D) % 2 == 1) F[D - 1][D - 1] = p[D * D - 1];
}

// ---------------------------------------------------------------------------
// One backward step of the covariance adjoint, in place on a symmetric
// matrix in shared memory (packed upper, sL[e * ST]):
//   L <- A (F^T L F) A^T + B,  A = I - e0 K^T,
//   B = (vSi / 2)(xb e0^T + e0 xb^T) + (c - vSi K^T xb) e0 e0^T.
// Returns K^T (F^T L F) K (the term of dl/dR).  F^T L F is accumulated over
// the rows a of L: row a of L F, then its outer contribution F[a][i] (LF)[a][j]
// to the upper triangle.
// ---------------------------------------------------------------------------
template <int D, int ST>
__device__ __forceinline__ double adj_cov_step(double* sL, const Mat<D>& F, const Vec<D>& K, double vSi, double c,
                                               const Vec<D>& xb, double kx) {
  double R[Sym<D>::N];
#pragma unroll
  for (int e = 0; e < Sym<D>::N; ++e) R[e] = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    double la[D];
#pragma unroll
    for (int b = 0; b < D; ++b) la[b] = sL[(a <= b ? pidx<D>(a, b) : pidx<D>(b, a)) * ST];
    double u[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = la[0] * F[0][j];
#pragma unroll
      for (int b = 1; b < D; ++b) s = fma(la[b], F[b][j], s);
      u[j] = s;
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) R[pidx<D>(i, j)] = fma(F[a][i], u[j], R[pidx<D>(i, j)]);
  }
  double w[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) s = fma(R[i <= j ? pidx<D>(i, j) : pidx<D>(j, i)], K[j], s);
    w[i] = s;
  }
  double kLk = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) kLk = fma(K[i], w[i], kLk);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      double val = R[pidx<D>(i, j)];
      if (i == 0 && j == 0) {
        val += -2.0 * w[0] + kLk + vSi * xb[0] + c - vSi * kx;
      } else if (i == 0) {
        val += -w[j] + 0.5 * vSi * xb[j];
      }
      sL[pidx<D>(i, j) * ST] = val;
    }
  return kLk;
}

// tr(S M) for symmetric S in shared memory (packed, stride ST) and symmetric
// M given packed in global memory (adjoint record layout)
template <int D, int ST>
__device__ __forceinline__ double adj_trace_smem_rec(const double* sS, const double* Mp) {
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      const double p = sS[pidx<D>(i, j) * ST] * Mp[pidx<D>(i, j)];
      s = (i == j) ? s + p : fma(2.0, p, s);
    }
  return s;
}

}  // namespace pssgp
