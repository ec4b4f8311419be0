/*
 * ssgp_oracle.c -- plain sequential CPU oracle for the state-space GP path of
 * "Temporal Gaussian Process Regression in Logarithmic Time" (Corenflos, Zhao,
 * Sarkka).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA library under paper_2102_09964_b300/ and must never be
 * used as a fallback for it.
 *
 * Everything is computed in long double (x87 extended precision) from double
 * inputs, with plain loops, no blocking and no reordering beyond what the
 * formulas state, so that it can be checked against the paper by eye.
 *
 * Layout conventions (all row-major, 0-based step index k = paper's k+1):
 *   F[k*d*d + i*d + j], Q[k*d*d + i*d + j]  -- transition INTO step k
 *        (paper: F_{k-1}, Q_{k-1} of the supplement's Eq. (ss-gp-formation));
 *        step 0 has no predecessor: stored as F_0 = 0, Q_0 = P_inf.
 *   m[k*d + i], P[k*d*d + i*d + j]           -- filter mean / covariance.
 *
 * Return codes: 0 ok, 1 singular/non-positive pivot, 2 unsorted times,
 * 3 bad argument.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef long double real;
#define DMAX 8
#define NMAX (2 * DMAX)

/* ----------------------------------------------------------------------- */
/* small dense helpers (n x n, row-major, n <= 16)                         */
/* ----------------------------------------------------------------------- */

/* C[n x p] = A[n x m] * B[m x p]  (C may alias A or B) */
static void mm(int n, int m, int p, const real *A, const real *B, real *C) {
  real T[NMAX * (2 * NMAX + 1)];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < p; ++j) {
      real s = 0.0L;
      for (int k = 0; k < m; ++k) s += A[i * m + k] * B[k * p + j];
      T[i * p + j] = s;
    }
  memcpy(C, T, sizeof(real) * n * p);
}

/* B <- A^T, A is n x m, B is m x n */
static void tr(int n, int m, const real *A, real *B) {
  real T[NMAX * NMAX];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < m; ++j) T[j * n + i] = A[i * m + j];
  memcpy(B, T, sizeof(real) * n * m);
}

static void eye(int n, real *A) {
  memset(A, 0, sizeof(real) * n * n);
  for (int i = 0; i < n; ++i) A[i * n + i] = 1.0L;
}

/* Solve A X = B in place (B <- A^{-1} B), A is n x n (destroyed), B n x m.
 * Gaussian elimination with partial pivoting.  Returns 1 if A is singular. */
static int solve(int n, real *A, real *B, int m) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[p * n + c])) p = r;
    if (A[p * n + c] == 0.0L) return 1;
    if (p != c) {
      for (int j = 0; j < n; ++j) { real t = A[c * n + j]; A[c * n + j] = A[p * n + j]; A[p * n + j] = t; }
      for (int j = 0; j < m; ++j) { real t = B[c * m + j]; B[c * m + j] = B[p * m + j]; B[p * m + j] = t; }
    }
    for (int r = c + 1; r < n; ++r) {
      real f = A[r * n + c] / A[c * n + c];
      if (f == 0.0L) continue;
      for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
      for (int j = 0; j < m; ++j) B[r * m + j] -= f * B[c * m + j];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    for (int j = 0; j < m; ++j) {
      real s = B[c * m + j];
      for (int k = c + 1; k < n; ++k) s -= A[c * n + k] * B[k * m + j];
      B[c * m + j] = s / A[c * n + c];
    }
  }
  return 0;
}

static void load(int n, int m, const double *src, real *dst) {
  for (int i = 0; i < n * m; ++i) dst[i] = (real)src[i];
}
static void store(int n, int m, const real *src, double *dst) {
  for (int i = 0; i < n * m; ++i) dst[i] = (double)src[i];
}
static void symmetrize(int n, real *A) {
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      real s = 0.5L * (A[i * n + j] + A[j * n + i]);
      A[i * n + j] = s; A[j * n + i] = s;
    }
}

/* Matrix exponential E = exp(A) of an n x n matrix: scale by 2^-s until the
 * 1-norm is <= 1/2, sum the Taylor series until the terms vanish at
 * long-double precision, then square s times. */
static void expm(int n, const real *A, real *E) {
  real nrm = 0.0L;
  for (int j = 0; j < n; ++j) {
    real c = 0.0L;
    for (int i = 0; i < n; ++i) c += fabsl(A[i * n + j]);
    if (c > nrm) nrm = c;
  }
  int s = 0;
  while (nrm > 0.5L) { nrm *= 0.5L; ++s; }
  real As[NMAX * NMAX], T[NMAX * NMAX];
  real sc = ldexpl(1.0L, -s);
  for (int i = 0; i < n * n; ++i) As[i] = A[i] * sc;
  eye(n, E);
  eye(n, T);
  for (int k = 1; k <= 60; ++k) {
    mm(n, n, n, T, As, T);
    real tmax = 0.0L, emax = 0.0L;
    for (int i = 0; i < n * n; ++i) {
      T[i] /= (real)k;
      E[i] += T[i];
      if (fabsl(T[i]) > tmax) tmax = fabsl(T[i]);
      if (fabsl(E[i]) > emax) emax = fabsl(E[i]);
    }
    if (k > 2 && tmax <= 1e-30L * emax) break;
  }
  for (int i = 0; i < s; ++i) mm(n, n, n, E, E, E);
}

/* ----------------------------------------------------------------------- */
/* Discretisation -- supplement Eq. (ss-gp-formation):                     */
/*   F = exp(h G),  Q = int_0^h exp((h-s)G) L q L^T exp((h-s)G)^T ds       */
/* evaluated with Van Loan's block exponential:                            */
/*   exp([[-G, W], [0, G^T]] h) = [[*, E12], [0, E22]],  F = E22^T,        */
/*   Q = F E12,  with W = L q L^T.                                         */
/* The -G block grows like exp(|G| h), so for long steps Van Loan is used   */
/* on h / 2^s (|G|_1 h / 2^s <= 1/2) and the result is doubled s times     */
/* with the exact semigroup identities of the same integral:                */
/*   F(2h) = F(h) F(h),  Q(2h) = F(h) Q(h) F(h)^T + Q(h).                  */
/* ----------------------------------------------------------------------- */
static void vanloan(int d, const real *G, const real *W, real h, real *F, real *Q);

static int discretize_one(int d, const real *G, const real *W, real h, real *F, real *Q) {
  real gn = 0.0L;
  for (int j = 0; j < d; ++j) {
    real c = 0.0L;
    for (int i = 0; i < d; ++i) c += fabsl(G[i * d + j]);
    if (c > gn) gn = c;
  }
  int s = 0;
  while (gn * ldexpl(h, -s) > 0.5L) ++s;
  vanloan(d, G, W, ldexpl(h, -s), F, Q);
  for (int r = 0; r < s; ++r) {
    real T[DMAX * DMAX], Ft[DMAX * DMAX], FQF[DMAX * DMAX];
    mm(d, d, d, F, Q, T);
    tr(d, d, F, Ft);
    mm(d, d, d, T, Ft, FQF);
    for (int i = 0; i < d * d; ++i) Q[i] += FQF[i];
    symmetrize(d, Q);
    mm(d, d, d, F, F, F);
  }
  return 0;
}

static void vanloan(int d, const real *G, const real *W, real h, real *F, real *Q) {
  int n = 2 * d;
  real C[NMAX * NMAX], E[NMAX * NMAX];
  memset(C, 0, sizeof(C));
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      C[i * n + j] = -G[i * d + j] * h;            /* -G h   */
      C[i * n + d + j] = W[i * d + j] * h;         /*  W h   */
      C[(d + i) * n + d + j] = G[j * d + i] * h;   /*  G^T h */
    }
  expm(n, C, E);
  real E12[DMAX * DMAX];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      F[i * d + j] = E[(d + j) * n + d + i];       /* F = E22^T */
      E12[i * d + j] = E[i * n + d + j];
    }
  mm(d, d, d, F, E12, Q);                          /* Q = F E12 */
  symmetrize(d, Q);
}

int orc_discretize(int d, const double *G_, const double *W_, const double *Pinf_,
                   const double *t, long n, double *F_, double *Q_) {
  if (d < 1 || d > DMAX || n < 1) return 3;
  for (long k = 1; k < n; ++k)
    if (!(t[k] >= t[k - 1])) return 2;
  real G[DMAX * DMAX], W[DMAX * DMAX], Pinf[DMAX * DMAX];
  load(d, d, G_, G); load(d, d, W_, W); load(d, d, Pinf_, Pinf);
  int dd = d * d;
  for (int i = 0; i < dd; ++i) { F_[i] = 0.0; Q_[i] = (double)Pinf[i]; }
#pragma omp parallel for schedule(static)
  for (long k = 1; k < n; ++k) {
    real F[DMAX * DMAX], Q[DMAX * DMAX];
    discretize_one(d, G, W, (real)t[k] - (real)t[k - 1], F, Q);
    store(d, d, F, F_ + k * dd);
    store(d, d, Q, Q_ + k * dd);
  }
  return 0;
}

/* ----------------------------------------------------------------------- */
/* Sequential Kalman filter with missing measurements.                     */
/*   no measurement  -- supplement Eq. (nomeas)                            */
/*   measurement     -- supplement Eq. (withmeas1)                         */
/*   first step: prior N(0, P_inf) (stationary start, Sec. 4.1)            */
/*   log-likelihood: prediction-error decomposition over observed steps,   */
/*     sum_k -1/2 [log(2 pi S_k) + v_k^2 / S_k]  (the "standard state-space */
/*     methods" the paper refers to in Sec. 2)                             */
/* ----------------------------------------------------------------------- */
int orc_kalman_filter(int d, const double *H_, const double *R, int R_per_step,
                      const double *Pinf_, const double *F_, const double *Q_,
                      const double *y, const unsigned char *mask, long n,
                      double *m_out, double *P_out, double *mp_out, double *Pp_out,
                      double *loglik) {
  if (d < 1 || d > DMAX || n < 1) return 3;
  const real twopi = 6.283185307179586476925286766559L;
  int dd = d * d;
  real H[DMAX], Pinf[DMAX * DMAX];
  load(1, d, H_, H); load(d, d, Pinf_, Pinf);
  real m[DMAX], P[DMAX * DMAX], mp[DMAX], Pp[DMAX * DMAX];
  real ll = 0.0L;
  for (long k = 0; k < n; ++k) {
    /* prediction */
    if (k == 0) {
      for (int i = 0; i < d; ++i) mp[i] = 0.0L;
      memcpy(Pp, Pinf, sizeof(real) * dd);
    } else {
      real F[DMAX * DMAX], Q[DMAX * DMAX], FP[DMAX * DMAX], Ft[DMAX * DMAX];
      load(d, d, F_ + k * dd, F); load(d, d, Q_ + k * dd, Q);
      mm(d, d, 1, F, m, mp);                       /* m^- = F m          */
      mm(d, d, d, F, P, FP);
      tr(d, d, F, Ft);
      mm(d, d, d, FP, Ft, Pp);                     /* P^- = F P F^T + Q  */
      for (int i = 0; i < dd; ++i) Pp[i] += Q[i];
      symmetrize(d, Pp);
    }
    if (mp_out) store(1, d, mp, mp_out + k * d);
    if (Pp_out) store(d, d, Pp, Pp_out + k * dd);
    /* update */
    if (mask[k]) {
      real Rk = (real)(R_per_step ? R[k] : R[0]);
      real PH[DMAX];
      for (int i = 0; i < d; ++i) {
        real s = 0.0L;
        for (int j = 0; j < d; ++j) s += Pp[i * d + j] * H[j];
        PH[i] = s;                                 /* P^- H^T            */
      }
      real S = Rk;
      for (int i = 0; i < d; ++i) S += H[i] * PH[i]; /* S = H P^- H^T + R */
      if (!(S > 0.0L)) return 1;
      real v = (real)y[k];
      for (int i = 0; i < d; ++i) v -= H[i] * mp[i]; /* v = y - H m^-     */
      real K[DMAX];
      for (int i = 0; i < d; ++i) K[i] = PH[i] / S;  /* K = P^- H^T / S   */
      for (int i = 0; i < d; ++i) m[i] = mp[i] + K[i] * v;
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) P[i * d + j] = Pp[i * d + j] - K[i] * S * K[j];
      symmetrize(d, P);
      ll += -0.5L * (logl(twopi * S) + v * v / S);
    } else {
      memcpy(m, mp, sizeof(real) * d);
      memcpy(P, Pp, sizeof(real) * dd);
    }
    store(1, d, m, m_out + k * d);
    store(d, d, P, P_out + k * dd);
  }
  if (loglik) *loglik = (double)ll;
  return 0;
}

/* ----------------------------------------------------------------------- */
/* Sequential Rauch-Tung-Striebel smoother -- supplement Eq. (smoother),   */
/* with the sign of the covariance correction as derived in the proof of   */
/* Prop. 2:  P^s_k = P_k + G_k (P^s_{k+1} - F P_k F^T - Q) G_k^T.          */
/* Here F, Q of step k+1 are the transition from step k to step k+1.       */
/* mp, Pp: the filter's predicted moments (F m_k, F P_k F^T + Q) of k+1.   */
/* The sequential Kalman filter started from a given state: the state at the
 * time before step 0 is N(x0, P0), and every step k, step 0 included, is
 * predicted through its own transition (F[k], Q[k]) and then updated as in
 * orc_kalman_filter (supplement Eqs. (nomeas), (withmeas1)).  This is the
 * filter of a piece of a longer series given the filter state at the piece's
 * start; with F[0] = 0 and Q[0] = P_inf it is orc_kalman_filter.  loglik:
 * the sum over the observed steps of log p(y_k | earlier y of the piece, start
 * state). */
int orc_kalman_filter_from(int d, const double *H_, const double *R, int R_per_step,
                           const double *x0_, const double *P0_, const double *F_, const double *Q_,
                           const double *y, const unsigned char *mask, long n,
                           double *m_out, double *P_out, double *mp_out, double *Pp_out,
                           double *loglik) {
  if (d < 1 || d > DMAX || n < 1) return 3;
  const real twopi = 6.283185307179586476925286766559L;
  int dd = d * d;
  real H[DMAX], m[DMAX], P[DMAX * DMAX];
  load(1, d, H_, H);
  load(1, d, x0_, m);
  load(d, d, P0_, P);
  real ll = 0.0L;
  for (long k = 0; k < n; ++k) {
    real F[DMAX * DMAX], Q[DMAX * DMAX], FP[DMAX * DMAX], Ft[DMAX * DMAX], mp[DMAX], Pp[DMAX * DMAX];
    load(d, d, F_ + k * dd, F); load(d, d, Q_ + k * dd, Q);
    mm(d, d, 1, F, m, mp);                         /* m^- = F m          */
    mm(d, d, d, F, P, FP);
    tr(d, d, F, Ft);
    mm(d, d, d, FP, Ft, Pp);                       /* P^- = F P F^T + Q  */
    for (int i = 0; i < dd; ++i) Pp[i] += Q[i];
    symmetrize(d, Pp);
    if (mp_out) store(1, d, mp, mp_out + k * d);
    if (Pp_out) store(d, d, Pp, Pp_out + k * dd);
    if (mask[k]) {
      real Rk = (real)(R_per_step ? R[k] : R[0]);
      real PH[DMAX], S = Rk, v = (real)y[k], K[DMAX];
      for (int i = 0; i < d; ++i) {
        real s = 0.0L;
        for (int j = 0; j < d; ++j) s += Pp[i * d + j] * H[j];
        PH[i] = s;
      }
      for (int i = 0; i < d; ++i) S += H[i] * PH[i];
      if (!(S > 0.0L)) return 1;
      for (int i = 0; i < d; ++i) v -= H[i] * mp[i];
      for (int i = 0; i < d; ++i) K[i] = PH[i] / S;
      for (int i = 0; i < d; ++i) m[i] = mp[i] + K[i] * v;
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) P[i * d + j] = Pp[i * d + j] - K[i] * S * K[j];
      symmetrize(d, P);
      ll += -0.5L * (logl(twopi * S) + v * v / S);
    } else {
      memcpy(m, mp, sizeof(real) * d);
      memcpy(P, Pp, sizeof(real) * dd);
    }
    store(1, d, m, m_out + k * d);
    store(d, d, P, P_out + k * dd);
  }
  if (loglik) *loglik = (double)ll;
  return 0;
}

/* ----------------------------------------------------------------------- */
int orc_rts_smoother(int d, const double *F_, const double *m_, const double *P_,
                     const double *mp_, const double *Pp_, long n,
                     double *ms_out, double *Ps_out) {
  if (d < 1 || d > DMAX || n < 1) return 3;
  int dd = d * d;
  real ms[DMAX], Ps[DMAX * DMAX];
  load(1, d, m_ + (n - 1) * d, ms);
  load(d, d, P_ + (n - 1) * dd, Ps);
  store(1, d, ms, ms_out + (n - 1) * d);
  store(d, d, Ps, Ps_out + (n - 1) * dd);
  for (long k = n - 2; k >= 0; --k) {
    real F[DMAX * DMAX], m[DMAX], P[DMAX * DMAX], mp[DMAX], Pp[DMAX * DMAX];
    load(d, d, F_ + (k + 1) * dd, F);
    load(1, d, m_ + k * d, m);
    load(d, d, P_ + k * dd, P);
    load(1, d, mp_ + (k + 1) * d, mp);
    load(d, d, Pp_ + (k + 1) * dd, Pp);
    /* G_k = P_k F^T (P^-)^{-1}  <=>  P^- G_k^T = F P_k */
    real X[DMAX * DMAX], Gk[DMAX * DMAX], A[DMAX * DMAX];
    mm(d, d, d, F, P, X);
    memcpy(A, Pp, sizeof(real) * dd);
    if (solve(d, A, X, d)) return 1;
    tr(d, d, X, Gk);
    real dm[DMAX], nms[DMAX];
    for (int i = 0; i < d; ++i) dm[i] = ms[i] - mp[i];
    mm(d, d, 1, Gk, dm, nms);
    for (int i = 0; i < d; ++i) nms[i] += m[i];
    real dP[DMAX * DMAX], T[DMAX * DMAX], Gt[DMAX * DMAX], nPs[DMAX * DMAX];
    for (int i = 0; i < dd; ++i) dP[i] = Ps[i] - Pp[i];
    mm(d, d, d, Gk, dP, T);
    tr(d, d, Gk, Gt);
    mm(d, d, d, T, Gt, nPs);
    for (int i = 0; i < dd; ++i) nPs[i] += P[i];
    symmetrize(d, nPs);
    memcpy(ms, nms, sizeof(real) * d);
    memcpy(Ps, nPs, sizeof(real) * dd);
    store(1, d, ms, ms_out + k * d);
    store(d, d, Ps, Ps_out + k * dd);
  }
  return 0;
}

/* ----------------------------------------------------------------------- */
/* Parallel-filter elements (A, b, C, eta, J) per step.                    */
/*   missing, k > 1:  A = F, b = 0, C = Q            (Sec. 3)              */
/*   missing, k = 1:  A = 0, b = 0, C = P_inf        (Sec. 3)              */
/*   missing, any k:  eta = 0, J = 0                 (Sec. 3)              */
/*   observed, k > 1: S = H Q H^T + R, K = Q H^T / S, A = (I - K H) F,     */
/*     b = K y, C = (I - K H) Q, eta = F^T H^T y / S,                      */
/*     J = F^T H^T H F / S                  (supplement, proof of Prop. 1) */
/*   observed, k = 1: the prior at t_1 does not depend on x_0, so A = 0,   */
/*     eta = 0, J = 0, and b, C are the update of N(0, P_inf) by y_1.      */
/* Element arrays: A, C, J are d x d per step, b and eta are d per step.   */
/* ----------------------------------------------------------------------- */
int orc_filter_elements(int d, const double *H_, const double *R, int R_per_step,
                        const double *Pinf_, const double *F_, const double *Q_,
                        const double *y, const unsigned char *mask, long n,
                        double *A_, double *b_, double *C_, double *eta_, double *J_) {
  if (d < 1 || d > DMAX || n < 1) return 3;
  int dd = d * d;
  real H[DMAX], Pinf[DMAX * DMAX];
  load(1, d, H_, H); load(d, d, Pinf_, Pinf);
  for (long k = 0; k < n; ++k) {
    real F[DMAX * DMAX], Q[DMAX * DMAX];
    real A[DMAX * DMAX], b[DMAX], C[DMAX * DMAX], eta[DMAX], J[DMAX * DMAX];
    if (k == 0) {
      memset(F, 0, sizeof(F));
      memcpy(Q, Pinf, sizeof(real) * dd);
    } else {
      load(d, d, F_ + k * dd, F);
      load(d, d, Q_ + k * dd, Q);
    }
    memset(b, 0, sizeof(b)); memset(eta, 0, sizeof(eta)); memset(J, 0, sizeof(J));
    if (!mask[k]) {
      memcpy(A, F, sizeof(real) * dd);            /* F (k>1) or 0 (k=1)        */
      memcpy(C, Q, sizeof(real) * dd);            /* Q (k>1) or P_inf (k=1)    */
    } else {
      real Rk = (real)(R_per_step ? R[k] : R[0]);
      real QH[DMAX], S = Rk;
      for (int i = 0; i < d; ++i) {
        real s = 0.0L;
        for (int j = 0; j < d; ++j) s += Q[i * d + j] * H[j];
        QH[i] = s;
      }
      for (int i = 0; i < d; ++i) S += H[i] * QH[i];
      if (!(S > 0.0L)) return 1;
      real K[DMAX], IKH[DMAX * DMAX];
      for (int i = 0; i < d; ++i) K[i] = QH[i] / S;
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) IKH[i * d + j] = (i == j ? 1.0L : 0.0L) - K[i] * H[j];
      mm(d, d, d, IKH, F, A);
      for (int i = 0; i < d; ++i) b[i] = K[i] * (real)y[k];
      mm(d, d, d, IKH, Q, C);
      symmetrize(d, C);
      if (k > 0) {
        real HF[DMAX];                              /* H F (row vector)          */
        for (int j = 0; j < d; ++j) {
          real s = 0.0L;
          for (int i = 0; i < d; ++i) s += H[i] * F[i * d + j];
          HF[j] = s;
        }
        for (int i = 0; i < d; ++i) eta[i] = HF[i] * (real)y[k] / S;
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j) J[i * d + j] = HF[i] * HF[j] / S;
      }
      if (k == 0) memset(A, 0, sizeof(A));
    }
    store(d, d, A, A_ + k * dd); store(1, d, b, b_ + k * d);
    store(d, d, C, C_ + k * dd); store(1, d, eta, eta_ + k * d);
    store(d, d, J, J_ + k * dd);
  }
  return 0;
}

/* ----------------------------------------------------------------------- */
/* The filtering operator (Sec. 3), (i) earlier, (j) later:                */
/*  A_ij = A_j (I + C_i J_j)^{-1} A_i                                      */
/*  b_ij = A_j (I + C_i J_j)^{-1} (b_i + C_i eta_j) + b_j                  */
/*  C_ij = A_j (I + C_i J_j)^{-1} C_i A_j^T + C_j                          */
/*  eta_ij = A_i^T (I + J_j C_i)^{-1} (eta_j - J_j b_i) + eta_i            */
/*  J_ij = A_i^T (I + J_j C_i)^{-1} J_j A_i + J_i                          */
/* The inverses are applied by solving with partial pivoting.              */
/* ----------------------------------------------------------------------- */
int orc_filter_combine(int d,
                       const double *Ai_, const double *bi_, const double *Ci_, const double *etai_, const double *Ji_,
                       const double *Aj_, const double *bj_, const double *Cj_, const double *etaj_, const double *Jj_,
                       double *A_, double *b_, double *C_, double *eta_, double *J_) {
  if (d < 1 || d > DMAX) return 3;
  int dd = d * d;
  real Ai[DMAX * DMAX], bi[DMAX], Ci[DMAX * DMAX], etai[DMAX], Ji[DMAX * DMAX];
  real Aj[DMAX * DMAX], bj[DMAX], Cj[DMAX * DMAX], etaj[DMAX], Jj[DMAX * DMAX];
  load(d, d, Ai_, Ai); load(1, d, bi_, bi); load(d, d, Ci_, Ci); load(1, d, etai_, etai); load(d, d, Ji_, Ji);
  load(d, d, Aj_, Aj); load(1, d, bj_, bj); load(d, d, Cj_, Cj); load(1, d, etaj_, etaj); load(d, d, Jj_, Jj);

  /* M1 = I + C_i J_j ; right-hand sides [A_i | b_i + C_i eta_j | C_i] */
  real M1[DMAX * DMAX];
  mm(d, d, d, Ci, Jj, M1);
  for (int i = 0; i < d; ++i) M1[i * d + i] += 1.0L;
  int m = 2 * d + 1;
  real RHS[DMAX * (2 * DMAX + 1)];
  real Ceta[DMAX];
  mm(d, d, 1, Ci, etaj, Ceta);
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j < d; ++j) RHS[i * m + j] = Ai[i * d + j];
    RHS[i * m + d] = bi[i] + Ceta[i];
    for (int j = 0; j < d; ++j) RHS[i * m + d + 1 + j] = Ci[i * d + j];
  }
  if (solve(d, M1, RHS, m)) return 1;
  real XA[DMAX * DMAX], xb[DMAX], XC[DMAX * DMAX];
  for (int i = 0; i < d; ++i) {
    for (int j = 0; j < d; ++j) XA[i * d + j] = RHS[i * m + j];
    xb[i] = RHS[i * m + d];
    for (int j = 0; j < d; ++j) XC[i * d + j] = RHS[i * m + d + 1 + j];
  }
  real A[DMAX * DMAX], b[DMAX], C[DMAX * DMAX], T[DMAX * DMAX], Ajt[DMAX * DMAX];
  mm(d, d, d, Aj, XA, A);
  mm(d, d, 1, Aj, xb, b);
  for (int i = 0; i < d; ++i) b[i] += bj[i];
  mm(d, d, d, Aj, XC, T);
  tr(d, d, Aj, Ajt);
  mm(d, d, d, T, Ajt, C);
  for (int i = 0; i < dd; ++i) C[i] += Cj[i];
  symmetrize(d, C);

  /* M2 = I + J_j C_i ; right-hand sides [eta_j - J_j b_i | J_j A_i] */
  real M2[DMAX * DMAX];
  mm(d, d, d, Jj, Ci, M2);
  for (int i = 0; i < d; ++i) M2[i * d + i] += 1.0L;
  int m2 = d + 1;
  real RHS2[DMAX * (DMAX + 1)], Jb[DMAX], JA[DMAX * DMAX];
  mm(d, d, 1, Jj, bi, Jb);
  mm(d, d, d, Jj, Ai, JA);
  for (int i = 0; i < d; ++i) {
    RHS2[i * m2] = etaj[i] - Jb[i];
    for (int j = 0; j < d; ++j) RHS2[i * m2 + 1 + j] = JA[i * d + j];
  }
  if (solve(d, M2, RHS2, m2)) return 1;
  real Ait[DMAX * DMAX], z[DMAX], Z[DMAX * DMAX], eta[DMAX], J[DMAX * DMAX];
  for (int i = 0; i < d; ++i) {
    z[i] = RHS2[i * m2];
    for (int j = 0; j < d; ++j) Z[i * d + j] = RHS2[i * m2 + 1 + j];
  }
  tr(d, d, Ai, Ait);
  mm(d, d, 1, Ait, z, eta);
  for (int i = 0; i < d; ++i) eta[i] += etai[i];
  mm(d, d, d, Ait, Z, J);
  for (int i = 0; i < dd; ++i) J[i] += Ji[i];
  symmetrize(d, J);

  store(d, d, A, A_); store(1, d, b, b_); store(d, d, C, C_);
  store(1, d, eta, eta_); store(d, d, J, J_);
  return 0;
}

/* ----------------------------------------------------------------------- */
/* Parallel-smoother elements (E, g, L) per step (supplement, Prop. 2):    */
/*   k < n:  E_k = P_k F^T (F P_k F^T + Q)^{-1}  (the smoother gain),      */
/*           g_k = m_k - E_k F m_k,   L_k = P_k - E_k F P_k,               */
/*           with F, Q the transition from step k to step k+1;             */
/*   k = n:  E = 0, g = m_n, L = P_n.                                       */
/* ----------------------------------------------------------------------- */
int orc_smoother_elements(int d, const double *F_, const double *Q_,
                          const double *m_, const double *P_, long n,
                          double *E_, double *g_, double *L_) {
  if (d < 1 || d > DMAX || n < 1) return 3;
  int dd = d * d;
  for (long k = 0; k < n; ++k) {
    real m[DMAX], P[DMAX * DMAX], E[DMAX * DMAX], g[DMAX], L[DMAX * DMAX];
    load(1, d, m_ + k * d, m);
    load(d, d, P_ + k * dd, P);
    if (k == n - 1) {
      memset(E, 0, sizeof(E));
      memcpy(g, m, sizeof(real) * d);
      memcpy(L, P, sizeof(real) * dd);
    } else {
      real F[DMAX * DMAX], Q[DMAX * DMAX], FP[DMAX * DMAX], Ft[DMAX * DMAX], Pp[DMAX * DMAX];
      load(d, d, F_ + (k + 1) * dd, F);
      load(d, d, Q_ + (k + 1) * dd, Q);
      mm(d, d, d, F, P, FP);
      tr(d, d, F, Ft);
      mm(d, d, d, FP, Ft, Pp);
      for (int i = 0; i < dd; ++i) Pp[i] += Q[i];
      symmetrize(d, Pp);
      real X[DMAX * DMAX];
      memcpy(X, FP, sizeof(real) * dd);           /* Pp E^T = F P */
      if (solve(d, Pp, X, d)) return 1;
      tr(d, d, X, E);
      real Fm[DMAX], EFm[DMAX], EFP[DMAX * DMAX];
      mm(d, d, 1, F, m, Fm);
      mm(d, d, 1, E, Fm, EFm);
      for (int i = 0; i < d; ++i) g[i] = m[i] - EFm[i];
      mm(d, d, d, E, FP, EFP);
      for (int i = 0; i < dd; ++i) L[i] = P[i] - EFP[i];
      symmetrize(d, L);
    }
    store(d, d, E, E_ + k * dd); store(1, d, g, g_ + k * d); store(d, d, L, L_ + k * dd);
  }
  return 0;
}

/* The smoothing operator (supplement, Prop. 2), (i) earlier, (j) later:    */
/*   (E_i, g_i, L_i) x (E_j, g_j, L_j) = (E_i E_j, E_i g_j + g_i,           */
/*                                        E_i L_j E_i^T + L_i)              */
int orc_smoother_combine(int d,
                         const double *Ei_, const double *gi_, const double *Li_,
                         const double *Ej_, const double *gj_, const double *Lj_,
                         double *E_, double *g_, double *L_) {
  if (d < 1 || d > DMAX) return 3;
  int dd = d * d;
  real Ei[DMAX * DMAX], gi[DMAX], Li[DMAX * DMAX], Ej[DMAX * DMAX], gj[DMAX], Lj[DMAX * DMAX];
  load(d, d, Ei_, Ei); load(1, d, gi_, gi); load(d, d, Li_, Li);
  load(d, d, Ej_, Ej); load(1, d, gj_, gj); load(d, d, Lj_, Lj);
  real E[DMAX * DMAX], g[DMAX], L[DMAX * DMAX], T[DMAX * DMAX], Eit[DMAX * DMAX];
  mm(d, d, d, Ei, Ej, E);
  mm(d, d, 1, Ei, gj, g);
  for (int i = 0; i < d; ++i) g[i] += gi[i];
  mm(d, d, d, Ei, Lj, T);
  tr(d, d, Ei, Eit);
  mm(d, d, d, T, Eit, L);
  for (int i = 0; i < dd; ++i) L[i] += Li[i];
  symmetrize(d, L);
  store(d, d, E, E_); store(1, d, g, g_); store(d, d, L, L_);
  return 0;
}

/* Library self-identification for the ctypes loader. */
int orc_version(void) { return 1; }

/* ----------------------------------------------------------------------- */
/* Forward-mode (tangent) derivative of the log marginal likelihood        */
/* (Sec. 2, parameter estimation by maximising the marginal likelihood).   */
/*                                                                         */
/* Discretisation tangents: the Frechet derivative of the matrix           */
/* exponential in direction B is the upper-right block of                  */
/*   exp([[A, B], [0, A]]),                                                */
/* applied to Van Loan's block A = [[-G, W], [0, G^T]] h with the tangent  */
/* B = [[-dG, dW], [0, dG^T]] h; then F = E22^T, Q = F E12 give            */
/* dF = dE22^T, dQ = dF E12 + F dE12.  Long steps are halved as in         */
/* discretize_one and doubled back with the differentiated identities      */
/*   F(2h) = F F,  Q(2h) = F Q F^T + Q.                                    */
/* ----------------------------------------------------------------------- */
#define BMAX (4 * DMAX)

/* C = A B, all n x n (n <= BMAX), C may alias A or B */
static void mm_big(int n, const real *A, const real *B, real *C) {
  static __thread real T[BMAX * BMAX];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      real s = 0.0L;
      for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
      T[i * n + j] = s;
    }
  memcpy(C, T, sizeof(real) * n * n);
}

/* exp(A) for n <= BMAX: the same scaling, Taylor sum and squaring as expm */
static void expm_big(int n, const real *A, real *E) {
  real nrm = 0.0L;
  for (int j = 0; j < n; ++j) {
    real c = 0.0L;
    for (int i = 0; i < n; ++i) c += fabsl(A[i * n + j]);
    if (c > nrm) nrm = c;
  }
  int s = 0;
  while (nrm > 0.5L) { nrm *= 0.5L; ++s; }
  static __thread real As[BMAX * BMAX], T[BMAX * BMAX];
  real sc = ldexpl(1.0L, -s);
  for (int i = 0; i < n * n; ++i) As[i] = A[i] * sc;
  memset(E, 0, sizeof(real) * n * n);
  memset(T, 0, sizeof(real) * n * n);
  for (int i = 0; i < n; ++i) { E[i * n + i] = 1.0L; T[i * n + i] = 1.0L; }
  for (int k = 1; k <= 80; ++k) {
    mm_big(n, T, As, T);
    real tmax = 0.0L, emax = 0.0L;
    for (int i = 0; i < n * n; ++i) {
      T[i] /= (real)k;
      E[i] += T[i];
      if (fabsl(T[i]) > tmax) tmax = fabsl(T[i]);
      if (fabsl(E[i]) > emax) emax = fabsl(E[i]);
    }
    if (k > 2 && tmax <= 1e-30L * emax) break;
  }
  for (int i = 0; i < s; ++i) mm_big(n, E, E, E);
}

static void vanloan_tangent(int d, const real *G, const real *W, const real *dG, const real *dW, real h,
                            real *F, real *Q, real *dF, real *dQ) {
  int n = 2 * d, N = 4 * d;
  real X[BMAX * BMAX], E[BMAX * BMAX];
  memset(X, 0, sizeof(X));
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      /* diagonal blocks: Van Loan's matrix C */
      for (int b = 0; b < 2; ++b) {
        int o = b * n;
        X[(o + i) * N + o + j] = -G[i * d + j] * h;
        X[(o + i) * N + o + d + j] = W[i * d + j] * h;
        X[(o + d + i) * N + o + d + j] = G[j * d + i] * h;
      }
      /* upper-right block: its tangent */
      X[i * N + n + j] = -dG[i * d + j] * h;
      X[i * N + n + d + j] = dW[i * d + j] * h;
      X[(d + i) * N + n + d + j] = dG[j * d + i] * h;
    }
  expm_big(N, X, E);
  real E12[DMAX * DMAX], dE12[DMAX * DMAX], T1[DMAX * DMAX], T2[DMAX * DMAX];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      F[i * d + j] = E[(d + j) * N + d + i];            /* F  = E22^T  */
      E12[i * d + j] = E[i * N + d + j];
      dF[i * d + j] = E[(d + j) * N + n + d + i];       /* dF = dE22^T */
      dE12[i * d + j] = E[i * N + n + d + j];
    }
  mm(d, d, d, F, E12, Q);                               /* Q  = F E12  */
  mm(d, d, d, dF, E12, T1);
  mm(d, d, d, F, dE12, T2);
  for (int i = 0; i < d * d; ++i) dQ[i] = T1[i] + T2[i];  /* dQ = dF E12 + F dE12 */
  symmetrize(d, Q);
  symmetrize(d, dQ);
}

static void discretize_tangent_one(int d, const real *G, const real *W, const real *dG, const real *dW, real h,
                                   real *F, real *Q, real *dF, real *dQ) {
  real gn = 0.0L;
  for (int j = 0; j < d; ++j) {
    real c = 0.0L;
    for (int i = 0; i < d; ++i) c += fabsl(G[i * d + j]);
    if (c > gn) gn = c;
  }
  int s = 0;
  while (gn * ldexpl(h, -s) > 0.5L) ++s;
  vanloan_tangent(d, G, W, dG, dW, ldexpl(h, -s), F, Q, dF, dQ);
  for (int r = 0; r < s; ++r) {
    real Ft[DMAX * DMAX], dFt[DMAX * DMAX], T[DMAX * DMAX], A1[DMAX * DMAX], A2[DMAX * DMAX],
        A3[DMAX * DMAX], A4[DMAX * DMAX];
    tr(d, d, F, Ft);
    tr(d, d, dF, dFt);
    /* dQ' = dF Q F^T + F dQ F^T + F Q dF^T + dQ */
    mm(d, d, d, dF, Q, T);  mm(d, d, d, T, Ft, A1);
    mm(d, d, d, F, dQ, T);  mm(d, d, d, T, Ft, A2);
    mm(d, d, d, F, Q, T);   mm(d, d, d, T, dFt, A3);
    /* Q' = F Q F^T + Q */
    mm(d, d, d, T, Ft, A4);
    for (int i = 0; i < d * d; ++i) {
      dQ[i] += A1[i] + A2[i] + A3[i];
      Q[i] += A4[i];
    }
    symmetrize(d, Q);
    symmetrize(d, dQ);
    /* dF' = dF F + F dF,  F' = F F */
    mm(d, d, d, dF, F, A1);
    mm(d, d, d, F, dF, A2);
    for (int i = 0; i < d * d; ++i) dF[i] = A1[i] + A2[i];
    mm(d, d, d, F, F, F);
  }
}

/* Per-step F, Q (as orc_discretize) and their tangents for one direction
 * (dG, dW, dPinf: derivatives of the model's G, W = L q L^T and P_inf). */
int orc_discretize_tangent(int d, const double *G_, const double *W_, const double *Pinf_, const double *dG_,
                           const double *dW_, const double *dPinf_, const double *t, long n, double *F_,
                           double *Q_, double *dF_, double *dQ_) {
  if (d < 1 || d > DMAX || n < 1) return 3;
  for (long k = 1; k < n; ++k)
    if (!(t[k] >= t[k - 1])) return 2;
  real G[DMAX * DMAX], W[DMAX * DMAX], dG[DMAX * DMAX], dW[DMAX * DMAX];
  load(d, d, G_, G); load(d, d, W_, W); load(d, d, dG_, dG); load(d, d, dW_, dW);
  int dd = d * d;
  for (int i = 0; i < dd; ++i) { F_[i] = 0.0; Q_[i] = Pinf_[i]; dF_[i] = 0.0; dQ_[i] = dPinf_[i]; }
#pragma omp parallel for schedule(static)
  for (long k = 1; k < n; ++k) {
    real F[DMAX * DMAX], Q[DMAX * DMAX], dF[DMAX * DMAX], dQ[DMAX * DMAX];
    discretize_tangent_one(d, G, W, dG, dW, (real)t[k] - (real)t[k - 1], F, Q, dF, dQ);
    store(d, d, F, F_ + k * dd); store(d, d, Q, Q_ + k * dd);
    store(d, d, dF, dF_ + k * dd); store(d, d, dQ, dQ_ + k * dd);
  }
  return 0;
}

/* The sequential Kalman filter of orc_kalman_filter carried with one
 * tangent direction: given per-step F, Q and their tangents dF, dQ (step 0:
 * F = 0, Q = P_inf, dQ = dP_inf) and the noise tangent dR (scalar, or per
 * step with R_per_step), returns the log-likelihood and its directional
 * derivative.  Differentiating each line of the filter:
 *   m^- = F m                 dm^- = dF m + F dm
 *   P^- = F P F^T + Q         dP^- = dF P F^T + F dP F^T + F P dF^T + dQ
 *   S = H P^- H^T + R         dS = H dP^- H^T + dR
 *   v = y - H m^-             dv = -H dm^-
 *   K = P^- H^T / S           dK = (dP^- H^T - K dS) / S
 *   m = m^- + K v             dm = dm^- + dK v + K dv
 *   P = P^- - K S K^T         dP = dP^- - dK S K^T - K dS K^T - K S dK^T
 *   l += -1/2 [log(2 pi S) + v^2 / S]
 *                             dl += -1/2 [dS / S + 2 v dv / S - v^2 dS / S^2]
 * dloglik_abs (nullable) receives the sum of the absolute values of the
 * per-step terms of dl: the scale against which the rounding of any order of
 * summing those terms is measured (a gradient near 0 is a cancellation). */
int orc_loglik_tangent(int d, const double *H_, const double *R, const double *dR, int R_per_step,
                       const double *F_, const double *Q_, const double *dF_, const double *dQ_,
                       const double *y, const unsigned char *mask, long n, double *loglik, double *dloglik,
                       double *dloglik_abs) {
  if (d < 1 || d > DMAX || n < 1) return 3;
  const real twopi = 6.283185307179586476925286766559L;
  int dd = d * d;
  real H[DMAX];
  load(1, d, H_, H);
  real m[DMAX] = {0}, P[DMAX * DMAX] = {0}, dm[DMAX] = {0}, dP[DMAX * DMAX] = {0};
  real ll = 0.0L, dll = 0.0L, dabs = 0.0L;
  for (long k = 0; k < n; ++k) {
    real F[DMAX * DMAX], Q[DMAX * DMAX], dF[DMAX * DMAX], dQ[DMAX * DMAX], Ft[DMAX * DMAX], dFt[DMAX * DMAX];
    load(d, d, F_ + k * dd, F); load(d, d, Q_ + k * dd, Q);
    load(d, d, dF_ + k * dd, dF); load(d, d, dQ_ + k * dd, dQ);
    tr(d, d, F, Ft);
    tr(d, d, dF, dFt);
    real mp[DMAX], dmp[DMAX], Pp[DMAX * DMAX], dPp[DMAX * DMAX], T[DMAX * DMAX], A[DMAX * DMAX];
    real t1[DMAX], t2[DMAX];
    mm(d, d, 1, F, m, mp);
    mm(d, d, 1, dF, m, t1);
    mm(d, d, 1, F, dm, t2);
    for (int i = 0; i < d; ++i) dmp[i] = t1[i] + t2[i];
    mm(d, d, d, F, P, T); mm(d, d, d, T, Ft, Pp);
    for (int i = 0; i < dd; ++i) Pp[i] += Q[i];
    for (int i = 0; i < dd; ++i) dPp[i] = dQ[i];
    mm(d, d, d, dF, P, T); mm(d, d, d, T, Ft, A);
    for (int i = 0; i < dd; ++i) dPp[i] += A[i];
    mm(d, d, d, F, dP, T); mm(d, d, d, T, Ft, A);
    for (int i = 0; i < dd; ++i) dPp[i] += A[i];
    mm(d, d, d, F, P, T); mm(d, d, d, T, dFt, A);
    for (int i = 0; i < dd; ++i) dPp[i] += A[i];
    symmetrize(d, Pp);
    symmetrize(d, dPp);
    if (mask[k]) {
      real Rk = (real)(R_per_step ? R[k] : R[0]);
      real dRk = (real)(R_per_step ? dR[k] : dR[0]);
      real PH[DMAX], dPH[DMAX];
      for (int i = 0; i < d; ++i) {
        real s = 0.0L, ds = 0.0L;
        for (int j = 0; j < d; ++j) { s += Pp[i * d + j] * H[j]; ds += dPp[i * d + j] * H[j]; }
        PH[i] = s; dPH[i] = ds;
      }
      real S = Rk, dS = dRk;
      for (int i = 0; i < d; ++i) { S += H[i] * PH[i]; dS += H[i] * dPH[i]; }
      if (!(S > 0.0L)) return 1;
      real v = (real)y[k], dv = 0.0L;
      for (int i = 0; i < d; ++i) { v -= H[i] * mp[i]; dv -= H[i] * dmp[i]; }
      real K[DMAX], dK[DMAX];
      for (int i = 0; i < d; ++i) { K[i] = PH[i] / S; dK[i] = (dPH[i] - K[i] * dS) / S; }
      for (int i = 0; i < d; ++i) {
        m[i] = mp[i] + K[i] * v;
        dm[i] = dmp[i] + dK[i] * v + K[i] * dv;
      }
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          P[i * d + j] = Pp[i * d + j] - K[i] * S * K[j];
          dP[i * d + j] = dPp[i * d + j] - dK[i] * S * K[j] - K[i] * dS * K[j] - K[i] * S * dK[j];
        }
      symmetrize(d, P);
      symmetrize(d, dP);
      ll += -0.5L * (logl(twopi * S) + v * v / S);
      const real dterm = -0.5L * (dS / S + 2.0L * v * dv / S - v * v * dS / (S * S));
      dll += dterm;
      dabs += fabsl(dterm);
    } else {
      memcpy(m, mp, sizeof(real) * d); memcpy(dm, dmp, sizeof(real) * d);
      memcpy(P, Pp, sizeof(real) * dd); memcpy(dP, dPp, sizeof(real) * dd);
    }
  }
  if (loglik) *loglik = (double)ll;
  if (dloglik) *dloglik = (double)dll;
  if (dloglik_abs) *dloglik_abs = (double)dabs;
  return 0;
}

/* ----------------------------------------------------------------------- */
/* Simulation from the state-space prior (the training data of the learned */
/* initialisation): random numbers from the counter-based generator        */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as */
/* easy as 1, 2, 3", SC 2011), written from its definition: ten rounds of  */
/*   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),                  */
/*                        hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))                  */
/* with the key advanced by the Weyl constants (W0, W1) between rounds.    */
/* ----------------------------------------------------------------------- */
#include <stdint.h>

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k[0];
  const uint32_t n1 = (uint32_t)p1;
  const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k[1];
  const uint32_t n3 = (uint32_t)p0;
  c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

static void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(c, k);
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) { philox4x32_10(ctr, key, out); }

/* a uniform in (0, 1) from two 32-bit words: the 53-bit integer
 * m = a * 2^21 + floor(b / 2^11), u = (m + 1/2) 2^-53 */
static real u53(uint32_t a, uint32_t b) {
  const uint64_t m = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
  return ((real)m + 0.5L) * ldexpl(1.0L, -53);
}

/* Draws of series `sid` at step k: call j of the generator has counter
 * (k, sid, j, 0) and key (seed_lo, seed_hi).  Call 0 gives the time
 * increment (its first uniform); call j >= 1 gives two standard normals by
 * Box-Muller: r = sqrt(-2 log u1), (r cos 2 pi u2, r sin 2 pi u2). */
static void draw_call(uint32_t k, uint32_t sid, uint32_t j, uint64_t seed, uint32_t w[4]) {
  const uint32_t ctr[4] = {k, sid, j, 0u};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  philox4x32_10(ctr, key, w);
}

void orc_normals(uint64_t seed, uint32_t sid, uint32_t k, int count, double *z) {
  const real twopi = 6.283185307179586476925286766559L;
  for (int j = 0; j < (count + 1) / 2; ++j) {
    uint32_t w[4];
    draw_call(k, sid, (uint32_t)(j + 1), seed, w);
    const real u1 = u53(w[0], w[1]), u2 = u53(w[2], w[3]);
    const real r = sqrtl(-2.0L * logl(u1));
    z[2 * j] = (double)(r * cosl(twopi * u2));
    if (2 * j + 1 < count) z[2 * j + 1] = (double)(r * sinl(twopi * u2));
  }
}

/* lower Cholesky factor of a symmetric positive semi-definite matrix; a
 * pivot at most 1e-10 times its diagonal entry (a direction with no
 * variance, e.g. a zero-length step) gives a zero column */
static void chol_psd(int d, const real *A, real *L) {
  memset(L, 0, sizeof(real) * d * d);
  for (int j = 0; j < d; ++j) {
    real p = A[j * d + j];
    for (int k = 0; k < j; ++k) p -= L[j * d + k] * L[j * d + k];
    if (!(p > 1e-10L * A[j * d + j])) continue;
    const real ljj = sqrtl(p);
    L[j * d + j] = ljj;
    for (int i = j + 1; i < d; ++i) {
      real s = A[i * d + j];
      for (int k = 0; k < j; ++k) s -= L[i * d + k] * L[j * d + k];
      L[i * d + j] = s / ljj;
    }
  }
}

/* One series of n steps from the prior of the model (G, W, P_inf, H) with
 * noise variance R: t_0 = 0, t_k = t_{k-1} - spacing log u_k (a Poisson
 * process of mean spacing `spacing`); x_0 = chol(P_inf) z_0,
 * x_k = F_k x_{k-1} + chol(Q_k) z_k (F_k, Q_k of the step, Van Loan as in
 * orc_discretize); y_k = H x_k + sqrt(R) z'_k, with (z_k, z'_k) the d + 1
 * normals of step k. */
int orc_simulate_series(int d, const double *G_, const double *W_, const double *Pinf_, const double *H_,
                        double R, long n, uint64_t seed, uint32_t sid, double spacing, double *t_out,
                        double *y_out) {
  if (d < 1 || d > DMAX || n < 0) return 3;
  real G[DMAX * DMAX], W[DMAX * DMAX], Pinf[DMAX * DMAX], H[DMAX], L[DMAX * DMAX];
  load(d, d, G_, G); load(d, d, W_, W); load(d, d, Pinf_, Pinf); load(1, d, H_, H);
  real x[DMAX];
  real t = 0.0L;
  for (long k = 0; k < n; ++k) {
    double z[DMAX + 2];
    orc_normals(seed, sid, (uint32_t)k, d + 1, z);
    if (k == 0) {
      chol_psd(d, Pinf, L);
      for (int i = 0; i < d; ++i) {
        real s = 0.0L;
        for (int j = 0; j <= i; ++j) s += L[i * d + j] * (real)z[j];
        x[i] = s;
      }
    } else {
      uint32_t w[4];
      draw_call((uint32_t)k, sid, 0u, seed, w);
      const real h = -(real)spacing * logl(u53(w[0], w[1]));
      t += h;
      real F[DMAX * DMAX], Q[DMAX * DMAX], xn[DMAX];
      discretize_one(d, G, W, h, F, Q);
      chol_psd(d, Q, L);
      for (int i = 0; i < d; ++i) {
        real s = 0.0L;
        for (int j = 0; j < d; ++j) s += F[i * d + j] * x[j];
        for (int j = 0; j <= i; ++j) s += L[i * d + j] * (real)z[j];
        xn[i] = s;
      }
      memcpy(x, xn, sizeof(real) * d);
    }
    real f = 0.0L;
    for (int i = 0; i < d; ++i) f += H[i] * x[i];
    t_out[k] = (double)t;
    y_out[k] = (double)(f + sqrtl((real)R) * (real)z[d]);
  }
  return 0;
}
