// pssgp_model.cpp -- host-side model formation for libpssgp (Sec. 2, 4.1, 4.2).
//
// kernel -> continuous SDE (G, L, q, H)   [Sec. 2, Eq. (ssmodel)]
//        -> stationary covariance P_inf   [Sec. 4.1, vectorised Lyapunov solve]
//        -> diagonal balancing D          [Sec. 4.2, Eq. (scaled-ssmodel)]
//        -> Taylor tables for the on-device discretisation of
//           supplement Eq. (ss-gp-formation).
// All of it is O(1) in the number of time steps and runs in long double.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "../../include/pssgp.h"

namespace {

typedef long double ld;
typedef std::complex<long double> cld;
constexpr int DM = PSSGP_DMAX;
const ld kPi = 3.141592653589793238462643383279502884L;

// Gaussian elimination with partial pivoting on an n x n system (n <= 64).
bool gauss_solve(int n, ld* A, ld* b) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[p * n + c])) p = r;
    if (A[p * n + c] == 0.0L) return false;
    if (p != c) {
      for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[p * n + j]);
      std::swap(b[c], b[p]);
    }
    for (int r = c + 1; r < n; ++r) {
      ld f = A[r * n + c] / A[c * n + c];
      for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
      b[r] -= f * b[c];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    ld s = b[c];
    for (int j = c + 1; j < n; ++j) s -= A[c * n + j] * b[j];
    b[c] = s / A[c * n + c];
  }
  return true;
}

// Stationary covariance: G P + P G^T + W = 0, written for the unknown
// vec(P) as (G (x) I + I (x) G) vec(P) = -vec(W) (Sec. 4.1).
bool lyapunov(int d, const ld* G, const ld* W, ld* P) {
  const int n = d * d;
  ld A[64 * 64];
  ld b[64];
  for (int i = 0; i < n * n; ++i) A[i] = 0.0L;
  // row (i,j): sum_k G[i][k] P[k][j] + sum_k P[i][k] G[j][k] = -W[i][j]
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      const int row = i * d + j;
      for (int k = 0; k < d; ++k) {
        A[row * n + k * d + j] += G[i * d + k];
        A[row * n + i * d + k] += G[j * d + k];
      }
      b[row] = -W[i * d + j];
    }
  if (!gauss_solve(n, A, b)) return false;
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) P[i * d + j] = 0.5L * (b[i * d + j] + b[j * d + i]);
  return true;
}

// Roots of the truncated exponential T_n(z) = sum_{k<=n} z^k / k! by the
// Aberth-Ehrlich simultaneous iteration.
bool truncated_exp_roots(int n, cld* z) {
  ld c[DM + 1];
  ld f = 1.0L;
  for (int k = 0; k <= n; ++k) { c[k] = 1.0L / f; f *= (ld)(k + 1); }
  const ld R = 0.6L * n + 1.0L;
  for (int i = 0; i < n; ++i) z[i] = std::polar(R, (2.0L * kPi * (i + 0.25L)) / n);
  for (int it = 0; it < 500; ++it) {
    ld worst = 0.0L;
    for (int i = 0; i < n; ++i) {
      cld p = c[n], dp = 0.0L;
      for (int k = n - 1; k >= 0; --k) { dp = dp * z[i] + p; p = p * z[i] + c[k]; }
      const cld ratio = p / dp;
      cld s = 0.0L;
      for (int j = 0; j < n; ++j) if (j != i) s += 1.0L / (z[i] - z[j]);
      const cld w = ratio / (1.0L - ratio * s);
      z[i] -= w;
      const ld rel = std::abs(w) / std::max(std::abs(z[i]), (ld)1e-30L);
      if (rel > worst) worst = rel;
    }
    if (worst < 1e-30L) break;
  }
  for (int i = 0; i < n; ++i) {
    cld p = c[n];
    for (int k = n - 1; k >= 0; --k) p = p * z[i] + c[k];
    if (!(std::abs(p) <= 1e-14L)) return false;
  }
  return true;
}

// Companion SDE of a monic Hurwitz polynomial a(s) = s^d + a_{d-1} s^{d-1} + ... + a_0
// driven by white noise of density q in the last coordinate; f = x_0.
void companion(int d, const ld* a, ld* G, ld* L, ld* H) {
  for (int i = 0; i < d * d; ++i) G[i] = 0.0L;
  for (int i = 0; i + 1 < d; ++i) G[i * d + i + 1] = 1.0L;
  for (int j = 0; j < d; ++j) G[(d - 1) * d + j] = -a[j];
  for (int i = 0; i < d; ++i) { L[i] = (i == d - 1) ? 1.0L : 0.0L; H[i] = (i == 0) ? 1.0L : 0.0L; }
}

// Parlett-Reinsch balancing with 1-norms and powers of two: diagonal D with
// D^{-1} G D having comparable off-diagonal row and column norms (Sec. 4.2,
// Osborne's method).  D[0] = 1.
void balance(int d, const ld* G, ld* Dv) {
  for (int i = 0; i < d; ++i) Dv[i] = 1.0L;
  for (int sweep = 0; sweep < 200; ++sweep) {
    bool done = true;
    for (int i = 0; i < d; ++i) {
      ld c = 0.0L, r = 0.0L;
      for (int j = 0; j < d; ++j) {
        if (j == i) continue;
        c += fabsl(G[j * d + i] * Dv[i] / Dv[j]);
        r += fabsl(G[i * d + j] * Dv[j] / Dv[i]);
      }
      if (c == 0.0L || r == 0.0L) continue;
      ld f = 1.0L, cc = c, rr = r;
      while (cc < rr / 2.0L) { cc *= 2.0L; rr /= 2.0L; f *= 2.0L; }
      while (cc > rr * 2.0L) { cc /= 2.0L; rr *= 2.0L; f /= 2.0L; }
      if (cc + rr < 0.95L * (c + r)) { Dv[i] *= f; done = false; }
    }
    if (done) break;
  }
  const ld d0 = Dv[0];
  for (int i = 0; i < d; ++i) Dv[i] /= d0;
}

ld factorial(int k) { ld f = 1.0L; for (int i = 2; i <= k; ++i) f *= i; return f; }

// Largest theta in [0, 1] with tail(theta) <= 2^-54, by bisection.
template <class Tail>
double threshold(Tail tail) {
  ld lo = 0.0L, hi = 1.0L;
  if (tail(hi) <= ldexpl(1.0L, -54)) return 1.0;
  for (int it = 0; it < 200; ++it) {
    const ld mid = 0.5L * (lo + hi);
    if (tail(mid) <= ldexpl(1.0L, -54)) lo = mid; else hi = mid;
  }
  return (double)lo;
}

int finish_model(int d, int kind, const ld* G0, const ld* L0, ld q, const ld* H0, int do_balance,
                 pssgp_model* out) {
  // H must be h0 e_0^T
  const ld h0 = H0[0];
  if (!(h0 != 0.0L) || !std::isfinite((double)h0)) return PSSGP_EKERNEL;
  for (int i = 1; i < d; ++i) if (H0[i] != 0.0L) return PSSGP_EKERNEL;
  for (int i = 0; i < d * d; ++i) if (!std::isfinite((double)G0[i])) return PSSGP_EKERNEL;
  if (!(q > 0.0L) || !std::isfinite((double)q)) return PSSGP_EKERNEL;
  ld W0[DM * DM], P0[DM * DM];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) W0[i * d + j] = L0[i] * q * L0[j];
  if (!lyapunov(d, G0, W0, P0)) return PSSGP_EMODEL;
  for (int i = 0; i < d; ++i) if (!(P0[i * d + i] > 0.0L)) return PSSGP_EMODEL;
  ld Db[DM];
  if (do_balance) balance(d, G0, Db); else for (int i = 0; i < d; ++i) Db[i] = 1.0L;
  ld Dt[DM];
  for (int i = 0; i < d; ++i) Dt[i] = Db[i] / h0;           // x = Dt z, H Dt = e_0^T
  ld G[DM * DM], W[DM * DM], P[DM * DM];
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      G[i * d + j] = G0[i * d + j] * Dt[j] / Dt[i];
      W[i * d + j] = W0[i * d + j] / (Dt[i] * Dt[j]);
      P[i * d + j] = P0[i * d + j] / (Dt[i] * Dt[j]);
    }
  std::memset(out, 0, sizeof(*out));
  out->d = d;
  out->kind = kind;
  for (int i = 0; i < d * d; ++i) { out->G[i] = (double)G[i]; out->W[i] = (double)W[i]; out->Pinf[i] = (double)P[i]; }
  for (int i = 0; i < d; ++i) out->D[i] = (double)Dt[i];
  ld gn = 0.0L;
  for (int j = 0; j < d; ++j) {
    ld c = 0.0L;
    for (int i = 0; i < d; ++i) c += fabsl(G[i * d + j]);
    if (c > gn) gn = c;
  }
  out->gnorm = (double)gn;
  // Taylor tables: F(h) = sum_m G^m h^m / m!,  Q(h) = sum_{m>=1} W_m h^m / m!
  // with W_1 = W, W_{m+1} = G W_m + W_m G^T (the h-derivatives of the integral
  // of Eq. (ss-gp-formation) at h = 0).
  ld Gp[DM * DM], T[DM * DM], Wm[DM * DM];
  for (int i = 0; i < d * d; ++i) Gp[i] = 0.0L;
  for (int i = 0; i < d; ++i) Gp[i * d + i] = 1.0L;
  for (int i = 0; i < d * d; ++i) Wm[i] = W[i];
  for (int m = 0; m < PSSGP_NTAYLOR; ++m) {
    const ld fm = factorial(m), fm1 = factorial(m + 1);
    for (int e = 0; e < d * d; ++e) {
      out->fc[e * PSSGP_NTAYLOR + m] = (double)(Gp[e] / fm);
      out->qc[e * PSSGP_NTAYLOR + m] = (double)(Wm[e] / fm1);
    }
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        ld s = 0.0L;
        for (int k = 0; k < d; ++k) s += Gp[i * d + k] * G[k * d + j];
        T[i * d + j] = s;
      }
    std::memcpy(Gp, T, sizeof(ld) * d * d);
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) {
        ld s = 0.0L;
        for (int k = 0; k < d; ++k) s += G[i * d + k] * Wm[k * d + j] + Wm[i * d + k] * G[j * d + k];
        T[i * d + j] = s;
      }
    std::memcpy(Wm, T, sizeof(ld) * d * d);
  }
  // exact norms ||G^m||_1 (m = 0..MN) and ||W_m||_1 (m = 1..MN+1) for the
  // truncation bounds of the two series
  constexpr int MN = 120;
  ld gnm[MN + 1], wnm[MN + 2];
  {
    auto norm1 = [d](const ld* A) {
      ld best = 0.0L;
      for (int j = 0; j < d; ++j) {
        ld c = 0.0L;
        for (int i = 0; i < d; ++i) c += fabsl(A[i * d + j]);
        best = std::max(best, c);
      }
      return best;
    };
    ld Pw[DM * DM], Ww[DM * DM], nP[DM * DM], nW[DM * DM];
    for (int i = 0; i < d * d; ++i) Pw[i] = 0.0L;
    for (int i = 0; i < d; ++i) Pw[i * d + i] = 1.0L;
    for (int i = 0; i < d * d; ++i) Ww[i] = W[i];
    wnm[0] = 0.0L;
    for (int m = 0; m <= MN; ++m) {
      gnm[m] = norm1(Pw);         // ||G^m||
      wnm[m + 1] = norm1(Ww);     // ||W_{m+1}||
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          ld a = 0.0L, bb = 0.0L;
          for (int k = 0; k < d; ++k) {
            a += Pw[i * d + k] * G[k * d + j];
            bb += G[i * d + k] * Ww[k * d + j] + Ww[i * d + k] * G[j * d + k];
          }
          nP[i * d + j] = a;
          nW[i * d + j] = bb;
        }
      std::memcpy(Pw, nP, sizeof(ld) * d * d);
      std::memcpy(Ww, nW, sizeof(ld) * d * d);
    }
  }
  const ld w1 = wnm[1];
  const ld eps = ldexpl(1.0L, -54);
  auto tail_f = [&](int K, ld h) {       // sum_{m >= K} ||G^m|| h^m / m!
    ld s = 0.0L, hm = powl(h, K), fm = factorial(K);
    for (int m = K; m <= MN; ++m) { s += gnm[m] * hm / fm; hm *= h; fm *= (m + 1); }
    return s;
  };
  auto tail_q = [&](int K, ld h) {       // sum_{m >= K} ||W_{m+1}|| h^m / (m+1)!  relative to ||W_1||
    ld s = 0.0L, hm = powl(h, K), fm = factorial(K + 1);
    for (int m = K; m < MN; ++m) { s += wnm[m + 1] * hm / fm; hm *= h; fm *= (m + 2); }
    return s / w1;
  };
  auto largest_h = [&](auto tail, int K, ld bound) {
    ld lo = 0.0L, hi = 1.0L;
    while (tail(K, hi) <= bound && hi < 1e6L) { lo = hi; hi *= 2.0L; }
    for (int it = 0; it < 200; ++it) {
      const ld mid = 0.5L * (lo + hi);
      if (tail(K, mid) <= bound) lo = mid; else hi = mid;
    }
    return lo;
  };
  out->hthr_f[0] = 0.0;
  out->hthr_q[0] = 0.0;
  for (int K = 1; K <= PSSGP_NTAYLOR; ++K) {
    out->hthr_f[K] = (double)(0.999L * largest_h(tail_f, K, eps));
    out->hthr_q[K] = (double)(0.999L * largest_h(tail_q, K, eps));
  }
  // split points of the mixed-precision sums: terms from K on below 2^-36 may
  // be summed in FP32 (Horner error at most 2 x 16 x 2^-24 of their size, i.e.
  // below 2^-55), if every coefficient is zero or within the FP32-safe range
  bool f32ok = true;
  for (int e = 0; e < d * d * PSSGP_NTAYLOR; ++e)
    for (const double c : {out->fc[e], out->qc[e]})
      if (c != 0.0 && !(std::fabs(c) >= 1e-30 && std::fabs(c) <= 1e30)) f32ok = false;
  const ld eps32 = ldexpl(1.0L, -36);
  out->hthr_f32[0] = 0.0;
  out->hthr_q32[0] = 0.0;
  for (int K = 1; K <= PSSGP_NTAYLOR; ++K) {
    out->hthr_f32[K] = f32ok ? (double)(0.999L * largest_h(tail_f, K, eps32)) : 0.0;
    out->hthr_q32[K] = f32ok ? (double)(0.999L * largest_h(tail_q, K, eps32)) : 0.0;
  }
  out->hmax = std::min(out->hthr_f[PSSGP_NTAYLOR], out->hthr_q[PSSGP_NTAYLOR]);
  if (!(out->hmax > 0.0)) return PSSGP_EMODEL;
  // companion structure of the balanced drift
  bool comp = d >= 2;
  for (int i = 0; i + 1 < d && comp; ++i)
    for (int j = 0; j < d; ++j)
      if ((j == i + 1) != (G[i * d + j] != 0.0L)) comp = false;
  out->companion = comp ? 1 : 0;
  if (comp) {
    for (int i = 0; i + 1 < d; ++i) {
      const ld c = 1.0L / G[i * d + i + 1];
      for (int j = 0; j < d; ++j) {
        out->rsup[i * d + j] = (j >= 1) ? (double)(G[(j - 1) * d + j] * c) : 0.0;
        out->rlast[i * d + j] = (double)(G[(d - 1) * d + j] * c);
      }
    }
  }
  return PSSGP_OK;
}

}  // namespace

extern "C" int pssgp_model_build(const pssgp_kernel* k, pssgp_model* out) {
  if (!k || !out) return PSSGP_EINVAL;
  const ld ell = k->lengthscale, s2 = k->variance;
  if (!(ell > 0.0L) || !(s2 > 0.0L) || !std::isfinite((double)ell) || !std::isfinite((double)s2))
    return PSSGP_EKERNEL;
  ld a[DM], G[DM * DM], L[DM], H[DM], q;
  int d;
  if (k->kind == PSSGP_MATERN12 || k->kind == PSSGP_MATERN32 || k->kind == PSSGP_MATERN52) {
    // Matern nu = p + 1/2: spectral density ~ (lam^2 + w^2)^{-(p+1)}, so
    // a(s) = (s + lam)^{p+1}, lam = sqrt(2 nu) / ell; q from the spectral
    // density's constant: 2 s2 lam, 4 s2 lam^3, 16/3 s2 lam^5.
    d = (k->kind == PSSGP_MATERN12) ? 1 : (k->kind == PSSGP_MATERN32) ? 2 : 3;
    const ld nu = d - 0.5L;
    const ld lam = sqrtl(2.0L * nu) / ell;
    for (int j = 0; j < d; ++j) {
      ld binom = 1.0L;
      for (int t = 0; t < j; ++t) binom = binom * (d - t) / (t + 1);
      a[j] = binom * powl(lam, d - j);
    }
    q = (d == 1) ? 2.0L * s2 * lam : (d == 2) ? 4.0L * s2 * lam * lam * lam
                                              : 16.0L / 3.0L * s2 * powl(lam, 5);
  } else if (k->kind == PSSGP_RBF) {
    // S(w) ~ s2 sqrt(2 pi) ell / T_n(ell^2 w^2 / 2).  With s = i w the
    // denominator is T_n(-ell^2 s^2 / 2); its roots are s^2 = -2 z / ell^2 for
    // the roots z of T_n; the stable factor takes s = -sqrt(-2 z / ell^2).
    d = k->order;
    if (d < 1 || d > DM) return PSSGP_EDIM;
    cld z[DM], s[DM];
    if (!truncated_exp_roots(d, z)) return PSSGP_EMODEL;
    for (int i = 0; i < d; ++i) {
      s[i] = -std::sqrt(-2.0L * z[i] / (ell * ell));
      if (!(s[i].real() < 0.0L)) return PSSGP_EMODEL;
    }
    // ascending coefficients of prod_i (s - s_i): multiply by (s - s_i) in turn
    cld asc[DM + 1];
    asc[0] = 1.0L;
    for (int j = 1; j <= d; ++j) asc[j] = 0.0L;
    for (int i = 0; i < d; ++i) {
      for (int j = i + 1; j >= 1; --j) asc[j] = asc[j - 1] - s[i] * asc[j];
      asc[0] = -s[i] * asc[0];
    }
    for (int j = 0; j < d; ++j) a[j] = asc[j].real();
    q = s2 * sqrtl(2.0L * kPi) * ell * factorial(d) / powl(ell * ell / 2.0L, d);
  } else {
    return PSSGP_EKERNEL;
  }
  companion(d, a, G, L, H);
  const int rc = finish_model(d, k->kind, G, L, q, H, k->balance, out);
  if (rc == PSSGP_OK) { out->lengthscale = k->lengthscale; out->variance = k->variance; }
  return rc;
}

extern "C" int pssgp_model_from_sde(int32_t d, const double* G_, const double* L_, double q_,
                                    const double* H_, int32_t do_balance, pssgp_model* out) {
  if (!G_ || !L_ || !H_ || !out) return PSSGP_EINVAL;
  if (d < 1 || d > DM) return PSSGP_EDIM;
  ld G[DM * DM], L[DM], H[DM];
  for (int i = 0; i < d * d; ++i) G[i] = G_[i];
  for (int i = 0; i < d; ++i) { L[i] = L_[i]; H[i] = H_[i]; }
  return finish_model(d, 0, G, L, (ld)q_, H, do_balance, out);
}

extern "C" size_t pssgp_model_bytes(void) { return sizeof(pssgp_model); }
