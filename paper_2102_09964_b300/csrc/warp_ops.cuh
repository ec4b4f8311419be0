// warp_ops.cuh -- warp-cooperative forms of the two operators, for the level-2
// scan over warp aggregates.  There only ~600 combines run per round, so
// latency, not throughput, decides: one warp evaluates one combine with the
// matrix entries spread over its lanes (a d x d product is d FMA
// instructions per pass of 32 entries instead of d^3 on one lane).  Operands
// live in shared memory; __syncwarp() orders the phases.
#pragma once
#include "scan_ops.cuh"

namespace pssgp {

// shared-memory doubles one warp needs for a filter combine
template <int D> struct WarpFilterSmem {
  static constexpr int NR = 2 * D + 2;
  static constexpr int N = 2 * FAggSize<D>::N + D * D + D * NR + 2 * D * D + 3 * D;
};
template <int D> struct WarpSmootherSmem { static constexpr int N = 2 * SAggSize<D>::N + D * D; };

// accessors into the packed aggregate layout of store_fagg / store_sagg
template <int D> struct FView {
  const double* p;
  __device__ double A(int i, int j) const { return p[i * D + j]; }
  __device__ double b(int i) const { return p[D * D + i]; }
  __device__ double C(int i, int j) const { return p[D * D + D + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))]; }
  __device__ double eta(int i) const { return p[D * D + D + Sym<D>::N + i]; }
  __device__ double J(int i, int j) const {
    return p[D * D + 2 * D + Sym<D>::N + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))];
  }
};
template <int D> struct SView {
  const double* p;
  __device__ double E(int i, int j) const { return p[i * D + j]; }
  __device__ double g(int i) const { return p[D * D + i]; }
  __device__ double L(int i, int j) const { return p[D * D + D + (i <= j ? pidx<D>(i, j) : pidx<D>(j, i))]; }
};

// warp argmax of a non-negative integer key (ties: lowest index)
__device__ __forceinline__ int warp_argmax(long long key, int idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (k2 > key || (k2 == key && i2 < idx)) { key = k2; idx = i2; }
  }
  return idx;
}

// Filtering operator of Sec. 3 by one warp: o = a (earlier) x b (later), with
// the same algebra as fagg_combine (one LU with partial pivoting of
// M = I + C_a J_b for all right-hand sides).  a, b: packed aggregates in
// shared memory; the result is written packed to `out` with stride `st`.
// Returns false (on every lane) if a pivot is zero or not finite.
template <int D>
__device__ bool warp_fagg_combine(const double* sa, const double* sb, double* work, double* out, int64_t st,
                                  int lane) {
  constexpr int NR = 2 * D + 2;
  const FView<D> a{sa}, b{sb};
  double* M = work;                 // D x D
  double* X = M + D * D;            // D x NR: [A_a | x_b | C_a | x_v]
  double* T = X + D * NR;           // D x D
  double* U = T + D * D;            // D x D
  double* v = U + D * D;            // D
  double* w = v + D;                // D
  double* invd = w + D;             // D
  // M = I + C_a J_b ; v = eta_b - J_b b_a
  for (int e = lane; e < D * D; e += 32) {
    const int i = e / D, j = e % D;
    double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(a.C(i, k), b.J(k, j), s);
    M[e] = s;
  }
  if (lane < D) {
    double s = b.eta(lane);
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(-b.J(lane, k), a.b(k), s);
    v[lane] = s;
  }
  __syncwarp();
  // right-hand sides
  for (int e = lane; e < D * NR; e += 32) {
    const int i = e / NR, j = e % NR;
    double x;
    if (j < D) {
      x = a.A(i, j);
    } else if (j == D) {
      x = a.b(i);
#pragma unroll
      for (int k = 0; k < D; ++k) x = fma(a.C(i, k), b.eta(k), x);
    } else if (j < 2 * D + 1) {
      x = a.C(i, j - D - 1);
    } else {
      x = 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) x = fma(a.C(i, k), v[k], x);
    }
    X[e] = x;
  }
  __syncwarp();
  // LU with partial pivoting; eliminations applied to X as they happen
  bool ok = true;
#pragma unroll 1
  for (int c = 0; c < D; ++c) {
    const long long key = (lane >= c && lane < D) ? abs_key(M[lane * D + c]) : -1LL;
    const int p = warp_argmax(key, lane);
    const long long best = __shfl_sync(0xffffffffu, key, p);
    if (best == 0 || best >= 0x7ff0000000000000LL) ok = false;
    if (p != c) {
      for (int j = lane; j < D + NR; j += 32) {
        if (j < D) { double t = M[c * D + j]; M[c * D + j] = M[p * D + j]; M[p * D + j] = t; }
        else { const int jj = j - D; double t = X[c * NR + jj]; X[c * NR + jj] = X[p * NR + jj]; X[p * NR + jj] = t; }
      }
    }
    __syncwarp();
    const double ip = __drcp_rn(M[c * D + c]);
    if (lane == 0) invd[c] = ip;
    const int rows = D - 1 - c;
    const int cols = (D - 1 - c) + NR;       // trailing M columns, then all of X
    for (int e = lane; e < rows * cols; e += 32) {
      const int r = c + 1 + e / cols, q = e % cols;
      const double l = M[r * D + c] * ip;
      if (q < D - 1 - c) {
        const int j = c + 1 + q;
        M[r * D + j] = fma(-l, M[c * D + j], M[r * D + j]);
      } else {
        const int j = q - (D - 1 - c);
        X[r * NR + j] = fma(-l, X[c * NR + j], X[r * NR + j]);
      }
    }
    __syncwarp();
  }
  // back substitution, columns of X in parallel
#pragma unroll 1
  for (int c = D - 1; c >= 0; --c) {
    if (lane < NR) {
      double s = X[c * NR + lane];
      for (int k = c + 1; k < D; ++k) s = fma(-M[c * D + k], X[k * NR + lane], s);
      X[c * NR + lane] = s * invd[c];
    }
    __syncwarp();
  }
  // products: A = A_b X_A, T = A_b X_C, b = A_b x_b + b_b, U = J_b X_A,
  // w = v - J_b x_v
  for (int e = lane; e < D * D; e += 32) {
    const int i = e / D, j = e % D;
    double sA = 0.0, sT = 0.0, sU = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      sA = fma(b.A(i, k), X[k * NR + j], sA);
      sT = fma(b.A(i, k), X[k * NR + D + 1 + j], sT);
      sU = fma(b.J(i, k), X[k * NR + j], sU);
    }
    out[(i * D + j) * st] = sA;
    T[e] = sT;
    U[e] = sU;
  }
  if (lane < D) {
    double sb = b.b(lane), sw = v[lane];
#pragma unroll
    for (int k = 0; k < D; ++k) {
      sb = fma(b.A(lane, k), X[k * NR + D], sb);
      sw = fma(-b.J(lane, k), X[k * NR + 2 * D + 1], sw);
    }
    out[(D * D + lane) * st] = sb;
    w[lane] = sw;
  }
  __syncwarp();
  // C = T A_b^T + C_b, J = A_a^T U + J_a (packed upper), eta = A_a^T w + eta_a
  for (int e = lane; e < Sym<D>::N; e += 32) {
    int i = 0, r = e;
    while (r >= D - i) { r -= D - i; ++i; }
    const int j = i + r;
    double sC = b.C(i, j), sJ = a.J(i, j);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      sC = fma(T[i * D + k], b.A(j, k), sC);
      sJ = fma(a.A(k, i), U[k * D + j], sJ);
    }
    out[(D * D + D + e) * st] = sC;
    out[(D * D + 2 * D + Sym<D>::N + e) * st] = sJ;
  }
  if (lane < D) {
    double s = a.eta(lane);
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(a.A(k, lane), w[k], s);
    out[(D * D + D + Sym<D>::N + lane) * st] = s;
  }
  return ok;
}

// Smoothing operator (supplement, Prop. 2) by one warp:
// (E_a E_b, E_a g_b + g_a, E_a L_b E_a^T + L_a).
template <int D>
__device__ void warp_sagg_combine(const double* sa, const double* sb, double* work, double* out, int64_t st,
                                  int lane) {
  const SView<D> a{sa}, b{sb};
  double* T = work;                 // E_a L_b
  for (int e = lane; e < D * D; e += 32) {
    const int i = e / D, j = e % D;
    double sE = 0.0, sT = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      sE = fma(a.E(i, k), b.E(k, j), sE);
      sT = fma(a.E(i, k), b.L(k, j), sT);
    }
    out[(i * D + j) * st] = sE;
    T[e] = sT;
  }
  if (lane < D) {
    double s = a.g(lane);
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(a.E(lane, k), b.g(k), s);
    out[(D * D + lane) * st] = s;
  }
  __syncwarp();
  for (int e = lane; e < Sym<D>::N; e += 32) {
    int i = 0, r = e;
    while (r >= D - i) { r -= D - i; ++i; }
    const int j = i + r;
    double s = a.L(i, j);
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(T[i * D + k], a.E(j, k), s);
    out[(D * D + D + e) * st] = s;
  }
}

}  // namespace pssgp
