// linalg.cuh -- register-resident small-matrix algebra for the scan kernels.
//
// Every routine is fully unrolled on the state dimension D (1..8), works on
// per-thread register arrays and issues only the FP64 operations the formula
// needs: the FP64 pipe of sm_103a retires one warp instruction per 64 cycles
// per SM sub-partition whatever the number of active lanes, so the operation
// count is the cost model.  Symmetric results are computed on the upper
// triangle and mirrored (a register copy, no FP64 work).  Comparisons that
// would otherwise run on the FP64 pipe are done on the integer bit patterns.
#pragma once
#include <cstdint>

namespace pssgp {

template <int D> using Mat = double[D][D];
template <int D> using Vec = double[D];

// true unless 0 < s < inf
__device__ __forceinline__ bool bad_pos(double s) {
  long long b = __double_as_longlong(s);
  return !(b > 0 && b < 0x7ff0000000000000LL);
}
__device__ __forceinline__ bool nonfinite(double s) {
  return ((__double_as_longlong(s) >> 52) & 0x7ff) == 0x7ff;
}
__device__ __forceinline__ bool negative_nonzero(double s) {
  long long b = __double_as_longlong(s);
  return b < 0 && (b & 0x7fffffffffffffffLL) != 0;
}
// |x| as an integer key, monotone in |x|
__device__ __forceinline__ long long abs_key(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

template <int D>
__device__ __forceinline__ void set_zero(Mat<D>& A) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) A[i][j] = 0.0;
}
template <int D>
__device__ __forceinline__ void set_eye(Mat<D>& A) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) A[i][j] = (i == j) ? 1.0 : 0.0;
}
template <int D>
__device__ __forceinline__ void copy(const Mat<D>& A, Mat<D>& B) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) B[i][j] = A[i][j];
}

// C = A B
template <int D>
__device__ __forceinline__ void mul(const Mat<D>& A, const Mat<D>& B, Mat<D>& C) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = A[i][0] * B[0][j];
#pragma unroll
      for (int k = 1; k < D; ++k) s = fma(A[i][k], B[k][j], s);
      C[i][j] = s;
    }
}
// y = A x
template <int D>
__device__ __forceinline__ void mulv(const Mat<D>& A, const Vec<D>& x, Vec<D>& y) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = A[i][0] * x[0];
#pragma unroll
    for (int k = 1; k < D; ++k) s = fma(A[i][k], x[k], s);
    y[i] = s;
  }
}
// y = A x + c
template <int D>
__device__ __forceinline__ void mulv_add(const Mat<D>& A, const Vec<D>& x, const Vec<D>& c, Vec<D>& y) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = c[i];
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(A[i][k], x[k], s);
    y[i] = s;
  }
}
// y = A^T x + c
template <int D>
__device__ __forceinline__ void mulTv_add(const Mat<D>& A, const Vec<D>& x, const Vec<D>& c, Vec<D>& y) {
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = c[i];
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(A[k][i], x[k], s);
    y[i] = s;
  }
}
// Y = T B^T + Q, symmetric result (upper triangle computed, mirrored);
// with T = B X this is B X B^T + Q.
template <int D>
__device__ __forceinline__ void mul_Bt_sym_add(const Mat<D>& T, const Mat<D>& B, const Mat<D>& Q, Mat<D>& Y) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      double s = Q[i][j];
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(T[i][k], B[j][k], s);
      Y[i][j] = s;
      Y[j][i] = s;
    }
}
// Y = A^T T + Q, symmetric result; with T = X A this is A^T X A + Q.
template <int D>
__device__ __forceinline__ void mul_At_sym_add(const Mat<D>& A, const Mat<D>& T, const Mat<D>& Q, Mat<D>& Y) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      double s = Q[i][j];
#pragma unroll
      for (int k = 0; k < D; ++k) s = fma(A[k][i], T[k][j], s);
      Y[i][j] = s;
      Y[j][i] = s;
    }
}

// In-place LU factorisation with partial pivoting of M, P M = L U, full rows
// exchanged with predicated selects so that M stays in registers.  perm[c] is
// the row exchanged with row c at step c; inv_diag[c] = 1 / U[c][c].
// Returns false if a pivot is zero or not finite.
template <int D>
__device__ __forceinline__ bool lu_factor(Mat<D>& M, int (&perm)[D], double (&inv_diag)[D]) {
  bool ok = true;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    int p = c;
    long long best = abs_key(M[c][c]);
#pragma unroll
    for (int r = c + 1; r < D; ++r) {
      long long k = abs_key(M[r][c]);
      if (k > best) { best = k; p = r; }
    }
    perm[c] = p;
#pragma unroll
    for (int r = c + 1; r < D; ++r) {
      if (p == r) {
#pragma unroll
        for (int j = 0; j < D; ++j) { double t = M[c][j]; M[c][j] = M[r][j]; M[r][j] = t; }
      }
    }
    if (best == 0 || best >= 0x7ff0000000000000LL) ok = false;
    double ip = __drcp_rn(M[c][c]);
    inv_diag[c] = ip;
#pragma unroll
    for (int r = c + 1; r < D; ++r) {
      double f = M[r][c] * ip;
      M[r][c] = f;
#pragma unroll
      for (int j = c + 1; j < D; ++j) M[r][j] = fma(-f, M[c][j], M[r][j]);
    }
  }
  return ok;
}
// Solve M X = B for NR right-hand-side columns held as B[D][NR], in place,
// with the factors of lu_factor: all row interchanges first (the factors hold
// the final row order), then unit-lower forward and upper back substitution.
template <int D, int NR>
__device__ __forceinline__ void lu_solve(const Mat<D>& LU, const int (&perm)[D], const double (&inv_diag)[D],
                                         double (&B)[D][NR]) {
#pragma unroll
  for (int c = 0; c < D; ++c) {
#pragma unroll
    for (int r = c + 1; r < D; ++r) {
      if (perm[c] == r) {
#pragma unroll
        for (int j = 0; j < NR; ++j) { double t = B[c][j]; B[c][j] = B[r][j]; B[r][j] = t; }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < D; ++c) {
#pragma unroll
    for (int r = c + 1; r < D; ++r)
#pragma unroll
      for (int j = 0; j < NR; ++j) B[r][j] = fma(-LU[r][c], B[c][j], B[r][j]);
  }
#pragma unroll
  for (int c = D - 1; c >= 0; --c) {
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      double s = B[c][j];
#pragma unroll
      for (int k = c + 1; k < D; ++k) s = fma(-LU[c][k], B[k][j], s);
      B[c][j] = s * inv_diag[c];
    }
  }
}

// Cholesky factor of a symmetric positive definite S: lower Lc with
// S = Lc Lc^T, and inv_d[i] = 1 / Lc[i][i].  Returns false if a pivot is not
// strictly positive and finite.
template <int D>
__device__ __forceinline__ bool cholesky(const Mat<D>& S, Mat<D>& Lc, double (&inv_d)[D]) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double s = S[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s = fma(-Lc[j][k], Lc[j][k], s);
    if (bad_pos(s)) ok = false;
    double r = rsqrt(s);
    inv_d[j] = r;
    Lc[j][j] = s * r;
#pragma unroll
    for (int i = j + 1; i < D; ++i) {
      double t = S[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) t = fma(-Lc[i][k], Lc[j][k], t);
      Lc[i][j] = t * r;
    }
#pragma unroll
    for (int i = 0; i < j; ++i) Lc[i][j] = 0.0;
  }
  return ok;
}

// Square-root-free factorisation S = Lu diag(d) Lu^T of a symmetric positive
// definite S, Lu unit lower triangular (entries below the diagonal are set,
// the rest are not used); rd[i] = 1 / d_i.  Returns false if a pivot d_i is
// not strictly positive and finite.  Z holds Lu[i][k] d_k for the dot
// products.
template <int D>
__device__ __forceinline__ bool ldlt(const Mat<D>& S, Mat<D>& Lu, double (&rd)[D]) {
  bool ok = true;
  Mat<D> Z;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double s = S[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s = fma(-Z[j][k], Lu[j][k], s);
    if (bad_pos(s)) ok = false;
    const double r = __drcp_rn(s);
    rd[j] = r;
#pragma unroll
    for (int i = j + 1; i < D; ++i) {
      double t = S[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) t = fma(-Z[i][k], Lu[j][k], t);
      Z[i][j] = t;
      Lu[i][j] = t * r;
    }
  }
  return ok;
}

}  // namespace pssgp
