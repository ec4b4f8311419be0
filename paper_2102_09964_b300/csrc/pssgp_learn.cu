// pssgp_learn.cu -- the learned initialisation of the batched marginal-
// likelihood fit (Sec. 2, parameter estimation): series simulated from the
// state-space prior itself, their log-periodogram features, and a small MLP
// (65 -> 256 -> 256 -> 3, BF16 tensor-core GEMMs with FP32 accumulation)
// trained on the device to propose initial log hyperparameters.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/pssgp.h"
#include "host_model.cuh"
#include "linalg.cuh"
#include "scan_ops.cuh"
#include "tc_gemm.cuh"

using namespace pssgp;

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) from its definition:
// ten rounds of (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1,
// lo(M0 c0)), the key advanced by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// uniform in (0, 1): m = a 2^21 + floor(b / 2^11) (53 bits), (m + 1/2) 2^-53
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  const unsigned long long m = ((unsigned long long)a << 21) | (unsigned long long)(b >> 11);
  return ((double)m + 0.5) * 1.1102230246251565404e-16;
}

// the draws of series sid at step k: call j has counter (k, sid, j, 0), key
// (seed_lo, seed_hi); call 0: time increment, call j >= 1: two normals
__device__ __forceinline__ U4 draw(uint32_t k, uint32_t sid, uint32_t j, unsigned long long seed) {
  return philox(U4{k, sid, j, 0u}, (uint32_t)seed, (uint32_t)(seed >> 32));
}

template <int N>
__device__ __forceinline__ void normals(uint32_t k, uint32_t sid, unsigned long long seed, double (&z)[N]) {
#pragma unroll
  for (int j = 0; j < (N + 1) / 2; ++j) {
    const U4 w = draw(k, sid, (uint32_t)(j + 1), seed);
    const double u1 = u53(w.x, w.y), u2 = u53(w.z, w.w);
    const double r = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    z[2 * j] = r * cs;
    if (2 * j + 1 < N) z[2 * j + 1] = r * sn;
  }
}

// lower Cholesky factor of a symmetric positive semi-definite matrix; a pivot
// at most 1e-10 times its diagonal entry gives a zero column
template <int D>
__device__ __forceinline__ void chol_psd(const Mat<D>& A, Mat<D>& L) {
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double p = A[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) p = fma(-L[j][k], L[j][k], p);
    const bool keep = p > 1e-10 * A[j][j];
    const double ljj = keep ? sqrt(p) : 0.0;
    const double inv = keep ? 1.0 / ljj : 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (i < j) { L[i][j] = 0.0; continue; }
      if (i == j) { L[j][j] = ljj; continue; }
      double s = A[i][j];
#pragma unroll
      for (int k = 0; k < j; ++k) s = fma(-L[i][k], L[j][k], s);
      L[i][j] = s * inv;
    }
  }
}

// one thread per series: t_0 = 0, t_k = t_{k-1} - spacing log u_k;
// x_0 = chol(q P_inf) z, x_k = F_k x_{k-1} + chol(Q_k) z (the model built at
// (l0, s20) rescaled to the series' (l, s2) as in the batched filter);
// y_k = z-coordinate 0 of x_k (f, as H D = e_0^T) + sqrt(R) z'
template <int D>
__global__ void __launch_bounds__(128) k_simulate_prior(const DevModel<D> m, double ell0, double var0,
                                                        const int64_t* offsets, int B, const double* params,
                                                        unsigned long long seed, double spacing, double* t_out,
                                                        double* y_out, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < B;
  int64_t a = 0, len = 0;
  double uscale = 1.0, qscale = 1.0, sqR = 0.0;
  if (live) {
    a = offsets[s];
    len = offsets[s + 1] - a;
    uscale = ell0 / params[3 * s];
    qscale = params[3 * s + 1] / var0;
    sqR = sqrt(params[3 * s + 2]);
  }
  // every lane of the warp runs the warp's longest series (discretize needs
  // the whole warp)
  int64_t lmax = len;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)lmax, o));
  Vec<D> x;
#pragma unroll
  for (int i = 0; i < D; ++i) x[i] = 0.0;
  double t = 0.0;
  int bits = 0;
#pragma unroll 1
  for (int64_t k = 0; k < lmax; ++k) {
    const bool act = k < len;
    double h = 0.0;
    if (act && k > 0) {
      const U4 w = draw((uint32_t)k, (uint32_t)s, 0u, seed);
      h = -spacing * log(u53(w.x, w.y));
    }
    Mat<D> F, Q, L;
    discretize<D>(m, h, k == 0, act, F, Q, uscale, qscale, true);
    double z[D + 1];
    normals<D + 1>((uint32_t)k, (uint32_t)s, seed, z);
    chol_psd<D>(Q, L);
    Vec<D> xn;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double acc = 0.0;
      if (k > 0) {
#pragma unroll
        for (int j = 0; j < D; ++j) acc = fma(F[i][j], x[j], acc);
      }
#pragma unroll
      for (int j = 0; j <= i; ++j) acc = fma(L[i][j], z[j], acc);
      xn[i] = acc;
    }
    if (act) {
#pragma unroll
      for (int i = 0; i < D; ++i) x[i] = xn[i];
      t += h;
      t_out[a + k] = t;
      const double y = fma(sqR, z[D], x[0]);
      if (nonfinite(y)) bits |= PSSGP_ENAN;
      y_out[a + k] = y;
    }
  }
  if (bits) atomicOr(status, bits);
}

// ---------------------------------------------------------------------------
// Features: 64-bin log periodogram and log sample variance (65 per series).
// For a series y_k, k < n (n >= 2), with mean ybar, s2 = sum (y - ybar)^2 / n
// and mean spacing dbar = (t_{n-1} - t_0) / (n - 1), on the regular grid k dbar:
//   A(w) = |sum_k (y_k - ybar) exp(-i w k dbar)|^2 / (n s2),
//   P_j = 1/4 sum_{q<4} A(w_lo r^(j + (q - 3/2) / 4)),  r = (w_hi / w_lo)^(1/63),
//   w_lo = 2 pi / 40.96, w_hi = 0.9 pi / 0.01;
// features log(P_j + 1e-8) (j < 64) and log(s2); zeros if n < 2 or s2 = 0.
// One warp per series; lane l owns bins l and l + 32 (8 sub-frequencies).
// On the regular grid the phase factor advances by a constant rotation per
// step (FP32 complex multiply) and is re-anchored from the FP64 phase
// w dbar k (reduced mod 2 pi) every 128 steps.  The sums run in FP32.
// ---------------------------------------------------------------------------
constexpr int NFEAT = 65;
constexpr int NFREQ = 64;

__device__ __forceinline__ double feat_freq(int j, int q) {
  const double wlo = 6.283185307179586477 / 40.96, whi = 0.9 * 3.141592653589793238 / 0.01;
  const double e = (double)j + ((double)q - 1.5) * 0.25;
  return wlo * exp(log(whi / wlo) * e / (double)(NFREQ - 1));
}

__global__ void __launch_bounds__(128) k_features(const int64_t* offsets, int B, const double* t, const double* y,
                                                  float* feat) {
  const int s = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= B) return;                      // whole warp
  const int64_t a = offsets[s], n = offsets[s + 1] - a;
  float* out = feat + (int64_t)s * NFEAT;
  double sy = 0.0;
  for (int64_t k = lane; k < n; k += 32) sy += y[a + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sy += __shfl_xor_sync(0xffffffffu, sy, o);
  const double ybar = n > 0 ? sy / (double)n : 0.0;
  double sv = 0.0;
  for (int64_t k = lane; k < n; k += 32) { const double d = y[a + k] - ybar; sv = fma(d, d, sv); }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
  const double s2 = n > 0 ? sv / (double)n : 0.0;
  if (n < 2 || !(s2 > 0.0)) {
    out[lane] = 0.0f;
    out[lane + 32] = 0.0f;
    if (lane == 0) out[NFREQ] = 0.0f;
    return;
  }
  const double dbar = (t[a + n - 1] - t[a]) / (double)(n - 1);
  const double inv2pi = 0.15915494309189533577, twopi = 6.283185307179586477;
  double wd[8];            // radians per step of sub-frequency (bin lane + 32 (f / 4), sub f % 4)
  float rr[8], ri[8], zr[8], zi[8], sr[8], si[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    wd[f] = feat_freq(lane + 32 * (f >> 2), f & 3) * dbar;
    double sn, cs;
    sincos(wd[f], &sn, &cs);
    rr[f] = (float)cs; ri[f] = (float)-sn;      // exp(-i wd)
    zr[f] = 1.f; zi[f] = 0.f; sr[f] = 0.f; si[f] = 0.f;
  }
  // each lane converts one value per 32 steps; the warp reads them back by
  // shuffles (the FP64 work is one subtraction and one conversion per step)
#pragma unroll 1
  for (int64_t k0 = 0; k0 < n; k0 += 32) {
    const float ycl = (k0 + lane < n) ? (float)(y[a + k0 + lane] - ybar) : 0.f;
    if ((k0 & 127) == 0 && k0 > 0) {           // re-anchor from the FP64 phase
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        double p = wd[f] * (double)k0;
        p = fma(-twopi, rint(p * inv2pi), p);
        float sn, cs;
        sincosf((float)p, &sn, &cs);
        zr[f] = cs; zi[f] = -sn;
      }
    }
    const int cnt = (int)min((int64_t)32, n - k0);
#pragma unroll 1
    for (int j = 0; j < cnt; ++j) {
      const float yc = __shfl_sync(0xffffffffu, ycl, j);
#pragma unroll
      for (int f = 0; f < 8; ++f) {
        sr[f] = fmaf(yc, zr[f], sr[f]);
        si[f] = fmaf(yc, zi[f], si[f]);
        const float r2 = zr[f] * rr[f] - zi[f] * ri[f];
        const float i2 = zr[f] * ri[f] + zi[f] * rr[f];
        zr[f] = r2; zi[f] = i2;
      }
    }
  }
  const double den = 4.0 * (double)n * s2;
  double p0 = 0.0, p1 = 0.0;
#pragma unroll
  for (int f = 0; f < 4; ++f) p0 += (double)sr[f] * sr[f] + (double)si[f] * si[f];
#pragma unroll
  for (int f = 4; f < 8; ++f) p1 += (double)sr[f] * sr[f] + (double)si[f] * si[f];
  out[lane] = (float)log(p0 / den + 1e-8);
  out[lane + 32] = (float)log(p1 / den + 1e-8);
  if (lane == 0) out[NFREQ] = (float)log(s2);
}

// ---------------------------------------------------------------------------
// BF16 GEMM with FP32 accumulation on the tensor cores:
//   C[M x N] = A[M x K] B[N x K]^T,  A and B row-major with K contiguous,
// K a multiple of 8 (16-byte rows).  Block tile 64 x 64, four warps of 32 x 32,
// K steps of 32 staged in shared memory; each warp issues
// mma.sync.m16n8k16.row.col.f32.bf16.bf16.f32 on fragments read from shared
// memory in the PTX ISA's fragment layout (group g = lane / 4, t = lane % 4:
// A rows g, g + 8 and columns 2t, 2t + 1, 2t + 8, 2t + 9; B column g and rows
// 2t, 2t + 1, 2t + 8, 2t + 9; C rows g, g + 8 and columns 2t, 2t + 1).
// Partial tiles are zero-filled; the epilogue gets (row, col, value) of every
// in-range element.
// ---------------------------------------------------------------------------
constexpr int GT = 64;          // block tile (M and N)
constexpr int GK = 32;          // K step
constexpr int GKP = GK + 8;     // padded shared-memory row (bf16 elements)

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

template <class Epi>
__global__ void __launch_bounds__(128) k_gemm_bf16(const __nv_bfloat16* A, const __nv_bfloat16* Bm, int M, int N,
                                                   int K, Epi epi) {
  __shared__ __align__(16) __nv_bfloat16 As[GT][GKP];
  __shared__ __align__(16) __nv_bfloat16 Bs[GT][GKP];
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GK) {
    // 64 rows x 4 vectors of 8 bf16 per operand: 2 vectors per thread each
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int v = threadIdx.x + r * 128;
      const int row = v >> 2, kk = (v & 3) * 8;
      uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
      if (m0 + row < M && k0 + kk < K) a = *reinterpret_cast<const uint4*>(A + (int64_t)(m0 + row) * K + k0 + kk);
      if (n0 + row < N && k0 + kk < K) b = *reinterpret_cast<const uint4*>(Bm + (int64_t)(n0 + row) * K + k0 + kk);
      *reinterpret_cast<uint4*>(&As[row][kk]) = a;
      *reinterpret_cast<uint4*>(&Bs[row][kk]) = b;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GK; ks += 16) {
      uint32_t af[2][4], bfr[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r0 = wm + 16 * i + g;
        af[i][0] = ld_pair(&As[r0][ks + 2 * tq]);
        af[i][1] = ld_pair(&As[r0 + 8][ks + 2 * tq]);
        af[i][2] = ld_pair(&As[r0][ks + 8 + 2 * tq]);
        af[i][3] = ld_pair(&As[r0 + 8][ks + 8 + 2 * tq]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c0 = wn + 8 * j + g;
        bfr[j][0] = ld_pair(&Bs[c0][ks + 2 * tq]);
        bfr[j][1] = ld_pair(&Bs[c0][ks + 8 + 2 * tq]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]), "r"(bfr[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int row = m0 + wm + 16 * i + g + ((c & 2) ? 8 : 0);
        const int col = n0 + wn + 8 * j + 2 * tq + (c & 1);
        if (row < M && col < N) epi(row, col, acc[i][j][c]);
      }
}

// epilogues
struct EpiF32 {          // plain FP32 store, leading dimension ld
  float* C; int ld;
  __device__ void operator()(int r, int c, float v) const { C[(int64_t)r * ld + c] = v; }
};
struct EpiBiasF32 {      // + bias, FP32 store
  float* C; int ld; const float* b;
  __device__ void operator()(int r, int c, float v) const { C[(int64_t)r * ld + c] = v + b[c]; }
};
struct EpiBiasReLU {     // relu(v + b) to bf16, row-major [M][N] and transposed [N][M]
  __nv_bfloat16* H; __nv_bfloat16* HT; int N, M; const float* b;
  __device__ void operator()(int r, int c, float v) const {
    const __nv_bfloat16 h = __float2bfloat16_rn(fmaxf(v + b[c], 0.f));
    H[(int64_t)r * N + c] = h;
    HT[(int64_t)c * M + r] = h;
  }
};
struct EpiReLUMask {     // v where the forward activation is positive, else 0;
  __nv_bfloat16* D; __nv_bfloat16* DT; int N, M; const __nv_bfloat16* Hf;  // to bf16, both layouts
  __device__ void operator()(int r, int c, float v) const {
    const float h = __bfloat162float(Hf[(int64_t)r * N + c]);
    const __nv_bfloat16 d = __float2bfloat16_rn(h > 0.f ? v : 0.f);
    D[(int64_t)r * N + c] = d;
    DT[(int64_t)c * M + r] = d;
  }
};

// ---------------------------------------------------------------------------
// The network: 65 -> 256 -> 256 -> 3 (ReLU), inputs and outputs standardised.
// State (one caller-owned device buffer, FP32 then BF16):
//   norm[144]: feature mean[65], sd[65], target mean[3], sd[3] (+ padding)
//   P[NP], Madam[NP], Vadam[NP]: FP32 parameters W1[256][80] (columns >= 65
//     zero), b1[256], W2[256][256], b2[256], W3[16][256] (rows >= 3 zero),
//     b3[16], and Adam's moments in the same layout
//   BF16 copies for the GEMMs: W1h[256][80], W2h[256][256], W2T = W2^T,
//     W3h[16][256], W3T = W3^T[256][16]
// ---------------------------------------------------------------------------
constexpr int HID = 256;
constexpr int KIN = 80;                 // 65 inputs padded to a multiple of 16
constexpr int NOUT = 16;                // 3 outputs padded
constexpr int OW1 = 0, OB1 = OW1 + HID * KIN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + NOUT * HID, NP = OB3 + NOUT;
constexpr int NNORM = 144;
constexpr int64_t SB_P = NNORM * 4, SB_M = SB_P + (int64_t)NP * 4, SB_V = SB_M + (int64_t)NP * 4,
                  SB_H = (SB_V + (int64_t)NP * 4 + 255) / 256 * 256;
constexpr int64_t HB_W1 = 0, HB_W2 = HB_W1 + HID * KIN, HB_W2T = HB_W2 + HID * HID, HB_W3 = HB_W2T + HID * HID,
                  HB_W3T = HB_W3 + NOUT * HID, HB_END = HB_W3T + HID * NOUT;
constexpr int64_t STATE_BYTES = SB_H + HB_END * 2;

struct Net {
  float* norm;
  float* P;
  float* Ma;
  float* Va;
  __nv_bfloat16 *W1h, *W2h, *W2T, *W3h, *W3T;
};
Net net_of(void* state) {
  char* b = static_cast<char*>(state);
  Net n;
  n.norm = reinterpret_cast<float*>(b);
  n.P = reinterpret_cast<float*>(b + SB_P);
  n.Ma = reinterpret_cast<float*>(b + SB_M);
  n.Va = reinterpret_cast<float*>(b + SB_V);
  __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(b + SB_H);
  n.W1h = h + HB_W1; n.W2h = h + HB_W2; n.W2T = h + HB_W2T; n.W3h = h + HB_W3; n.W3T = h + HB_W3T;
  return n;
}

// activations of a minibatch of M rows
struct Acts {
  __nv_bfloat16 *X, *XT, *H1, *H1T, *H2, *H2T, *dOh, *dOT, *dZ2, *dZ2T, *dZ1, *dZ1T;
  float *Out, *dOut, *lossp;
  int* err;                // set by a tensor-core GEMM whose waits timed out
  int64_t bytes;
};
Acts acts_of(void* ws, int64_t M) {
  Acts a;
  int64_t o = 0;
  char* b = static_cast<char*>(ws);
  auto bf = [&](int64_t n) { __nv_bfloat16* p = reinterpret_cast<__nv_bfloat16*>(b + o); o += (n * 2 + 255) / 256 * 256; return p; };
  auto fl = [&](int64_t n) { float* p = reinterpret_cast<float*>(b + o); o += (n * 4 + 255) / 256 * 256; return p; };
  a.X = bf(M * KIN); a.XT = bf(M * KIN);
  a.H1 = bf(M * HID); a.H1T = bf(M * HID); a.H2 = bf(M * HID); a.H2T = bf(M * HID);
  a.dOh = bf(M * NOUT); a.dOT = bf(M * NOUT);
  a.dZ2 = bf(M * HID); a.dZ2T = bf(M * HID); a.dZ1 = bf(M * HID); a.dZ1T = bf(M * HID);
  a.Out = fl(M * NOUT); a.dOut = fl(M * NOUT); a.lossp = fl(M);
  a.err = reinterpret_cast<int*>(fl(64));
  a.bytes = o;
  return a;
}

// standardised inputs to bf16, both layouts (columns >= 65 zero)
__global__ void k_mlp_input(const float* feat, int64_t M, const float* norm, __nv_bfloat16* X, __nv_bfloat16* XT) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * KIN) return;
  const int64_t r = i / KIN;
  const int c = (int)(i % KIN);
  float v = 0.f;
  if (c < NFEAT) v = (feat[r * NFEAT + c] - norm[c]) / norm[NFEAT + c];
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  X[i] = h;
  XT[(int64_t)c * M + r] = h;
}

// loss 1/(2M) sum (out - target_std)^2 over the 3 outputs; dOut = (out - t)/M
__global__ void k_mlp_loss(const float* Out, const double* theta, int64_t M, const float* norm, float* dOut,
                           __nv_bfloat16* dOh, __nv_bfloat16* dOT, float* lossp) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  float l = 0.f;
#pragma unroll
  for (int o = 0; o < NOUT; ++o) {
    float d = 0.f;
    if (o < 3) {
      const float tn = (float)((theta[r * 3 + o] - (double)norm[2 * NFEAT + o]) / (double)norm[2 * NFEAT + 3 + o]);
      const float e = Out[r * NOUT + o] - tn;
      l = fmaf(e, e, l);
      d = e / (float)M;
    }
    dOut[r * NOUT + o] = d;
    const __nv_bfloat16 h = __float2bfloat16_rn(d);
    dOh[r * NOUT + o] = h;
    dOT[(int64_t)o * M + r] = h;
  }
  lossp[r] = 0.5f * l / (float)M;
}

// column sums (fixed order per column): out[c] = sum_r X[r][c]
__device__ __forceinline__ float as_float(float v) { return v; }
__device__ __forceinline__ float as_float(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class T>
__global__ void k_colsum(const T* X, int64_t M, int N, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  float s = 0.f;
  for (int64_t r = 0; r < M; ++r) s += as_float(X[r * N + c]);
  out[c] = s;
}

// fixed-order sum of n floats by one block into out[0]
__global__ void k_sum1(const float* v, int64_t n, float* out) {
  __shared__ float sm[256];
  float s = 0.f;
  for (int64_t i = threadIdx.x; i < n; i += 256) s += v[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sm[0];
}

// bf16 copies of the weights (row-major and transposed)
__global__ void k_mlp_refresh(Net n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < HID * KIN) n.W1h[i] = __float2bfloat16_rn(n.P[OW1 + i]);
  if (i < HID * HID) {
    const int r = i / HID, c = i % HID;
    const __nv_bfloat16 h = __float2bfloat16_rn(n.P[OW2 + i]);
    n.W2h[i] = h;
    n.W2T[c * HID + r] = h;
  }
  if (i < NOUT * HID) {
    const int r = i / HID, c = i % HID;
    const __nv_bfloat16 h = __float2bfloat16_rn(n.P[OW3 + i]);
    n.W3h[i] = h;
    n.W3T[c * NOUT + r] = h;
  }
}

// Adam on the FP32 parameters (descent on the loss)
__global__ void k_mlp_adam(float* P, const float* G, float* Ma, float* Va, float lr, float b1t, float b2t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  const float g = G[i];
  const float m = 0.9f * Ma[i] + 0.1f * g;
  const float v = 0.999f * Va[i] + 0.001f * g * g;
  Ma[i] = m;
  Va[i] = v;
  P[i] -= lr * (m / b1t) / (sqrtf(v / b2t) + 1e-8f);
}

// He-uniform initialisation from the counter-based generator: parameter i
// uses call (i, 0x6d6c7000, 0, 0) of Philox4x32-10 with the given seed;
// W ~ U(-sqrt(6 / fan_in), sqrt(6 / fan_in)), biases and padding 0
__global__ void k_mlp_init(float* P, float* Ma, float* Va, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NP) return;
  const U4 w = philox(U4{(uint32_t)i, 0x6d6c7000u, 0u, 0u}, (uint32_t)seed, (uint32_t)(seed >> 32));
  const float u = (float)(2.0 * u53(w.x, w.y) - 1.0);
  float v = 0.f;
  if (i < OB1) { const int c = (i - OW1) % KIN; if (c < NFEAT) v = u * sqrtf(6.f / NFEAT); }
  else if (i >= OW2 && i < OB2) v = u * sqrtf(6.f / HID);
  else if (i >= OW3 && i < OB3) { const int r = (i - OW3) / HID; if (r < 3) v = u * sqrtf(6.f / HID); }
  P[i] = v;
  Ma[i] = 0.f;
  Va[i] = 0.f;
}

// column mean and standard deviation (FP64 sums, one block per column, fixed
// order); the standard deviation is floored at 1e-6
template <class T>
__global__ void k_colstats(const T* X, int64_t M, int ld, float* mean, float* sd) {
  __shared__ double s1[256], s2[256];
  const int c = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int64_t r = threadIdx.x; r < M; r += 256) { const double v = (double)X[r * ld + c]; a += v; b = fma(v, v, b); }
  s1[threadIdx.x] = a; s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) { s1[threadIdx.x] += s1[threadIdx.x + w]; s2[threadIdx.x] += s2[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mu = s1[0] / (double)M;
    const double var = fmax(s2[0] / (double)M - mu * mu, 0.0);
    mean[c] = (float)mu;
    sd[c] = (float)fmax(sqrt(var), 1e-6);
  }
}

// network outputs to log hyperparameters; a row with a non-finite feature
// (the ReLU, fmaxf, would hide it), a non-finite output or one more than 4
// standard deviations of the training targets from their mean falls back to
// the plain default 0 (l = s2 = R = 1) in all three
__global__ void k_mlp_decode(const float* Out, const float* feat, int64_t M, const float* norm, double* theta) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= M) return;
  double th[3];
  bool ok = true;
  for (int c = 0; c < NFEAT; ++c) ok = ok && isfinite(feat[r * NFEAT + c]);
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    const float z = Out[r * NOUT + o];
    ok = ok && isfinite(z) && fabsf(z) <= 4.0f;
    th[o] = (double)z * (double)norm[2 * NFEAT + 3 + o] + (double)norm[2 * NFEAT + o];
  }
#pragma unroll
  for (int o = 0; o < 3; ++o) theta[r * 3 + o] = ok ? th[o] : 0.0;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// tensor map of a K-contiguous bf16 matrix [rows][K]: boxes of 64 K-elements
// (one 128-byte swizzle row) by box_rows rows, zero fill outside
bool tile_map(CUtensorMap* map, const __nv_bfloat16* ptr, int rows, int K, int box_rows) {
  const EncodeTiledFn fn = encode_tiled();
  if (!fn || (reinterpret_cast<uintptr_t>(ptr) & 15) || (K * 2) % 16 != 0 || rows < 1 || K < 1) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(ptr), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 0: tcgen05 with TMA (default); 1: the mma.sync kernel (checked baseline)
int g_gemm_path = 0;

// C = A B^T through the epilogue; returns false if a tensor map cannot be made
template <class Epi>
bool gemm_path(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K, Epi e, int path, int* err,
               cudaStream_t s) {
  if (path == 1) {
    const dim3 grid((unsigned)((N + GT - 1) / GT), (unsigned)((M + GT - 1) / GT));
    k_gemm_bf16<Epi><<<grid, 128, 0, s>>>(A, B, M, N, K, e);
    return true;
  }
  CUtensorMap ma, mb;
  if (!tile_map(&ma, A, M, K, tc::BM) || !tile_map(&mb, B, N, K, tc::BN)) return false;
  cudaFuncSetAttribute(tc::k_gemm_tc<Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES);
  const dim3 grid((unsigned)((N + tc::BN - 1) / tc::BN), (unsigned)((M + tc::BM - 1) / tc::BM));
  tc::k_gemm_tc<Epi><<<grid, 128, tc::SMEM_BYTES, s>>>(ma, mb, M, N, K, e, err);
  return true;
}

thread_local bool t_gemm_ok = true;   // cleared when a tensor map could not be made

template <class Epi>
void gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, int M, int N, int K, Epi e, int* err, cudaStream_t s) {
  if (!gemm_path(A, B, M, N, K, e, g_gemm_path, err, s)) t_gemm_ok = false;
}

unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

void forward(const Net& n, const Acts& a, const float* feat, int M, cudaStream_t s) {
  k_mlp_input<<<blocks((int64_t)M * KIN, 256), 256, 0, s>>>(feat, M, n.norm, a.X, a.XT);
  gemm(a.X, n.W1h, M, HID, KIN, EpiBiasReLU{a.H1, a.H1T, HID, M, n.P + OB1}, a.err, s);
  gemm(a.H1, n.W2h, M, HID, HID, EpiBiasReLU{a.H2, a.H2T, HID, M, n.P + OB2}, a.err, s);
  gemm(a.H2, n.W3h, M, NOUT, HID, EpiBiasF32{a.Out, NOUT, n.P + OB3}, a.err, s);
}

void backward(const Net& n, const Acts& a, const double* theta, int M, float* G, float* loss, cudaStream_t s) {
  k_mlp_loss<<<blocks(M, 256), 256, 0, s>>>(a.Out, theta, M, n.norm, a.dOut, a.dOh, a.dOT, a.lossp);
  if (loss) k_sum1<<<1, 256, 0, s>>>(a.lossp, M, loss);
  gemm(a.dOT, a.H2T, NOUT, HID, M, EpiF32{G + OW3, HID}, a.err, s);                       // dW3 = dOut^T H2
  k_colsum<float><<<1, NOUT, 0, s>>>(a.dOut, M, NOUT, G + OB3);
  gemm(a.dOh, n.W3T, M, HID, NOUT, EpiReLUMask{a.dZ2, a.dZ2T, HID, M, a.H2}, a.err, s);    // dZ2 = dOut W3 .* [H2 > 0]
  gemm(a.dZ2T, a.H1T, HID, HID, M, EpiF32{G + OW2, HID}, a.err, s);                        // dW2 = dZ2^T H1
  k_colsum<__nv_bfloat16><<<1, HID, 0, s>>>(a.dZ2, M, HID, G + OB2);
  gemm(a.dZ2, n.W2T, M, HID, HID, EpiReLUMask{a.dZ1, a.dZ1T, HID, M, a.H1}, a.err, s);     // dZ1 = dZ2 W2 .* [H1 > 0]
  gemm(a.dZ1T, a.XT, HID, KIN, M, EpiF32{G + OW1, KIN}, a.err, s);                         // dW1 = dZ1^T X
  k_colsum<__nv_bfloat16><<<1, HID, 0, s>>>(a.dZ1, M, HID, G + OB1);
}

int rc_of(cudaError_t e) { return e == cudaSuccess ? PSSGP_OK : PSSGP_ECUDA; }

}  // namespace

extern "C" int pssgp_simulate_prior(const pssgp_model* model, const int64_t* offsets, int32_t B,
                                    const double* params, uint64_t seed, double spacing, double* t, double* y,
                                    int32_t* status, void* stream) {
  if (!model_ok(model) || !offsets || !params || !t || !y || !status || B < 1 || !(spacing > 0.0))
    return PSSGP_EINVAL;
  const double ell0 = model->lengthscale, var0 = model->variance;
  if (!(ell0 > 0.0) || !(var0 > 0.0) || !std::isfinite(ell0) || !std::isfinite(var0)) return PSSGP_EMODEL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) return PSSGP_ECUDA;
  const unsigned g = blocks(B, 128);
  switch (model->d) {
#define PSSGP_SIM(DD) case DD: k_simulate_prior<DD><<<g, 128, 0, s>>>(dev_model<DD>(model), ell0, var0, offsets, B, \
                                 params, (unsigned long long)seed, spacing, t, y, status); break;
    PSSGP_SIM(1) PSSGP_SIM(2) PSSGP_SIM(3) PSSGP_SIM(4) PSSGP_SIM(5) PSSGP_SIM(6) PSSGP_SIM(7) PSSGP_SIM(8)
#undef PSSGP_SIM
    default: return PSSGP_EDIM;
  }
  return rc_of(cudaGetLastError());
}

extern "C" int pssgp_features(const int64_t* offsets, int32_t B, const double* t, const double* y, float* feat,
                              void* stream) {
  if (!offsets || !t || !y || !feat || B < 1) return PSSGP_EINVAL;
  (void)cudaGetLastError();
  k_features<<<blocks((int64_t)B * 32, 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(offsets, B, t, y, feat);
  return rc_of(cudaGetLastError());
}

extern "C" size_t pssgp_mlp_state_bytes(void) { return (size_t)STATE_BYTES; }
extern "C" int32_t pssgp_mlp_param_count(void) { return NP; }

extern "C" size_t pssgp_mlp_workspace_size(int32_t rows) {
  if (rows < 1) return 0;
  return (size_t)acts_of(nullptr, rows).bytes;
}

extern "C" int pssgp_mlp_init(void* state, uint64_t seed, const float* feat, int64_t nrows, const double* theta,
                              void* stream) {
  if (!state || !feat || !theta || nrows < 2) return PSSGP_EINVAL;
  if ((reinterpret_cast<uintptr_t>(state) & 255) != 0) return PSSGP_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();
  Net n = net_of(state);
  if (cudaMemsetAsync(n.norm, 0, NNORM * 4, s) != cudaSuccess) return PSSGP_ECUDA;
  k_colstats<float><<<NFEAT, 256, 0, s>>>(feat, nrows, NFEAT, n.norm, n.norm + NFEAT);
  k_colstats<double><<<3, 256, 0, s>>>(theta, nrows, 3, n.norm + 2 * NFEAT, n.norm + 2 * NFEAT + 3);
  k_mlp_init<<<blocks(NP, 256), 256, 0, s>>>(n.P, n.Ma, n.Va, (unsigned long long)seed);
  k_mlp_refresh<<<blocks(HID * HID, 256), 256, 0, s>>>(n);
  return rc_of(cudaGetLastError());
}

extern "C" int pssgp_mlp_set_params(void* state, const float* params, const float* norm, void* stream) {
  if (!state || !params || !norm) return PSSGP_EINVAL;
  if ((reinterpret_cast<uintptr_t>(state) & 255) != 0) return PSSGP_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();
  Net n = net_of(state);
  if (cudaMemcpyAsync(n.norm, norm, NNORM * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(n.P, params, (size_t)NP * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(n.Ma, 0, (size_t)NP * 4, s) != cudaSuccess ||
      cudaMemsetAsync(n.Va, 0, (size_t)NP * 4, s) != cudaSuccess)
    return PSSGP_ECUDA;
  k_mlp_refresh<<<blocks(HID * HID, 256), 256, 0, s>>>(n);
  return rc_of(cudaGetLastError());
}

extern "C" int pssgp_mlp_grad(void* state, const float* feat, const double* theta, int32_t rows, float* grad,
                              float* loss, float* out, void* ws, size_t ws_bytes, void* stream) {
  if (!state || !feat || !theta || !grad || !ws || rows < 1 || rows % 8 != 0) return PSSGP_EINVAL;
  const Acts a = acts_of(ws, rows);
  if ((int64_t)ws_bytes < a.bytes || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return PSSGP_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();
  const Net n = net_of(state);
  t_gemm_ok = true;
  if (cudaMemsetAsync(a.err, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  forward(n, a, feat, rows, s);
  backward(n, a, theta, rows, grad, loss, s);
  if (!t_gemm_ok) return PSSGP_ECUDA;
  if (out && cudaMemcpyAsync(out, a.Out, (size_t)rows * NOUT * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return PSSGP_ECUDA;
  return rc_of(cudaGetLastError());
}

extern "C" int pssgp_mlp_adam(void* state, const float* grad, float lr, int32_t step, void* stream) {
  if (!state || !grad || step < 1 || !(lr > 0.f)) return PSSGP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();
  Net n = net_of(state);
  const float b1t = 1.f - powf(0.9f, (float)step), b2t = 1.f - powf(0.999f, (float)step);
  k_mlp_adam<<<blocks(NP, 256), 256, 0, s>>>(n.P, grad, n.Ma, n.Va, lr, b1t, b2t);
  k_mlp_refresh<<<blocks(HID * HID, 256), 256, 0, s>>>(n);
  return rc_of(cudaGetLastError());
}

extern "C" int pssgp_mlp_predict(const void* state, const float* feat, int32_t rows, double* theta, void* ws,
                                 size_t ws_bytes, void* stream) {
  if (!state || !feat || !theta || !ws || rows < 1) return PSSGP_EINVAL;
  const Acts a = acts_of(ws, rows);
  if ((int64_t)ws_bytes < a.bytes || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return PSSGP_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();
  const Net n = net_of(const_cast<void*>(state));
  t_gemm_ok = true;
  if (cudaMemsetAsync(a.err, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  forward(n, a, feat, rows, s);
  if (!t_gemm_ok) return PSSGP_ECUDA;
  k_mlp_decode<<<blocks(rows, 256), 256, 0, s>>>(a.Out, feat, rows, n.norm, theta);
  return rc_of(cudaGetLastError());
}

extern "C" int pssgp_mlp_set_gemm(int32_t path) {
  if (path != 0 && path != 1) return PSSGP_EINVAL;
  g_gemm_path = path;
  return PSSGP_OK;
}

extern "C" int pssgp_debug_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N, int32_t K, float* C,
                                     int32_t path, int32_t* err, void* stream) {
  if (!A || !B || !C || !err || M < 1 || N < 1 || K < 1 || (path != 0 && path != 1)) return PSSGP_EINVAL;
  if (K % 8 != 0) return PSSGP_EINVAL;   // 16-byte rows
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  (void)cudaGetLastError();
  if (cudaMemsetAsync(err, 0, sizeof(int32_t), s) != cudaSuccess) return PSSGP_ECUDA;
  if (!gemm_path(static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B), M, N, K,
                 EpiF32{C, N}, path, err, s))
    return PSSGP_ECUDA;
  return rc_of(cudaGetLastError());
}
