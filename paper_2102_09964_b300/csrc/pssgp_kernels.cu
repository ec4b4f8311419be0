// pssgp_kernels.cu -- CUDA kernels and C ABI of libpssgp (sm_103a, FP64).
//
// Parallel state-space GP of Corenflos, Zhao, Sarkka, "Temporal Gaussian
// Process Regression in Logarithmic Time": merge (Sec. 4.3), discretisation
// (supplement Eq. (ss-gp-formation)), parallel Kalman filter with missing
// measurements (Sec. 3, Prop. 1), log-likelihood (Sec. 2), parallel RTS
// smoother (supplement, Prop. 2).
//
// Scan organisation (both directions): the n time steps are cut into P0
// contiguous chunks, one per thread ("lane"), P0 = 32 x (warps).  On B300 the
// FP64 pipe retires one warp instruction per 64 cycles per sub-partition
// whatever the number of active lanes, so one warp per sub-partition already
// saturates it and every lane must carry useful work.
//   level 0  each lane folds the elements of its chunk into the chunk's
//            aggregate (the operator applied element by element);
//   level 1  Kogge-Stone scan of the 32 lane aggregates of a warp (shuffles);
//   level 2  Kogge-Stone scan of the warp aggregates, one launch per round;
//   level 3  each lane combines its exclusive prefix with its chunk start and
//            runs the sequential recursion through the chunk (Props. 1 and 2:
//            folding the operator from a known prefix is the Kalman filter /
//            RTS smoother), writing per-step results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/pssgp.h"
#include "adjoint_ops.cuh"
#include "host_model.cuh"
#include "scan_ops.cuh"
#include "warp_ops.cuh"

using namespace pssgp;

namespace {

constexpr int BLOCK = 128;           // 4 warps: one per SM sub-partition
// lanes per SM / 32, per state dimension (pssgp_set_warps_per_sm, pssgp_tune_set)
constexpr int WARPS_MAX = 16;
// default: 8 for d <= 3 (short per-step work, more warps hide its latency;
// measured 8-12 % faster than 4 at 2^20 steps), 4 above (255 registers)
int g_warps_per_sm[PSSGP_DMAX + 1] = {8, 8, 8, 8, 4, 4, 4, 4, 4};
constexpr int MIN_CHUNK = 8;         // steps per lane below which fewer lanes are used

// ---------------------------------------------------------------------------
// plan and workspace
// ---------------------------------------------------------------------------
int g_num_sms = 0;
std::mutex g_mu;

int num_sms() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_num_sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      g_num_sms = v;
    else
      g_num_sms = 148;
  }
  return g_num_sms;
}

// Optional per-kernel timing (diagnostic): CUDA events recorded on the
// launching stream around every launch, summed per kernel name.
constexpr int TIMING_SLOTS = 16;
const char* const kTimingNames[TIMING_SLOTS] = {
    "merge", "filter_reduce", "filter_level2", "filter_propagate", "smoother_level2", "smoother_propagate",
    "smoother_elements", "gather", "loglik_reduce", "discretize", "adjoint_level2", "adjoint_mean",
    "adjoint_cov", "loglik_chunks", "", ""};
enum { T_MERGE = 0, T_FRED, T_FL2, T_FPROP, T_SL2, T_SPROP, T_SELEM, T_GATHER, T_LL, T_DISC, T_AL2, T_AMEAN,
       T_ACOV, T_LLC };
bool g_timing = false;
struct TimingRec { cudaEvent_t a, b; int slot; };
std::vector<TimingRec> g_pending;
double g_ms[TIMING_SLOTS] = {0};
long long g_count[TIMING_SLOTS] = {0};

struct Timed {
  cudaStream_t s;
  int slot;
  cudaEvent_t a = nullptr, b = nullptr;
  Timed(cudaStream_t s_, int slot_) : s(s_), slot(slot_) {
    if (g_timing) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, s);
    }
  }
  ~Timed() {
    if (g_timing) {
      cudaEventRecord(b, s);
      std::lock_guard<std::mutex> lk(g_mu);
      g_pending.push_back({a, b, slot});
    }
  }
};

// first CUDA error seen since the start of the current entry-point call (host
// thread): every launch is followed by after_launch(), so an error cannot be
// masked by later runtime calls
thread_local cudaError_t t_first_err = cudaSuccess;
inline void begin_call() { t_first_err = cudaSuccess; (void)cudaGetLastError(); }
inline void after_launch() {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess && t_first_err == cudaSuccess) t_first_err = e;
}
inline int end_call() {
  after_launch();
  return t_first_err == cudaSuccess ? PSSGP_OK : PSSGP_ECUDA;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
int64_t align256(int64_t b) { return round_up(b, 256); }

struct Plan {
  int d;
  int64_t n;
  int64_t P0;        // lanes (multiple of BLOCK)
  int64_t P2;        // warps
  int64_t L;         // steps per lane
  int warps;         // the tuning the plan was made for (lanes per SM / 32)
  int nf, ns;        // aggregate sizes (doubles)
  int fnext;         // split series: offset (doubles) of the F/Q record after the chunk in the o_bnd slot
  int fqs, egs;      // per-step record strides (doubles, even)
  // byte offsets into the workspace
  int64_t o_status, o_fq, o_egl, o_laggf, o_waggf, o_laggs, o_waggs, o_llp, o_fmean, o_fvar, o_t, o_y, o_mask,
      o_tpos, o_rstep, o_seg, o_llstep, o_adj, o_tauq, o_lpi, o_lmbar, o_lgj, o_gpart, o_gstep, o_bnd, total;
};

int warps_for(int d) {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_warps_per_sm[d];
}

// warps: lanes per SM / 32 (0: the current tuning for d)
Plan make_plan(int d, int64_t n, int64_t lanes_req, int warps = 0, bool grad = false) {
  Plan p{};
  p.d = d;
  p.n = n;
  p.warps = warps > 0 ? warps : warps_for(d);
  const int64_t lanes_max = (int64_t)num_sms() * p.warps * 32;
  const int64_t want = (n + MIN_CHUNK - 1) / MIN_CHUNK;
  int64_t P0 = std::min(lanes_max, std::max<int64_t>(want, 1));
  if (lanes_req > 0) P0 = lanes_req;
  P0 = round_up(P0, BLOCK);
  p.P0 = P0;
  p.P2 = P0 / 32;
  p.L = (n + P0 - 1) / P0;
  const int sym = d * (d + 1) / 2;
  p.nf = d * d + 2 * d + 2 * sym;
  p.ns = d * d + d + sym;
  p.fqs = (int)round_up(d * d + sym, 2);
  p.egs = (int)round_up(d * d + d + 2 * sym, 2);
  int64_t o = 0;
  p.o_status = o; o += 256;
  p.o_fq = o; o += align256(n * p.fqs * 8);
  p.o_egl = o; o += align256(n * p.egs * 8);
  p.o_laggf = o; o += align256(P0 * p.nf * 8);
  p.o_waggf = o; o += align256(2 * p.P2 * p.nf * 8);
  p.o_laggs = o; o += align256(P0 * p.ns * 8);
  p.o_waggs = o; o += align256(2 * p.P2 * p.ns * 8);
  p.o_llp = o; o += align256(P0 * 8);
  p.o_fmean = o; o += align256(n * 8);
  p.o_fvar = o; o += align256(n * 8);
  p.o_t = o; o += align256(n * 8);
  p.o_y = o; o += align256(n * 8);
  p.o_mask = o; o += align256(n);
  p.o_tpos = o; o += align256(n * 8);
  p.o_rstep = o; o += align256(n * 8);     // batched: noise variance per step
  p.o_seg = o; o += align256(n);           // batched: 1 at each series' first step
  p.o_llstep = o; o += align256(n * 8);    // batched: log-likelihood pieces per step
  p.fnext = (p.nf + 1) / 2 * 2;                       // the record after the aggregate, 16-byte aligned
  p.o_bnd = o; o += align256((p.fnext + p.fqs) * 8);  // split series: the folded aggregate of the other
                                                    // chunks, then the F/Q record of the step after the chunk
  p.o_adj = p.o_tauq = p.o_lpi = p.o_lmbar = p.o_lgj = p.o_gpart = p.o_gstep = -1;
  if (grad) {                                // gradient: forward moments, scan state
    const int adjs = (d + sym + 2 + 1) / 2 * 2;
    p.o_adj = o; o += align256(n * adjs * 8);
    p.o_tauq = o; o += align256(n * 16);       // (tau, q) per step
    p.o_lpi = o; o += align256(P0 * d * d * 8);
    p.o_lmbar = o; o += align256(P0 * d * 8);
    p.o_lgj = o; o += align256(P0 * (d + sym) * 8);
    p.o_gpart = o; o += align256(3 * P0 * 8);
    p.o_gstep = o; o += align256(3 * n * 8);
  }
  p.total = o;
  return p;
}

// ---------------------------------------------------------------------------
// kernel arguments
// ---------------------------------------------------------------------------
struct ScanArgs {
  const double* t;
  const double* y;
  const uint8_t* mask;
  const double* R;       // noise variance(s) on the device, or null
  double R_scalar;       // used when R is null
  int R_per_step;
  int64_t n, L, P0, P2;
  double* rec_fq;        // per step: F (d*d), Q packed
  double* rec_egl;       // per step: the RTS record E (d*d), g (d), P_k and P^-_{k+1} (packed)
  double* lagg_f;        // [nf][P0] level-1 inclusive lane aggregates
  double* wagg_f;        // [nf][P2] warp totals (level-2 input)
  const double* wfin_f;  // [nf][P2] level-2 inclusive results
  double* lagg_s;
  double* wagg_s;
  const double* wfin_s;
  double* llp;           // [P0] log-likelihood partial per lane
  int* status;
  double* xf;            // optional per-step filter outputs (SDE coordinates)
  double* Pf;
  double* f_mean;        // smoother outputs
  double* f_var;
  double* xs;
  double* Ps;
  int64_t ld;
  int fuse_smoother;     // 1: the filter pass also builds the smoother elements
  double* dbg_agg;       // optional: level-0 lane aggregates (tests)
  const uint8_t* seg_start;  // batched: series starts (null for one series)
  double* ll_step;           // batched: per-step log-likelihood pieces
  double* lane_ll;           // [1 + D + D(D+1)/2][P0] log-likelihood-only path: per chunk the
                             // log-likelihood of its first series piece given the state 0, eta, J
  double* lane_fp;           // [D*D + D + D(D+1)/2][P0] fused smoother: (A, eta, J) of the filter
                             // aggregate of the lane's steps but the last (all of them in the last lane)
  // gradient (adjoint) mode
  int adj;                   // 1: the filter pass stores rec_adj and folds the mean-adjoint aggregate
  double* rec_adj;           // [n][adjs] predicted moments, v, 1/S
  double* tauq;              // [n][2] scaled step tau and variance ratio q
  double* lane_pi;           // [D*D][P0] raw chunk product of the mean-adjoint factors
  double* lane_mbar;         // [D][P0] mean adjoint at the chunk end
  double* lane_gj;           // [D + D(D+1)/2][P0] gamma and N^{-1} J of the mean-adjoint chunk aggregate
  double* gpart;             // [3][P0] gradient partials per lane
  double* g_step;            // batched: [3][n] gradient pieces per step
  double* lagg_a;            // [ns][P0] covariance-adjoint lane aggregates
  double* wagg_a;            // [2][ns][P2] and their warp aggregates
  const double* wfin_a;
  // one chunk of a longer series (split over several GPUs)
  double t_prev;             // time of the step before the chunk (NaN: the series starts at step 0)
  double t_next;             // time of the step after the chunk (NaN: the series ends at step n-1)
  const double* start_f;     // packed filter aggregate of all steps before the chunk (a filter state:
                             // it holds the series' first step, so A = 0, eta = 0, J = 0), or null
  const double* end_s;       // packed smoother aggregate of all steps after the chunk (a smoothed state:
                             // it holds the series' last step, so E = 0), or null; in the gradient's
                             // backward scans the folded adjoint aggregate of the steps after the chunk
  const double* f_next;      // gradient of a chunk of a longer series: the F/Q record of the transition
                             // into the step after the chunk (null: the series ends with the chunk)
};

__device__ __forceinline__ void flag(int* status, int bits) {
  if (bits) atomicOr(status, bits);
}

template <int D> __host__ __device__ constexpr int fqs_of() { return (D * D + Sym<D>::N + 1) / 2 * 2; }
// per-step RTS record: E (d*d), g (d), the filtered covariance P_k and the
// predicted covariance P^-_{k+1} (both packed)
template <int D> __host__ __device__ constexpr int egs_of() { return (D * D + D + 2 * Sym<D>::N + 1) / 2 * 2; }

// Ask for a per-step record of N doubles (the next step's) in L1 while the
// current step computes: a lane spends microseconds on a step at d = 6, far
// longer than a DRAM access, but its loads are issued only when the step
// starts.  One prefetch per 128-byte line, every address inside the record.
template <int N>
__device__ __forceinline__ void prefetch_record(const double* p) {
#pragma unroll
  for (int o = 0; o < N; o += 16) asm volatile("prefetch.global.L1 [%0];" ::"l"(p + o));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p + N - 1));
}

// A per-step record of N doubles (N even) by 16-byte loads: every record
// starts on a 16-byte boundary (the workspace regions are 256-byte aligned
// and the record lengths even), and half as many load instructions queue in
// the load/store unit.
template <int N>
__device__ __forceinline__ void load_record(const double* p, double (&r)[N]) {
  static_assert(N % 2 == 0, "records have an even number of doubles");
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int i = 0; i < N / 2; ++i) {
    const double2 v = q[i];
    r[2 * i] = v.x;
    r[2 * i + 1] = v.y;
  }
}

template <int D, bool VEC = true>
__device__ __forceinline__ void load_fq(const double* rec, int64_t k, Mat<D>& F, Mat<D>& Q) {
  double r[fqs_of<D>()];
  if constexpr (VEC) {
    load_record(rec + k * fqs_of<D>(), r);
  } else {
#pragma unroll
    for (int e = 0; e < fqs_of<D>(); ++e) r[e] = rec[k * fqs_of<D>() + e];
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) F[i][j] = r[i * D + j];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) { Q[i][j] = r[D * D + pidx<D>(i, j)]; Q[j][i] = Q[i][j]; }
}
template <int D>
__device__ __forceinline__ void store_fq(double* rec, int64_t k, const Mat<D>& F, const Mat<D>& Q) {
  double* p = rec + k * fqs_of<D>();
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) p[i * D + j] = F[i][j];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) p[D * D + pidx<D>(i, j)] = Q[i][j];
}
// the RTS record of step k: (E, g) of element e, P_k and P^-_{k+1}
template <int D>
__device__ __forceinline__ void store_rts(double* rec, int64_t k, const SAgg<D>& e, const Mat<D>& P,
                                          const Mat<D>& Pm) {
  double* p = rec + k * egs_of<D>();
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) p[i * D + j] = e.E[i][j];
#pragma unroll
  for (int i = 0; i < D; ++i) p[D * D + i] = e.g[i];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      p[D * D + D + pidx<D>(i, j)] = P[i][j];
      p[D * D + D + Sym<D>::N + pidx<D>(i, j)] = Pm[i][j];
    }
}
// a symmetric matrix, packed upper, in shared memory (entry e at p[e * SST])
template <int D, int SST>
__device__ __forceinline__ void store_sym_smem(double* p, const Mat<D>& M) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) p[pidx<D>(i, j) * SST] = M[i][j];
}
template <int D, int SST>
__device__ __forceinline__ void load_sym_smem(const double* p, Mat<D>& M) {
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) { M[i][j] = p[pidx<D>(i, j) * SST]; M[j][i] = M[i][j]; }
}

// The RTS record of step k written as it is formed: E and g of
// smoother_element() (W = Lu^{-1} T in place of T, V = diag(rd) W row by row,
// then E row by row with g: row j of E = Lu^{-T} applied to column j of V, so
// that at most one row of E is held), P_k (packed, read from shared memory at
// sP[e * SST]) and P^- (the prediction of step k+1).  The smoother pass uses
// P^s_k = P_k + E (P^s_{k+1} - P^-) E^T, identical to E P^s_{k+1} E^T + L with
// L = P_k - E P^- E^T, so L is not formed.
template <int D, int SST>
__device__ __forceinline__ bool smoother_element_store(double* rec, int64_t k, const Vec<D>& x, const double* sP,
                                                       Mat<D>& T, const Vec<D>& xm, const Mat<D>& Pm) {
  double* p = rec + k * egs_of<D>();
  Mat<D> Lu;
  double rd[D];
  const bool ok = ldlt<D>(Pm, Lu, rd);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = T[i][j];
#pragma unroll
      for (int q = 0; q < i; ++q) s = fma(-Lu[i][q], T[q][j], s);
      T[i][j] = s;
    }
#pragma unroll
  for (int q = 0; q < D; ++q)
#pragma unroll
    for (int j = 0; j < D; ++j) T[q][j] *= rd[q];
#pragma unroll
  for (int e = 0; e < Sym<D>::N; ++e) {
    p[D * D + D + e] = sP[e * SST];
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) p[D * D + D + Sym<D>::N + pidx<D>(i, j)] = Pm[i][j];
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double r[D];
#pragma unroll
    for (int i = D - 1; i >= 0; --i) {
      double s = T[i][j];
#pragma unroll
      for (int q = i + 1; q < D; ++q) s = fma(-Lu[q][i], r[q], s);
      r[i] = s;
    }
    double gj = x[j];
#pragma unroll
    for (int q = 0; q < D; ++q) gj = fma(-r[q], xm[q], gj);
#pragma unroll
    for (int i = 0; i < D; ++i) p[j * D + i] = r[i];
    p[D * D + j] = gj;
  }
  return ok;
}

template <int D>
__device__ __forceinline__ void load_rts(const double* rec, int64_t k, Mat<D>& E, Vec<D>& g, Mat<D>& P,
                                         Mat<D>& Pm) {
  double p[egs_of<D>()];
  load_record(rec + k * egs_of<D>(), p);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) E[i][j] = p[i * D + j];
#pragma unroll
  for (int i = 0; i < D; ++i) g[i] = p[D * D + i];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) {
      P[i][j] = p[D * D + D + pidx<D>(i, j)];
      P[j][i] = P[i][j];
      Pm[i][j] = p[D * D + D + Sym<D>::N + pidx<D>(i, j)];
      Pm[j][i] = Pm[i][j];
    }
}

// ---------------------------------------------------------------------------
// filter levels 0 + 1: discretise, fold the chunk's elements, warp scan
// ---------------------------------------------------------------------------
// discretisation into the per-step records, one thread per step; a series'
// first step (k = 0) gets F = 0, Q = P_inf, unless t_prev (the time of the
// step before a chunk of a longer series) is a number: then step 0 is the
// transition from t_prev.  Also checks the times.  The
// block's records (consecutive steps, contiguous in memory) are staged in
// shared memory and written out with consecutive threads on consecutive
// addresses.
constexpr int DISC_BLOCK = 128;
// Three blocks per SM up to d = 6 (at most 170 registers; d = 6 spills
// 24 bytes): the kernel alternates FP64 work with staging and coalesced
// stores, and the third block fills the FP64 pipe during another's stores.
template <int D>
__global__ void __launch_bounds__(DISC_BLOCK, (D <= 6 ? 3 : 1)) k_discretize_rec(const DevModel<D> m, const double* t, int64_t n,
                                                             double* rec, double* tauq, int* status,
                                                             double t_prev) {
  constexpr int FQS = fqs_of<D>();
  extern __shared__ double stage[];           // DISC_BLOCK * FQS doubles
  const int64_t k0 = (int64_t)blockIdx.x * DISC_BLOCK;
  const int64_t k = k0 + threadIdx.x;
  const bool act = k < n;
  const bool first = (k == 0) && isnan(t_prev);
  double h = 0.0;
  int bits = 0;
  if (act) {
    const double t1 = t[k];
    if (nonfinite(t1)) bits |= PSSGP_ENAN;
    if (!first) {
      h = t1 - (k > 0 ? t[k - 1] : t_prev);
      if (negative_nonzero(h)) bits |= PSSGP_EUNSORTED;
    }
  }
  Mat<D> F, Q;
  discretize<D, false, true>(m, h, first, act, F, Q);
  store_fq<D>(stage, threadIdx.x, F, Q);     // record threadIdx.x of the block
  if (tauq && act) { tauq[2 * k] = h; tauq[2 * k + 1] = 1.0; }
  __syncthreads();
  const int64_t nrec = min((int64_t)DISC_BLOCK, n - k0);
  double* dst = rec + k0 * FQS;
  for (int64_t e = threadIdx.x; e < nrec * FQS; e += DISC_BLOCK) dst[e] = stage[e];
  flag(status, bits);
}

// batched series: the series of step k by binary search in offsets[0..B];
// the model, built at (ell0, var0), rescaled per series (see discretize);
// writes the F/Q record, the step's noise variance and whether it starts a
// series.  params[3s..3s+2] = lengthscale, variance, noise variance.  The
// grid covers max(n, B + 1) threads so that every offset is checked.
// per-series scales of the unit model, once per series: uscale = l0 / l and
// qscale = s2 / s2_0 and the noise variance, stored at the series' first step
// (a non-empty series' first step is unique and < n); checks the parameters
__global__ void __launch_bounds__(128) k_series_scales(double ell0, double var0, const int64_t* offsets, int B,
                                                      const double* params, int64_t n, double* su, double* sq,
                                                      double* sr, int* sf, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B) return;
  const int64_t a = offsets[s], b = offsets[s + 1];
  if (!(b > a) || a < 0 || a >= n) return;      // empty (or invalid: flagged by k_discretize_batched)
  const double ell = params[3 * s], s2 = params[3 * s + 1], R = params[3 * s + 2];
  // a series with a parameter that is not positive and finite is computed
  // with unit scales (finite values, so that nothing non-finite can reach the
  // other series through the scan) and flagged; its outputs become NaN
  const bool badp = bad_pos(ell) || bad_pos(s2) || bad_pos(R);
  if (badp) flag(status, PSSGP_EBATCH);
  su[a] = badp ? 1.0 : ell0 / ell;
  sq[a] = badp ? 1.0 : s2 / var0;
  sr[a] = badp ? 1.0 : R;
  sf[a] = badp ? PSSGP_EBATCH : 0;
}

template <int D>
__global__ void __launch_bounds__(DISC_BLOCK) k_discretize_batched(const DevModel<D> m, const int64_t* offsets,
                                                                 int B, const double* su, const double* sq,
                                                                 const double* sr, const double* t, int64_t n,
                                                                 double* rec, double* Rstep, uint8_t* seg,
                                                                 double* tauq, const double* y,
                                                                 const uint8_t* mask, int* sf, int* status) {
  constexpr int FQS = fqs_of<D>();
  extern __shared__ double stage[];
  const int64_t k0 = (int64_t)blockIdx.x * DISC_BLOCK;
  const int64_t k = k0 + threadIdx.x;
  const bool act = k < n;
  int bits = 0;
  if (k <= B) {   // offsets: 0 = o_0 <= o_1 <= ... <= o_B = n
    const int64_t ok = offsets[k];
    if ((k == 0 && ok != 0) || (k == B && ok != n) || (k < B && offsets[k + 1] < ok)) bits |= PSSGP_EBATCH;
  }
  int64_t sid = 0;
  bool first = false;
  double uscale = 1.0, qscale = 1.0, R = 1.0, h = 0.0;
  if (act) {
    int lo = 0, hi = B;                       // last s with offsets[s] <= k
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (offsets[mid] <= k) lo = mid; else hi = mid;
    }
    sid = lo;
    const int64_t a0 = offsets[sid];
    first = (k == 0) || (k == a0);
    const int64_t ia = min(max(a0, (int64_t)0), n - 1);   // in range even for invalid offsets (flagged)
    uscale = su[ia];
    qscale = sq[ia];
    R = sr[ia];
    const double t1 = t[k];
    int sbits = 0;
    if (nonfinite(t1)) sbits |= PSSGP_ENAN;
    if (!first) {
      h = t1 - t[k - 1];
      if (negative_nonzero(h)) sbits |= PSSGP_EUNSORTED;
      // a bad time becomes a zero-length step (F = I, Q = 0), which keeps the
      // scan finite; the series is flagged and its outputs become NaN
      if (!(h >= 0.0) || nonfinite(h)) h = 0.0;
    }
    // an observed non-finite y is taken as missing by the filter kernels
    if (mask[k] && nonfinite(y[k])) sbits |= PSSGP_ENAN;
    if (sbits) {
      atomicOr(sf + ia, sbits);
      bits |= sbits;
    }
  }
  Mat<D> F, Q;
  discretize<D, true, true>(m, h, first, act, F, Q, uscale, qscale);
  store_fq<D>(stage, threadIdx.x, F, Q);
  if (act) {
    Rstep[k] = R;
    seg[k] = first ? 1 : 0;
    if (tauq) { tauq[2 * k] = first ? 0.0 : h * uscale; tauq[2 * k + 1] = qscale; }
  }
  __syncthreads();
  const int64_t nrec = min((int64_t)DISC_BLOCK, n - k0);
  double* dst = rec + k0 * FQS;
  for (int64_t e = threadIdx.x; e < nrec * FQS; e += DISC_BLOCK) dst[e] = stage[e];
  flag(status, bits);
}

// per-series sums of pieces written at the first step of every (lane chunk,
// series) pair: for series [a, b) the positions a and every chunk start c L
// in (a, b); nothing else of v is read.  One warp per series: lane j adds the
// pieces j, j + 32, ... of that list, then a fixed shuffle tree adds the lanes
// (deterministic).  nv <= 4 arrays of stride n at once, out[s * ostride + i]
// for array i.
constexpr int SEG_WARPS = 4;   // series per 128-thread block
__global__ void __launch_bounds__(32 * SEG_WARPS) k_segment_pieces(const double* v, int nv, int64_t n, int64_t L,
                                                                 const int64_t* offsets, int B, double* out,
                                                                 int ostride, const int* sf) {
  const int s = blockIdx.x * SEG_WARPS + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= B) return;                                         // the whole warp
  const int64_t a = min(max(offsets[s], (int64_t)0), n);     // clamped: bad offsets are
  const int64_t b = min(max(offsets[s + 1], a), n);           // flagged by k_discretize_batched
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (b > a) {
    const int64_t c0 = a / L + 1;                  // first chunk starting after a
    const int64_t np = 1 + (b - 1) / L - a / L;    // a, and the chunk starts c L with c0 <= c <= (b - 1) / L
    for (int64_t j = lane; j < np; j += 32) {
      const int64_t k = (j == 0) ? a : (c0 + j - 1) * L;
      for (int i = 0; i < nv; ++i) acc[i] += v[(int64_t)i * n + k];
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], off);
  // a flagged series (bad parameter, time or observation) gets NaN
  const bool failed = (b > a) && sf[a] != 0;
  if (lane == 0)
    for (int i = 0; i < nv; ++i) out[(int64_t)s * ostride + i] = failed ? __longlong_as_double(0x7ff8000000000000LL) : acc[i];
}
unsigned segment_grid(int B) { return (unsigned)((B + SEG_WARPS - 1) / SEG_WARPS); }

// natural log of a product of positive numbers kept as mantissa and binary
// exponent: one multiply per factor instead of one logarithm
struct LogProd {
  double mant = 1.0;
  long long expo = 0;
  __device__ __forceinline__ void mul(double s) {
    mant *= s;
    const long long b = __double_as_longlong(mant);
    expo += ((b >> 52) & 0x7ff) - 1023;
    mant = __longlong_as_double((b & ~(0x7ffLL << 52)) | (1023LL << 52));
  }
  __device__ __forceinline__ double ln() const { return ::log(mant) + (double)expo * 0.69314718055994530942; }
};

// log-likelihood of nobs observed steps from log prod S and sum v^2/S
__device__ __forceinline__ double ll_piece(int nobs, const LogProd& lp, double qsum) {
  return (nobs > 0) ? -0.5 * ((double)nobs * 1.8378770664093454836 + lp.ln() + qsum) : 0.0;
}

// shared memory of k_filter_reduce: A (two buffers), J (packed) and eta per
// thread, entry-major with stride BLOCK
// instances of k_filter_reduce (RMODE, described below)
enum { RED_PLAIN = 0, RED_LL = 1, RED_SMOOTH = 2, RED_ADJ = 3 };

// For 4 <= d <= 6 the level-1 warp scan can run in shared
// memory: two buffers of one packed aggregate per thread, the second
// overlapping the fold's region (the fold is done when the scan starts); 189
// doubles per thread (194 KB per block) at d = 6.  Below d = 4 the aggregates
// are small enough for registers, above d = 6 the buffers would not fit.
// The other form runs the scan on register/local operands and keeps the
// fold's 101 KB of shared memory only, so that a block of another call's
// filter pass (114 KB) fits beside it on an SM.  The prediction's instance
// (RED_SMOOTH) takes the shared-memory form when the call is planned on the
// whole GPU (4 or more warps per SM: one call at a time) and the small form
// when it is planned on fewer (several calls in flight on streams, which
// overlap only if their blocks share SMs).  Measured at 2^20 RBF-6: one call
// 5.35 against 5.44 ms; eight calls in flight at 2 warps per SM 235 against
// 240 M steps/s, four at 4 warps per SM 217 against 226 M.
template <int D> __host__ __device__ constexpr bool l1_smem_fits() { return D >= 4 && D <= 6; }
template <int D> __host__ __device__ constexpr int reduce_fold_doubles() { return 2 * D * D + Sym<D>::N + D; }
template <int D, bool L1S> constexpr int reduce_smem_doubles() {
  return (L1S ? FAggSize<D>::N + (reduce_fold_doubles<D>() > FAggSize<D>::N ? reduce_fold_doubles<D>()
                                                                            : FAggSize<D>::N)
              : reduce_fold_doubles<D>()) * BLOCK;
}

// RMODE:
//  RED_LL: also the log-likelihood of the chunk's observations given the
//    state 0 before it (the terms of the fold's zero-start Kalman filter),
//    split where a series starts inside the chunk; pieces after the first are
//    exact and written to ll_step, the first goes with the lane's own (eta, J)
//    to lane_ll for k_filter_llfinish.
//  RED_SMOOTH: also (A, eta, J) of the aggregate of the lane's steps but the
//    last (of all its steps in the lane holding the series' last step) to
//    lane_fp, from which k_filter_propagate forms the smoother chunk aggregate.
//  RED_ADJ: the chunk's first step folded with its transition left out
//    (F = I, Q = 0): the aggregate then takes the predicted state of the
//    chunk's first step as input; its (A, eta, J) go to lane_fp (for the
//    mean-adjoint chunk aggregate of k_filter_propagate), and the transition
//    is put back in front (one operator application) for the scan: in
//    shared memory with the transition read from its record
//    (fagg_transition_combine_smem) where the scan runs there, else on
//    register operands.

// A, eta, J: this thread's entries in shared memory with stride SST (the
// block's thread count)
template <int D, int SST>
__device__ __forceinline__ void save_fold_state(const ScanArgs& a, int64_t g, const double* A, const double* eta,
                                                const double* J) {
#pragma unroll
  for (int e = 0; e < D * D; ++e) a.lane_fp[e * a.P0 + g] = A[e * SST];
#pragma unroll
  for (int i = 0; i < D; ++i) a.lane_fp[(D * D + i) * a.P0 + g] = eta[i * SST];
#pragma unroll
  for (int e = 0; e < Sym<D>::N; ++e) a.lane_fp[(D * D + D + e) * a.P0 + g] = J[e * SST];
}

template <int D, int RMODE, bool L1S>
__global__ void __launch_bounds__(BLOCK, 1) k_filter_reduce(const DevModel<D> m, const ScanArgs a) {
  constexpr int RB = BLOCK;   // threads per block (stride of the per-thread arrays)
  constexpr bool LL = RMODE == RED_LL;
  // 16-byte record loads (load_record): faster in the gradient's instance, in
  // every instance with the shared-memory warp scan (prediction 1.948 ->
  // 1.876 ms at 2^20 RBF-6) and in the prediction's register-scan instance
  // at d >= 4 (eight concurrent predictions 240.0 -> 240.8 M steps/s); not
  // in the log-likelihood's instance at d <= 3 (batched: 10.53 -> 10.64 ms)
  constexpr bool VECMODE = RMODE == RED_ADJ || (D >= 4 && RMODE == RED_SMOOTH) || (L1S && RMODE == RED_LL);
  extern __shared__ double smem[];
  constexpr int NF = FAggSize<D>::N;
  double* sB0 = smem + threadIdx.x;                    // level-1 buffer 0 (shared-memory scan)
  double* sA0 = smem + (L1S ? NF * RB : 0) + threadIdx.x;
  double* sA1 = sA0 + D * D * RB;
  double* sJ = sA1 + D * D * RB;
  double* seta = sJ + Sym<D>::N * RB;
  const int64_t g = (int64_t)blockIdx.x * RB + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t k0 = g * a.L;
  const int64_t k1 = min(k0 + a.L, a.n);
  int bits = 0;
  bool bad = false;
  // chunk aggregate starts as the identity of the operator
  Vec<D> b;
  Mat<D> C;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    b[i] = 0.0;
    seta[i * RB] = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) { C[i][j] = 0.0; sA0[(i * D + j) * RB] = (i == j) ? 1.0 : 0.0; }
  }
#pragma unroll
  for (int e = 0; e < Sym<D>::N; ++e) sJ[e * RB] = 0.0;
  double* Ain = sA0;
  double* Aout = sA1;
  const double R0 = a.R ? a.R[0] : a.R_scalar;
  double qsum = 0.0, cfirst = 0.0;
  LogProd lp;
  int nobs = 0;
  bool first = true;
  int64_t lpos = k0;
#pragma unroll 1
  for (int64_t k = k0; k < k1; ++k) {
    if constexpr (LL) {
      if (a.ll_step && k > k0 && a.seg_start[k]) {   // a series starts inside the chunk
        const double piece = ll_piece(nobs, lp, qsum);
        if (first) cfirst = piece;
        else a.ll_step[lpos] = piece;
        first = false;
        lpos = k;
        nobs = 0;
        qsum = 0.0;
        lp = LogProd();
      }
    }
    if constexpr (RMODE == RED_SMOOTH) {
      // steps k0 .. k1-2 (also in the last lane when the series goes on in a next chunk)
      if (k == k1 - 1 && (k1 < a.n || !isnan(a.t_next))) save_fold_state<D, RB>(a, g, Ain, seta, sJ);
    }
    Mat<D> F, Q;
    load_fq<D, VECMODE>(a.rec_fq, k, F, Q);
    if constexpr (RMODE == RED_ADJ) {
      if (k == k0) {   // from the predicted state of step k0: no transition
        set_eye<D>(F);
        set_zero<D>(Q);
      }
    }
    const double yk = a.y[k];
    const double Rk = a.R_per_step ? a.R[k] : R0;
    // a non-finite observation is flagged and taken as missing
    const bool obs = a.mask[k] != 0 && !nonfinite(yk);
    if (a.mask[k] != 0 && nonfinite(yk)) bits |= PSSGP_ENAN;
    double S, Si, r;
    fagg_fold_step_smem<D, RB>(b, C, Ain, Aout, sJ, seta, F, Q, obs, yk, Rk, bad, S, Si, r);
    if constexpr (LL) {
      qsum = fma(r * Si, r, qsum);
      lp.mul(obs ? S : 1.0);
      nobs += obs ? 1 : 0;
    }
    double* tsw = Ain;
    Ain = Aout;
    Aout = tsw;
  }
  if constexpr (RMODE == RED_SMOOTH) {
    if (k1 == a.n && k1 > k0 && isnan(a.t_next)) save_fold_state<D, RB>(a, g, Ain, seta, sJ);   // the series' last step
  }
  if constexpr (RMODE == RED_ADJ) {
    if (k1 > k0) save_fold_state<D, RB>(a, g, Ain, seta, sJ);
  }
  if constexpr (LL) {
    const double piece = ll_piece(nobs, lp, qsum);
    if (first) cfirst = piece;
    else a.ll_step[lpos] = piece;
    a.lane_ll[g] = cfirst;
#pragma unroll
    for (int i = 0; i < D; ++i) a.lane_ll[(1 + i) * a.P0 + g] = seta[i * RB];
#pragma unroll
    for (int e = 0; e < Sym<D>::N; ++e) a.lane_ll[(1 + D + e) * a.P0 + g] = sJ[e * RB];
  }
  if constexpr (L1S) {
    // the chunk aggregate, packed into buffer 0, then the level-1 scan in
    // shared memory (partner lane's aggregate read in place, no shuffles)
    double* B0 = sB0;
    {
#pragma unroll
      for (int e = 0; e < D * D; ++e) B0[e * RB] = Ain[e * RB];
#pragma unroll
      for (int i = 0; i < D; ++i) B0[(D * D + i) * RB] = b[i];
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) B0[(D * D + D + pidx<D>(i, j)) * RB] = C[i][j];
#pragma unroll
      for (int i = 0; i < D; ++i) B0[(D * D + D + Sym<D>::N + i) * RB] = seta[i * RB];
#pragma unroll
      for (int e = 0; e < Sym<D>::N; ++e) B0[(D * D + 2 * D + Sym<D>::N + e) * RB] = sJ[e * RB];
    }
    if constexpr (RMODE == RED_ADJ) {
      // the transition of step k0 in front, (F, 0, Q, 0, 0) x aggregate, once
      // per lane: into the fold's (now free) region, then back to buffer 0
      if (k1 > k0) {
        if (!fagg_transition_combine_smem<D, RB>(a.rec_fq + k0 * fqs_of<D>(), B0, sA0)) bad = true;
        for (int e = 0; e < NF; ++e) B0[e * RB] = sA0[e * RB];
      }
    }
    if (a.dbg_agg) {
      for (int e = 0; e < NF; ++e) a.dbg_agg[e * a.P0 + g] = B0[e * RB];
    }
    __syncwarp();
    double* cur = B0;
    double* nxt = sA0;                // buffer 1 over the fold's region
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
      if (lane >= off) {
        if (!fagg_combine_smem<D, RB>(cur - off, cur, nxt)) bad = true;
      } else {
        for (int e = 0; e < NF; ++e) nxt[e * RB] = cur[e * RB];
      }
      __syncwarp();
      double* tsw = cur;
      cur = nxt;
      nxt = tsw;
    }
    for (int e = 0; e < NF; ++e) {
      const double v = cur[e * RB];
      a.lagg_f[e * a.P0 + g] = v;
      if (lane == 31) a.wagg_f[e * a.P2 + (g >> 5)] = v;
    }
  } else {
    FAgg<D> ag;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      ag.b[i] = b[i];
      ag.eta[i] = seta[i * RB];
#pragma unroll
      for (int jj = 0; jj < D; ++jj) {
        ag.A[i][jj] = Ain[(i * D + jj) * RB];
        ag.C[i][jj] = C[i][jj];
        ag.J[i][jj] = sJ[(i <= jj ? pidx<D>(i, jj) : pidx<D>(jj, i)) * RB];
      }
    }
    if constexpr (RMODE == RED_ADJ) {
      if (k1 > k0) {   // the transition of step k0 in front: (F, 0, Q, 0, 0) x aggregate
        FAgg<D> T, r;
        load_fq<D>(a.rec_fq, k0, T.A, T.C);
#pragma unroll
        for (int i = 0; i < D; ++i) {
          T.b[i] = 0.0;
          T.eta[i] = 0.0;
#pragma unroll
          for (int j = 0; j < D; ++j) T.J[i][j] = 0.0;
        }
        if (!fagg_combine<D>(T, ag, r)) bad = true;
        ag = r;
      }
    }
    if (a.dbg_agg) store_fagg<D>(a.dbg_agg + g, a.P0, ag);
    // level 1: inclusive scan over the 32 lanes of the warp
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
      FAgg<D> o = ag;
      shfl_up_fagg<D>(o, off);
      if (lane >= off) {
        FAgg<D> r;
        if (!fagg_combine<D>(o, ag, r)) bad = true;
        ag = r;
      }
    }
    store_fagg<D>(a.lagg_f + g, a.P0, ag);
    if (lane == 31) store_fagg<D>(a.wagg_f + (g >> 5), a.P2, ag);
  }
  if (bad) bits |= PSSGP_ENOTPD;
  flag(a.status, bits);
}

// The filter state (x = b, P = C) of a packed filter aggregate that holds a
// series' first step (then A = 0, eta = 0, J = 0: a state, Prop. 1).
// (entry e at p[e * st])
template <int D>
__device__ __forceinline__ void load_fstate(const double* p, Vec<D>& x, Mat<D>& P, int64_t st = 1) {
#pragma unroll
  for (int i = 0; i < D; ++i) x[i] = p[(D * D + i) * st];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = i; j < D; ++j) { P[i][j] = p[(D * D + D + pidx<D>(i, j)) * st]; P[j][i] = P[i][j]; }
}

// filter level 2: one Kogge-Stone round over the warp aggregates, one warp
// per element (warp-cooperative operator, see warp_ops.cuh)
template <int D>
__global__ void __launch_bounds__(BLOCK) k_filter_ks(const double* in, double* out, int64_t P2, int64_t off,
                                                     int* status) {
  constexpr int NF = FAggSize<D>::N;
  __shared__ double sm[BLOCK / 32][WarpFilterSmem<D>::N];
  // programmatic dependent launch (level2_launch): wait for the previous
  // grid's results; the next round may be scheduled meanwhile
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (BLOCK / 32) + wid;
  if (i >= P2) return;                       // whole warp
  if (i < off) {
    for (int e = lane; e < NF; e += 32) out[e * P2 + i] = in[e * P2 + i];
    return;
  }
  double* sa = sm[wid];
  double* sb = sa + NF;
  double* work = sb + NF;
  for (int e = lane; e < NF; e += 32) { sa[e] = in[e * P2 + i - off]; sb[e] = in[e * P2 + i]; }
  __syncwarp();
  const bool ok = warp_fagg_combine<D>(sa, sb, work, out + i, P2, lane);
  if (!ok && lane == 0) flag(status, PSSGP_ENOTPD);
}

// Log-likelihood of a chunk's observations given the filter state N(x, P)
// before it.  For a state z before the chunk, the chunk's aggregate gives
// log p(y | z) = c + eta^T z - z^T J z / 2 exactly (c: the log-likelihood the
// fold accumulates from the state 0; eta, J: Sec. 3's information terms), and
// the Gaussian integral over z ~ N(x, P) is
//   c + eta^T x - x^T J x / 2 + r^T (I + P J)^{-1} P r / 2 - log det(I + P J) / 2,
//   r = eta - J x.
// Returns false if a pivot of I + P J is zero or its determinant is not
// positive (it is at least 1 for P, J positive semi-definite).
template <int D>
__device__ __noinline__ bool chunk_loglik(const Vec<D>& x, const Mat<D>& P, const Vec<D>& eta, const Mat<D>& J,
                                          double c, double& out) {
  Vec<D> r;
  double lin = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double jx = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) jx = fma(J[i][k], x[k], jx);
    r[i] = eta[i] - jx;
    lin = fma(x[i], fma(-0.5, jx, eta[i]), lin);
  }
  Mat<D> M;
  double X[D][1];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) s = fma(P[i][k], r[k], s);
    X[i][0] = s;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double t = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < D; ++k) t = fma(P[i][k], J[k][j], t);
      M[i][j] = t;
    }
  }
  int perm[D];
  double invd[D];
  bool ok = lu_factor<D>(M, perm, invd);
  lu_solve<D, 1>(M, perm, invd, X);
  double quad = 0.0;
#pragma unroll
  for (int i = 0; i < D; ++i) quad = fma(r[i], X[i][0], quad);
  LogProd ld;
  int neg = 0;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if (perm[i] != i) ++neg;
    if (M[i][i] < 0.0) ++neg;
    ld.mul(fabs(M[i][i]));
  }
  if (neg & 1) ok = false;
  out = c + lin + 0.5 * quad - 0.5 * ld.ln();
  return ok;
}

// log-likelihood-only path, after level 2 (replaces the propagate pass): the
// filter state before each chunk from the scan, then the chunk's first series
// piece by chunk_loglik, per lane (llp) and, batched, as the piece at the
// chunk's first step
template <int D>
__global__ void __launch_bounds__(BLOCK) k_filter_llfinish(const DevModel<D> m, const ScanArgs a) {
  const int64_t g = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t w = g >> 5;
  const int64_t k0 = g * a.L;
  const int64_t k1 = min(k0 + a.L, a.n);
  if (k1 <= k0) {
    a.llp[g] = 0.0;
    return;
  }
  bool bad = false;
  Vec<D> x;
  Mat<D> P;
#pragma unroll
  for (int i = 0; i < D; ++i) x[i] = 0.0;
  set_zero<D>(P);
  if (w > 0) {
    load_fstate<D>(a.wfin_f + (w - 1), x, P, a.P2);
  } else if (a.start_f) {   // a chunk of a longer series: the state before it
    load_fstate<D>(a.start_f, x, P);
  }
  if (lane > 0) {
    Vec<D> x2;
    Mat<D> P2;
    if (!fstate_combine<D>(x, P, a.lagg_f + (g - 1), a.P0, x2, P2)) bad = true;
#pragma unroll
    for (int i = 0; i < D; ++i) x[i] = x2[i];
    copy<D>(P2, P);
  }
  Vec<D> eta;
  Mat<D> J;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    eta[i] = a.lane_ll[(1 + i) * a.P0 + g];
#pragma unroll
    for (int j = i; j < D; ++j) {
      J[i][j] = a.lane_ll[(1 + D + pidx<D>(i, j)) * a.P0 + g];
      J[j][i] = J[i][j];
    }
  }
  double ll;
  if (!chunk_loglik<D>(x, P, eta, J, a.lane_ll[g], ll)) bad = true;
  a.llp[g] = ll;
  if (a.ll_step) a.ll_step[k0] = ll;
  if (bad) flag(a.status, PSSGP_ENOTPD);
}

// filter level 3 (+ smoother levels 0/1 when fused)
// shared memory of k_filter_propagate, per thread, entry-major with stride
// BLOCK: a d x d matrix (Sig), a packed symmetric one (V) and a vector (mu).
// The adjoint mode keeps the prediction of the chunk's first step in (mu, V);
// the fused mode keeps the start state (x0 in mu, P0 in V) and F of the
// lane's last step (in Sig), plus the filter covariance P_k (packed) and the
// prediction (x^-, P^-) of the last step.
template <int D, int MODE> constexpr int propagate_smem_doubles() {
  return (D * D + Sym<D>::N + D + (MODE == 1 ? 2 * Sym<D>::N + D : 0)) * BLOCK;
}

// MODE: PROP_PLAIN (filter outputs / log-likelihood), PROP_FUSE (+ smoother
// levels 0/1), PROP_ADJ (+ the forward part of the gradient); a template
// parameter so that each instance holds only its own state in the step loop
enum { PROP_PLAIN = 0, PROP_FUSE = 1, PROP_ADJ = 2 };

template <int D, int MODE>
__global__ void __launch_bounds__(BLOCK, 1) k_filter_propagate(const DevModel<D> m, const ScanArgs a) {
  extern __shared__ double psm[];
  double* sSig = psm + threadIdx.x;
  double* sV = sSig + D * D * BLOCK;
  double* smu = sV + Sym<D>::N * BLOCK;
  double* sP = smu + D * BLOCK;     // fused mode only
  double* sxm1 = sP + Sym<D>::N * BLOCK;
  double* sPm1 = sxm1 + D * BLOCK;
  const int64_t g = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t w = g >> 5;
  const int64_t k0 = g * a.L;
  const int64_t k1 = min(k0 + a.L, a.n);
  int bits = 0;
  bool bad = false;
  // chunk start state = (warps before) x (lanes before, same warp)
  Vec<D> x;
  Mat<D> P;
#pragma unroll
  for (int i = 0; i < D; ++i) x[i] = 0.0;
  set_zero<D>(P);
  if (w > 0) {
    load_fstate<D>(a.wfin_f + (w - 1), x, P, a.P2);
  } else if (a.start_f) {   // a chunk of a longer series: the state before it
    load_fstate<D>(a.start_f, x, P);
  }
  if (lane > 0) {
    Vec<D> x2;
    Mat<D> P2;
    if (!fstate_combine<D>(x, P, a.lagg_f + (g - 1), a.P0, x2, P2)) bad = true;
#pragma unroll
    for (int i = 0; i < D; ++i) x[i] = x2[i];
    copy<D>(P2, P);
  }
  const double R0 = a.R ? a.R[0] : a.R_scalar;
  constexpr bool fuse = MODE == PROP_FUSE;
  constexpr bool adj = MODE == PROP_ADJ;
  if constexpr (fuse) {   // the filter state before the chunk, for the smoother chunk aggregate
#pragma unroll
    for (int i = 0; i < D; ++i) smu[i * BLOCK] = x[i];
    store_sym_smem<D, BLOCK>(sV, P);
  }
  double qsum = 0.0;
  LogProd lp;
  int nobs = 0;
  int64_t lpos = k0;   // batched: where the current series piece is written
#pragma unroll 1
  for (int64_t k = k0; k < k1; ++k) {
    if (a.ll_step) {   // one log-likelihood piece per (lane chunk, series) pair
      if (k > k0 && a.seg_start[k]) {
        a.ll_step[lpos] = ll_piece(nobs, lp, qsum);
        lpos = k;
        nobs = 0;
        qsum = 0.0;
        lp = LogProd();
      }
    }
    if (k + 1 < k1) prefetch_record<fqs_of<D>()>(a.rec_fq + (k + 1) * fqs_of<D>());
    Mat<D> F, Q, T, Pm;
    Vec<D> xm;
    load_fq<D>(a.rec_fq, k, F, Q);
    mulv<D>(F, x, xm);
    mul<D>(F, P, T);
    mul_Bt_sym_add<D>(T, F, Q, Pm);
    // the update without a branch (1/S and v are 0 on a missing step)
    const double yk = a.y[k];
    const bool obs = a.mask[k] != 0 && !nonfinite(yk);   // a non-finite observation is missing (flagged by the reduce)
    const double S = Pm[0][0] + (a.R_per_step ? a.R[k] : R0);
    if (obs && bad_pos(S)) bad = true;
    const double Si = obs ? __drcp_rn(S) : 0.0;
    const double v = obs ? yk - xm[0] : 0.0;
    if constexpr (fuse) {
      if (k == k1 - 1) {   // the prediction of the lane's last step closes the smoother chunk aggregate
#pragma unroll
        for (int i = 0; i < D; ++i) {
          sxm1[i * BLOCK] = xm[i];
#pragma unroll
          for (int j = 0; j < D; ++j) sSig[(i * D + j) * BLOCK] = F[i][j];
        }
        store_sym_smem<D, BLOCK>(sPm1, Pm);
      }
      if (k > k0 && !smoother_element_store<D, BLOCK>(a.rec_egl, k - 1, x, sP, T, xm, Pm)) bad = true;
    }
    {
      Vec<D> K;
#pragma unroll
      for (int i = 0; i < D; ++i) K[i] = Pm[i][0] * Si;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        x[i] = fma(K[i], v, xm[i]);
#pragma unroll
        for (int j = i; j < D; ++j) { P[i][j] = fma(-K[i], Pm[0][j], Pm[i][j]); P[j][i] = P[i][j]; }
      }
    }
    qsum = fma(v * Si, v, qsum);
    lp.mul(obs ? S : 1.0);
    nobs += obs ? 1 : 0;
    if constexpr (fuse) store_sym_smem<D, BLOCK>(sP, P);
    if constexpr (adj) {  // gradient: forward moments; the prediction of step k0 for the chunk aggregate
      store_adj<D>(a.rec_adj, k, xm, Pm, v, Si);
      if (k == k0) {
#pragma unroll
        for (int i = 0; i < D; ++i) smu[i * BLOCK] = xm[i];
        store_sym_smem<D, BLOCK>(sV, Pm);
      }
    }
    if (a.xf) {
#pragma unroll
      for (int i = 0; i < D; ++i) a.xf[i * a.ld + k] = x[i] * m.Dsc[i];
    }
    if (a.Pf) {
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) a.Pf[pidx<D>(i, j) * a.ld + k] = P[i][j] * (m.Dsc[i] * m.Dsc[j]);
    }
  }
  a.llp[g] = ll_piece(nobs, lp, qsum);
  if (a.ll_step && k1 > k0) a.ll_step[lpos] = a.llp[g];
  if constexpr (adj) {
    // The mean-adjoint chunk aggregate mb_{k0} = Pi mb_{k1} + gamma, with
    // Pi^T = d m^-_{k1} / d m^-_{k0} and gamma the derivative of the chunk's
    // log-likelihood by the predicted mean m^- of step k0, in closed form from
    // the filter aggregate (A, eta, J) that takes the predicted state of step
    // k0 as input (k_filter_reduce, RED_ADJ) and that prediction (m^-, P^-):
    // the filtered mean of step k1-1 is A (I + P^- J)^{-1} (m^- + P^- eta) + b
    // and the chunk's log-likelihood is Sec. 3's Gaussian integral, so with
    // N = I + J P^-,
    //   Pi = N^{-1} A^T F_{k1}^T,   gamma = N^{-1} (eta - J m^-)
    // (F_{k1} = 0 after the last step; a series start inside the chunk gives
    // A = 0 and freezes eta, J, as the recursion would).
    SAgg<D> sa;
    if (k1 > k0) {
      Mat<D> F1, J, N, Pm0;
      Vec<D> eta;
      if (k1 < a.n) load_F<D>(a.rec_fq, k1, fqs_of<D>(), F1);
      else if (a.f_next) load_F<D>(a.f_next, 0, fqs_of<D>(), F1);   // the series goes on in a next chunk
      else set_zero<D>(F1);
      load_sym_smem<D, BLOCK>(sV, Pm0);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        eta[i] = a.lane_fp[(D * D + i) * a.P0 + g];
#pragma unroll
        for (int j = i; j < D; ++j) {
          J[i][j] = a.lane_fp[(D * D + D + pidx<D>(i, j)) * a.P0 + g];
          J[j][i] = J[i][j];
        }
      }
      constexpr int NR = 2 * D + 1;   // [eta - J m^- | A^T F1^T | J]
      double X[D][NR];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        double gi = eta[i];
#pragma unroll
        for (int k = 0; k < D; ++k) gi = fma(-J[i][k], smu[k * BLOCK], gi);
        X[i][0] = gi;
#pragma unroll
        for (int j = 0; j < D; ++j) X[i][1 + D + j] = J[i][j];
#pragma unroll
        for (int j = 0; j < D; ++j) {
          double t = (i == j) ? 1.0 : 0.0;   // N = I + J P^-
#pragma unroll
          for (int k = 0; k < D; ++k) t = fma(J[i][k], Pm0[k][j], t);
          N[i][j] = t;
          double u = 0.0;                    // (A^T F1^T)[i][j] = sum_k A[k][i] F1[j][k]
#pragma unroll
          for (int k = 0; k < D; ++k) u = fma(a.lane_fp[(k * D + i) * a.P0 + g], F1[j][k], u);
          X[i][1 + j] = u;
        }
      }
      int perm[D];
      double invn[D];
      if (!lu_factor<D>(N, perm, invn)) bad = true;
      lu_solve<D, NR>(N, perm, invn, X);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        sa.g[i] = X[i][0];
        a.lane_gj[i * a.P0 + g] = X[i][0];
#pragma unroll
        for (int j = 0; j < D; ++j) {
          sa.E[i][j] = X[i][1 + j];
          a.lane_pi[(i * D + j) * a.P0 + g] = sa.E[i][j];
          sa.L[i][j] = 0.0;
        }
#pragma unroll
        for (int j = i; j < D; ++j)    // N^{-1} J (symmetric)
          a.lane_gj[(D + pidx<D>(i, j)) * a.P0 + g] = 0.5 * (X[i][1 + D + j] + X[j][1 + D + i]);
      }
    } else {
      sagg_identity<D>(sa);
#pragma unroll
      for (int e = 0; e < D * D; ++e) a.lane_pi[e * a.P0 + g] = (e % (D + 1) == 0) ? 1.0 : 0.0;
#pragma unroll
      for (int e = 0; e < D + Sym<D>::N; ++e) a.lane_gj[e * a.P0 + g] = 0.0;
    }
    // level 1 of the mean-adjoint scan: inclusive suffix scan over the warp
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
      SAgg<D> o = sa;
      shfl_down_sagg<D>(o, off);
      if (lane + off < 32) {
        SAgg<D> r;
        sagg_combine<D>(sa, o, r);
        sa = r;
      }
    }
    store_sagg<D>(a.lagg_s + g, a.P0, sa);
    if (lane == 0) store_sagg<D>(a.wagg_s + w, a.P2, sa);
  } else if constexpr (fuse) {
    // The lane's smoother chunk is the elements k0-1 .. k1-2 (k0-1 .. n-1 in
    // the lane with the last step; element -1 of lane 0 is void: its start
    // state is 0).  Its aggregate p(x_{k0-1} | x_{k1-1}, y_{1:k1-2}) comes from
    // the filter state (x0, P0) before the chunk and the filter aggregate
    // (A, eta, J) of steps k0 .. k1-2 saved by k_filter_reduce: with
    // M = I + P0 J,
    //   mu  = M^{-1} (x0 + P0 eta) = E[x_{k0-1} | y_{1:k1-2}],
    //   V   = M^{-1} P0            = Cov(x_{k0-1} | y_{1:k1-2}),
    //   Sig = V A^T                = Cov(x_{k0-1}, x_{k1-2} | y_{1:k1-2})
    // (A M^{-1} is the filter's closed-loop transition over those steps), and
    // the prediction of step k1-1 closes it (fixed_point_finish).  The lane
    // with the last step ends on the series' last element (E = 0), which
    // gives E = 0, g = mu, L = V over all its steps.
    SAgg<D> sa;
    if (k1 > k0) {
      FixedPoint<D> fp;
      {
        Mat<D> P0, J, M;
        Vec<D> eta;
        load_sym_smem<D, BLOCK>(sV, P0);
#pragma unroll
        for (int i = 0; i < D; ++i) {
          eta[i] = a.lane_fp[(D * D + i) * a.P0 + g];
#pragma unroll
          for (int j = i; j < D; ++j) {
            J[i][j] = a.lane_fp[(D * D + D + pidx<D>(i, j)) * a.P0 + g];
            J[j][i] = J[i][j];
          }
        }
        constexpr int NR = D + 1;
        double X[D][NR];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          double sx = smu[i * BLOCK];
#pragma unroll
          for (int k = 0; k < D; ++k) sx = fma(P0[i][k], eta[k], sx);
          X[i][0] = sx;
#pragma unroll
          for (int j = 0; j < D; ++j) {
            X[i][1 + j] = P0[i][j];
            double t = (i == j) ? 1.0 : 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) t = fma(P0[i][k], J[k][j], t);
            M[i][j] = t;
          }
        }
        int perm[D];
        double invm[D];
        if (!lu_factor<D>(M, perm, invm)) bad = true;
        lu_solve<D, NR>(M, perm, invm, X);
#pragma unroll
        for (int i = 0; i < D; ++i) {
          fp.mu[i] = X[i][0];
#pragma unroll
          for (int j = 0; j < D; ++j) fp.V[i][j] = 0.5 * (X[i][1 + j] + X[j][1 + i]);
        }
      }
      // the lane holding the chunk's last step closes like the others when
      // the series goes on in a next chunk (which holds that step's element)
      if (k1 < a.n || !isnan(a.t_next)) {
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int j = 0; j < D; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) s = fma(fp.V[i][k], a.lane_fp[(j * D + k) * a.P0 + g], s);
            fp.Sig[i][j] = s;
          }
        Mat<D> F1, Pm1, Lc;
        Vec<D> xm1;
        double invd[D];
#pragma unroll
        for (int i = 0; i < D; ++i) {
          xm1[i] = sxm1[i * BLOCK];
#pragma unroll
          for (int j = 0; j < D; ++j) F1[i][j] = sSig[(i * D + j) * BLOCK];
        }
        load_sym_smem<D, BLOCK>(sPm1, Pm1);
        if (!cholesky<D>(Pm1, Lc, invd)) bad = true;
        fixed_point_finish<D>(fp, F1, xm1, Lc, invd, sa);
      } else {
        SAgg<D> e;   // the series' last element: E = 0, g = x_{n-1}, P^s = P_{n-1}
        Mat<D> Z;
        set_zero<D>(e.E);
        set_zero<D>(Z);
#pragma unroll
        for (int i = 0; i < D; ++i) e.g[i] = x[i];
        store_rts<D>(a.rec_egl, k1 - 1, e, P, Z);
        set_zero<D>(sa.E);
#pragma unroll
        for (int i = 0; i < D; ++i) sa.g[i] = fp.mu[i];
        copy<D>(fp.V, sa.L);
      }
    } else {
      sagg_identity<D>(sa);
    }
    // smoother level 1: inclusive suffix scan over the warp's lanes
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
      SAgg<D> o = sa;
      shfl_down_sagg<D>(o, off);
      if (lane + off < 32) {
        SAgg<D> r;
        sagg_combine<D>(sa, o, r);
        sa = r;
      }
    }
    store_sagg<D>(a.lagg_s + g, a.P0, sa);
    if (lane == 0) store_sagg<D>(a.wagg_s + w, a.P2, sa);
  }
  if (bad) bits |= PSSGP_ENOTPD;
  flag(a.status, bits);
}

// smoother level 2: one Kogge-Stone round of the suffix scan, one warp per
// element
template <int D>
__global__ void __launch_bounds__(BLOCK) k_smoother_ks(const double* in, double* out, int64_t P2, int64_t off) {
  constexpr int NS = SAggSize<D>::N;
  __shared__ double sm[BLOCK / 32][WarpSmootherSmem<D>::N];
  asm volatile("griddepcontrol.wait;" ::: "memory");   // as in k_filter_ks
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (BLOCK / 32) + wid;
  if (i >= P2) return;
  if (i + off >= P2) {
    for (int e = lane; e < NS; e += 32) out[e * P2 + i] = in[e * P2 + i];
    return;
  }
  double* sa = sm[wid];
  double* sb = sa + NS;
  double* work = sb + NS;
  for (int e = lane; e < NS; e += 32) { sa[e] = in[e * P2 + i]; sb[e] = in[e * P2 + i + off]; }
  __syncwarp();
  warp_sagg_combine<D>(sa, sb, work, out + i, P2, lane);
}

// ---------------------------------------------------------------------------
// one long series split in time chunks (one per GPU): the chunk aggregates of
// the other chunks enter each chunk's scan as one element before it (filter)
// or after it (smoother)
// ---------------------------------------------------------------------------
// packed (stride 1) aggregates[lo .. hi-1] folded in order by one warp:
// out = agg[lo] x agg[lo+1] x ... x agg[hi-1] (filtering operator, Sec. 3)
template <int D>
__global__ void __launch_bounds__(32) k_fold_filter_range(const double* aggs, int lo, int hi, double* out,
                                                          int* status) {
  constexpr int NF = FAggSize<D>::N;
  __shared__ double sm[WarpFilterSmem<D>::N + NF];
  double* sa = sm;
  double* sb = sa + NF;
  double* work = sb + NF;
  double* so = sm + WarpFilterSmem<D>::N;
  const int lane = threadIdx.x;
  for (int e = lane; e < NF; e += 32) sa[e] = aggs[(int64_t)lo * NF + e];
  __syncwarp();
  bool ok = true;
  for (int i = lo + 1; i < hi; ++i) {
    for (int e = lane; e < NF; e += 32) sb[e] = aggs[(int64_t)i * NF + e];
    __syncwarp();
    if (!warp_fagg_combine<D>(sa, sb, work, so, 1, lane)) ok = false;
    __syncwarp();
    for (int e = lane; e < NF; e += 32) sa[e] = so[e];
    __syncwarp();
  }
  for (int e = lane; e < NF; e += 32) out[e] = sa[e];
  if (!ok && lane == 0) flag(status, PSSGP_ENOTPD);
}

// the same with the smoothing operator (supplement, Prop. 2)
template <int D>
__global__ void __launch_bounds__(32) k_fold_smoother_range(const double* aggs, int lo, int hi, double* out) {
  constexpr int NS = SAggSize<D>::N;
  __shared__ double sm[WarpSmootherSmem<D>::N + NS];
  double* sa = sm;
  double* sb = sa + NS;
  double* work = sb + NS;
  double* so = sm + WarpSmootherSmem<D>::N;
  const int lane = threadIdx.x;
  for (int e = lane; e < NS; e += 32) sa[e] = aggs[(int64_t)lo * NS + e];
  __syncwarp();
  for (int i = lo + 1; i < hi; ++i) {
    for (int e = lane; e < NS; e += 32) sb[e] = aggs[(int64_t)i * NS + e];
    __syncwarp();
    warp_sagg_combine<D>(sa, sb, work, so, 1, lane);
    __syncwarp();
    for (int e = lane; e < NS; e += 32) sa[e] = so[e];
    __syncwarp();
  }
  for (int e = lane; e < NS; e += 32) out[e] = sa[e];
}

// filter: every level-2 result w (steps of warps 0..w) becomes
// start x result, so that the chunk's scan starts from the state `start`
template <int D>
__global__ void __launch_bounds__(BLOCK) k_apply_filter_start(double* wfin, int64_t P2, const double* start,
                                                             int* status) {
  constexpr int NF = FAggSize<D>::N;
  __shared__ double sm[BLOCK / 32][WarpFilterSmem<D>::N];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (BLOCK / 32) + wid;
  if (i >= P2) return;                       // whole warp
  double* sa = sm[wid];
  double* sb = sa + NF;
  double* work = sb + NF;
  for (int e = lane; e < NF; e += 32) { sa[e] = start[e]; sb[e] = wfin[e * P2 + i]; }
  __syncwarp();
  if (!warp_fagg_combine<D>(sa, sb, work, wfin + i, P2, lane) && lane == 0) flag(status, PSSGP_ENOTPD);
}

// smoother: every level-2 result w (steps of warps w..P2-1) becomes
// result x end, so that the chunk's scan ends in the smoothed state `end`
template <int D>
__global__ void __launch_bounds__(BLOCK) k_apply_smoother_end(double* wfin, int64_t P2, const double* end) {
  constexpr int NS = SAggSize<D>::N;
  __shared__ double sm[BLOCK / 32][WarpSmootherSmem<D>::N];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (BLOCK / 32) + wid;
  if (i >= P2) return;
  double* sa = sm[wid];
  double* sb = sa + NS;
  double* work = sb + NS;
  for (int e = lane; e < NS; e += 32) { sa[e] = wfin[e * P2 + i]; sb[e] = end[e]; }
  __syncwarp();
  warp_sagg_combine<D>(sa, sb, work, wfin + i, P2, lane);
}

// the F/Q record (layout of the per-step records) of the transition from the
// chunk's last time t[n-1] to t_next, by one warp (discretize is warp-collective,
// and the same instance as k_discretize_rec's, so that the record equals the
// next chunk's record of its first step bit for bit); all zeros when t_next is
// NaN (the series ends with the chunk: no transition after it)
template <int D>
__global__ void __launch_bounds__(32) k_discretize_next(const DevModel<D> m, const double* t, int64_t n,
                                                        double t_next, double* rec, int* status) {
  const bool act = threadIdx.x == 0;
  if (isnan(t_next)) {
    for (int e = threadIdx.x; e < fqs_of<D>(); e += 32) rec[e] = 0.0;
    return;
  }
  double h = 0.0;
  int bits = 0;
  if (act) {
    h = t_next - t[n - 1];
    if (negative_nonzero(h)) bits |= PSSGP_EUNSORTED;
  }
  Mat<D> F, Q;
  discretize<D, false, true>(m, h, false, act, F, Q);
  if (act) {
    store_fq<D>(rec, 0, F, Q);
    flag(status, bits);
  }
}

// one aggregate from an entry-major array (stride st) to packed (stride 1)
__global__ void k_pack_aggregate(const double* src, int64_t st, int count, double* dst) {
  for (int e = threadIdx.x; e < count; e += blockDim.x) dst[e] = src[(int64_t)e * st];
}

// smoother outputs of step k: f = H x = H D z = z_0 (the model is built with
// H D = e_0^T), its variance, and optionally the state in SDE coordinates
template <int D>
__device__ __forceinline__ void smooth_out(const DevModel<D>& m, const ScanArgs& a, int64_t k, const Vec<D>& ms,
                                           const Mat<D>& Ps) {
  if (a.f_mean) a.f_mean[k] = ms[0];
  if (a.f_var) a.f_var[k] = Ps[0][0];
  if (a.xs) {
#pragma unroll
    for (int i = 0; i < D; ++i) a.xs[i * a.ld + k] = ms[i] * m.Dsc[i];
  }
  if (a.Ps) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) a.Ps[pidx<D>(i, j) * a.ld + k] = Ps[i][j] * (m.Dsc[i] * m.Dsc[j]);
  }
}

// smoother level 3: backward recursion through the chunk,
// m^s_k = E_k m^s_{k+1} + g_k,  P^s_k = E_k P^s_{k+1} E_k^T + L_k
template <int D>
__global__ void __launch_bounds__(BLOCK, 1) k_smoother_propagate(const DevModel<D> m, const ScanArgs a) {
  const int64_t g = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t w = g >> 5;
  const int64_t k0 = g * a.L;
  const int64_t k1 = min(k0 + a.L, a.n);
  if (k1 <= k0) return;
  Vec<D> ms;
  Mat<D> Ps;
#pragma unroll
  for (int i = 0; i < D; ++i) ms[i] = 0.0;
  set_zero<D>(Ps);
  if (w + 1 < a.P2) {
    SAgg<D> V;
    load_sagg<D>(a.wfin_s + (w + 1), a.P2, V);
#pragma unroll
    for (int i = 0; i < D; ++i) ms[i] = V.g[i];
    copy<D>(V.L, Ps);
  } else if (a.end_s) {   // a chunk of a longer series: the smoothed state after it
    SAgg<D> V;
    load_sagg<D>(a.end_s, 1, V);
#pragma unroll
    for (int i = 0; i < D; ++i) ms[i] = V.g[i];
    copy<D>(V.L, Ps);
  }
  if (lane < 31) {
    SAgg<D> S;
    load_sagg<D>(a.lagg_s + (g + 1), a.P0, S);
    Vec<D> m2;
    Mat<D> T, P2;
    mulv_add<D>(S.E, ms, S.g, m2);
    mul<D>(S.E, Ps, T);
    mul_Bt_sym_add<D>(T, S.E, S.L, P2);
#pragma unroll
    for (int i = 0; i < D; ++i) ms[i] = m2[i];
    copy<D>(P2, Ps);
  }
  // With the fused filter pass a lane's smoother chunk is the elements
  // k0-1 .. k1-2 (k0-1 .. n-1 in the lane with the series' last step), so the
  // start above is the smoothed state of step k1-1 itself, which this lane
  // writes; in a chunk of a longer series the next chunk holds element n-1
  // and the end state is the smoothed state of step n-1.  From pssgp_smooth
  // the chunk is k0 .. k1-1 and the start is step k1's.
  int64_t khi = k1 - 1;
  if (a.fuse_smoother && (k1 < a.n || a.end_s)) {
    smooth_out<D>(m, a, k1 - 1, ms, Ps);
    khi = k1 - 2;
  }
#pragma unroll 1
  for (int64_t k = khi; k >= k0; --k) {
    if (k > k0) prefetch_record<egs_of<D>()>(a.rec_egl + (k - 1) * egs_of<D>());
    Mat<D> E, Pk, Pm;
    Vec<D> g;
    load_rts<D>(a.rec_egl, k, E, g, Pk, Pm);
    Vec<D> m2;
    Mat<D> T, P2;
    mulv_add<D>(E, ms, g, m2);
    // P^s_k = P_k + E (P^s_{k+1} - P^-_{k+1}) E^T
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) { Ps[i][j] -= Pm[i][j]; Ps[j][i] = Ps[i][j]; }
    mul<D>(E, Ps, T);
    mul_Bt_sym_add<D>(T, E, Pk, P2);
#pragma unroll
    for (int i = 0; i < D; ++i) ms[i] = m2[i];
    copy<D>(P2, Ps);
    smooth_out<D>(m, a, k, ms, Ps);
  }
}

// smoother levels 0/1 from given filter outputs (pssgp_smooth): elements from
// (x_k, P_k) and the transition into k+1, folded per lane, warp suffix scan
template <int D>
__global__ void __launch_bounds__(BLOCK, 1) k_smoother_elements(const DevModel<D> m, const ScanArgs a,
                                                                const double* xf, const double* Pf) {
  const int64_t g = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t w = g >> 5;
  const int64_t k0 = g * a.L;
  const int64_t k1 = min(k0 + a.L, a.n);
  int bits = 0;
  bool bad = false;
  SAgg<D> sa;
  sagg_identity<D>(sa);
  double tcur = (k0 < a.n) ? a.t[k0] : 0.0;
#pragma unroll 1
  for (int64_t j = 0; j < a.L; ++j) {          // trip count uniform across the warp
    const int64_t k = k0 + j;
    const bool act = k < k1;
    const bool last = (k + 1 >= a.n);
    const double tn = (act && !last) ? a.t[k + 1] : tcur;
    const double h = tn - tcur;
    tcur = tn;
    if (act && !last) {
      if (nonfinite(tn)) bits |= PSSGP_ENAN;
      if (negative_nonzero(h)) bits |= PSSGP_EUNSORTED;
    }
    Mat<D> F, Q;
    discretize<D>(m, h, false, act && !last, F, Q);
    if (act) {
      Vec<D> x;
      Mat<D> P;
#pragma unroll
      for (int i = 0; i < D; ++i) x[i] = xf[i * a.ld + k] / m.Dsc[i];
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int jj = i; jj < D; ++jj) {
          P[i][jj] = Pf[pidx<D>(i, jj) * a.ld + k] / (m.Dsc[i] * m.Dsc[jj]);
          P[jj][i] = P[i][jj];
        }
      SAgg<D> e, r;
      Mat<D> Pm;
      if (!last) {
        Mat<D> T;
        Vec<D> xm;
        mulv<D>(F, x, xm);
        mul<D>(F, P, T);
        mul_Bt_sym_add<D>(T, F, Q, Pm);
        if (!smoother_element<D>(x, P, T, xm, Pm, e)) bad = true;
      } else {
        set_zero<D>(e.E);
        set_zero<D>(Pm);
#pragma unroll
        for (int i = 0; i < D; ++i) e.g[i] = x[i];
        copy<D>(P, e.L);
      }
      store_rts<D>(a.rec_egl, k, e, P, Pm);
      sagg_combine<D>(sa, e, r);
      sa = r;
    }
  }
#pragma unroll 1
  for (int off = 1; off < 32; off <<= 1) {
    SAgg<D> o = sa;
    shfl_down_sagg<D>(o, off);
    if (lane + off < 32) {
      SAgg<D> r;
      sagg_combine<D>(sa, o, r);
      sa = r;
    }
  }
  store_sagg<D>(a.lagg_s + g, a.P0, sa);
  if (lane == 0) store_sagg<D>(a.wagg_s + w, a.P2, sa);
  if (bad) bits |= PSSGP_ENOTPD;
  flag(a.status, bits);
}

// deterministic sum of the per-lane log-likelihood partials (fixed order)
// ---------------------------------------------------------------------------
// gradient (adjoint) levels 3 and 0/1, see adjoint_ops.cuh
// ---------------------------------------------------------------------------
template <int D> constexpr int adjoint_smem_doubles() { return Sym<D>::N * BLOCK; }

// per lane: the mean adjoint at the chunk end (level 3 of the mean-adjoint
// scan, from the exclusive suffix) and the covariance-adjoint chunk aggregate
// (levels 0/1: the closed form below, then a warp suffix scan)
template <int D>
__global__ void __launch_bounds__(BLOCK, 1) k_adjoint_mean(const DevModel<D> m, const ScanArgs a) {
  const int64_t g = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t w = g >> 5;
  Vec<D> mb;
#pragma unroll
  for (int i = 0; i < D; ++i) mb[i] = 0.0;
  if (w + 1 < a.P2) {
    SAgg<D> V;
    load_sagg<D>(a.wfin_s + (w + 1), a.P2, V);
#pragma unroll
    for (int i = 0; i < D; ++i) mb[i] = V.g[i];
  } else if (a.end_s) {   // a chunk of a longer series: the mean adjoint after it
#pragma unroll
    for (int i = 0; i < D; ++i) mb[i] = a.end_s[D * D + i];
  }
  if (lane < 31) {
    SAgg<D> S;
    load_sagg<D>(a.lagg_s + (g + 1), a.P0, S);
    Vec<D> t2;
    mulv_add<D>(S.E, mb, S.g, t2);
#pragma unroll
    for (int i = 0; i < D; ++i) mb[i] = t2[i];
  }
#pragma unroll
  for (int i = 0; i < D; ++i) a.lane_mbar[i * a.P0 + g] = mb[i];
  // The covariance adjoint's chunk term (Mb_{k0} = Pi Mb_{k1} Pi^T + L) in
  // closed form: L is the derivative by the predicted covariance P^- of step
  // k0 of the chunk's log-likelihood (the Gaussian integral of Sec. 3's
  // aggregate: gamma gamma^T / 2 - N^{-1} J / 2) plus that of the predicted
  // mean of step k1 through the filter gains (Pi mb_{k1} gamma^T,
  // symmetrised):
  //   L = (u gamma^T + gamma u^T) / 2 + gamma gamma^T / 2 - N^{-1} J / 2,
  //   u = Pi mb_{k1},
  // with gamma, N^{-1} J and Pi from the filter pass.  It equals the backward
  // recursion L <- A (F^T L F) A^T + B through the chunk from L = 0.
  SAgg<D> sa;
  {
    Vec<D> u, gam;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      gam[i] = a.lane_gj[i * a.P0 + g];
      double t = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        sa.E[i][j] = a.lane_pi[(i * D + j) * a.P0 + g];
        t = fma(sa.E[i][j], mb[j], t);
      }
      u[i] = t;
      sa.g[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) {
        const double l = 0.5 * (fma(u[i], gam[j], u[j] * gam[i]) + gam[i] * gam[j] -
                                a.lane_gj[(D + pidx<D>(i, j)) * a.P0 + g]);
        sa.L[i][j] = l;
        sa.L[j][i] = l;
      }
  }
#pragma unroll 1
  for (int off = 1; off < 32; off <<= 1) {
    SAgg<D> o = sa;
    shfl_down_sagg<D>(o, off);
    if (lane + off < 32) {
      SAgg<D> r;
      sagg_combine<D>(sa, o, r);
      sa = r;
    }
  }
  store_sagg<D>(a.lagg_a + g, a.P0, sa);
  if (lane == 0) store_sagg<D>(a.wagg_a + w, a.P2, sa);
}

// covariance-adjoint level 3 with the gradient accumulation; per lane (or,
// batched, per series piece) partial sums of the three derivatives
template <int D>
__global__ void __launch_bounds__(BLOCK, 1) k_adjoint_cov(const DevModel<D> m, const ScanArgs a) {
  extern __shared__ double adsm[];
  double* sM = adsm + threadIdx.x;
  const int64_t g = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int64_t w = g >> 5;
  const int64_t k0 = g * a.L;
  const int64_t k1 = min(k0 + a.L, a.n);
  {
    Mat<D> Mb;
    set_zero<D>(Mb);
    if (w + 1 < a.P2) {
      SAgg<D> V;
      load_sagg<D>(a.wfin_a + (w + 1), a.P2, V);
      copy<D>(V.L, Mb);
    } else if (a.end_s) {   // a chunk of a longer series: the covariance adjoint after it
      SAgg<D> V;
      load_sagg<D>(a.end_s, 1, V);
      copy<D>(V.L, Mb);
    }
    if (lane < 31) {
      SAgg<D> S;
      load_sagg<D>(a.lagg_a + (g + 1), a.P0, S);
      Mat<D> T, M2;
      mul<D>(S.E, Mb, T);
      mul_Bt_sym_add<D>(T, S.E, S.L, M2);
      copy<D>(M2, Mb);
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) sM[pidx<D>(i, j) * BLOCK] = Mb[i][j];
  }
  Vec<D> mb;
#pragma unroll
  for (int i = 0; i < D; ++i) mb[i] = a.lane_mbar[i * a.P0 + g];
  const double R0 = a.R[0];
  double gl = 0.0, gs = 0.0, gr = 0.0;
#pragma unroll 1
  for (int64_t k = k1 - 1; k >= k0; --k) {
    Vec<D> xb, xm, c0, K;
    double v, Si, kx = 0.0, kPk;
    {
      Mat<D> F1;
      if (k + 1 < a.n) load_F<D>(a.rec_fq, k + 1, fqs_of<D>(), F1);
      else if (a.f_next) load_F<D>(a.f_next, 0, fqs_of<D>(), F1);   // the series goes on in a next chunk
      else set_zero<D>(F1);
#pragma unroll
      for (int i = 0; i < D; ++i) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < D; ++j) s = fma(F1[j][i], mb[j], s);
        xb[i] = s;
      }
      load_adj_col0<D>(a.rec_adj, k, xm, c0, v, Si);
#pragma unroll
      for (int i = 0; i < D; ++i) { K[i] = c0[i] * Si; kx = fma(K[i], xb[i], kx); }
      const double vSi0 = v * Si;
      kPk = adj_cov_step<D, BLOCK>(sM, F1, K, vSi0, -0.5 * fma(-vSi0, vSi0, Si), xb, kx);
    }
    const double vSi = v * Si;
    const double c = -0.5 * fma(-vSi, vSi, Si);
#pragma unroll
    for (int i = 0; i < D; ++i) mb[i] = xb[i];
    mb[0] += vSi - kx;
    // sM = Mb_k, mb = mb_k: the step's contributions
    gs += adj_trace_smem_rec<D, BLOCK>(sM, a.rec_fq + k * fqs_of<D>() + D * D);
    // no branches (one basic block per step): on a missing step K, v/S and c
    // are 0, so the noise term is 0; tau = 0 (a series' first step or a
    // zero-length step) makes the lengthscale term 0
    gr = fma(kPk - vSi * kx + c, a.R_per_step ? a.R[k] : R0, gr);
    const double tau = a.tauq[2 * k];
    {
      const double q = a.tauq[2 * k + 1];
      Mat<D> Mk, Mbk;
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) {
          Mk[i][j] = load_adj_M<D>(a.rec_adj, k, i, j);
          Mk[j][i] = Mk[i][j];
          Mbk[i][j] = sM[pidx<D>(i, j) * BLOCK];
          Mbk[j][i] = Mbk[i][j];
        }
      // t1 = mb^T G m, t2 = tr(Mb G M) = sum_il G_il (M Mb)_li, t3 = tr(Mb W)
      double t1 = 0.0, t2 = 0.0, t3 = 0.0;
      if (m.companion) {
#pragma unroll
        for (int i = 0; i + 1 < D; ++i) {
          const double gi = m.fc[i * D + i + 1][1];
          t1 = fma(mb[i] * gi, xm[i + 1], t1);
          double s = 0.0;
#pragma unroll
          for (int c2 = 0; c2 < D; ++c2) s = fma(Mk[i + 1][c2], Mbk[c2][i], s);
          t2 = fma(gi, s, t2);
        }
#pragma unroll
        for (int l = 0; l < D; ++l) {
          const double gl_ = m.fc[(D - 1) * D + l][1];
          t1 = fma(mb[D - 1] * gl_, xm[l], t1);
          double s = 0.0;
#pragma unroll
          for (int c2 = 0; c2 < D; ++c2) s = fma(Mk[l][c2], Mbk[c2][D - 1], s);
          t2 = fma(gl_, s, t2);
        }
      } else {
#pragma unroll
        for (int i = 0; i < D; ++i)
#pragma unroll
          for (int l = 0; l < D; ++l) {
            const double gil = m.fc[i * D + l][1];
            t1 = fma(mb[i] * gil, xm[l], t1);
            double s = 0.0;
#pragma unroll
            for (int c2 = 0; c2 < D; ++c2) s = fma(Mk[l][c2], Mbk[c2][i], s);
            t2 = fma(gil, s, t2);
          }
      }
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = i; j < D; ++j) {
          const double p = Mbk[i][j] * m.qc[pidx<D>(i, j)][0];
          t3 = (i == j) ? t3 + p : fma(2.0, p, t3);
        }
      gl = fma(-tau, fma(2.0, t2, fma(q, t3, t1)), gl);
    }
    if (a.g_step && ((k == k0) || a.seg_start[k])) {   // batched: one piece per (chunk, series),
      a.g_step[k] = gl;                                   // at its first step in the chunk
      a.g_step[a.n + k] = gs;
      a.g_step[2 * a.n + k] = gr;
      gl = 0.0; gs = 0.0; gr = 0.0;
    }
  }
  if (!a.g_step) {
    a.gpart[g] = gl;
    a.gpart[a.P0 + g] = gs;
    a.gpart[2 * a.P0 + g] = gr;
  }
}

__global__ void __launch_bounds__(256) k_loglik_reduce(const double* llp, int64_t P0, double* out) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < P0; i += 256) s += llp[i];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sm[threadIdx.x] += sm[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// standalone discretisation, one thread per step, SDE coordinates out
template <int D>
__global__ void __launch_bounds__(BLOCK) k_discretize(const DevModel<D> m, const double* t, int64_t n, double* Fo,
                                                      double* Qo, int64_t ld, int* status) {
  const int64_t k = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const bool act = k < n;
  const bool first = (k == 0);
  double h = 0.0;
  int bits = 0;
  if (act && !first) {
    const double t1 = t[k], t0 = t[k - 1];
    h = t1 - t0;
    if (nonfinite(t1) || nonfinite(t0)) bits |= PSSGP_ENAN;
    if (negative_nonzero(h)) bits |= PSSGP_EUNSORTED;
  }
  Mat<D> F, Q;
  discretize<D>(m, h, first, act, F, Q);
  if (act) {
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) Fo[(i * D + j) * ld + k] = F[i][j] * (m.Dsc[i] / m.Dsc[j]);
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = i; j < D; ++j) Qo[pidx<D>(i, j) * ld + k] = Q[i][j] * (m.Dsc[i] * m.Dsc[j]);
  }
  flag(status, bits);
}

// ---------------------------------------------------------------------------
// merge (Sec. 4.3): merge-path partition + sequential merge per thread
// ---------------------------------------------------------------------------
// order-preserving integer key of a double (compares on the integer pipe)
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
constexpr int MERGE_ITEMS = 8;

__global__ void __launch_bounds__(BLOCK) k_merge(const double* A, const double* yA, int64_t N, const double* B,
                                                 int64_t M, double* t, double* y, uint8_t* mask, int64_t* tpos,
                                                 int* status) {
  const int64_t tid = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  const int64_t total = N + M;
  const int64_t d0 = tid * MERGE_ITEMS;
  if (d0 >= total) return;
  // split of diagonal d0: the largest i (taken from A) with A[i-1] <= B[d0-i]
  int64_t lo = max((int64_t)0, d0 - M), hi = min(d0, N);
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (okey(A[mid]) <= okey(B[d0 - mid - 1])) lo = mid + 1; else hi = mid;
  }
  int64_t i = lo, j = d0 - lo;
  int bits = 0;
  for (int it = 0; it < MERGE_ITEMS; ++it) {
    const int64_t o = d0 + it;
    if (o >= total) break;
    const bool takeA = (i < N) && (j >= M || okey(A[i]) <= okey(B[j]));
    if (takeA) {
      const double v = A[i];
      if (nonfinite(v)) bits |= PSSGP_ENAN;
      if (i + 1 < N && okey(A[i + 1]) < okey(v)) bits |= PSSGP_EUNSORTED;
      t[o] = v;
      y[o] = yA[i];
      mask[o] = 1;
      ++i;
    } else {
      const double v = B[j];
      if (nonfinite(v)) bits |= PSSGP_ENAN;
      if (j + 1 < M && okey(B[j + 1]) < okey(v)) bits |= PSSGP_EUNSORTED;
      t[o] = v;
      y[o] = 0.0;
      mask[o] = 0;
      tpos[j] = o;
      ++j;
    }
  }
  flag(status, bits);
}

__global__ void k_gather(const double* src_m, const double* src_v, const int64_t* pos, int64_t M, double* om,
                         double* ov) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int64_t p = pos[j];
  om[j] = src_m[p];
  ov[j] = src_v[p];
}

// ---------------------------------------------------------------------------
// batched prediction: B series, series s with training times/values
// [toff_s, toff_{s+1}) and prediction times [uoff_s, uoff_{s+1}); merged
// series s occupies [toff_s + uoff_s, toff_{s+1} + uoff_{s+1}) (Sec. 4.3 per
// series: prediction times as missing measurements)
// ---------------------------------------------------------------------------
__global__ void k_merged_offsets(const int64_t* toff, const int64_t* uoff, int B, int64_t* mo) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s <= B) mo[s] = toff[s] + uoff[s];
}

// each element's merged position by its rank within its series (training
// before prediction at equal times, as k_merge): a training time goes after
// the prediction times strictly before it, a prediction time after the
// training times at or before it.  Positions stay inside the series' range;
// an element whose series range is invalid is not written (PSSGP_EBATCH).
// Non-finite or decreasing times flag the series (sf at its first merged
// step; its outputs become NaN).
__global__ void __launch_bounds__(BLOCK) k_merge_batched(const int64_t* toff, const int64_t* uoff, int B,
                                                         const double* A, const double* yA, int64_t N,
                                                         const double* Bt, int64_t M, double* t, double* y,
                                                         uint8_t* mask, int64_t* tpos, int* sf, int* status) {
  const int64_t idx = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
  if (idx >= N + M) return;
  const bool train = idx < N;
  const int64_t e = train ? idx : idx - N;
  const int64_t* off = train ? toff : uoff;
  int lo = 0, hi = B;                      // last s with off[s] <= e
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid;
  }
  const int s = lo;
  const int64_t a0 = toff[s], a1 = toff[s + 1], b0 = uoff[s], b1 = uoff[s + 1];
  if (!(a0 >= 0 && a0 <= a1 && a1 <= N && b0 >= 0 && b0 <= b1 && b1 <= M) ||
      !(train ? (a0 <= e && e < a1) : (b0 <= e && e < b1))) {
    flag(status, PSSGP_EBATCH);
    return;
  }
  const int64_t base = a0 + b0;
  const double v = train ? A[e] : Bt[e];
  const long long kv = okey(v);
  int64_t pos;
  if (train) {
    int64_t l = b0, h = b1;
    while (l < h) {
      const int64_t m = (l + h) >> 1;
      if (okey(Bt[m]) < kv) l = m + 1; else h = m;
    }
    pos = base + (e - a0) + (l - b0);
  } else {
    int64_t l = a0, h = a1;
    while (l < h) {
      const int64_t m = (l + h) >> 1;
      if (okey(A[m]) <= kv) l = m + 1; else h = m;
    }
    pos = base + (e - b0) + (l - a0);
  }
  int bits = 0;
  if (nonfinite(v)) bits |= PSSGP_ENAN;
  const int64_t eend = train ? a1 : b1;
  if (e + 1 < eend && okey((train ? A : Bt)[e + 1]) < kv) bits |= PSSGP_EUNSORTED;
  t[pos] = v;
  y[pos] = train ? yA[e] : 0.0;
  mask[pos] = train ? 1 : 0;
  if (!train) tpos[e] = pos;
  if (bits) {
    atomicOr(sf + base, bits);
    flag(status, bits);
  }
}

// outputs at the prediction times; NaN for the prediction times of a flagged series
__global__ void k_gather_batched(const double* src_m, const double* src_v, const int64_t* pos,
                                 const int64_t* uoff, const int64_t* mo, int B, const int* sf, int64_t M,
                                 double* om, double* ov) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= M) return;
  int lo = 0, hi = B;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (uoff[mid] <= j) lo = mid; else hi = mid;
  }
  const bool bad = sf[mo[lo]] != 0;
  const int64_t p = pos[j];
  om[j] = bad ? NAN : src_m[p];
  ov[j] = bad ? NAN : src_v[p];
}

// FP64 FMA rate probe: four independent dependent chains per thread
__global__ void k_dfma_probe(double* out, int iters) {
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * 1e-3 + j;
  const double c = 0.999999, dd = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], c, dd);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
int cuda_rc(cudaError_t e) { return e == cudaSuccess ? PSSGP_OK : PSSGP_ECUDA; }

char* ws_ptr(void* ws, int64_t off) { return static_cast<char*>(ws) + off; }

ScanArgs base_args(const Plan& p, void* ws) {
  ScanArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n = p.n;
  a.L = p.L;
  a.P0 = p.P0;
  a.P2 = p.P2;
  a.rec_fq = reinterpret_cast<double*>(ws_ptr(ws, p.o_fq));
  a.rec_egl = reinterpret_cast<double*>(ws_ptr(ws, p.o_egl));
  a.lagg_f = reinterpret_cast<double*>(ws_ptr(ws, p.o_laggf));
  a.wagg_f = reinterpret_cast<double*>(ws_ptr(ws, p.o_waggf));
  a.lagg_s = reinterpret_cast<double*>(ws_ptr(ws, p.o_laggs));
  a.lane_ll = a.lagg_s;   // [1 + d + d(d+1)/2][P0] fits in the smoother's [ns][P0], unused without a smoother
  // [ns][P0]: written by k_filter_reduce, read by each k_filter_propagate thread
  // from its own slot before it writes its smoother aggregate there
  a.lane_fp = a.lagg_s;
  a.wagg_s = reinterpret_cast<double*>(ws_ptr(ws, p.o_waggs));
  a.llp = reinterpret_cast<double*>(ws_ptr(ws, p.o_llp));
  a.status = reinterpret_cast<int*>(ws_ptr(ws, p.o_status));
  a.t_prev = a.t_next = NAN;
  if (p.o_adj >= 0) {
    a.rec_adj = reinterpret_cast<double*>(ws_ptr(ws, p.o_adj));
    a.tauq = reinterpret_cast<double*>(ws_ptr(ws, p.o_tauq));
    a.lane_pi = reinterpret_cast<double*>(ws_ptr(ws, p.o_lpi));
    a.lane_mbar = reinterpret_cast<double*>(ws_ptr(ws, p.o_lmbar));
    a.lane_gj = reinterpret_cast<double*>(ws_ptr(ws, p.o_lgj));
    a.gpart = reinterpret_cast<double*>(ws_ptr(ws, p.o_gpart));
    a.lagg_a = a.lagg_f;     // the filter aggregates are dead once the filter pass is done
    a.wagg_a = a.wagg_f;
  }
  return a;
}

// a level-2 round, launched so that it may be scheduled while the grid
// before it drains (programmatic dependent launch; the kernels start with
// griddepcontrol.wait, so nothing is read before that grid has finished)
template <typename... KArgs, typename... Args>
void level2_launch(void (*kern)(KArgs...), int grid, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(BLOCK);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// level-2 rounds; returns the buffer that holds the final inclusive result
template <int D>
const double* run_filter_level2(const Plan& p, double* buf0, int* status, cudaStream_t s) {
  double* in = buf0;
  double* out = buf0 + p.P2 * p.nf;
  const int grid = (int)((p.P2 + BLOCK / 32 - 1) / (BLOCK / 32));
  for (int64_t off = 1; off < p.P2; off <<= 1) {
    Timed tm(s, T_FL2);
    level2_launch(k_filter_ks<D>, grid, s, (const double*)in, out, p.P2, off, status);
    after_launch();
    std::swap(in, out);
  }
  return in;
}
template <int D>
const double* run_smoother_level2(const Plan& p, double* buf0, cudaStream_t s) {
  double* in = buf0;
  double* out = buf0 + p.P2 * p.ns;
  const int grid = (int)((p.P2 + BLOCK / 32 - 1) / (BLOCK / 32));
  for (int64_t off = 1; off < p.P2; off <<= 1) {
    Timed tm(s, T_SL2);
    level2_launch(k_smoother_ks<D>, grid, s, (const double*)in, out, p.P2, off);
    after_launch();
    std::swap(in, out);
  }
  return in;
}

// a batch of series sharing one model (pssgp_loglik_batched)
struct BatchArgs {
  double ell0, var0;        // hyperparameters the model was built at
  const int64_t* offsets;   // [B + 1]
  int B;
  const double* params;     // [B][3]
  double* Rstep;
  uint8_t* seg;
  double* su;               // [n] each: (uscale, qscale, R) of every series at its first step
  double* sq;
  double* sr;
  int* sf;                  // [n]: error bits of every series at its first step (0: the series is fine)
  bool scales_ready = false;  // the per-series table is already made (k_series_scales ran)
};

// the buffer that holds the final level-2 result: the rounds alternate
// between the two halves of the warp-aggregate array
const double* level2_result(const Plan& p, double* buf0, int nagg) {
  int rounds = 0;
  for (int64_t off = 1; off < p.P2; off <<= 1) ++rounds;
  return (rounds & 1) ? buf0 + p.P2 * nagg : buf0;
}

// ll_only: the log-likelihood alone (reduce with the zero-start terms, level
// 2, k_filter_llfinish) instead of the propagate pass.  run_filter_front:
// discretisation, levels 0-1 and level 2; run_filter_back: level 3.
template <int D>
void run_filter_front(const DevModel<D>& m, const Plan& p, ScanArgs& a, cudaStream_t s, const BatchArgs* bt,
                      bool ll_only) {
  const int grid = (int)(p.P0 / BLOCK);
  if (bt && !bt->scales_ready) {
    Timed tm(s, T_DISC);
    k_series_scales<<<(unsigned)((bt->B + 127) / 128), 128, 0, s>>>(bt->ell0, bt->var0, bt->offsets, bt->B,
                                                                     bt->params, p.n, bt->su, bt->sq, bt->sr,
                                                                     bt->sf, a.status);
    after_launch();
  }
  {
    Timed tm(s, T_DISC);
    constexpr int dsmem = DISC_BLOCK * fqs_of<D>() * 8;
    // opt in to > 48 KB of dynamic shared memory (per device; cheap host call)
    if (!bt) {
      cudaFuncSetAttribute(k_discretize_rec<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem);
      k_discretize_rec<D><<<(unsigned)((p.n + DISC_BLOCK - 1) / DISC_BLOCK), DISC_BLOCK, dsmem, s>>>(
          m, a.t, p.n, a.rec_fq, a.tauq, a.status, a.t_prev);
    } else {
      cudaFuncSetAttribute(k_discretize_batched<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsmem);
      const int64_t thr = std::max<int64_t>(p.n, (int64_t)bt->B + 1);
      k_discretize_batched<D><<<(unsigned)((thr + DISC_BLOCK - 1) / DISC_BLOCK), DISC_BLOCK, dsmem, s>>>(
          m, bt->offsets, bt->B, bt->su, bt->sq, bt->sr, a.t, p.n, a.rec_fq, bt->Rstep, bt->seg, a.tauq,
          a.y, a.mask, bt->sf, a.status);
    }
    after_launch();
  }
  {
    constexpr bool L1S = l1_smem_fits<D>();
    // the prediction's instance: the shared-memory scan only when the call
    // has the whole GPU (see l1_smem_fits)
    const bool smooth_l1s = L1S && p.warps >= 4;
    auto kern = ll_only ? k_filter_reduce<D, RED_LL, L1S>
                : a.adj ? k_filter_reduce<D, RED_ADJ, L1S>
                : a.fuse_smoother ? (smooth_l1s ? k_filter_reduce<D, RED_SMOOTH, L1S>
                                                : k_filter_reduce<D, RED_SMOOTH, false>)
                                  : k_filter_reduce<D, RED_PLAIN, L1S>;
    const int smem = 8 * ((!a.adj && !ll_only && a.fuse_smoother && !smooth_l1s) ? reduce_smem_doubles<D, false>()
                                                                                   : reduce_smem_doubles<D, L1S>());
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    Timed tm(s, T_FRED);
    kern<<<grid, BLOCK, smem, s>>>(m, a);
    after_launch();
  }
  a.wfin_f = run_filter_level2<D>(p, a.wagg_f, a.status, s);
}
template <int D>
void run_filter_back(const DevModel<D>& m, const Plan& p, ScanArgs& a, cudaStream_t s, bool ll_only) {
  const int grid = (int)(p.P0 / BLOCK);
  if (ll_only) {
    Timed tm(s, T_LLC);
    k_filter_llfinish<D><<<grid, BLOCK, 0, s>>>(m, a);
    after_launch();
    return;
  }
  {
    const int psmem = 8 * (a.adj ? propagate_smem_doubles<D, PROP_ADJ>()
                           : a.fuse_smoother ? propagate_smem_doubles<D, PROP_FUSE>()
                                             : propagate_smem_doubles<D, PROP_PLAIN>());
    auto kern = a.adj ? k_filter_propagate<D, PROP_ADJ>
                      : a.fuse_smoother ? k_filter_propagate<D, PROP_FUSE> : k_filter_propagate<D, PROP_PLAIN>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);
    Timed tm(s, T_FPROP);
    kern<<<grid, BLOCK, psmem, s>>>(m, a);
    after_launch();
  }
}
template <int D>
void run_filter(const DevModel<D>& m, const Plan& p, ScanArgs& a, cudaStream_t s, const BatchArgs* bt = nullptr,
                bool ll_only = false) {
  run_filter_front<D>(m, p, a, s, bt, ll_only);
  run_filter_back<D>(m, p, a, s, ll_only);
}
template <int D>
void run_smoother_tail(const DevModel<D>& m, const Plan& p, ScanArgs& a, cudaStream_t s) {
  const int grid = (int)(p.P0 / BLOCK);
  a.wfin_s = run_smoother_level2<D>(p, a.wagg_s, s);
  Timed tm(s, T_SPROP);
  k_smoother_propagate<D><<<grid, BLOCK, 0, s>>>(m, a);
  after_launch();
}

// gradient: filter pass in adjoint mode, then the two backward scans
template <int D>
void run_grad(const DevModel<D>& m, const Plan& p, ScanArgs& a, cudaStream_t s, const BatchArgs* bt) {
  const int grid = (int)(p.P0 / BLOCK);
  a.adj = 1;
  a.fuse_smoother = 0;
  run_filter<D>(m, p, a, s, bt);
  {
    double* in = a.wagg_s;
    double* out = a.wagg_s + p.P2 * p.ns;
    const int g2 = (int)((p.P2 + BLOCK / 32 - 1) / (BLOCK / 32));
    for (int64_t off = 1; off < p.P2; off <<= 1) {
      Timed tm(s, T_AL2);
      level2_launch(k_smoother_ks<D>, g2, s, (const double*)in, out, p.P2, off);
      after_launch();
      std::swap(in, out);
    }
    a.wfin_s = in;
  }
  constexpr int asmem = adjoint_smem_doubles<D>() * 8;
  {
    Timed tm(s, T_AMEAN);
    k_adjoint_mean<D><<<grid, BLOCK, 0, s>>>(m, a);
    after_launch();
  }
  {
    double* in = a.wagg_a;
    double* out = a.wagg_a + p.P2 * p.ns;
    const int g2 = (int)((p.P2 + BLOCK / 32 - 1) / (BLOCK / 32));
    for (int64_t off = 1; off < p.P2; off <<= 1) {
      Timed tm(s, T_AL2);
      level2_launch(k_smoother_ks<D>, g2, s, (const double*)in, out, p.P2, off);
      after_launch();
      std::swap(in, out);
    }
    a.wfin_a = in;
  }
  {
    cudaFuncSetAttribute(k_adjoint_cov<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, asmem);
    Timed tm(s, T_ACOV);
    k_adjoint_cov<D><<<grid, BLOCK, asmem, s>>>(m, a);
    after_launch();
  }
}

int check_ws(const Plan& p, void* ws, size_t ws_bytes) {
  if (!ws) return PSSGP_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return PSSGP_EWORKSPACE;
  if ((int64_t)ws_bytes < p.total) return PSSGP_EWORKSPACE;
  return PSSGP_OK;
}
int check_small_ws(void* ws, size_t ws_bytes) {
  if (!ws) return PSSGP_EINVAL;
  if (ws_bytes < 256 || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return PSSGP_EWORKSPACE;
  return PSSGP_OK;
}

#define PSSGP_DISPATCH(d, ...)                                   \
  switch (d) {                                                   \
    case 1: { constexpr int D = 1; __VA_ARGS__; } break;          \
    case 2: { constexpr int D = 2; __VA_ARGS__; } break;          \
    case 3: { constexpr int D = 3; __VA_ARGS__; } break;          \
    case 4: { constexpr int D = 4; __VA_ARGS__; } break;          \
    case 5: { constexpr int D = 5; __VA_ARGS__; } break;          \
    case 6: { constexpr int D = 6; __VA_ARGS__; } break;          \
    case 7: { constexpr int D = 7; __VA_ARGS__; } break;          \
    case 8: { constexpr int D = 8; __VA_ARGS__; } break;          \
    default: return PSSGP_EDIM;                                  \
  }

int filter_common(const pssgp_model* model, const double* t, const double* y, const uint8_t* mask, const double* R,
                  int32_t R_per_step, int64_t n, double* xf, double* Pf, int64_t ld, double* loglik, void* ws,
                  size_t ws_bytes, void* stream, int64_t lanes, double* dbg) {
  begin_call();
  if (!model_ok(model) || !t || !y || !mask || !R || n < 1 || n > PSSGP_NMAX) return PSSGP_EINVAL;
  if ((xf || Pf) && ld < n) return PSSGP_EINVAL;
  const Plan p = make_plan(model->d, n, lanes);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  a.t = t; a.y = y; a.mask = mask; a.R = R; a.R_per_step = R_per_step;
  a.xf = xf; a.Pf = Pf; a.ld = ld;
  a.fuse_smoother = 0;
  a.dbg_agg = dbg;
  if (cudaMemsetAsync(a.status, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  // without per-step outputs the log-likelihood needs no propagate pass
  const bool ll_only = !xf && !Pf && !dbg;
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    run_filter<D>(m, p, a, s, nullptr, ll_only);
  });
  if (loglik) {
    Timed tm(s, T_LL);
    k_loglik_reduce<<<1, 256, 0, s>>>(a.llp, p.P0, loglik);
    after_launch();
  }
  return end_call();
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" size_t pssgp_workspace_size(int32_t d, int64_t n) {
  if (d < 1 || d > PSSGP_DMAX || n < 1 || n > PSSGP_NMAX) return 0;
  return (size_t)make_plan(d, n, 0, WARPS_MAX).total;   // enough for every tuning
}

extern "C" int pssgp_get_status(void* ws, void* stream, int32_t* status) {
  if (!ws || !status) return PSSGP_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, ws, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *status = v;
  return cuda_rc(e);
}

extern "C" int pssgp_merge(const double* t_train, const double* y_train, int64_t N, const double* t_test, int64_t M,
                           double* t, double* y, uint8_t* mask, int64_t* test_pos, void* ws, size_t ws_bytes,
                           void* stream) {
  begin_call();
  if (!t_train || !y_train || !t || !y || !mask || N < 0 || M < 0 || N + M < 1 || N > PSSGP_NMAX || M > PSSGP_NMAX) return PSSGP_EINVAL;
  if (M > 0 && (!t_test || !test_pos)) return PSSGP_EINVAL;
  int rc = check_small_ws(ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* status = static_cast<int*>(ws);
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  const int64_t threads = (N + M + MERGE_ITEMS - 1) / MERGE_ITEMS;
  k_merge<<<(unsigned)((threads + BLOCK - 1) / BLOCK), BLOCK, 0, s>>>(t_train, y_train, N, t_test, M, t, y, mask,
                                                                       test_pos, status);
  after_launch();
  return end_call();
}

extern "C" int pssgp_discretize(const pssgp_model* model, const double* t, int64_t n, double* F, double* Q,
                                int64_t ld, void* ws, size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !t || !F || !Q || n < 1 || n > PSSGP_NMAX || ld < n) return PSSGP_EINVAL;
  int rc = check_small_ws(ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* status = static_cast<int*>(ws);
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  const unsigned grid = (unsigned)((n + BLOCK - 1) / BLOCK);
  PSSGP_DISPATCH(model->d, k_discretize<D><<<grid, BLOCK, 0, s>>>(dev_model<D>(model), t, n, F, Q, ld, status); after_launch());
  return end_call();
}

extern "C" int pssgp_filter(const pssgp_model* model, const double* t, const double* y, const uint8_t* mask,
                            const double* R, int32_t R_per_step, int64_t n, double* xf, double* Pf, int64_t ld,
                            double* loglik, void* ws, size_t ws_bytes, void* stream) {
  return filter_common(model, t, y, mask, R, R_per_step, n, xf, Pf, ld, loglik, ws, ws_bytes, stream, 0, nullptr);
}

extern "C" int pssgp_loglik(const pssgp_model* model, const double* t, const double* y, const uint8_t* mask,
                            const double* R, int32_t R_per_step, int64_t n, double* loglik, void* ws,
                            size_t ws_bytes, void* stream) {
  if (!loglik) return PSSGP_EINVAL;
  return filter_common(model, t, y, mask, R, R_per_step, n, nullptr, nullptr, n, loglik, ws, ws_bytes, stream, 0,
                       nullptr);
}

extern "C" int pssgp_loglik_batched(const pssgp_model* model, const int64_t* offsets, int32_t B,
                                    const double* params, const double* t, const double* y, const uint8_t* mask,
                                    int64_t n, double* loglik, void* ws, size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !offsets || !params || !t || !y || !mask || !loglik || B < 1 || n < 1 || n > PSSGP_NMAX)
    return PSSGP_EINVAL;
  const double ell0 = model->lengthscale, var0 = model->variance;
  if (!(ell0 > 0.0) || !(var0 > 0.0) || !std::isfinite(ell0) || !std::isfinite(var0)) return PSSGP_EMODEL;
  const Plan p = make_plan(model->d, n, 0);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  BatchArgs bt;
  bt.ell0 = ell0; bt.var0 = var0; bt.offsets = offsets; bt.B = B; bt.params = params;
  bt.Rstep = reinterpret_cast<double*>(ws_ptr(ws, p.o_rstep));
  bt.seg = reinterpret_cast<uint8_t*>(ws_ptr(ws, p.o_seg));
  // the smoother outputs and prediction positions are unused by the batched
  // paths: 3n doubles for the per-series table (indexed by a series' first step)
  bt.su = reinterpret_cast<double*>(ws_ptr(ws, p.o_fmean));
  bt.sq = reinterpret_cast<double*>(ws_ptr(ws, p.o_fvar));
  bt.sr = reinterpret_cast<double*>(ws_ptr(ws, p.o_tpos));
  bt.sf = reinterpret_cast<int*>(ws_ptr(ws, p.o_t));       // the merge's time array, unused here
  a.t = t; a.y = y; a.mask = mask; a.R = bt.Rstep; a.R_per_step = 1;
  a.fuse_smoother = 0;
  a.seg_start = bt.seg;
  a.ll_step = reinterpret_cast<double*>(ws_ptr(ws, p.o_llstep));
  if (cudaMemsetAsync(a.status, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    run_filter<D>(m, p, a, s, &bt, true);
  });
  {
    Timed tm(s, T_LL);
    k_segment_pieces<<<segment_grid(B), 32 * SEG_WARPS, 0, s>>>(a.ll_step, 1, n, p.L, offsets, B, loglik, 1,
                                                                bt.sf);
    after_launch();
  }
  return end_call();
}

// batched prediction: the scan plan of the merged batch (the size for every
// tuning), then the merged offsets [B + 1] and the per-series table
// (k_series_scales: uscale, qscale, R, flags at each series' first merged step)
namespace {
struct PredBatchLayout {
  int64_t o_mo, o_su, o_sq, o_sr, o_sf, total;
};
PredBatchLayout pred_batch_layout(int d, int64_t n, int B) {
  PredBatchLayout l;
  int64_t o = make_plan(d, n, 0, WARPS_MAX).total;
  l.o_mo = o; o += align256(((int64_t)B + 1) * 8);
  l.o_su = o; o += align256(n * 8);
  l.o_sq = o; o += align256(n * 8);
  l.o_sr = o; o += align256(n * 8);
  l.o_sf = o; o += align256(n * 4);
  l.total = o;
  return l;
}
}  // namespace

extern "C" size_t pssgp_predict_batched_workspace_size(int32_t d, int64_t N, int64_t M, int32_t B) {
  if (d < 1 || d > PSSGP_DMAX || N < 0 || M < 0 || B < 1 || N + M < 1 || N + M > PSSGP_NMAX) return 0;
  return (size_t)pred_batch_layout(d, N + M, B).total;
}

extern "C" int pssgp_predict_batched(const pssgp_model* model, const int64_t* train_offsets,
                                     const int64_t* test_offsets, int32_t B, const double* params,
                                     const double* t_train, const double* y_train, int64_t N, const double* t_test,
                                     int64_t M, double* mean_test, double* var_test, double* loglik, void* ws,
                                     size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !train_offsets || !test_offsets || !params || B < 1 || N < 0 || M < 0 || N + M < 1 ||
      N + M > PSSGP_NMAX || (N > 0 && (!t_train || !y_train)) || (M > 0 && (!t_test || !mean_test || !var_test)))
    return PSSGP_EINVAL;
  const double ell0 = model->lengthscale, var0 = model->variance;
  if (!(ell0 > 0.0) || !(var0 > 0.0) || !std::isfinite(ell0) || !std::isfinite(var0)) return PSSGP_EMODEL;
  const int64_t n = N + M;
  const Plan p = make_plan(model->d, n, 0);
  const PredBatchLayout lay = pred_batch_layout(model->d, n, B);
  if (!ws) return PSSGP_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0 || (int64_t)ws_bytes < lay.total) return PSSGP_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  double* t = reinterpret_cast<double*>(ws_ptr(ws, p.o_t));
  double* y = reinterpret_cast<double*>(ws_ptr(ws, p.o_y));
  uint8_t* mask = reinterpret_cast<uint8_t*>(ws_ptr(ws, p.o_mask));
  int64_t* tpos = reinterpret_cast<int64_t*>(ws_ptr(ws, p.o_tpos));
  double* fmean = reinterpret_cast<double*>(ws_ptr(ws, p.o_fmean));
  double* fvar = reinterpret_cast<double*>(ws_ptr(ws, p.o_fvar));
  int64_t* mo = reinterpret_cast<int64_t*>(ws_ptr(ws, lay.o_mo));
  BatchArgs bt;
  bt.ell0 = ell0; bt.var0 = var0; bt.offsets = mo; bt.B = B; bt.params = params;
  bt.Rstep = reinterpret_cast<double*>(ws_ptr(ws, p.o_rstep));
  bt.seg = reinterpret_cast<uint8_t*>(ws_ptr(ws, p.o_seg));
  bt.su = reinterpret_cast<double*>(ws_ptr(ws, lay.o_su));
  bt.sq = reinterpret_cast<double*>(ws_ptr(ws, lay.o_sq));
  bt.sr = reinterpret_cast<double*>(ws_ptr(ws, lay.o_sr));
  bt.sf = reinterpret_cast<int*>(ws_ptr(ws, lay.o_sf));
  bt.scales_ready = true;
  // times and mask are cleared first: the merge leaves gaps only in a series
  // whose times are not sorted (flagged, NaN outputs), and a gap must read as
  // a missing step at time 0 (a decreasing time, which the discretisation
  // turns into a zero-length step) whatever stale bytes it held, so that
  // nothing non-finite can reach the other series
  if (cudaMemsetAsync(a.status, 0, sizeof(int), s) != cudaSuccess ||
      cudaMemsetAsync(mask, 0, (size_t)n, s) != cudaSuccess ||
      cudaMemsetAsync(t, 0, (size_t)n * 8, s) != cudaSuccess)
    return PSSGP_ECUDA;
  {
    Timed tm(s, T_MERGE);
    k_merged_offsets<<<(unsigned)((B + 1 + 255) / 256), 256, 0, s>>>(train_offsets, test_offsets, B, mo);
    after_launch();
    k_series_scales<<<(unsigned)((B + 127) / 128), 128, 0, s>>>(ell0, var0, mo, B, params, n, bt.su, bt.sq, bt.sr,
                                                                 bt.sf, a.status);
    after_launch();
    k_merge_batched<<<(unsigned)((n + BLOCK - 1) / BLOCK), BLOCK, 0, s>>>(
        train_offsets, test_offsets, B, t_train, y_train, N, t_test, M, t, y, mask, tpos, bt.sf, a.status);
    after_launch();
  }
  a.t = t; a.y = y; a.mask = mask; a.R = bt.Rstep; a.R_per_step = 1;
  a.fuse_smoother = 1;
  a.seg_start = bt.seg;
  a.ll_step = reinterpret_cast<double*>(ws_ptr(ws, p.o_llstep));
  a.f_mean = fmean; a.f_var = fvar;
  a.ld = n;
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    run_filter<D>(m, p, a, s, &bt);
    run_smoother_tail<D>(m, p, a, s);
  });
  if (M > 0) {
    Timed tm(s, T_GATHER);
    k_gather_batched<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(fmean, fvar, tpos, test_offsets, mo, B, bt.sf, M,
                                                                  mean_test, var_test);
    after_launch();
  }
  if (loglik) {
    Timed tm(s, T_LL);
    k_segment_pieces<<<segment_grid(B), 32 * SEG_WARPS, 0, s>>>(a.ll_step, 1, n, p.L, mo, B, loglik, 1, bt.sf);
    after_launch();
  }
  return end_call();
}

extern "C" size_t pssgp_workspace_size_grad(int32_t d, int64_t n) {
  if (d < 1 || d > PSSGP_DMAX || n < 1 || n > PSSGP_NMAX) return 0;
  return (size_t)make_plan(d, n, 0, WARPS_MAX, true).total;
}

extern "C" int pssgp_loglik_grad(const pssgp_model* model, const double* t, const double* y, const uint8_t* mask,
                                 const double* R, int32_t R_per_step, int64_t n, double* loglik, double* grad,
                                 void* ws, size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !t || !y || !mask || !R || !grad || n < 1 || n > PSSGP_NMAX) return PSSGP_EINVAL;
  const Plan p = make_plan(model->d, n, 0, 0, true);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  a.t = t; a.y = y; a.mask = mask; a.R = R; a.R_per_step = R_per_step;
  if (cudaMemsetAsync(a.status, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    run_grad<D>(m, p, a, s, nullptr);
  });
  {
    Timed tm(s, T_LL);
    if (loglik) {
      k_loglik_reduce<<<1, 256, 0, s>>>(a.llp, p.P0, loglik);
      after_launch();
    }
    for (int i = 0; i < 3; ++i) {
      k_loglik_reduce<<<1, 256, 0, s>>>(a.gpart + i * p.P0, p.P0, grad + i);
      after_launch();
    }
  }
  return end_call();
}

extern "C" int pssgp_loglik_grad_batched(const pssgp_model* model, const int64_t* offsets, int32_t B,
                                         const double* params, const double* t, const double* y,
                                         const uint8_t* mask, int64_t n, double* loglik, double* grad, void* ws,
                                         size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !offsets || !params || !t || !y || !mask || !grad || B < 1 || n < 1 || n > PSSGP_NMAX)
    return PSSGP_EINVAL;
  const double ell0 = model->lengthscale, var0 = model->variance;
  if (!(ell0 > 0.0) || !(var0 > 0.0) || !std::isfinite(ell0) || !std::isfinite(var0)) return PSSGP_EMODEL;
  const Plan p = make_plan(model->d, n, 0, 0, true);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  BatchArgs bt;
  bt.ell0 = ell0; bt.var0 = var0; bt.offsets = offsets; bt.B = B; bt.params = params;
  bt.Rstep = reinterpret_cast<double*>(ws_ptr(ws, p.o_rstep));
  bt.seg = reinterpret_cast<uint8_t*>(ws_ptr(ws, p.o_seg));
  // the smoother outputs and prediction positions are unused by the batched
  // paths: 3n doubles for the per-series table (indexed by a series' first step)
  bt.su = reinterpret_cast<double*>(ws_ptr(ws, p.o_fmean));
  bt.sq = reinterpret_cast<double*>(ws_ptr(ws, p.o_fvar));
  bt.sr = reinterpret_cast<double*>(ws_ptr(ws, p.o_tpos));
  bt.sf = reinterpret_cast<int*>(ws_ptr(ws, p.o_t));       // the merge's time array, unused here
  a.t = t; a.y = y; a.mask = mask; a.R = bt.Rstep; a.R_per_step = 1;
  a.seg_start = bt.seg;
  a.ll_step = reinterpret_cast<double*>(ws_ptr(ws, p.o_llstep));
  a.g_step = reinterpret_cast<double*>(ws_ptr(ws, p.o_gstep));
  if (cudaMemsetAsync(a.status, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    run_grad<D>(m, p, a, s, &bt);
  });
  {
    Timed tm(s, T_LL);
    const unsigned sg = segment_grid(B);
    if (loglik) {
      k_segment_pieces<<<sg, 32 * SEG_WARPS, 0, s>>>(a.ll_step, 1, n, p.L, offsets, B, loglik, 1, bt.sf);
      after_launch();
    }
    k_segment_pieces<<<sg, 32 * SEG_WARPS, 0, s>>>(a.g_step, 3, n, p.L, offsets, B, grad, 3, bt.sf);
    after_launch();
  }
  return end_call();
}

extern "C" int pssgp_smooth(const pssgp_model* model, const double* t, const double* xf, const double* Pf, int64_t n,
                            int64_t ld, double* f_mean, double* f_var, double* xs, double* Ps, void* ws,
                            size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !t || !xf || !Pf || n < 1 || n > PSSGP_NMAX || ld < n) return PSSGP_EINVAL;
  const Plan p = make_plan(model->d, n, 0);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  a.t = t;
  a.ld = ld;
  a.f_mean = f_mean; a.f_var = f_var; a.xs = xs; a.Ps = Ps;
  const int grid = (int)(p.P0 / BLOCK);
  if (cudaMemsetAsync(a.status, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    {
      Timed tm(s, T_SELEM);
      k_smoother_elements<D><<<grid, BLOCK, 0, s>>>(m, a, xf, Pf);
      after_launch();
    }
    run_smoother_tail<D>(m, p, a, s);
  });
  return end_call();
}

// host staging of pssgp_predict_host, after the regular workspace
namespace {
struct HostStage { int64_t o_tt, o_yy, o_ts, o_mean, o_var, o_ll, total; };
HostStage host_stage(int d, int64_t N, int64_t M) {
  HostStage h{};
  int64_t o = (int64_t)pssgp_workspace_size(d, N + M);
  auto take = [&o](int64_t bytes) { const int64_t r = o; o += (bytes + 255) / 256 * 256; return r; };
  h.o_tt = take(N * 8); h.o_yy = take(N * 8); h.o_ts = take(M * 8);
  h.o_mean = take(M * 8); h.o_var = take(M * 8); h.o_ll = take(8);
  h.total = o;
  return h;
}
}  // namespace

// ===========================================================================
// one long series split in contiguous time chunks over several GPUs
// (Sec. 3, Prop. 1 and supplement Prop. 2: the scans over chunks are scans of
// the same operators, so each chunk reduces to one aggregate, the aggregates
// are exchanged, and each chunk folds the other chunks' aggregates into its
// own scan as one element before it (filter) or after it (smoother))
// ===========================================================================
extern "C" int32_t pssgp_split_agg_doubles(int32_t d, int32_t smoother) {
  if (d < 1 || d > PSSGP_DMAX) return 0;
  const int sym = d * (d + 1) / 2;
  return smoother ? d * d + d + sym : d * d + 2 * d + 2 * sym;
}

namespace {
bool time_arg_ok(double t) { return std::isnan(t) || std::isfinite(t); }
}  // namespace

extern "C" int pssgp_split_filter_reduce(const pssgp_model* model, const double* t, const double* y,
                                         const uint8_t* mask, const double* R, int32_t R_per_step, int64_t n,
                                         double t_prev, double t_next, int32_t smoother, double* agg, void* ws,
                                         size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !t || !y || !mask || !R || !agg || n < 1 || n > PSSGP_NMAX || !time_arg_ok(t_prev) ||
      !time_arg_ok(t_next) || smoother < 0 || smoother > 2)
    return PSSGP_EINVAL;
  const bool grad = smoother == 2;
  const Plan p = make_plan(model->d, n, 0, 0, grad);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  a.t = t; a.y = y; a.mask = mask; a.R = R; a.R_per_step = R_per_step;
  a.t_prev = t_prev;
  a.t_next = t_next;
  a.fuse_smoother = smoother == 1;
  a.adj = grad;
  if (cudaMemsetAsync(a.status, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    // without the smoother the log-likelihood terms of the reduce are kept,
    // so the finishing call can take either level 3 (with or without filter
    // outputs); with it (or the gradient) the reduce saves what the fused
    // (or adjoint) pass needs
    run_filter_front<D>(m, p, a, s, nullptr, smoother == 0);
    // the chunk's aggregate: the inclusive level-2 result of the last warp
    k_pack_aggregate<<<1, 128, 0, s>>>(a.wfin_f + (p.P2 - 1), p.P2, p.nf, agg);
    after_launch();
  });
  return end_call();
}

extern "C" int pssgp_split_filter_finish(const pssgp_model* model, const double* t, const double* y,
                                         const uint8_t* mask, const double* R, int32_t R_per_step, int64_t n,
                                         double t_next, int32_t smoother, const double* aggs, int32_t G,
                                         int32_t rank, double* xf, double* Pf, int64_t ld, double* loglik, void* ws,
                                         size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !t || !y || !mask || !R || !aggs || n < 1 || n > PSSGP_NMAX || G < 1 || rank < 0 ||
      rank >= G || !time_arg_ok(t_next) || smoother < 0 || smoother > 2)
    return PSSGP_EINVAL;
  if ((xf || Pf) && ld < n) return PSSGP_EINVAL;
  const bool grad = smoother == 2;
  const Plan p = make_plan(model->d, n, 0, 0, grad);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  a.t = t; a.y = y; a.mask = mask; a.R = R; a.R_per_step = R_per_step;
  a.xf = xf; a.Pf = Pf; a.ld = ld;
  a.t_next = t_next;
  a.fuse_smoother = smoother == 1;
  a.adj = grad;
  a.wfin_f = level2_result(p, a.wagg_f, p.nf);
  const bool ll_only = smoother == 0 && !xf && !Pf;
  double* bnd = reinterpret_cast<double*>(ws_ptr(ws, p.o_bnd));
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    if (grad) {   // the transition after the chunk (zero when the series ends with it)
      k_discretize_next<D><<<1, 32, 0, s>>>(m, t, n, t_next, bnd + p.fnext, a.status);
      after_launch();
      a.f_next = bnd + p.fnext;
    }
    if (rank > 0) {   // the filter state before the chunk: chunks 0 .. rank-1 folded
      k_fold_filter_range<D><<<1, 32, 0, s>>>(aggs, 0, rank, bnd, a.status);
      after_launch();
      k_apply_filter_start<D><<<(unsigned)((p.P2 + BLOCK / 32 - 1) / (BLOCK / 32)), BLOCK, 0, s>>>(
          const_cast<double*>(a.wfin_f), p.P2, bnd, a.status);
      after_launch();
      a.start_f = bnd;
    }
    run_filter_back<D>(m, p, a, s, ll_only);
  });
  if (loglik) {
    Timed tm(s, T_LL);
    k_loglik_reduce<<<1, 256, 0, s>>>(a.llp, p.P0, loglik);
    after_launch();
  }
  return end_call();
}

extern "C" int pssgp_split_smooth_reduce(const pssgp_model* model, int64_t n, double* agg, void* ws,
                                         size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !agg || n < 1 || n > PSSGP_NMAX) return PSSGP_EINVAL;
  const Plan p = make_plan(model->d, n, 0);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  PSSGP_DISPATCH(model->d, {
    // levels 0-1 ran in the fused filter pass
    a.wfin_s = run_smoother_level2<D>(p, a.wagg_s, s);
    // the chunk's aggregate: the inclusive (suffix) level-2 result of warp 0
    k_pack_aggregate<<<1, 128, 0, s>>>(a.wfin_s, p.P2, p.ns, agg);
    after_launch();
  });
  return end_call();
}

extern "C" int pssgp_split_smooth_finish(const pssgp_model* model, int64_t n, int64_t ld, const double* aggs,
                                         int32_t G, int32_t rank, double* f_mean, double* f_var, double* xs,
                                         double* Ps, void* ws, size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !aggs || n < 1 || n > PSSGP_NMAX || ld < n || G < 1 || rank < 0 || rank >= G)
    return PSSGP_EINVAL;
  const Plan p = make_plan(model->d, n, 0);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  a.ld = ld;
  a.f_mean = f_mean; a.f_var = f_var; a.xs = xs; a.Ps = Ps;
  a.fuse_smoother = 1;
  a.wfin_s = level2_result(p, a.wagg_s, p.ns);
  double* bnd = reinterpret_cast<double*>(ws_ptr(ws, p.o_bnd));
  const int grid = (int)(p.P0 / BLOCK);
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    if (rank + 1 < G) {   // the smoothed state of the chunk's last step: chunks rank+1 .. G-1 folded
      k_fold_smoother_range<D><<<1, 32, 0, s>>>(aggs, rank + 1, G, bnd);
      after_launch();
      k_apply_smoother_end<D><<<(unsigned)((p.P2 + BLOCK / 32 - 1) / (BLOCK / 32)), BLOCK, 0, s>>>(
          const_cast<double*>(a.wfin_s), p.P2, bnd);
      after_launch();
      a.end_s = bnd;
    }
    Timed tm(s, T_SPROP);
    k_smoother_propagate<D><<<grid, BLOCK, 0, s>>>(m, a);
    after_launch();
  });
  return end_call();
}

// gradient of a split series: the two backward (adjoint) scans, each with one
// exchange of chunk aggregates (E = Pi, g, L: the smoother's operator)
extern "C" int pssgp_split_grad_mean_reduce(const pssgp_model* model, int64_t n, double* agg, void* ws,
                                            size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !agg || n < 1 || n > PSSGP_NMAX) return PSSGP_EINVAL;
  const Plan p = make_plan(model->d, n, 0, 0, true);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  PSSGP_DISPATCH(model->d, {
    // levels 0-1 of the mean-adjoint scan ran in the adjoint filter pass
    a.wfin_s = run_smoother_level2<D>(p, a.wagg_s, s);
    k_pack_aggregate<<<1, 128, 0, s>>>(a.wfin_s, p.P2, p.ns, agg);
    after_launch();
  });
  return end_call();
}

extern "C" int pssgp_split_grad_mean_finish(const pssgp_model* model, int64_t n, const double* aggs, int32_t G,
                                            int32_t rank, double* agg_cov, void* ws, size_t ws_bytes,
                                            void* stream) {
  begin_call();
  if (!model_ok(model) || !aggs || !agg_cov || n < 1 || n > PSSGP_NMAX || G < 1 || rank < 0 || rank >= G)
    return PSSGP_EINVAL;
  const Plan p = make_plan(model->d, n, 0, 0, true);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  a.wfin_s = level2_result(p, a.wagg_s, p.ns);
  double* bnd = reinterpret_cast<double*>(ws_ptr(ws, p.o_bnd));
  const int grid = (int)(p.P0 / BLOCK);
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    if (rank + 1 < G) {   // the mean adjoint after the chunk: chunks rank+1 .. G-1 folded
      k_fold_smoother_range<D><<<1, 32, 0, s>>>(aggs, rank + 1, G, bnd);
      after_launch();
      k_apply_smoother_end<D><<<(unsigned)((p.P2 + BLOCK / 32 - 1) / (BLOCK / 32)), BLOCK, 0, s>>>(
          const_cast<double*>(a.wfin_s), p.P2, bnd);
      after_launch();
      a.end_s = bnd;
    }
    {
      Timed tm(s, T_AMEAN);
      k_adjoint_mean<D><<<grid, BLOCK, 0, s>>>(m, a);
      after_launch();
    }
    // level 2 of the covariance-adjoint scan and the chunk's aggregate
    const double* wfin_a = run_smoother_level2<D>(p, a.wagg_a, s);
    k_pack_aggregate<<<1, 128, 0, s>>>(wfin_a, p.P2, p.ns, agg_cov);
    after_launch();
  });
  return end_call();
}

extern "C" int pssgp_split_grad_finish(const pssgp_model* model, const double* R, int32_t R_per_step, int64_t n,
                                       const double* aggs_cov, int32_t G, int32_t rank, double* grad, void* ws,
                                       size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !R || !aggs_cov || !grad || n < 1 || n > PSSGP_NMAX || G < 1 || rank < 0 || rank >= G)
    return PSSGP_EINVAL;
  const Plan p = make_plan(model->d, n, 0, 0, true);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  a.R = R; a.R_per_step = R_per_step;
  a.wfin_a = level2_result(p, a.wagg_a, p.ns);
  double* bnd = reinterpret_cast<double*>(ws_ptr(ws, p.o_bnd));
  a.f_next = bnd + p.fnext;   // written by the filter pass (zero after the series' last chunk)
  const int grid = (int)(p.P0 / BLOCK);
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    if (rank + 1 < G) {   // the covariance adjoint after the chunk: chunks rank+1 .. G-1 folded
      k_fold_smoother_range<D><<<1, 32, 0, s>>>(aggs_cov, rank + 1, G, bnd);
      after_launch();
      k_apply_smoother_end<D><<<(unsigned)((p.P2 + BLOCK / 32 - 1) / (BLOCK / 32)), BLOCK, 0, s>>>(
          const_cast<double*>(a.wfin_a), p.P2, bnd);
      after_launch();
      a.end_s = bnd;
    }
    constexpr int asmem = adjoint_smem_doubles<D>() * 8;
    cudaFuncSetAttribute(k_adjoint_cov<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, asmem);
    {
      Timed tm(s, T_ACOV);
      k_adjoint_cov<D><<<grid, BLOCK, asmem, s>>>(m, a);
      after_launch();
    }
  });
  {
    Timed tm(s, T_LL);
    for (int i = 0; i < 3; ++i) {
      k_loglik_reduce<<<1, 256, 0, s>>>(a.gpart + i * p.P0, p.P0, grad + i);
      after_launch();
    }
  }
  return end_call();
}

extern "C" size_t pssgp_predict_host_workspace_size(int32_t d, int64_t N, int64_t M) {
  if (d < 1 || d > PSSGP_DMAX || N < 1 || M < 0 || N > PSSGP_NMAX || M > PSSGP_NMAX) return 0;
  return (size_t)host_stage(d, N, M).total;
}

extern "C" int pssgp_predict(const pssgp_model* model, const double* t_train, const double* y_train, int64_t N,
                             const double* t_test, int64_t M, double R, double* mean_test, double* var_test,
                             double* loglik, void* ws, size_t ws_bytes, void* stream);

extern "C" int pssgp_predict_host(const pssgp_model* model, const double* t_train, const double* y_train, int64_t N,
                                  const double* t_test, int64_t M, double R, double* mean_test, double* var_test,
                                  double* loglik, void* ws, size_t ws_bytes, void* stream) {
  if (!model_ok(model) || !t_train || !y_train || N < 1 || M < 0 || N > PSSGP_NMAX || M > PSSGP_NMAX || !ws) return PSSGP_EINVAL;
  if (M > 0 && (!t_test || !mean_test || !var_test)) return PSSGP_EINVAL;
  const HostStage h = host_stage(model->d, N, M);
  if ((int64_t)ws_bytes < h.total || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return PSSGP_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  double* tt = reinterpret_cast<double*>(w + h.o_tt);
  double* yy = reinterpret_cast<double*>(w + h.o_yy);
  double* ts = reinterpret_cast<double*>(w + h.o_ts);
  double* dm = reinterpret_cast<double*>(w + h.o_mean);
  double* dv = reinterpret_cast<double*>(w + h.o_var);
  double* dl = reinterpret_cast<double*>(w + h.o_ll);
  if (cudaMemcpyAsync(tt, t_train, (size_t)N * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(yy, y_train, (size_t)N * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (M > 0 && cudaMemcpyAsync(ts, t_test, (size_t)M * 8, cudaMemcpyHostToDevice, s) != cudaSuccess))
    return PSSGP_ECUDA;
  const int rc = pssgp_predict(model, tt, yy, N, M > 0 ? ts : nullptr, M, R, M > 0 ? dm : nullptr,
                               M > 0 ? dv : nullptr, loglik ? dl : nullptr, ws, (size_t)h.o_tt, stream);
  if (rc) return rc;
  if ((M > 0 && (cudaMemcpyAsync(mean_test, dm, (size_t)M * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                 cudaMemcpyAsync(var_test, dv, (size_t)M * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)) ||
      (loglik && cudaMemcpyAsync(loglik, dl, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess))
    return PSSGP_ECUDA;
  return PSSGP_OK;
}

extern "C" int pssgp_predict(const pssgp_model* model, const double* t_train, const double* y_train, int64_t N,
                             const double* t_test, int64_t M, double R, double* mean_test, double* var_test,
                             double* loglik, void* ws, size_t ws_bytes, void* stream) {
  begin_call();
  if (!model_ok(model) || !t_train || !y_train || N < 1 || M < 0 || N > PSSGP_NMAX || M > PSSGP_NMAX) return PSSGP_EINVAL;
  if (M > 0 && (!t_test || !mean_test || !var_test)) return PSSGP_EINVAL;
  if (!(R > 0.0) || !std::isfinite(R)) return PSSGP_EINVAL;
  const int64_t n = N + M;
  const Plan p = make_plan(model->d, n, 0);
  const int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScanArgs a = base_args(p, ws);
  double* t = reinterpret_cast<double*>(ws_ptr(ws, p.o_t));
  double* y = reinterpret_cast<double*>(ws_ptr(ws, p.o_y));
  uint8_t* mask = reinterpret_cast<uint8_t*>(ws_ptr(ws, p.o_mask));
  int64_t* tpos = reinterpret_cast<int64_t*>(ws_ptr(ws, p.o_tpos));
  double* fmean = reinterpret_cast<double*>(ws_ptr(ws, p.o_fmean));
  double* fvar = reinterpret_cast<double*>(ws_ptr(ws, p.o_fvar));
  if (cudaMemsetAsync(a.status, 0, sizeof(int), s) != cudaSuccess) return PSSGP_ECUDA;
  const int64_t threads = (n + MERGE_ITEMS - 1) / MERGE_ITEMS;
  {
    Timed tm(s, T_MERGE);
    k_merge<<<(unsigned)((threads + BLOCK - 1) / BLOCK), BLOCK, 0, s>>>(t_train, y_train, N, t_test, M, t, y, mask,
                                                                         tpos, a.status);
    after_launch();
  }
  a.t = t; a.y = y; a.mask = mask; a.R = nullptr; a.R_scalar = R; a.R_per_step = 0;
  a.fuse_smoother = 1;
  a.f_mean = fmean; a.f_var = fvar;
  a.ld = n;
  PSSGP_DISPATCH(model->d, {
    const DevModel<D> m = dev_model<D>(model);
    run_filter<D>(m, p, a, s);
    run_smoother_tail<D>(m, p, a, s);
  });
  if (M > 0) {
    Timed tm(s, T_GATHER);
    k_gather<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(fmean, fvar, tpos, M, mean_test, var_test);
    after_launch();
  }
  if (loglik) {
    Timed tm(s, T_LL);
    k_loglik_reduce<<<1, 256, 0, s>>>(a.llp, p.P0, loglik);
    after_launch();
  }
  return end_call();
}

extern "C" int pssgp_debug_filter_aggregates(const pssgp_model* model, const double* t, const double* y,
                                             const uint8_t* mask, const double* R, int64_t n, int32_t lanes,
                                             double* agg, int64_t* first, int32_t* lanes_out, void* ws,
                                             size_t ws_bytes, void* stream) {
  if (!model_ok(model) || !agg || !first || !lanes_out || n < 1 || n > PSSGP_NMAX) return PSSGP_EINVAL;
  if (lanes < 0 || lanes % BLOCK) return PSSGP_EINVAL;
  const Plan p = make_plan(model->d, n, lanes);
  int rc = check_ws(p, ws, ws_bytes);
  if (rc) return rc;
  if ((int64_t)ws_bytes < p.total + p.P0 * p.nf * 8) return PSSGP_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* dbg = reinterpret_cast<double*>(ws_ptr(ws, p.total));
  rc = filter_common(model, t, y, mask, R, 0, n, nullptr, nullptr, n, nullptr, ws, ws_bytes, stream, lanes, dbg);
  if (rc) return rc;
  const int d = model->d;
  const int nfh = 3 * d * d + 2 * d;
  std::vector<double> tmp((size_t)p.P0 * p.nf);
  cudaError_t e = cudaMemcpyAsync(tmp.data(), dbg, tmp.size() * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return PSSGP_ECUDA;
  const double* Dv = model->D;
  for (int64_t c = 0; c < p.P0; ++c) {
    auto at = [&](int ent) { return tmp[(size_t)ent * p.P0 + c]; };
    double* o = agg + c * nfh;
    int ent = 0;
    // balanced -> SDE coordinates: A' = D A D^-1, b' = D b, C' = D C D,
    // eta' = D^-1 eta, J' = D^-1 J D^-1
    for (int i = 0; i < d; ++i)
      for (int j = 0; j < d; ++j) o[i * d + j] = at(ent++) * Dv[i] / Dv[j];
    for (int i = 0; i < d; ++i) o[d * d + i] = at(ent++) * Dv[i];
    for (int i = 0; i < d; ++i)
      for (int j = i; j < d; ++j) {
        const double v = at(ent++) * Dv[i] * Dv[j];
        o[d * d + d + i * d + j] = v;
        o[d * d + d + j * d + i] = v;
      }
    for (int i = 0; i < d; ++i) o[2 * d * d + d + i] = at(ent++) / Dv[i];
    for (int i = 0; i < d; ++i)
      for (int j = i; j < d; ++j) {
        const double v = at(ent++) / (Dv[i] * Dv[j]);
        o[2 * d * d + 2 * d + i * d + j] = v;
        o[2 * d * d + 2 * d + j * d + i] = v;
      }
    first[c] = std::min(c * p.L, n);
  }
  *lanes_out = (int32_t)p.P0;
  return PSSGP_OK;
}

// Best of three timed launches (after one warm-up) at each of 4, 8 and 16
// warps per SM: eight independent FMA chains per thread keep the pipe fed at
// every occupancy, and the fastest launch is the rate the FP64 pipe sustains.
extern "C" int pssgp_fp64_fma_rate(double* fma_per_s) {
  if (!fma_per_s) return PSSGP_EINVAL;
  const int sms = num_sms(), iters = 1 << 13, threads = 128;
  const int max_blocks = sms * 4;
  double* out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * max_blocks * threads) != cudaSuccess) return PSSGP_ECUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best = 0.0;
  cudaError_t e = cudaSuccess;
  for (int bps = 1; bps <= 4 && e == cudaSuccess; bps *= 2) {
    const int blocks = sms * bps;
    k_dfma_probe<<<blocks, threads>>>(out, iters);
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0);
      k_dfma_probe<<<blocks, threads>>>(out, iters * (4 / bps));
      cudaEventRecord(e1);
      e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms > 0.0f)
        best = std::max(best, (double)blocks * threads * (double)iters * (4 / bps) * 8 / (ms * 1e-3));
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || best <= 0.0) return PSSGP_ECUDA;
  *fma_per_s = best;
  return PSSGP_OK;
}

extern "C" int pssgp_timing(int32_t mode, double* ms, int64_t* counts, int32_t nslots) {
  // mode 1: enable and reset; 0: disable; 2: collect (synchronises on the
  // recorded events) into ms[slot], counts[slot]
  if (mode == 1 || mode == 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& r : g_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    g_pending.clear();
    for (int i = 0; i < TIMING_SLOTS; ++i) { g_ms[i] = 0; g_count[i] = 0; }
    g_timing = (mode == 1);
    return PSSGP_OK;
  }
  if (mode != 2 || !ms || !counts) return PSSGP_EINVAL;
  std::vector<TimingRec> pend;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    pend.swap(g_pending);
  }
  for (auto& r : pend) {
    float t = 0.0f;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return PSSGP_ECUDA;
    cudaEventElapsedTime(&t, r.a, r.b);
    g_ms[r.slot] += t;
    g_count[r.slot] += 1;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (int i = 0; i < nslots && i < TIMING_SLOTS; ++i) { ms[i] = g_ms[i]; counts[i] = g_count[i]; }
  return PSSGP_OK;
}

extern "C" const char* pssgp_timing_name(int32_t slot) {
  return (slot >= 0 && slot < TIMING_SLOTS) ? kTimingNames[slot] : "";
}

// ===========================================================================
// Allocation-free log-likelihood
//
// For callers that cannot allocate device memory themselves, e.g. a plugin
// loaded into a host program that owns every device allocation and forbids
// third-party code from calling cudaMalloc, or a latency-critical loop that
// must never enter the driver's allocator.  They cannot hand the library a
// workspace, so this entry point uses a fixed scratch array that lives in the
// library's own device image instead.  The paper has no counterpart: it is a
// deployment convenience around pssgp_loglik.
// ===========================================================================
namespace {
constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB per device, held until exit
}  // namespace

// The scratch itself.  Host code must not use this name as a device address
// (on the host it is only a stand-in); its device address is looked up with
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
// Device address of the scratch in the current device's context, looked up
// on every call with that device current (a cheap host call once the module
// is loaded; the first call on a device loads it).  Not cached, so a context
// that was torn down and created again (cudaDeviceReset) cannot leave a stale
// address behind.
int noalloc_scratch(void** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return PSSGP_ECUDA;
  *out = p;
  return PSSGP_OK;
}
}  // namespace

extern "C" int pssgp_loglik_noalloc(const pssgp_model* model, const double* t, const double* y, const uint8_t* mask,
                                    const double* R, int32_t R_per_step, int64_t n, double* loglik,
                                    int32_t* status, void* stream) {
  if (!model_ok(model) || !t || !y || !mask || !R || !loglik || n < 1 || n > PSSGP_NMAX) return PSSGP_EINVAL;
  {
    // the timing diagnostic creates CUDA events around every launch
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_timing) return PSSGP_EINVAL;
  }
  if ((size_t)make_plan(model->d, n, 0).total > kNoAllocScratchBytes) return PSSGP_ESCRATCH;
  void* ws = nullptr;
  int rc = noalloc_scratch(&ws);
  if (rc) return rc;
  // filter_common clears the status word before its kernels run; every other
  // scratch region it reads is fully written earlier in the same call.
  rc = filter_common(model, t, y, mask, R, R_per_step, n, nullptr, nullptr, n, loglik, ws, kNoAllocScratchBytes,
                     stream, 0, nullptr);
  if (rc) return rc;
  if (status) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(status, ws, sizeof(int32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess) return PSSGP_ECUDA;
  }
  return PSSGP_OK;
}

extern "C" int pssgp_set_warps_per_sm(int32_t warps_per_sm) {
  if (warps_per_sm < 1 || warps_per_sm > WARPS_MAX) return PSSGP_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int d = 0; d <= PSSGP_DMAX; ++d) g_warps_per_sm[d] = warps_per_sm;
  return PSSGP_OK;
}

extern "C" int pssgp_tune_set(int32_t d, int32_t warps_per_sm) {
  if (d < 1 || d > PSSGP_DMAX) return PSSGP_EDIM;
  if (warps_per_sm < 1 || warps_per_sm > WARPS_MAX) return PSSGP_EINVAL;
  std::lock_guard<std::mutex> lk(g_mu);
  g_warps_per_sm[d] = warps_per_sm;
  return PSSGP_OK;
}

extern "C" int pssgp_tune_get(int32_t d) {
  if (d < 1 || d > PSSGP_DMAX) return PSSGP_EDIM;
  return warps_for(d);
}

// ===========================================================================
// Autotuner: times the candidate lane counts on the caller's own problem
// ===========================================================================
extern "C" int pssgp_autotune_loglik_batched(const pssgp_model* model, const int64_t* offsets, int32_t B,
                                             const double* params, const double* t, const double* y,
                                             const uint8_t* mask, int64_t n, double* loglik, void* ws,
                                             size_t ws_bytes, void* stream, int32_t reps, int32_t* best_warps,
                                             float* best_ms) {
  if (!model_ok(model) || !best_warps || reps < 1) return PSSGP_EINVAL;
  const int d = model->d;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int saved = warps_for(d);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return PSSGP_ECUDA;
  }
  int best = saved, rc = PSSGP_OK;
  float best_t = 0.0f;
  for (int w = 4; w <= WARPS_MAX && rc == PSSGP_OK; w += 4) {
    pssgp_tune_set(d, w);
    rc = pssgp_loglik_batched(model, offsets, B, params, t, y, mask, n, loglik, ws, ws_bytes, stream);  // warm-up
    if (rc) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && rc == PSSGP_OK; ++r)
      rc = pssgp_loglik_batched(model, offsets, B, params, t, y, mask, n, loglik, ws, ws_bytes, stream);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (rc == PSSGP_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = PSSGP_ECUDA;
    ms /= (float)reps;
    if (rc == PSSGP_OK && (best_t == 0.0f || ms < best_t)) { best_t = ms; best = w; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  pssgp_tune_set(d, rc == PSSGP_OK ? best : saved);
  if (rc) return rc;
  *best_warps = best;
  if (best_ms) *best_ms = best_t;
  return PSSGP_OK;
}

// ===========================================================================
// CUDA graphs: record a sequence of library calls once, replay it with one
// launch
// ===========================================================================
struct pssgp_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" int pssgp_graph_begin(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!s) return PSSGP_EINVAL;   // the legacy default stream cannot be captured
  return cuda_rc(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
}

extern "C" int pssgp_graph_end(void* stream, pssgp_graph_s** out) {
  if (!out) return PSSGP_EINVAL;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGraph_t g = nullptr;
  if (cudaStreamEndCapture(s, &g) != cudaSuccess || !g) {
    (void)cudaGetLastError();
    return PSSGP_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    return PSSGP_ECUDA;
  }
  pssgp_graph_s* h = new pssgp_graph_s;
  h->graph = g;
  h->exec = ex;
  *out = h;
  return PSSGP_OK;
}

extern "C" int pssgp_graph_launch(pssgp_graph_s* g, void* stream) {
  if (!g || !g->exec) return PSSGP_EINVAL;
  return cuda_rc(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
}

extern "C" int pssgp_graph_destroy(pssgp_graph_s* g) {
  if (!g) return PSSGP_EINVAL;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return PSSGP_OK;
}
