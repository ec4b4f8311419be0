// pssgp_fit.cu -- batched maximum-marginal-likelihood fit of the
// hyperparameters of many independent series (the parameter estimation of
// Sec. 2, "by maximising the marginal likelihood"), driven natively on the
// device: every iteration is one pssgp_loglik_grad_batched call on the
// series still being fitted and one Adam ascent step per series; converged
// series are frozen and, every check_every iterations, removed from the
// concatenation the scans run over.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/pssgp.h"

namespace {

constexpr int FIT_BLOCK = 256;

int64_t align256(int64_t x) { return (x + 255) / 256 * 256; }

struct FitLayout {
  int64_t o_gws, gws_bytes, o_t, o_y, o_mask, o_noff, o_ooff, o_idx, o_par, o_ll, o_g, o_m, o_v, o_llp, o_cnt,
      o_done, o_lb, total;
};

FitLayout fit_layout(int d, int64_t n, int B) {
  FitLayout L{};
  int64_t o = 0;
  L.o_gws = o;
  L.gws_bytes = (int64_t)pssgp_workspace_size_grad(d, std::max<int64_t>(n, 1));
  o += align256(L.gws_bytes);
  L.o_t = o; o += align256(n * 8);
  L.o_y = o; o += align256(n * 8);
  L.o_mask = o; o += align256(n);
  L.o_noff = o; o += align256((int64_t)(B + 1) * 8);   // offsets of the compacted concatenation
  L.o_ooff = o; o += align256((int64_t)(B + 1) * 8);   // the caller's offsets, on the device
  L.o_idx = o; o += align256((int64_t)B * 4);          // compacted position -> series
  L.o_par = o; o += align256((int64_t)B * 24);
  L.o_ll = o; o += align256((int64_t)B * 8);
  L.o_g = o; o += align256((int64_t)B * 24);
  L.o_m = o; o += align256((int64_t)B * 24);           // Adam moments
  L.o_v = o; o += align256((int64_t)B * 24);
  L.o_llp = o; o += align256((int64_t)B * 8);          // previous log-likelihood
  L.o_cnt = o; o += align256((int64_t)B * 4);          // iterations in a row below tol
  L.o_done = o; o += align256((int64_t)B);
  L.o_lb = o; o += align256((int64_t)B * 512);         // L-BFGS state per series
  L.total = o;
  return L;
}

// copy the steps of the active series into the compacted arrays: the series of
// compacted step k by binary search in the new offsets
__global__ void k_fit_gather(int64_t n_new, const int64_t* noff, int Ba, const int* idx, const int64_t* ooff,
                             const double* t, const double* y, const uint8_t* mask, double* tc, double* yc,
                             uint8_t* mc) {
  const int64_t k = (int64_t)blockIdx.x * FIT_BLOCK + threadIdx.x;
  if (k >= n_new) return;
  int lo = 0, hi = Ba;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (noff[mid] <= k) lo = mid; else hi = mid;
  }
  const int64_t src = ooff[idx[lo]] + (k - noff[lo]);
  tc[k] = t[src];
  yc[k] = y[src];
  mc[k] = mask[src];
}

// parameters of the active series from theta (log values)
__global__ void k_fit_params(int Ba, const int* idx, const double* theta, double* par) {
  const int j = blockIdx.x * FIT_BLOCK + threadIdx.x;
  if (j >= Ba) return;
  const int s = idx[j];
#pragma unroll
  for (int c = 0; c < 3; ++c) par[3 * j + c] = exp(theta[3 * s + c]);
}

// one Adam ascent step per active series, with the convergence test on the
// log-likelihood just evaluated (at the current theta)
__global__ void k_fit_update(int Ba, const int* idx, const int64_t* ooff, const double* ll, const double* g,
                             double* theta, double* m1, double* m2, double* llp, int* cnt, uint8_t* done,
                             int32_t* iters, double* ll_out, double* par, int it, pssgp_fit_options o) {
  const int j = blockIdx.x * FIT_BLOCK + threadIdx.x;
  if (j >= Ba) return;
  const int s = idx[j];
  if (done[s]) return;
  const double l = ll[j];
  const double ns = fmax((double)(ooff[s + 1] - ooff[s]), 1.0);
  int c = cnt[s];
  if (it > 0) c = (fabs(l - llp[s]) / ns < o.tol) ? c + 1 : 0;
  cnt[s] = c;
  llp[s] = l;
  const bool bad = !isfinite(l) || !isfinite(g[3 * j]) || !isfinite(g[3 * j + 1]) || !isfinite(g[3 * j + 2]);
  if (c >= o.patience || it + 1 >= o.max_iter || bad) {
    done[s] = bad ? 2 : 1;
    iters[s] = it + 1;
    ll_out[s] = l;
    return;
  }
  const double b1t = 1.0 - pow(o.beta1, (double)(it + 1));
  const double b2t = 1.0 - pow(o.beta2, (double)(it + 1));
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const double gq = g[3 * j + q];
    const double a = o.beta1 * m1[3 * s + q] + (1.0 - o.beta1) * gq;
    const double b = o.beta2 * m2[3 * s + q] + (1.0 - o.beta2) * gq * gq;
    m1[3 * s + q] = a;
    m2[3 * s + q] = b;
    const double th = theta[3 * s + q] + o.lr * (a / b1t) / (sqrt(b / b2t) + o.eps);
    theta[3 * s + q] = th;
    par[3 * j + q] = exp(th);
  }
  iters[s] = it + 1;
  ll_out[s] = l;
}

// ---------------------------------------------------------------------------
// L-BFGS (limited-memory BFGS with an Armijo backtracking line search) per
// series on f = -loglik, in the log hyperparameters.  Each loop iteration
// evaluates every active series at its trial point; this kernel then either
// accepts the trial (history update, convergence test, new direction by the
// two-loop recursion, trial at step 1) or shortens the step.
// ---------------------------------------------------------------------------
constexpr int LB_M = 6;
struct LbfgsState {
  double tht[3];          // trial point
  double g[3];            // gradient of f at the accepted point
  double p[3];            // search direction
  double S[LB_M][3], Y[LB_M][3], rho[LB_M];
  double f, f0, alpha, gp0;
  int nh, head, stage, pad;
};

static_assert(sizeof(LbfgsState) <= 512, "L-BFGS state slot");

// trial parameters of the active series (the start point before the first
// evaluation)
__global__ void k_fit_params_lbfgs(int Ba, const int* idx, const double* theta, const LbfgsState* state,
                                   double* par) {
  const int j = blockIdx.x * FIT_BLOCK + threadIdx.x;
  if (j >= Ba) return;
  const int s = idx[j];
  const LbfgsState& st = state[s];
#pragma unroll
  for (int c = 0; c < 3; ++c) par[3 * j + c] = exp(st.stage ? st.tht[c] : theta[3 * s + c]);
}

__device__ void lb_direction(LbfgsState& st) {
  double q[3] = {st.g[0], st.g[1], st.g[2]}, a[LB_M];
  for (int c = 0; c < st.nh; ++c) {                  // newest to oldest
    const int i = (st.head - 1 - c + LB_M) % LB_M;
    a[i] = st.rho[i] * (st.S[i][0] * q[0] + st.S[i][1] * q[1] + st.S[i][2] * q[2]);
    for (int k = 0; k < 3; ++k) q[k] -= a[i] * st.Y[i][k];
  }
  double gam = 0.0;
  if (st.nh > 0) {
    const int i = (st.head - 1 + LB_M) % LB_M;
    const double yy = st.Y[i][0] * st.Y[i][0] + st.Y[i][1] * st.Y[i][1] + st.Y[i][2] * st.Y[i][2];
    gam = 1.0 / (st.rho[i] * yy);                    // s^T y / y^T y
  } else {
    const double gi = fmax(fabs(st.g[0]), fmax(fabs(st.g[1]), fabs(st.g[2])));
    gam = gi > 0.0 ? 0.5 / gi : 1.0;                 // first step: at most 0.5 in every log parameter
  }
  for (int k = 0; k < 3; ++k) q[k] *= gam;
  for (int c = st.nh - 1; c >= 0; --c) {             // oldest to newest
    const int i = (st.head - 1 - c + LB_M) % LB_M;
    const double b = st.rho[i] * (st.Y[i][0] * q[0] + st.Y[i][1] * q[1] + st.Y[i][2] * q[2]);
    for (int k = 0; k < 3; ++k) q[k] += st.S[i][k] * (a[i] - b);
  }
  for (int k = 0; k < 3; ++k) st.p[k] = -q[k];
  double gp = st.g[0] * st.p[0] + st.g[1] * st.p[1] + st.g[2] * st.p[2];
  if (!(gp < 0.0)) {                                 // not a descent direction: restart
    st.nh = 0;
    st.head = 0;
    const double gi = fmax(fabs(st.g[0]), fmax(fabs(st.g[1]), fabs(st.g[2])));
    for (int k = 0; k < 3; ++k) st.p[k] = gi > 0.0 ? -0.5 * st.g[k] / gi : 0.0;
  }
  const double pm = fmax(fabs(st.p[0]), fmax(fabs(st.p[1]), fabs(st.p[2])));
  if (pm > 2.0)                                      // at most a factor e^2 per step
    for (int k = 0; k < 3; ++k) st.p[k] *= 2.0 / pm;
}

__global__ void k_fit_lbfgs(int Ba, const int* idx, const int64_t* ooff, const double* ll, const double* g,
                            double* theta, LbfgsState* state, int* cnt, uint8_t* done, int32_t* iters,
                            double* ll_out, double* par, int it, pssgp_fit_options o) {
  const int j = blockIdx.x * FIT_BLOCK + threadIdx.x;
  if (j >= Ba) return;
  const int s = idx[j];
  if (done[s]) return;
  LbfgsState st = state[s];
  const double ns = fmax((double)(ooff[s + 1] - ooff[s]), 1.0);
  const double ft = -ll[j];
  const double gt[3] = {-g[3 * j], -g[3 * j + 1], -g[3 * j + 2]};
  const bool fin = isfinite(ft) && isfinite(gt[0]) && isfinite(gt[1]) && isfinite(gt[2]);
  iters[s] = it + 1;
  bool finish = false;
  if (st.stage == 0) {                               // first evaluation, at the start point
    if (!fin) { done[s] = 2; ll_out[s] = ll[j]; return; }
    for (int k = 0; k < 3; ++k) { st.tht[k] = theta[3 * s + k]; st.g[k] = gt[k]; }
    st.f = ft;
    st.nh = 0;
    st.head = 0;
    lb_direction(st);
  } else if (fin && ft <= st.f0 + 1e-4 * st.alpha * st.gp0) {   // Armijo: accept
    double sv[3], yv[3], sy = 0.0, ss = 0.0, yy = 0.0;
    for (int k = 0; k < 3; ++k) {
      sv[k] = st.tht[k] - theta[3 * s + k];
      yv[k] = gt[k] - st.g[k];
      sy += sv[k] * yv[k]; ss += sv[k] * sv[k]; yy += yv[k] * yv[k];
    }
    if (sy > 1e-12 * sqrt(ss * yy)) {
      const int h = st.head;
      for (int k = 0; k < 3; ++k) { st.S[h][k] = sv[k]; st.Y[h][k] = yv[k]; }
      st.rho[h] = 1.0 / sy;
      st.head = (h + 1) % LB_M;
      st.nh = min(st.nh + 1, LB_M);
    }
    int c = cnt[s];
    c = (fabs(ft - st.f) / ns < o.tol) ? c + 1 : 0;
    cnt[s] = c;
    for (int k = 0; k < 3; ++k) { theta[3 * s + k] = st.tht[k]; st.g[k] = gt[k]; }
    st.f = ft;
    if (c >= o.patience) finish = true;
    else lb_direction(st);
  } else {                                           // reject: shorter step
    const double a = st.alpha;
    double an = 0.5 * a;
    if (fin) {                                       // minimiser of the quadratic through f0, gp0, ft
      const double den = 2.0 * (ft - st.f0 - st.gp0 * a);
      if (den > 0.0) an = fmin(fmax(-st.gp0 * a * a / den, 0.1 * a), 0.5 * a);
    }
    if (an < 1e-10) {
      if (st.nh > 0) { st.nh = 0; st.head = 0; lb_direction(st); }   // retry along the gradient
      else finish = true;
    } else {
      st.alpha = an;
      for (int k = 0; k < 3; ++k) st.tht[k] = theta[3 * s + k] + an * st.p[k];
      for (int k = 0; k < 3; ++k) par[3 * j + k] = exp(st.tht[k]);
      if (it + 1 >= o.max_iter) finish = true;
      if (!finish) { state[s] = st; ll_out[s] = -st.f; return; }
    }
  }
  if (finish || it + 1 >= o.max_iter) {
    done[s] = 1;
    ll_out[s] = -st.f;
    state[s] = st;
    return;
  }
  // new line search along p from the accepted point
  st.stage = 1;
  st.alpha = 1.0;
  st.f0 = st.f;
  st.gp0 = st.g[0] * st.p[0] + st.g[1] * st.p[1] + st.g[2] * st.p[2];
  for (int k = 0; k < 3; ++k) {
    st.tht[k] = theta[3 * s + k] + st.p[k];
    par[3 * j + k] = exp(st.tht[k]);
  }
  state[s] = st;
  ll_out[s] = -st.f;
}

}  // namespace

extern "C" size_t pssgp_fit_workspace_size(int32_t d, int64_t n, int32_t B) {
  if (d < 1 || d > PSSGP_DMAX || n < 1 || n > PSSGP_NMAX || B < 1) return 0;
  return (size_t)fit_layout(d, n, B).total;
}

extern "C" int pssgp_fit_batched(const pssgp_model* model, const int64_t* offsets_host, int32_t B, const double* t,
                                 const double* y, const uint8_t* mask, int64_t n, double* theta, double* loglik,
                                 int32_t* iters, const pssgp_fit_options* opt, void* ws, size_t ws_bytes,
                                 void* stream, int32_t* iterations_run) {
  if (!model || !offsets_host || !t || !y || !mask || !theta || !loglik || !iters || !opt || !ws || B < 1 || n < 1 || n > PSSGP_NMAX)
    return PSSGP_EINVAL;
  if (opt->max_iter < 1 || opt->patience < 1 || opt->check_every < 1 || !(opt->lr > 0.0) || !(opt->tol >= 0.0) ||
      (opt->method != PSSGP_FIT_ADAM && opt->method != PSSGP_FIT_LBFGS))
    return PSSGP_EINVAL;
  if (offsets_host[0] != 0 || offsets_host[B] != n) return PSSGP_EINVAL;
  for (int s = 0; s < B; ++s)
    if (offsets_host[s + 1] < offsets_host[s]) return PSSGP_EINVAL;
  const FitLayout L = fit_layout(model->d, n, B);
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0 || (int64_t)ws_bytes < L.total) return PSSGP_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  void* gws = w + L.o_gws;
  double* tc = reinterpret_cast<double*>(w + L.o_t);
  double* yc = reinterpret_cast<double*>(w + L.o_y);
  uint8_t* mc = reinterpret_cast<uint8_t*>(w + L.o_mask);
  int64_t* noff = reinterpret_cast<int64_t*>(w + L.o_noff);
  int64_t* ooff = reinterpret_cast<int64_t*>(w + L.o_ooff);
  int* idx = reinterpret_cast<int*>(w + L.o_idx);
  double* par = reinterpret_cast<double*>(w + L.o_par);
  double* ll = reinterpret_cast<double*>(w + L.o_ll);
  double* g = reinterpret_cast<double*>(w + L.o_g);
  double* m1 = reinterpret_cast<double*>(w + L.o_m);
  double* m2 = reinterpret_cast<double*>(w + L.o_v);
  double* llp = reinterpret_cast<double*>(w + L.o_llp);
  int* cnt = reinterpret_cast<int*>(w + L.o_cnt);
  uint8_t* done = reinterpret_cast<uint8_t*>(w + L.o_done);
  LbfgsState* lbs = reinterpret_cast<LbfgsState*>(w + L.o_lb);
  const bool lbfgs = opt->method == PSSGP_FIT_LBFGS;

  auto ok = [](cudaError_t e) { return e == cudaSuccess; };
  if (!ok(cudaMemcpyAsync(ooff, offsets_host, (size_t)(B + 1) * 8, cudaMemcpyHostToDevice, s)) ||
      !ok(cudaMemsetAsync(m1, 0, (size_t)B * 24, s)) || !ok(cudaMemsetAsync(m2, 0, (size_t)B * 24, s)) ||
      !ok(cudaMemsetAsync(cnt, 0, (size_t)B * 4, s)) || !ok(cudaMemsetAsync(iters, 0, (size_t)B * 4, s)) ||
      !ok(cudaMemsetAsync(loglik, 0, (size_t)B * 8, s)) || !ok(cudaMemsetAsync(lbs, 0, (size_t)B * 512, s)))
    return PSSGP_ECUDA;
  // empty series are done from the start (log-likelihood 0, no iterations)
  std::vector<uint8_t> hdone(B);
  for (int q = 0; q < B; ++q) hdone[q] = (offsets_host[q + 1] == offsets_host[q]) ? 1 : 0;
  if (!ok(cudaMemcpyAsync(done, hdone.data(), (size_t)B, cudaMemcpyHostToDevice, s))) return PSSGP_ECUDA;

  std::vector<int> hidx;
  std::vector<int64_t> hnoff;
  int Ba = 0;
  int64_t n_new = 0;
  auto compact = [&]() -> int {
    hidx.clear();
    hnoff.assign(1, 0);
    for (int q = 0; q < B; ++q)
      if (!hdone[q]) {
        hidx.push_back(q);
        hnoff.push_back(hnoff.back() + (offsets_host[q + 1] - offsets_host[q]));
      }
    Ba = (int)hidx.size();
    n_new = hnoff.back();
    if (Ba == 0) return PSSGP_OK;
    // synchronous copies from pageable host memory: the vectors may change
    // before an asynchronous copy would have read them
    if (!ok(cudaStreamSynchronize(s)) ||
        !ok(cudaMemcpy(idx, hidx.data(), (size_t)Ba * 4, cudaMemcpyHostToDevice)) ||
        !ok(cudaMemcpy(noff, hnoff.data(), (size_t)(Ba + 1) * 8, cudaMemcpyHostToDevice)))
      return PSSGP_ECUDA;
    k_fit_gather<<<(unsigned)((n_new + FIT_BLOCK - 1) / FIT_BLOCK), FIT_BLOCK, 0, s>>>(n_new, noff, Ba, idx, ooff,
                                                                                       t, y, mask, tc, yc, mc);
    if (!ok(cudaGetLastError())) return PSSGP_ECUDA;
    if (lbfgs)
      k_fit_params_lbfgs<<<(unsigned)((Ba + FIT_BLOCK - 1) / FIT_BLOCK), FIT_BLOCK, 0, s>>>(Ba, idx, theta, lbs, par);
    else
      k_fit_params<<<(unsigned)((Ba + FIT_BLOCK - 1) / FIT_BLOCK), FIT_BLOCK, 0, s>>>(Ba, idx, theta, par);
    return ok(cudaGetLastError()) ? PSSGP_OK : PSSGP_ECUDA;
  };
  int rc = compact();
  if (rc) return rc;
  int it = 0;
  for (; it < opt->max_iter && Ba > 0; ++it) {
    rc = pssgp_loglik_grad_batched(model, noff, Ba, par, tc, yc, mc, n_new, ll, g, gws, (size_t)L.gws_bytes, stream);
    if (rc) return rc;
    if (lbfgs)
      k_fit_lbfgs<<<(unsigned)((Ba + FIT_BLOCK - 1) / FIT_BLOCK), FIT_BLOCK, 0, s>>>(
          Ba, idx, ooff, ll, g, theta, lbs, cnt, done, iters, loglik, par, it, *opt);
    else
      k_fit_update<<<(unsigned)((Ba + FIT_BLOCK - 1) / FIT_BLOCK), FIT_BLOCK, 0, s>>>(
          Ba, idx, ooff, ll, g, theta, m1, m2, llp, cnt, done, iters, loglik, par, it, *opt);
    if (!ok(cudaGetLastError())) return PSSGP_ECUDA;
    if ((it + 1) % opt->check_every == 0 || it + 1 == opt->max_iter) {
      std::vector<uint8_t> now(B);
      if (!ok(cudaMemcpyAsync(now.data(), done, (size_t)B, cudaMemcpyDeviceToHost, s)) ||
          !ok(cudaStreamSynchronize(s)))
        return PSSGP_ECUDA;
      int changed = 0;
      for (int q = 0; q < B; ++q)
        if (now[q] && !hdone[q]) { hdone[q] = 1; ++changed; }
      if (changed) {
        rc = compact();
        if (rc) return rc;
      }
    }
  }
  if (iterations_run) *iterations_run = it;
  return ok(cudaStreamSynchronize(s)) ? PSSGP_OK : PSSGP_ECUDA;
}
