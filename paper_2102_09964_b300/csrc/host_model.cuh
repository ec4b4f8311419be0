// host_model.cuh -- host-side conversion of a pssgp_model (pssgp.h) into the
// kernels' constant-bank model DevModel<D> (scan_ops.cuh).
#pragma once
#include <cmath>
#include <cstring>

#include "../../include/pssgp.h"
#include "scan_ops.cuh"

namespace pssgp {

template <int D>
inline DevModel<D> dev_model(const pssgp_model* pm) {
  DevModel<D> m;
  std::memset(&m, 0, sizeof(m));
  for (int i = 0; i < D; ++i)
    for (int j = i; j < D; ++j) m.Pinf[pidx<D>(i, j)] = pm->Pinf[i * D + j];
  for (int i = 0; i < D; ++i) m.Dsc[i] = pm->D[i];
  for (int e = 0; e < D * D; ++e)
    for (int t = 0; t < NT; ++t) m.fc[e][t] = pm->fc[e * PSSGP_NTAYLOR + t];
  for (int i = 0; i < D; ++i)
    for (int j = i; j < D; ++j)
      for (int t = 0; t < NT; ++t) m.qc[pidx<D>(i, j)][t] = pm->qc[(i * D + j) * PSSGP_NTAYLOR + t];
  // thresholds rounded toward zero in float so that a float step never passes a
  // bound that the double value would fail
  for (int t = 0; t <= NT; ++t) {
    m.hthr_f[t] = std::nextafter((float)pm->hthr_f[t], 0.0f);
    m.hthr_q[t] = std::nextafter((float)pm->hthr_q[t], 0.0f);
  }
  m.hmax = std::nextafter((float)pm->hmax, 0.0f);
  for (int e = 0; e < D * D; ++e)
    for (int t = 0; t < NT; ++t) m.fc32[e][t] = (float)pm->fc[e * PSSGP_NTAYLOR + t];
  for (int i = 0; i < D; ++i)
    for (int j = i; j < D; ++j)
      for (int t = 0; t < NT; ++t) m.qc32[pidx<D>(i, j)][t] = (float)pm->qc[(i * D + j) * PSSGP_NTAYLOR + t];
  for (int t = 0; t <= NT; ++t) {
    m.hthr_f32[t] = std::nextafter((float)pm->hthr_f32[t], 0.0f);
    m.hthr_q32[t] = std::nextafter((float)pm->hthr_q32[t], 0.0f);
  }
  m.companion = pm->companion;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) { m.rsup[i][j] = pm->rsup[i * D + j]; m.rlast[i][j] = pm->rlast[i * D + j]; }
  // rows 1..d-1 of Q from row 0 (companion_q_rows): companion drift and a
  // diffusion with the single entry W[d-1][d-1]
  bool rank1 = true;
  for (int e = 0; e + 1 < D * D; ++e) rank1 = rank1 && pm->W[e] == 0.0;
  m.qrows = (pm->companion && rank1 && pm->W[D * D - 1] > 0.0) ? 1 : 0;
  for (int i = 0; i + 1 < D; ++i) m.wg[i] = m.qrows ? pm->W[D * D - 1] / pm->G[i * D + i + 1] : 0.0;
  return m;
}

inline bool model_ok(const pssgp_model* pm) {
  return pm && pm->d >= 1 && pm->d <= PSSGP_DMAX && pm->hmax > 0.0 && pm->D[0] != 0.0;
}

}  // namespace pssgp
