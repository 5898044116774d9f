// Learned multiplier: network layout and launchers (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lgf_internal.h"

namespace lgf {

// 8 -> 64 -> 64 -> 64 -> 1, flat parameter layout (row-major [out][in]):
constexpr int MLP_NIN = 8, MLP_NH = 64;
constexpr int MLP_OFF_W1 = 0, MLP_OFF_B1 = 512, MLP_OFF_W2 = 576, MLP_OFF_B2 = 4672;
constexpr int MLP_OFF_W3 = 4736, MLP_OFF_B3 = 8832, MLP_OFF_W4 = 8896, MLP_OFF_B4 = 8960;
constexpr int MLP_NPARAM = 8961;
constexpr int MLP_NSTAT = 7;               // mode-log sums per (bucket, class)
constexpr float MLP_M_LO = 0.25f, MLP_M_HI = 2.0f;  // clamp of the multiplier
constexpr float MLP_ITER_SCALE = 10000.f;  // iter_frac = min(iter / 10000, 1)
constexpr int MLP_NBUCKET = 40;            // theta buckets of the mode log

// Momentum classes of a lattice: f_mu = min(k_mu, L_mu - k_mu) in [0, L/2];
// class = ((ft H2 + fz) H1 + fy) H0 + fx with H_mu = L_mu/2 + 1.
struct MlpGeom {
  int H[4];
  int off[4];      // offsets of the per-direction p2 tables
  int64_t nclass;
  float m_lo, m_hi;
  double theta_on;  // the table is applied only to steps from links with theta < theta_on
};

// bucket index of the mode log: b = clamp(4 - 2 * bucket(theta), 0, 39)
// with bucket(theta) = floor(2 log10 theta) / 2.
__host__ __device__ inline int mlp_bucket_index(double theta) {
  if (!(theta > 0.0)) return MLP_NBUCKET - 1;
  const double b = floor(2.0 * log10(theta)) * 0.5;
  int i = (int)(4.0 - 2.0 * b);
  return i < 0 ? 0 : (i >= MLP_NBUCKET ? MLP_NBUCKET - 1 : i);
}

cudaError_t launch_mlp_eval(const uint16_t* P, const float* X, int64_t n, float* out, cudaStream_t s);
// Multiplier of every momentum class for the step that starts from the
// current links (iteration k = st->iter), written to mtab + (k & 1) * nclass
// (the table of step k - 2 before: its entries turn the observed contraction
// into the plain-filter one).  snap: the two Fourier-space divergence
// snapshots [2][4][V] (BF16 pairs) that the filter passes write, slot k & 1 at step
// k; with st->snaps >= 2 the class contraction of the last step is formed
// from slots (k - 1) & 1 (divergence k - 1) and k & 1 (divergence k - 2).
// A step that redoes a rejected one, or starts from links with
// theta >= mg.theta_on, writes m = 1 (the plain filter it uses).
cudaError_t launch_mlp_multiplier(const uint16_t* P, const MlpGeom& mg, const Geom& g, const float* p2, DevState* st,
                                  float* mtab, const uint32_t* snap, cudaStream_t s);
size_t mlp_train_smem();
cudaError_t launch_mlp_grad(const float* P, const float* X, const float* Y, const float* Wt, int64_t n, int64_t batch,
                            uint64_t seed, int step, float inv_sw, float* part_g, double* part_l, int nblocks,
                            float* grad, double* loss, cudaStream_t s);
cudaError_t launch_adam(float* P, float* mom, float* vel, const float* grad, float lr, int t, cudaStream_t s);
cudaError_t launch_f32_to_bf16(const float* in, uint16_t* out, int n, cudaStream_t s);

// Per-mode statistics of consecutive Fourier-space divergences (see lgf_mlp.cu).
struct LogState {
  double theta_prev;   // theta of the links whose D^ is stored as "previous"
  double theta_prev2;  // theta one step earlier (0 if none)
  int iter_prev;
  int have_prev;
  int have_prev2;      // the divergence before "previous" is stored too
};

// Seventh feature: the last step's contraction, clamp(log10(theta/theta_prev), -2, 1)/2
// (0 when there is no previous step).
__host__ __device__ inline float mlp_rate_feature(double theta, double theta_prev) {
  if (!(theta > 0.0) || !(theta_prev > 0.0)) return 0.f;
  double r = log10(theta / theta_prev);
  r = r < -2.0 ? -2.0 : (r > 1.0 ? 1.0 : r);
  return (float)(0.5 * r);
}
// prev2 (may hold anything while ls->have_prev2 == 0): the divergence one
// step before prev, for the class contraction of the previous step.
template <typename R>
cudaError_t launch_mode_log(const Geom& g, const MlpGeom& mg, const C2<R>* cur, const C2<R>* prev,
                            const C2<R>* prev2, const LogState* ls, double* stats, cudaStream_t s);
cudaError_t launch_log_state_update(LogState* ls, const DevState* st, cudaStream_t s);

}  // namespace lgf
