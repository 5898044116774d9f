// C-ABI of the lgf library (include/lgf.h): handle management, the
// Algorithm 1 controller (arXiv:1206.0675 Sec. 2) with its loop captured in a
// CUDA graph whose WHILE node is driven by the measurement kernel, and the
// FP32 -> FP64 precision switch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lgf.h"
#include "lgf_internal.h"
#include "lgf_mem.h"
#include "lgf_mlp.h"

using namespace lgf;

namespace {

constexpr double kSU3Tol = 1e-10;       // input validation threshold

// One precision "lane" of the handle: the buffers and the captured loop graph
// of either the FP64 or the FP32 arithmetic.
template <typename R> struct Lane {
  C2<R>* U = nullptr;      // links [4][rows][3][V]
  C2<R>* U2 = nullptr;     // second link buffer (FP32 lanes)
  bool fused = false;      // update and measurement run as one kernel, links ping-pong between U and U2
  C2<R>* g = nullptr;      // gauge transform of the last step [grows][3][V]
  C2<R>* D = nullptr;      // packed divergence / FFT workspace [4][V]
  R* K = nullptr;          // filter table [V]
  C2<R>* tw = nullptr;     // twiddles
  short* pos = nullptr;    // digit-reversal position tables
  C2<R>* G = nullptr;      // accumulated transform [3][3][V] (optional)
  int rows = 3, grows = 3;
  FFTPlan plan{};
  double alpha = NAN;      // alpha the filter table holds
  int decomp = FFT_2D2D;   // decomposition of the 4D transform (lgf_set_fft_decomposition, lgf_autotune)
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  // overrelaxation loop graph and the parameters captured in it
  cudaGraphExec_t or_exec = nullptr;
  cudaGraph_t or_graph = nullptr;
  double or_omega = NAN;
  int or_check = 0;
  bool active = false;
  // learned multiplier and mode log
  float* mtab = nullptr;   // multiplier per momentum class
  float* p2f = nullptr;    // per-direction p2 tables for the network features
  MlpGeom mg{};
  C2<R>* Dlog = nullptr;   // Fourier-space divergence of the current / previous / earlier step (mode log)
  C2<R>* Dprev = nullptr;
  C2<R>* Dprev2 = nullptr;
};

// Per-kernel CUDA-event timing of lgf_step (ring of in-flight steps).
// Categories: 0 pass A, 1 pass B, 2 pass C, 3 update, 4 measure, 5 learned
// extras (undo of a rejected step, its re-measurement, network inference).
// With the 1D x 4 or 3D + 1D decompositions, category 0 holds the forward
// passes, 1 the pass with the filter and 2 the inverse passes and g.
struct TimingRing {
  // kMaxK: the longest body -- the three learned extras, the eight kernels
  // of the 1D x 4 transform and g, update and measurement (13)
  static constexpr int kSlots = 64, kMaxK = 16, kCat = 6;
  cudaEvent_t ev[kSlots][kMaxK + 1] = {};
  int cat[kSlots][kMaxK] = {};
  int nk[kSlots] = {};
  bool pending[kSlots] = {};
  int next = 0;
  double sum_ms[kCat] = {};
  long steps = 0;
  bool enabled = false;
};

}  // namespace

namespace {
// NVTX range over one library call or phase (visible in Nsight timelines;
// no cost when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

struct lgf_ctx {
  Geom geom{};
  lgf_precision prec = LGF_FP64;
  uint32_t flags = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  int device = 0;
  std::string err;
  bool broken = false;
  bool have_links = false;
  bool have_g = false;
  int phase = 64;  // arithmetic of the current configuration
  DeviceMemory mem;               // every device buffer of the handle
  Lane<double> d;
  Lane<float> f;
  double* U0 = nullptr;           // FP64 AoS copy of the input (LGF_MIXED)
  double* stage = nullptr;        // device AoS staging [4 V 18]
  double* partials = nullptr;
  DevState* st = nullptr;
  DevState* st_host = nullptr;    // pinned
  unsigned long long* defect = nullptr;
  unsigned long long* defect_host = nullptr;
  double* sin2 = nullptr;
  int lmax = 0;
  double p2max = 0;
  double* hist_F = nullptr;
  double* hist_T = nullptr;
  int* hist_flags = nullptr;
  double* hist_defect = nullptr;
  int hist_cap = 0;
  double* user_F = nullptr;
  double* user_T = nullptr;
  int32_t* user_flags = nullptr;
  double* user_defect = nullptr;
  double defect_bound64 = 1e-10;  // link unitarity defect that makes lgf_fix reunitarise (FP64 phases)
  double defect_bound32 = 1e-4;   // the same for FP32 phases
  int repairs = 0;                // reunitarisations of the links during the last lgf_fix
  TimingRing timing;
  // lgf_set_links from host memory: the copy runs in kSetChunks pieces on the
  // handle's stream and the SU(3) check of each piece on cap_stream as soon as
  // it has arrived, so that the check overlaps the copy of the next piece
  static constexpr int kSetChunks = 8;
  cudaEvent_t set_ev[kSetChunks + 1] = {};
  double switch_theta = 1e-9;     // FP32 -> FP64 switch level of LGF_MIXED
  bool learned = false;           // LGF_LEARNED
  float* mtab = nullptr;          // learned multiplier tables of even and odd steps [2][nclass]
  uint32_t* snap = nullptr;       // Fourier-space divergence snapshots of even and odd steps [2][4][V], BF16 pairs
  uint16_t* mlp_w = nullptr;      // BF16 network parameters (device)
  bool logging = false;           // per-mode statistics of every lgf_step
  bool log_primed = false;
  LogState* ls = nullptr;
  double* stats = nullptr;        // [MLP_NBUCKET][nclass][4]
};

namespace {

lgf_status fail(lgf_ctx* h, lgf_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

lgf_status fail_cuda(lgf_ctx* h, cudaError_t e, const char* what) {
  if (h) {
    h->broken = true;
    h->err = std::string(what) + ": " + cudaGetErrorString(e);
  }
  return e == cudaErrorMemoryAllocation ? LGF_E_NOMEM : LGF_E_CUDA;
}

#define LGF_CK(h, call)                                 \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return fail_cuda(h, e_, #call); \
  } while (0)

bool extent_ok(int L) {
  if (L < 2 || L > 128) return false;
  while (L % 2 == 0) L /= 2;
  while (L % 3 == 0) L /= 3;
  return L == 1;
}


template <typename R> void drop_graph(Lane<R>& L) {
  if (L.exec) cudaGraphExecDestroy(L.exec);
  if (L.graph) cudaGraphDestroy(L.graph);
  L.exec = nullptr;
  L.graph = nullptr;
}

// A new decomposition or plan invalidates the captured loop body.
template <typename R> void set_decomp(Lane<R>& L, int decomposition) {
  if (L.decomp == decomposition) return;
  drop_graph(L);
  L.decomp = decomposition;
}

template <typename R> void drop_or_graph(Lane<R>& L) {
  if (L.or_exec) cudaGraphExecDestroy(L.or_exec);
  if (L.or_graph) cudaGraphDestroy(L.or_graph);
  L.or_exec = nullptr;
  L.or_graph = nullptr;
}

template <typename R> void free_lane(lgf_ctx* h, Lane<R>& L) {
  drop_graph(L);
  drop_or_graph(L);
  for (void* p : {(void*)L.U, (void*)L.U2, (void*)L.g, (void*)L.D, (void*)L.K, (void*)L.tw, (void*)L.pos,
                  (void*)L.G, (void*)L.p2f, (void*)L.Dlog, (void*)L.Dprev, (void*)L.Dprev2})
    h->mem.put(p);
  L = Lane<R>();
}

template <typename R> lgf_status alloc_lane(lgf_ctx* h, Lane<R>& L, int rows, int grows, bool withG) {
  const int64_t V = h->geom.V;
  L.rows = rows;
  L.grows = grows;
  LGF_CK(h, h->mem.get(&L.U, (size_t)4 * rows * 3 * V));
  // FP32 lanes stream HBM in the update and the measurement: fuse them
  // (the undo of a rejected learned step then works on whichever of the two
  // link buffers holds the current links)
  if (sizeof(R) == sizeof(float)) {
    LGF_CK(h, h->mem.get(&L.U2, (size_t)4 * rows * 3 * V));
    L.fused = true;
  }
  LGF_CK(h, h->mem.get(&L.g, (size_t)grows * 3 * V));
  LGF_CK(h, h->mem.get(&L.D, (size_t)4 * V));
  LGF_CK(h, h->mem.get(&L.K, (size_t)V));
  const int nt = h->geom.L[0] + h->geom.L[1] + h->geom.L[2] + h->geom.L[3];
  LGF_CK(h, h->mem.get(&L.tw, (size_t)nt));
  if (withG) LGF_CK(h, h->mem.get(&L.G, (size_t)9 * V));
  if (configure_fft_plan(h->geom.L, (int)sizeof(R), &L.plan) != cudaSuccess)
    return fail(h, LGF_E_UNSUPPORTED, "lattice planes do not fit the shared-memory FFT passes");
  // twiddles W_N^m = exp(-2 pi i m/N), computed in FP64 on the host
  std::vector<C2<R>> tw(nt);
  int off = 0;
  for (int mu = 0; mu < 4; ++mu) {
    const int N = h->geom.L[mu];
    for (int m = 0; m < N; ++m) {
      const double a = -2.0 * M_PI * (double)m / (double)N;
      tw[off + m] = mkc<R>((R)std::cos(a), (R)std::sin(a));
    }
    off += N;
  }
  LGF_CK(h, cudaMemcpyAsync(L.tw, tw.data(), nt * sizeof(C2<R>), cudaMemcpyHostToDevice, h->stream));
  std::vector<short> pos(nt);
  fft_positions(L.plan, pos.data());
  LGF_CK(h, h->mem.get(&L.pos, (size_t)nt));
  LGF_CK(h, cudaMemcpyAsync(L.pos, pos.data(), nt * sizeof(short), cudaMemcpyHostToDevice, h->stream));
  // momentum classes and their per-direction p2 = 4 sin^2(pi f / L), f <= L/2
  std::vector<float> p2;
  L.mg.nclass = 1;
  for (int mu = 0; mu < 4; ++mu) {
    const int N = h->geom.L[mu];
    L.mg.H[mu] = N / 2 + 1;
    L.mg.off[mu] = (int)p2.size();
    L.mg.nclass *= L.mg.H[mu];
    for (int f = 0; f <= N / 2; ++f) {
      const double sv = std::sin(M_PI * (double)f / (double)N);
      p2.push_back((float)(4.0 * sv * sv));
    }
  }
  L.mg.m_lo = MLP_M_LO;
  L.mg.m_hi = MLP_M_HI;
  L.mg.theta_on = INFINITY;  // every step (lgf_set_learned_theta)
  LGF_CK(h, h->mem.get(&L.p2f, p2.size()));
  LGF_CK(h, cudaMemcpyAsync(L.p2f, p2.data(), p2.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  if (h->learned) {
    // one pair of multiplier tables and divergence snapshots per handle,
    // shared by both lanes of a mixed handle (the contraction feature spans
    // the precision switch)
    if (!h->mtab) {
      LGF_CK(h, h->mem.get(&h->mtab, (size_t)2 * L.mg.nclass));
      std::vector<float> ones((size_t)2 * L.mg.nclass, 1.f);
      LGF_CK(h, cudaMemcpyAsync(h->mtab, ones.data(), ones.size() * sizeof(float), cudaMemcpyHostToDevice,
                                h->stream));
      LGF_CK(h, cudaStreamSynchronize(h->stream));
      LGF_CK(h, h->mem.get(&h->snap, (size_t)2 * 4 * V));
    }
    L.mtab = h->mtab;
  }
  L.active = true;
  return LGF_OK;
}

// Filter table for the requested alpha (recomputed only when alpha changes).
template <typename R> lgf_status ensure_filter(lgf_ctx* h, Lane<R>& L, double alpha) {
  if (L.alpha == alpha) return LGF_OK;
  LGF_CK(h, launch_filter_table<R>(h->geom, h->sin2, h->lmax, alpha, h->p2max, (h->flags & LGF_PLAIN_SD) ? 1 : 0,
                                    L.K, h->stream));
  L.alpha = alpha;
  return LGF_OK;
}

// Measurement of the current links of a lane.
template <typename R> cudaError_t enqueue_measure(lgf_ctx* h, Lane<R>& L, int count_iter,
                                                   unsigned long long cond, int use_cond, cudaStream_t s,
                                                   int only_if_revert = 0, unsigned long long cond_undo = 0) {
  if (L.rows == 3)
    return launch_measure<R, 3>(h->geom, L.U, L.D, h->partials, h->st, count_iter, cond, use_cond, s,
                                only_if_revert, Batch(), L.U2, cond_undo);
  return launch_measure<R, 2>(h->geom, L.U, L.D, h->partials, h->st, count_iter, cond, use_cond, s, only_if_revert,
                              Batch(), L.U2, cond_undo);
}

// Gauge-transform step of a lane given the divergence in L.D (from the last
// measurement), followed by the next measurement: FFT passes A, B, C(+g),
// update, measure.
// The kernels of one body, in order, with their timing category.  Plain:
// pass A, pass B, pass C (+g), update, measure.  Learned: undo of a rejected
// step, its re-measurement and the network inference come first (each does
// nothing unless it has work), then the plain sequence with the multiplier.
// 1D x 4: forward x, y, z; forward t, filter, inverse t; inverse z, y, x; g.
// 3D + 1D: forward (x,y,z); t with the filter; inverse (x,y,z); g.
// A fused lane runs K_UM (update and measurement in one kernel) in place of
// K_UPD and K_MEAS.
enum { K_A = 0, K_B, K_C, K_UPD, K_MEAS, K_REVERT, K_RESTORE, K_MLP,
       K_F1X, K_F1Y, K_F1Z, K_T1, K_I1Z, K_I1Y, K_I1X, K_F3, K_I3, K_GD, K_UM };

constexpr int kLongestBody = 3 + 8 + 2;
static_assert(TimingRing::kMaxK >= kLongestBody, "the timing ring must hold the longest body");

// Parts of a body: the undo pair of a learned handle (undo of a rejected
// step and its re-measurement) and the rest.
enum { PART_ALL = 0, PART_UNDO = 1, PART_STEP = 2 };

// ks must hold TimingRing::kMaxK entries.
template <typename R> int body_kernels(const lgf_ctx* h, const Lane<R>& L, int* ks, int part = PART_ALL) {
  int n = 0;
  if (h->learned && part != PART_STEP) {
    ks[n++] = K_REVERT;
    ks[n++] = K_RESTORE;
  }
  if (part == PART_UNDO) return n;
  if (h->learned) ks[n++] = K_MLP;
  if (L.decomp == FFT_1D4) {
    for (int k : {K_F1X, K_F1Y, K_F1Z, K_T1, K_I1Z, K_I1Y, K_I1X, K_GD}) ks[n++] = k;
  } else if (L.decomp == FFT_3D1D) {
    for (int k : {K_F3, K_T1, K_I3, K_GD}) ks[n++] = k;
  } else {
    ks[n++] = K_A;
    ks[n++] = K_B;
    ks[n++] = K_C;
  }
  if (L.fused) {
    ks[n++] = K_UM;
  } else {
    ks[n++] = K_UPD;
    ks[n++] = K_MEAS;
  }
  return n;
}

inline int kernel_category(int k) {
  if (k <= K_MEAS) return k;
  if (k == K_UM) return K_UPD;
  if (k == K_F1X || k == K_F1Y || k == K_F1Z || k == K_F3) return 0;
  if (k == K_T1) return 1;
  if (k >= K_I1Z) return 2;
  return 5;
}

inline int exact_exp(const lgf_ctx* h) { return (h->flags & LGF_EXACT_EXP) ? 1 : 0; }

// The learned extras of the pass that carries the filter (none without LGF_LEARNED).
template <typename R> LearnedIO learned_io(const lgf_ctx* h, const Lane<R>& L) {
  LearnedIO io;
  if (!h->learned) return io;
  io.mtab = L.mtab;
  io.snap = h->snap;
  io.st = h->st;
  io.nclass = L.mg.nclass;
  return io;
}

// Passes of the 1D x 4 and 3D + 1D decompositions, and g from their output.
template <typename R> cudaError_t enqueue_alt_fft(lgf_ctx* h, Lane<R>& L, int k, cudaStream_t s) {
  const Geom& g = h->geom;
  switch (k) {
    case K_F1X: return launch_fft_line<R>(g, L.plan, 0, L.D, L.tw, L.pos, L.K, -1, 4, s);
    case K_F1Y: return launch_fft_line<R>(g, L.plan, 1, L.D, L.tw, L.pos, L.K, -1, 4, s);
    case K_F1Z: return launch_fft_line<R>(g, L.plan, 2, L.D, L.tw, L.pos, L.K, -1, 4, s);
    case K_T1: return launch_fft_line<R>(g, L.plan, 3, L.D, L.tw, L.pos, L.K, 0, 4, s, Batch(), learned_io(h, L));
    case K_I1Z: return launch_fft_line<R>(g, L.plan, 2, L.D, L.tw, L.pos, L.K, +1, 4, s);
    case K_I1Y: return launch_fft_line<R>(g, L.plan, 1, L.D, L.tw, L.pos, L.K, +1, 4, s);
    case K_I1X: return launch_fft_line<R>(g, L.plan, 0, L.D, L.tw, L.pos, L.K, +1, 4, s);
    case K_F3: return launch_fft_xyz<R>(g, L.plan, L.D, L.tw, L.pos, -1, 4, s);
    case K_I3: return launch_fft_xyz<R>(g, L.plan, L.D, L.tw, L.pos, +1, 4, s);
    default:
      if (L.grows == 3) return launch_gauge_from_delta<R, R, 3>(g, L.D, L.g, L.G, s, Batch(), exact_exp(h));
      return launch_gauge_from_delta<R, R, 2>(g, L.D, L.g, L.G, s, Batch(), exact_exp(h));
  }
}

// cond: the WHILE handle of a captured loop (use_cond != 0); cond_undo: the
// handle of the conditional node that runs the undo pair (0 = none), set by
// every counted measurement to whether its step was rejected.
template <typename R> cudaError_t enqueue_kernel(lgf_ctx* h, Lane<R>& L, int k, unsigned long long cond,
                                                  int use_cond, cudaStream_t s, unsigned long long cond_undo = 0);

template <> cudaError_t enqueue_kernel<double>(lgf_ctx* h, Lane<double>& L, int k, unsigned long long cond,
                                               int use_cond, cudaStream_t s, unsigned long long cond_undo) {
  const Geom& g = h->geom;
  switch (k) {
    case K_A: return launch_fft_xy<double>(g, L.plan, L.D, L.tw, L.pos, -1, 4, s);
    case K_B: return launch_fft_zt<double>(g, L.plan, L.D, L.tw, L.pos, L.K, 0, 4, s, learned_io(h, L));
    case K_C:
      return launch_fft_xy_inv_gauge<double, double, 3>(g, L.plan, L.D, L.tw, L.pos, L.g, L.G, s, Batch(),
                                                        exact_exp(h));
    case K_UPD:
      return L.rows == 3 ? launch_update<double, 3, 3>(g, L.U, L.g, s) : launch_update<double, 2, 3>(g, L.U, L.g, s);
    case K_MEAS: return enqueue_measure<double>(h, L, 1, cond, use_cond, s, 0, cond_undo);
    case K_REVERT:
      return L.rows == 3 ? launch_revert<double, 3, 3>(g, L.U, L.g, L.G, h->st, s, L.U2)
                         : launch_revert<double, 2, 3>(g, L.U, L.g, L.G, h->st, s, L.U2);
    case K_RESTORE: return enqueue_measure<double>(h, L, -1, 0, 0, s, 1);
    case K_MLP: return launch_mlp_multiplier(h->mlp_w, L.mg, g, L.p2f, h->st, L.mtab, h->snap, s);
    default: return enqueue_alt_fft<double>(h, L, k, s);
  }
}

template <> cudaError_t enqueue_kernel<float>(lgf_ctx* h, Lane<float>& L, int k, unsigned long long cond,
                                              int use_cond, cudaStream_t s, unsigned long long cond_undo) {
  const Geom& g = h->geom;
  switch (k) {
    case K_A: return launch_fft_xy<float>(g, L.plan, L.D, L.tw, L.pos, -1, 4, s);
    case K_B: return launch_fft_zt<float>(g, L.plan, L.D, L.tw, L.pos, L.K, 0, 4, s, learned_io(h, L));
    case K_C:
      return L.grows == 2 ? launch_fft_xy_inv_gauge<float, float, 2>(g, L.plan, L.D, L.tw, L.pos, L.g, L.G, s,
                                                                     Batch(), exact_exp(h))
                          : launch_fft_xy_inv_gauge<float, float, 3>(g, L.plan, L.D, L.tw, L.pos, L.g, L.G, s,
                                                                     Batch(), exact_exp(h));
    case K_UPD: return L.grows == 2 ? launch_update<float, 2, 2>(g, L.U, L.g, s) : launch_update<float, 3, 3>(g, L.U, L.g, s);
    case K_UM:
      return L.grows == 2
                 ? launch_update_measure<float, 2, 2>(g, L.U, L.U2, L.g, L.D, h->partials, h->st, cond, use_cond, s,
                                                      cond_undo)
                 : launch_update_measure<float, 3, 3>(g, L.U, L.U2, L.g, L.D, h->partials, h->st, cond, use_cond, s,
                                                      cond_undo);
    case K_MEAS: return enqueue_measure<float>(h, L, 1, cond, use_cond, s, 0, cond_undo);
    case K_REVERT:
      return L.grows == 2 ? launch_revert<float, 2, 2>(g, L.U, L.g, L.G, h->st, s, L.U2)
                          : launch_revert<float, 3, 3>(g, L.U, L.g, L.G, h->st, s, L.U2);
    case K_RESTORE: return enqueue_measure<float>(h, L, -1, 0, 0, s, 1);
    case K_MLP: return launch_mlp_multiplier(h->mlp_w, L.mg, g, L.p2f, h->st, L.mtab, h->snap, s);
    default: return enqueue_alt_fft<float>(h, L, k, s);
  }
}

cudaError_t timing_collect(TimingRing& T, int slot) {
  if (!T.pending[slot]) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(T.ev[slot][T.nk[slot]]);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < T.nk[slot]; ++k) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, T.ev[slot][k], T.ev[slot][k + 1]);
    if (e != cudaSuccess) return e;
    T.sum_ms[T.cat[slot][k]] += ms;
  }
  T.steps += 1;
  T.pending[slot] = false;
  return cudaSuccess;
}

// Gauge-transform step of a lane given the divergence in L.D (from the last
// measurement), followed by the next measurement: FFT passes A, B, C(+g),
// update, measure.  With timing enabled (and outside graph capture) every
// kernel is bracketed by CUDA events on the launching stream.
template <typename R> cudaError_t enqueue_body(lgf_ctx* h, Lane<R>& L, unsigned long long cond, int use_cond,
                                                cudaStream_t s, int part = PART_ALL,
                                                unsigned long long cond_undo = 0) {
  TimingRing& T = h->timing;
  const bool timed = T.enabled && !use_cond;
  int slot = 0;
  cudaError_t e;
  if (timed) {
    slot = T.next;
    T.next = (T.next + 1) % TimingRing::kSlots;
    if ((e = timing_collect(T, slot)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(T.ev[slot][0], s)) != cudaSuccess) return e;
  }
  int ks[TimingRing::kMaxK];
  const int nk = body_kernels<R>(h, L, ks, part);
  for (int i = 0; i < nk; ++i) {
    if ((e = enqueue_kernel<R>(h, L, ks[i], cond, use_cond, s, cond_undo)) != cudaSuccess) return e;
    if (timed) {
      T.cat[slot][i] = kernel_category(ks[i]);
      if ((e = cudaEventRecord(T.ev[slot][i + 1], s)) != cudaSuccess) return e;
    }
  }
  if (timed) {
    T.nk[slot] = nk;
    T.pending[slot] = true;
  }
  return cudaSuccess;
}

// Build (once) the graph  WHILE(cond) { body }  for a lane.
template <typename R> lgf_status ensure_graph(lgf_ctx* h, Lane<R>& L) {
  if (L.exec) return LGF_OK;
  cudaGraph_t graph;
  LGF_CK(h, cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  LGF_CK(h, cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  LGF_CK(h, cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  // Learned handles: the undo pair sits in an IF node at the top of the body,
  // taken only after a rejected step (the measurement sets its handle), so
  // that accepted steps launch neither kernel.
  cudaGraphNode_t undo_node = nullptr;
  unsigned long long undo_h = 0;
  if (h->learned) {
    cudaGraphConditionalHandle hu;
    LGF_CK(h, cudaGraphConditionalHandleCreate(&hu, graph, 0, cudaGraphCondAssignDefault));
    cudaGraphNodeParams up = {cudaGraphNodeTypeConditional};
    up.conditional.handle = hu;
    up.conditional.type = cudaGraphCondTypeIf;
    up.conditional.size = 1;
    LGF_CK(h, cudaGraphAddNode(&undo_node, body, nullptr, nullptr, 0, &up));
    LGF_CK(h, cudaStreamBeginCaptureToGraph(h->cap_stream, up.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                            cudaStreamCaptureModeRelaxed));
    cudaError_t eu = enqueue_body<R>(h, L, (unsigned long long)cond, 1, h->cap_stream, PART_UNDO);
    cudaGraph_t cu = nullptr;
    cudaError_t eu2 = cudaStreamEndCapture(h->cap_stream, &cu);
    if (eu != cudaSuccess) return fail_cuda(h, eu, "capture of the undo pair");
    if (eu2 != cudaSuccess) return fail_cuda(h, eu2, "cudaStreamEndCapture");
    undo_h = (unsigned long long)hu;
  }
  LGF_CK(h, cudaStreamBeginCaptureToGraph(h->cap_stream, body, undo_node ? &undo_node : nullptr, nullptr,
                                          undo_node ? 1 : 0, cudaStreamCaptureModeRelaxed));
  cudaError_t e = enqueue_body<R>(h, L, (unsigned long long)cond, 1, h->cap_stream,
                                  h->learned ? PART_STEP : PART_ALL, undo_h);
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &captured);
  if (e != cudaSuccess) return fail_cuda(h, e, "capture of the iteration body");
  if (e2 != cudaSuccess) return fail_cuda(h, e2, "cudaStreamEndCapture");
  LGF_CK(h, cudaGraphInstantiate(&L.exec, graph, 0));
  L.graph = graph;
  return LGF_OK;
}

// n overrelaxation sweeps (even colour, then odd) of a lane's current links,
// with G <- g G where the lane tracks G.
template <typename R> cudaError_t enqueue_or_sweeps(lgf_ctx* h, Lane<R>& L, double omega, int n, cudaStream_t s) {
  C2<R>* U1 = L.fused ? L.U2 : nullptr;
  for (int k = 0; k < n; ++k)
    for (int parity = 0; parity < 2; ++parity) {
      cudaError_t e = L.rows == 3 ? launch_or_half_sweep<R, 3>(h->geom, L.U, U1, h->st, L.G, parity, omega, s)
                                  : launch_or_half_sweep<R, 2>(h->geom, L.U, U1, h->st, L.G, parity, omega, s);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

// Build (once per omega and check_every) the overrelaxation loop graph
// WHILE(theta >= tol && sweeps < max) { check_every sweeps; measure }.
template <typename R> lgf_status ensure_or_graph(lgf_ctx* h, Lane<R>& L, double omega, int check_every) {
  if (L.or_exec && L.or_omega == omega && L.or_check == check_every) return LGF_OK;
  drop_or_graph(L);
  cudaGraph_t graph;
  LGF_CK(h, cudaGraphCreate(&graph, 0));
  L.or_graph = graph;
  cudaGraphConditionalHandle cond;
  LGF_CK(h, cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  LGF_CK(h, cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
  LGF_CK(h, cudaStreamBeginCaptureToGraph(h->cap_stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed));
  cudaError_t e = enqueue_or_sweeps<R>(h, L, omega, check_every, h->cap_stream);
  if (e == cudaSuccess) e = enqueue_measure<R>(h, L, check_every, (unsigned long long)cond, 1, h->cap_stream);
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &captured);
  if (e != cudaSuccess) return fail_cuda(h, e, "capture of the overrelaxation body");
  if (e2 != cudaSuccess) return fail_cuda(h, e2, "cudaStreamEndCapture");
  LGF_CK(h, cudaGraphInstantiate(&L.or_exec, graph, 0));
  L.or_omega = omega;
  L.or_check = check_every;
  return LGF_OK;
}

lgf_status sync_state(lgf_ctx* h) {
  LGF_CK(h, cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  return LGF_OK;
}

lgf_status check_handle(lgf_ctx* h) {
  if (!h) return LGF_E_ARG;
  if (h->broken) return LGF_E_CUDA;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return fail_cuda(h, e, "cudaSetDevice");
  return LGF_OK;
}

lgf_status measure_current(lgf_ctx* h) {
  cudaError_t e = (h->phase == 64) ? enqueue_measure<double>(h, h->d, 0, 0, 0, h->stream)
                                   : enqueue_measure<float>(h, h->f, 0, 0, 0, h->stream);
  if (e != cudaSuccess) return fail_cuda(h, e, "measure");
  return LGF_OK;
}

// FP32 -> FP64 switch: G64 = proj_SU3(G32) in FP64, U64 = G64 U0 G64^dag(x+mu).
lgf_status switch_to_fp64(lgf_ctx* h) {
  const Geom& g = h->geom;
  LGF_CK(h, launch_project_sites_f32_to_f64(g, h->f.G, h->d.g, h->stream));
  if (h->d.rows == 3) {
    LGF_CK(h, (launch_links_from_aos<double, 3>(g, h->U0, h->d.U, h->stream)));
    LGF_CK(h, (launch_update<double, 3, 3>(g, h->d.U, h->d.g, h->stream)));
  } else {
    LGF_CK(h, (launch_links_from_aos<double, 2>(g, h->U0, h->d.U, h->stream)));
    LGF_CK(h, (launch_update<double, 2, 3>(g, h->d.U, h->d.g, h->stream)));
  }
  if (h->d.G) LGF_CK(h, cudaMemcpyAsync(h->d.G, h->d.g, sizeof(double2) * 9 * g.V, cudaMemcpyDeviceToDevice,
                                        h->stream));
  h->phase = 64;
  lgf_status s = measure_current(h);
  return s;
}

lgf_status copy_out(lgf_ctx* h, const double* dev_src, double* dst, size_t n_doubles, int where) {
  if (where == LGF_DEVICE) {
    if (dev_src != dst)
      LGF_CK(h, cudaMemcpyAsync(dst, dev_src, n_doubles * 8, cudaMemcpyDeviceToDevice, h->stream));
  } else {
    LGF_CK(h, cudaMemcpyAsync(dst, dev_src, n_doubles * 8, cudaMemcpyDeviceToHost, h->stream));
  }
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  return LGF_OK;
}

// Gram-Schmidt reunitarisation of the lane's current links after a measured
// unitarity defect passed the bound, then a fresh measurement of them.
template <typename R> lgf_status repair_links(lgf_ctx* h, Lane<R>& L) {
  C2<R>* cur = (L.fused && h->st_host->ubuf) ? L.U2 : L.U;
  if (L.rows == 3) LGF_CK(h, (launch_reunitarize_links<R, 3>(h->geom, cur, h->st, h->stream)));
  else LGF_CK(h, (launch_reunitarize_links<R, 2>(h->geom, cur, h->st, h->stream)));
  LGF_CK(h, enqueue_measure<R>(h, L, 0, 0, 0, h->stream));
  h->repairs += 1;
  return sync_state(h);
}

// The device loop of a lane until theta < tol or max_iter updates: the
// Fourier-accelerated body, or with or_check > 0 the overrelaxation body of
// or_check sweeps with parameter or_omega.
template <typename R> lgf_status run_loop(lgf_ctx* h, Lane<R>& L, double tol, int max_iter, int reset,
                                          double or_omega = 0.0, int or_check = 0) {
  const bool f64 = sizeof(R) == sizeof(double);
  LGF_CK(h, launch_set_state(h->st, tol, max_iter, reset, h->hist_cap, h->hist_F, h->hist_T, h->stream,
                             h->hist_flags, h->hist_defect, f64 ? h->defect_bound64 : h->defect_bound32,
                             f64 ? TRACE_FP64 : 0));
  lgf_status s = sync_state(h);
  if (s != LGF_OK) return s;
  int last_repair_iter = -1;
  for (;;) {
    const DevState& S = *h->st_host;
    if (S.status == ST_DEFECT) {
      // the links drifted from SU(3) (rounding compounded over many steps far
      // from the fixed point): reunitarise them and carry on
      if (S.iter == last_repair_iter)
        return fail(h, LGF_E_NONFINITE, "link unitarity is lost within one step of a reunitarisation");
      last_repair_iter = S.iter;
      if ((s = repair_links<R>(h, L)) != LGF_OK) return s;
      continue;
    }
    if (!(std::isfinite(S.F) && std::isfinite(S.theta))) return LGF_OK;
    if ((S.theta < tol || S.iter >= max_iter) && !S.revert) return LGF_OK;
    s = or_check > 0 ? ensure_or_graph<R>(h, L, or_omega, or_check) : ensure_graph<R>(h, L);
    if (s != LGF_OK) return s;
    // the graph's undo node is off at launch: a rejected step left over from
    // an earlier launch (stopped by the defect guard) is undone here first
    if (h->learned && S.revert) {
      cudaError_t eu = enqueue_body<R>(h, L, 0, 0, h->stream, PART_UNDO);
      if (eu != cudaSuccess) return fail_cuda(h, eu, "undo of a rejected step");
    }
    LGF_CK(h, cudaGraphLaunch(or_check > 0 ? L.or_exec : L.exec, h->stream));
    if ((s = sync_state(h)) != LGF_OK) return s;
  }
}

// Mode log of one step: D^ of the divergence just measured, compared with the
// one of the previous step.
template <typename R> cudaError_t log_modes(lgf_ctx* h, Lane<R>& L, bool prime_only) {
  const Geom& g = h->geom;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(L.Dlog, L.D, sizeof(C2<R>) * 4 * g.V, cudaMemcpyDeviceToDevice, h->stream)) != cudaSuccess)
    return e;
  if ((e = launch_fft_xy<R>(g, L.plan, L.Dlog, L.tw, L.pos, -1, 4, h->stream)) != cudaSuccess) return e;
  if ((e = launch_fft_zt<R>(g, L.plan, L.Dlog, L.tw, L.pos, L.K, -1, 4, h->stream)) != cudaSuccess) return e;
  if (!prime_only &&
      (e = launch_mode_log<R>(g, L.mg, L.Dlog, L.Dprev, L.Dprev2, h->ls, h->stats, h->stream)) != cudaSuccess)
    return e;
  if ((e = launch_log_state_update(h->ls, h->st, h->stream)) != cudaSuccess) return e;
  // rotate: current -> previous -> the one before
  std::swap(L.Dprev2, L.Dprev);
  std::swap(L.Dlog, L.Dprev);
  return cudaSuccess;
}

template <typename R> lgf_status step_lane(lgf_ctx* h, Lane<R>& L, double alpha) {
  lgf_status s = ensure_filter<R>(h, L, alpha);
  if (s != LGF_OK) return s;
  cudaError_t e;
  if (h->logging && !h->log_primed) {
    if ((e = log_modes<R>(h, L, true)) != cudaSuccess) return fail_cuda(h, e, "mode log");
    h->log_primed = true;
  }
  // a learned handle synchronised after its last call, so the host knows
  // whether a rejected step still waits for its undo (normally not: it is
  // redone below); otherwise the body skips the undo pair
  const bool pending = h->learned && h->st_host->revert;
  if ((e = enqueue_body<R>(h, L, 0, 0, h->stream, (h->learned && !pending) ? PART_STEP : PART_ALL)) != cudaSuccess)
    return fail_cuda(h, e, "lgf_step");
  if (h->learned) {
    // a rejected learned step is undone and redone with the plain filter now
    if ((s = sync_state(h)) != LGF_OK) return s;
    if (h->st_host->revert && (e = enqueue_body<R>(h, L, 0, 0, h->stream, PART_ALL)) != cudaSuccess)
      return fail_cuda(h, e, "lgf_step redo");
  }
  if (h->logging && (e = log_modes<R>(h, L, false)) != cudaSuccess) return fail_cuda(h, e, "mode log");
  return LGF_OK;
}

struct MlpScratch {
  float* part_g = nullptr;
  double* part_l = nullptr;
  float* grad = nullptr;
  double* loss = nullptr;
  int nb = 0;
  cudaError_t alloc(int nblocks, int nloss, cudaStream_t s) {
    nb = nblocks;
    cudaError_t e = cudaMallocAsync((void**)&part_g, sizeof(float) * (size_t)nb * MLP_NPARAM, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&part_l, sizeof(double) * nb, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&grad, sizeof(float) * MLP_NPARAM, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&loss, sizeof(double) * (size_t)(nloss > 0 ? nloss : 1), s);
    return e;
  }
  void release(cudaStream_t s) {
    if (part_g) cudaFreeAsync(part_g, s);
    if (part_l) cudaFreeAsync(part_l, s);
    if (grad) cudaFreeAsync(grad, s);
    if (loss) cudaFreeAsync(loss, s);
  }
};

lgf_status finish_fix(lgf_ctx* h, double theta_tol, int32_t* iters, double* F, double* theta);

// Overrelaxation needs a checkerboard (every extent even); the learned
// multiplier belongs to the Fourier-accelerated filter and is not combined
// with it.
lgf_status or_supported(lgf_ctx* h) {
  for (int mu = 0; mu < 4; ++mu)
    if (h->geom.L[mu] % 2 != 0)
      return fail(h, LGF_E_UNSUPPORTED, "overrelaxation needs every extent even (checkerboard colours)");
  if (h->learned) return fail(h, LGF_E_UNSUPPORTED, "overrelaxation does not run on LGF_LEARNED handles");
  return LGF_OK;
}
}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

const char* lgf_status_string(lgf_status s) {
  switch (s) {
    case LGF_OK: return "ok";
    case LGF_E_ARG: return "invalid argument";
    case LGF_E_NOMEM: return "out of memory";
    case LGF_E_CUDA: return "CUDA error";
    case LGF_E_STATE: return "invalid state";
    case LGF_E_NONFINITE: return "non-finite value";
    case LGF_E_NOTCONV: return "not converged";
    case LGF_E_TIMEOUT: return "timeout";
    case LGF_E_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* lgf_last_error(lgf_handle h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

lgf_status lgf_destroy(lgf_handle h) {
  if (!h) return LGF_OK;
  cudaSetDevice(h->device);
  if (h->stream || h->cap_stream) cudaStreamSynchronize(h->stream);
  free_lane(h, h->d);
  free_lane(h, h->f);
  h->mem.put_all();  // U0, stage, partials, state, tables, histories, network, mode log
  cudaStreamSynchronize(h->stream);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->defect_host) cudaFreeHost(h->defect_host);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (cudaEvent_t e : h->set_ev)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < TimingRing::kSlots; ++i)
    for (int k = 0; k <= TimingRing::kMaxK; ++k)
      if (h->timing.ev[i][k]) cudaEventDestroy(h->timing.ev[i][k]);
  delete h;
  return LGF_OK;
}

lgf_status lgf_create(const int32_t extents[4], lgf_precision prec, uint32_t flags, void* cuda_stream,
                      lgf_handle* out) {
  return lgf_create_with_allocator(extents, prec, flags, cuda_stream, nullptr, out);
}

lgf_status lgf_create_with_allocator(const int32_t extents[4], lgf_precision prec, uint32_t flags,
                                     void* cuda_stream, const lgf_allocator* allocator, lgf_handle* out) {
  if (!extents || !out) return LGF_E_ARG;
  *out = nullptr;
  if (allocator && (!allocator->alloc || !allocator->free)) return LGF_E_ARG;
  if (prec != LGF_FP64 && prec != LGF_FP32 && prec != LGF_MIXED) return LGF_E_ARG;
  if (flags & ~(uint32_t)(LGF_STORE12 | LGF_TRACK_G | LGF_PLAIN_SD | LGF_LEARNED | LGF_EXACT_EXP)) return LGF_E_ARG;
  for (int mu = 0; mu < 4; ++mu)
    if (!extent_ok(extents[mu])) return LGF_E_UNSUPPORTED;
  lgf_ctx* h = new (std::nothrow) lgf_ctx();
  if (!h) return LGF_E_NOMEM;
  try {
    h->prec = prec;
    h->flags = flags;
    h->learned = (flags & LGF_LEARNED) != 0;
    h->stream = (cudaStream_t)cuda_stream;
    h->mem.stream = h->stream;
    if (allocator) h->mem.user = *allocator;
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return LGF_E_CUDA; }
    Geom& g = h->geom;
    g.V = 1;
    for (int mu = 0; mu < 4; ++mu) {
      g.L[mu] = extents[mu];
      g.stride[mu] = g.V;
      g.V *= extents[mu];
    }
    lgf_status s = LGF_OK;
    const bool store12 = (flags & LGF_STORE12) != 0;
    const bool track = (flags & LGF_TRACK_G) != 0;
    if (prec == LGF_FP64) {
      s = alloc_lane<double>(h, h->d, store12 ? 2 : 3, 3, track);
      h->phase = 64;
    } else if (prec == LGF_FP32) {
      s = alloc_lane<float>(h, h->f, store12 ? 2 : 3, store12 ? 2 : 3, track);
      h->phase = 32;
    } else {
      // FP32 phase in the requested storage; the FP64 phase keeps 18 reals
      // (it is bound by FP64 arithmetic, which 12-real storage increases).
      s = alloc_lane<float>(h, h->f, store12 ? 2 : 3, store12 ? 2 : 3, true);
      if (s == LGF_OK) s = alloc_lane<double>(h, h->d, 3, 3, track);
      if (s == LGF_OK) {
        cudaError_t e = h->mem.get(&h->U0, (size_t)4 * 18 * g.V);
        if (e != cudaSuccess) s = fail_cuda(h, e, "allocation of U0");
      }
      h->phase = 32;
    }
    if (s == LGF_OK) {
      cudaError_t e = cudaSuccess;
      if (e == cudaSuccess) e = h->mem.get(&h->stage, (size_t)4 * 18 * g.V);
      if (e == cudaSuccess) e = h->mem.get(&h->partials, (size_t)MEASURE_PARTIALS * measure_blocks(g.V));
      if (e == cudaSuccess) e = h->mem.get(&h->st, 1);
      if (e == cudaSuccess) e = cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream);
      if (e == cudaSuccess) e = h->mem.get(&h->defect, 1);
      if (e == cudaSuccess) e = cudaMallocHost((void**)&h->st_host, sizeof(DevState));
      if (e == cudaSuccess) e = cudaMallocHost((void**)&h->defect_host, sizeof(unsigned long long));
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
      for (cudaEvent_t& ev : h->set_ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      h->lmax = 0;
      for (int mu = 0; mu < 4; ++mu) h->lmax = std::max(h->lmax, g.L[mu]);
      std::vector<double> sin2((size_t)4 * h->lmax, 0.0);
      h->p2max = 0;
      for (int mu = 0; mu < 4; ++mu) {
        for (int k = 0; k < g.L[mu]; ++k) {
          const double sv = std::sin(M_PI * (double)k / (double)g.L[mu]);
          sin2[(size_t)mu * h->lmax + k] = 4.0 * sv * sv;
        }
        const double sm = std::sin(M_PI * (double)(g.L[mu] / 2) / (double)g.L[mu]);
        h->p2max += 4.0 * sm * sm;
      }
      if (e == cudaSuccess) e = h->mem.get(&h->sin2, sin2.size());
      if (e == cudaSuccess) e = cudaMemcpyAsync(h->sin2, sin2.data(), sin2.size() * 8, cudaMemcpyHostToDevice, h->stream);
      // stream-ordered buffers become usable by every stream once this returns
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) s = fail_cuda(h, e, "lgf_create allocation");
    }
    if (h->mem.misaligned) s = LGF_E_ARG;  // the caller's allocator returned memory not 256-byte aligned
    if (s != LGF_OK) {
      lgf_destroy(h);
      return s;
    }
    std::memset(h->st_host, 0, sizeof(DevState));
    *out = h;
    return LGF_OK;
  } catch (...) {
    lgf_destroy(h);
    return LGF_E_NOMEM;
  }
}

lgf_status lgf_set_links(lgf_handle h, const double* U, int where) {
  NvtxRange nvtx_("lgf_set_links");
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!U || (where != LGF_HOST && where != LGF_DEVICE)) return fail(h, LGF_E_ARG, "bad links pointer or location");
  try {
    const Geom& g = h->geom;
    const size_t n = (size_t)4 * 18 * g.V;
    const double* src = U;
    if (where == LGF_HOST) {
      // piece k of the links: copy on the handle's stream, check on cap_stream
      // after the copy's event; the stream waits for the last check
      const int64_t nmat = 4 * g.V, per = (nmat + lgf_ctx::kSetChunks - 1) / lgf_ctx::kSetChunks;
      LGF_CK(h, cudaMemsetAsync(h->defect, 0, sizeof(unsigned long long), h->stream));
      LGF_CK(h, cudaEventRecord(h->set_ev[lgf_ctx::kSetChunks], h->stream));
      LGF_CK(h, cudaStreamWaitEvent(h->cap_stream, h->set_ev[lgf_ctx::kSetChunks], 0));
      for (int k = 0; k < lgf_ctx::kSetChunks; ++k) {
        const int64_t m0 = k * per, m1 = std::min(nmat, m0 + per);
        if (m1 <= m0) break;
        const size_t off = (size_t)m0 * 18;
        LGF_CK(h, cudaMemcpyAsync(h->stage + off, U + off, (size_t)(m1 - m0) * 18 * 8, cudaMemcpyHostToDevice,
                                  h->stream));
        LGF_CK(h, cudaEventRecord(h->set_ev[k], h->stream));
        LGF_CK(h, cudaStreamWaitEvent(h->cap_stream, h->set_ev[k], 0));
        LGF_CK(h, launch_su3_defect(h->stage + off, m1 - m0, h->defect, h->cap_stream, /*reset=*/0));
      }
      LGF_CK(h, cudaEventRecord(h->set_ev[lgf_ctx::kSetChunks], h->cap_stream));
      LGF_CK(h, cudaStreamWaitEvent(h->stream, h->set_ev[lgf_ctx::kSetChunks], 0));
      src = h->stage;
    } else {
      LGF_CK(h, launch_su3_defect(src, 4 * g.V, h->defect, h->stream));
    }
    LGF_CK(h, cudaMemcpyAsync(h->defect_host, h->defect, 8, cudaMemcpyDeviceToHost, h->stream));
    LGF_CK(h, cudaStreamSynchronize(h->stream));
    double defect;
    std::memcpy(&defect, h->defect_host, 8);
    if (!std::isfinite(defect)) return fail(h, LGF_E_NONFINITE, "input links contain non-finite values");
    if (defect > kSU3Tol) {
      char buf[128];
      std::snprintf(buf, sizeof(buf), "input links are not in SU(3): defect %.3e > %.1e", defect, kSU3Tol);
      return fail(h, LGF_E_ARG, buf);
    }
    if (h->prec == LGF_FP64) {
      if (h->d.rows == 3) LGF_CK(h, (launch_links_from_aos<double, 3>(g, src, h->d.U, h->stream)));
      else LGF_CK(h, (launch_links_from_aos<double, 2>(g, src, h->d.U, h->stream)));
      if (h->d.G) LGF_CK(h, (launch_set_identity<double, 3>(g, h->d.G, h->stream)));
      h->phase = 64;
    } else {
      if (h->f.rows == 3) LGF_CK(h, (launch_links_from_aos<float, 3>(g, src, h->f.U, h->stream)));
      else LGF_CK(h, (launch_links_from_aos<float, 2>(g, src, h->f.U, h->stream)));
      LGF_CK(h, cudaMemsetAsync(&h->st->ubuf, 0, sizeof(int), h->stream));  // the links are in buffer U
      if (h->f.G) LGF_CK(h, (launch_set_identity<float, 3>(g, h->f.G, h->stream)));
      if (h->prec == LGF_MIXED) {
        LGF_CK(h, cudaMemcpyAsync(h->U0, src, n * 8, cudaMemcpyDeviceToDevice, h->stream));
        if (h->d.G) LGF_CK(h, (launch_set_identity<double, 3>(g, h->d.G, h->stream)));
      }
      h->phase = 32;
    }
    LGF_CK(h, launch_set_state(h->st, 0.0, 0, 1, 0, nullptr, nullptr, h->stream));
    s = measure_current(h);
    if (s != LGF_OK) return s;
    s = sync_state(h);
    if (s != LGF_OK) return s;
    h->have_links = true;
    h->have_g = false;
    return LGF_OK;
  } catch (...) {
    return fail(h, LGF_E_NOMEM, "host allocation failed");
  }
}

lgf_status lgf_get_links(lgf_handle h, double* U, int where) {
  NvtxRange nvtx_("lgf_get_links");
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!U || (where != LGF_HOST && where != LGF_DEVICE)) return fail(h, LGF_E_ARG, "bad links pointer or location");
  if (!h->have_links) return fail(h, LGF_E_STATE, "no links set");
  const Geom& g = h->geom;
  double* dst = where == LGF_DEVICE ? U : h->stage;
  if (h->phase == 64) {
    if (h->d.rows == 3) LGF_CK(h, (launch_links_to_aos<double, 3>(g, h->d.U, dst, h->stream)));
    else LGF_CK(h, (launch_links_to_aos<double, 2>(g, h->d.U, dst, h->stream)));
  } else {
    s = sync_state(h);  // which buffer of a fused lane holds the current links
    if (s != LGF_OK) return s;
    const float2* cur = (h->f.fused && h->st_host->ubuf) ? h->f.U2 : h->f.U;
    if (h->f.rows == 3) LGF_CK(h, (launch_links_to_aos<float, 3>(g, cur, dst, h->stream)));
    else LGF_CK(h, (launch_links_to_aos<float, 2>(g, cur, dst, h->stream)));
  }
  return copy_out(h, dst, U, (size_t)4 * 18 * g.V, where);
}

lgf_status lgf_step(lgf_handle h, double alpha) {
  NvtxRange nvtx_("lgf_step");
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!h->have_links) return fail(h, LGF_E_STATE, "no links set");
  if (!std::isfinite(alpha)) return fail(h, LGF_E_ARG, "alpha must be finite");
  if (h->learned && !h->mlp_w) return fail(h, LGF_E_STATE, "LGF_LEARNED handle without a loaded preconditioner");
  if (h->prec == LGF_MIXED && h->phase == 32) {
    // every step from links with theta below the switch level runs in FP64,
    // as in lgf_fix
    if ((s = sync_state(h)) != LGF_OK) return s;
    const double th = h->st_host->theta;
    if (std::isfinite(th) && th < h->switch_theta && (s = switch_to_fp64(h)) != LGF_OK) return s;
  }
  s = h->phase == 64 ? step_lane<double>(h, h->d, alpha) : step_lane<float>(h, h->f, alpha);
  if (s != LGF_OK) return s;
  h->have_g = true;
  return LGF_OK;
}

lgf_status lgf_measure(lgf_handle h, double* F, double* theta) {
  NvtxRange nvtx_("lgf_measure");
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!h->have_links) return fail(h, LGF_E_STATE, "no links set");
  s = sync_state(h);
  if (s != LGF_OK) return s;
  if (F) *F = h->st_host->F;
  if (theta) *theta = h->st_host->theta;
  if (!(std::isfinite(h->st_host->F) && std::isfinite(h->st_host->theta)))
    return fail(h, LGF_E_NONFINITE, "F or theta is not finite");
  return LGF_OK;
}

lgf_status lgf_fix(lgf_handle h, double theta_tol, int32_t max_iter, double alpha, int32_t* iters, double* F,
                   double* theta) {
  NvtxRange nvtx_("lgf_fix");
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!h->have_links) return fail(h, LGF_E_STATE, "no links set");
  if (!(theta_tol >= 0.0) || max_iter < 0 || !std::isfinite(alpha)) return fail(h, LGF_E_ARG, "bad fix arguments");
  if (h->learned && !h->mlp_w) return fail(h, LGF_E_STATE, "LGF_LEARNED handle without a loaded preconditioner");
  h->repairs = 0;
  if (h->phase == 32) {
    NvtxRange phase32("FP32 phase");
    if ((s = ensure_filter<float>(h, h->f, alpha)) != LGF_OK) return s;
    const double tol1 = h->prec == LGF_MIXED ? std::max(theta_tol, h->switch_theta) : theta_tol;
    if ((s = run_loop<float>(h, h->f, tol1, max_iter, 1)) != LGF_OK) return s;
    h->have_g = h->have_g || h->st_host->iter > 0;
    const DevState& S = *h->st_host;
    if (h->prec == LGF_MIXED && std::isfinite(S.theta) && S.theta < tol1 && theta_tol < tol1 &&
        S.iter < max_iter) {
      if ((s = switch_to_fp64(h)) != LGF_OK) return s;
    }
  } else {
    LGF_CK(h, launch_set_state(h->st, theta_tol, max_iter, 1, h->hist_cap, h->hist_F, h->hist_T, h->stream,
                               h->hist_flags, h->hist_defect, h->defect_bound64, TRACE_FP64));
  }
  if (h->phase == 64) {
    NvtxRange phase64("FP64 phase");
    if ((s = ensure_filter<double>(h, h->d, alpha)) != LGF_OK) return s;
    if ((s = run_loop<double>(h, h->d, theta_tol, max_iter, 0)) != LGF_OK) return s;
    h->have_g = h->have_g || h->st_host->iter > 0;
  }
  return finish_fix(h, theta_tol, iters, F, theta);
}

lgf_status lgf_or_sweep(lgf_handle h, double omega, int32_t nsweeps) {
  NvtxRange nvtx_("lgf_or_sweep");
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!h->have_links) return fail(h, LGF_E_STATE, "no links set");
  if (!(omega >= 1.0 && omega < 2.0) || nsweeps < 0) return fail(h, LGF_E_ARG, "need 1 <= omega < 2, nsweeps >= 0");
  if ((s = or_supported(h)) != LGF_OK) return s;
  if (h->prec == LGF_MIXED && h->phase == 32) {
    // sweeps from links with theta below the switch level run in FP64
    if ((s = sync_state(h)) != LGF_OK) return s;
    const double th = h->st_host->theta;
    if (std::isfinite(th) && th < h->switch_theta && (s = switch_to_fp64(h)) != LGF_OK) return s;
  }
  cudaError_t e = h->phase == 64 ? enqueue_or_sweeps<double>(h, h->d, omega, nsweeps, h->stream)
                                 : enqueue_or_sweeps<float>(h, h->f, omega, nsweeps, h->stream);
  if (e == cudaSuccess)
    e = h->phase == 64 ? enqueue_measure<double>(h, h->d, nsweeps, 0, 0, h->stream)
                       : enqueue_measure<float>(h, h->f, nsweeps, 0, 0, h->stream);
  if (e != cudaSuccess) return fail_cuda(h, e, "lgf_or_sweep");
  h->have_g = false;  // g of the last Fourier-accelerated step no longer describes the links
  return LGF_OK;
}

lgf_status lgf_or_fix(lgf_handle h, double theta_tol, int32_t max_sweeps, double omega, int32_t check_every,
                      int32_t* sweeps, double* F, double* theta) {
  NvtxRange nvtx_("lgf_or_fix");
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!h->have_links) return fail(h, LGF_E_STATE, "no links set");
  if (!(theta_tol >= 0.0) || max_sweeps < 0 || !(omega >= 1.0 && omega < 2.0) || check_every < 1)
    return fail(h, LGF_E_ARG, "bad overrelaxation fix arguments");
  if ((s = or_supported(h)) != LGF_OK) return s;
  h->repairs = 0;
  if (h->phase == 32) {
    NvtxRange phase32("FP32 phase");
    const double tol1 = h->prec == LGF_MIXED ? std::max(theta_tol, h->switch_theta) : theta_tol;
    if ((s = run_loop<float>(h, h->f, tol1, max_sweeps, 1, omega, check_every)) != LGF_OK) return s;
    const DevState& S = *h->st_host;
    if (h->prec == LGF_MIXED && std::isfinite(S.theta) && S.theta < tol1 && theta_tol < tol1 &&
        S.iter < max_sweeps) {
      if ((s = switch_to_fp64(h)) != LGF_OK) return s;
    }
  } else {
    LGF_CK(h, launch_set_state(h->st, theta_tol, max_sweeps, 1, h->hist_cap, h->hist_F, h->hist_T, h->stream,
                               h->hist_flags, h->hist_defect, h->defect_bound64, TRACE_FP64));
  }
  if (h->phase == 64) {
    NvtxRange phase64("FP64 phase");
    if ((s = run_loop<double>(h, h->d, theta_tol, max_sweeps, 0, omega, check_every)) != LGF_OK) return s;
  }
  h->have_g = false;
  return finish_fix(h, theta_tol, sweeps, F, theta);
}

}  // extern "C"

namespace {
// Results of a finished fix (either method): counts, F, theta, the trace
// copied to the caller's buffers, and the status.
lgf_status finish_fix(lgf_ctx* h, double theta_tol, int32_t* iters, double* F, double* theta) {
  const DevState& S = *h->st_host;
  if (iters) *iters = S.iter;
  if (F) *F = S.F;
  if (theta) *theta = S.theta;
  if (h->hist_cap > 0 && h->user_F && h->user_T) {
    const int n = std::min(h->hist_cap, S.iter + 1);
    LGF_CK(h, cudaMemcpyAsync(h->user_F, h->hist_F, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream));
    LGF_CK(h, cudaMemcpyAsync(h->user_T, h->hist_T, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream));
    if (h->user_flags)
      LGF_CK(h, cudaMemcpyAsync(h->user_flags, h->hist_flags, (size_t)n * 4, cudaMemcpyDeviceToHost, h->stream));
    if (h->user_defect)
      LGF_CK(h, cudaMemcpyAsync(h->user_defect, h->hist_defect, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream));
    LGF_CK(h, cudaStreamSynchronize(h->stream));
  }
  if (!(std::isfinite(S.F) && std::isfinite(S.theta)) || S.status == ST_NONFINITE)
    return fail(h, LGF_E_NONFINITE, "F or theta became non-finite");
  if (S.theta >= theta_tol) return fail(h, LGF_E_NOTCONV, "max_iter reached before theta < tol");
  return LGF_OK;
}
}  // namespace

extern "C" {

lgf_status lgf_get_transform(lgf_handle h, double* G, int where) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!G || (where != LGF_HOST && where != LGF_DEVICE)) return fail(h, LGF_E_ARG, "bad pointer or location");
  if (!h->have_links) return fail(h, LGF_E_STATE, "no links set");
  const Geom& g = h->geom;
  double* dst = where == LGF_DEVICE ? G : h->stage;
  if (h->phase == 64 && h->d.G) {
    LGF_CK(h, (launch_sites_to_aos<double, 3>(g, h->d.G, dst, h->stream)));
  } else if (h->phase == 32 && h->f.G && (h->flags & LGF_TRACK_G)) {
    LGF_CK(h, (launch_sites_to_aos<float, 3>(g, h->f.G, dst, h->stream)));
  } else {
    return fail(h, LGF_E_STATE, "the handle does not track G (create it with LGF_TRACK_G)");
  }
  return copy_out(h, dst, G, (size_t)18 * g.V, where);
}

lgf_status lgf_get_gauge(lgf_handle h, double* gout, int where) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!gout || (where != LGF_HOST && where != LGF_DEVICE)) return fail(h, LGF_E_ARG, "bad pointer or location");
  if (!h->have_g) return fail(h, LGF_E_STATE, "no step has been taken");
  const Geom& g = h->geom;
  double* dst = where == LGF_DEVICE ? gout : h->stage;
  if (h->phase == 64) {
    LGF_CK(h, (launch_sites_to_aos<double, 3>(g, h->d.g, dst, h->stream)));
  } else if (h->f.grows == 2) {
    LGF_CK(h, (launch_sites_to_aos<float, 2>(g, h->f.g, dst, h->stream)));
  } else {
    LGF_CK(h, (launch_sites_to_aos<float, 3>(g, h->f.g, dst, h->stream)));
  }
  return copy_out(h, dst, gout, (size_t)18 * g.V, where);
}

lgf_status lgf_get_divergence(lgf_handle h, double* D, int where) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!D || (where != LGF_HOST && where != LGF_DEVICE)) return fail(h, LGF_E_ARG, "bad pointer or location");
  if (!h->have_links) return fail(h, LGF_E_STATE, "no links set");
  const Geom& g = h->geom;
  double* dst = where == LGF_DEVICE ? D : h->stage;
  if (h->phase == 64) LGF_CK(h, launch_delta_to_aos<double>(g, h->d.D, dst, h->stream));
  else LGF_CK(h, launch_delta_to_aos<float>(g, h->f.D, dst, h->stream));
  return copy_out(h, dst, D, (size_t)18 * g.V, where);
}

lgf_status lgf_set_trace_ex(lgf_handle h, double* F_hist, double* theta_hist, int32_t* flags_hist,
                            double* defect_hist, int32_t cap) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (cap < 0 || (cap > 0 && (!F_hist || !theta_hist))) return fail(h, LGF_E_ARG, "bad trace arguments");
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  h->mem.put(h->hist_F);
  h->mem.put(h->hist_T);
  h->mem.put(h->hist_flags);
  h->mem.put(h->hist_defect);
  h->hist_F = h->hist_T = h->hist_defect = nullptr;
  h->hist_flags = nullptr;
  h->hist_cap = 0;
  h->user_F = h->user_T = h->user_defect = nullptr;
  h->user_flags = nullptr;
  if (cap > 0) {
    LGF_CK(h, h->mem.get(&h->hist_F, (size_t)cap));
    LGF_CK(h, h->mem.get(&h->hist_T, (size_t)cap));
    LGF_CK(h, h->mem.get(&h->hist_flags, (size_t)cap));
    LGF_CK(h, h->mem.get(&h->hist_defect, (size_t)cap));
    h->hist_cap = cap;
    h->user_F = F_hist;
    h->user_T = theta_hist;
    h->user_flags = flags_hist;
    h->user_defect = defect_hist;
  }
  // the device state must never point at freed history buffers
  LGF_CK(h, launch_set_state(h->st, 0.0, 0, 0, h->hist_cap, h->hist_F, h->hist_T, h->stream, h->hist_flags,
                             h->hist_defect));
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  return LGF_OK;
}

lgf_status lgf_set_trace(lgf_handle h, double* F_hist, double* theta_hist, int32_t cap) {
  return lgf_set_trace_ex(h, F_hist, theta_hist, nullptr, nullptr, cap);
}

lgf_status lgf_set_defect_bound(lgf_handle h, double bound_fp64, double bound_fp32) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!(bound_fp64 >= 0.0) || !(bound_fp32 >= 0.0)) return fail(h, LGF_E_ARG, "bounds must be >= 0");
  h->defect_bound64 = bound_fp64;
  h->defect_bound32 = bound_fp32;
  return LGF_OK;
}

lgf_status lgf_get_link_defect(lgf_handle h, double* defect, int32_t* repairs) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if ((s = sync_state(h)) != LGF_OK) return s;
  if (defect) *defect = h->st_host->defect;
  if (repairs) *repairs = h->repairs;
  return LGF_OK;
}

lgf_status lgf_fft4(lgf_handle h, double* data, int32_t nfields, int32_t sign, int where) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!data || nfields != 4 || (sign != -1 && sign != 1) || (where != LGF_HOST && where != LGF_DEVICE))
    return fail(h, LGF_E_ARG, "bad fft4 arguments");
  const Geom& g = h->geom;
  const size_t n = (size_t)4 * 2 * g.V;
  double* buf = h->stage;
  if (where == LGF_HOST) LGF_CK(h, cudaMemcpyAsync(buf, data, n * 8, cudaMemcpyHostToDevice, h->stream));
  else LGF_CK(h, cudaMemcpyAsync(buf, data, n * 8, cudaMemcpyDeviceToDevice, h->stream));
  if (h->phase == 64) {
    Lane<double>& L = h->d;
    LGF_CK(h, cudaMemcpyAsync(L.D, buf, n * 8, cudaMemcpyDeviceToDevice, h->stream));
    LGF_CK(h, launch_fft_xy<double>(g, L.plan, L.D, L.tw, L.pos, sign, 4, h->stream));
    LGF_CK(h, launch_fft_zt<double>(g, L.plan, L.D, L.tw, L.pos, L.K, sign, 4, h->stream));
    LGF_CK(h, cudaMemcpyAsync(buf, L.D, n * 8, cudaMemcpyDeviceToDevice, h->stream));
  } else {
    Lane<float>& L = h->f;
    LGF_CK(h, launch_c2_f64_to_f32(reinterpret_cast<const double2*>(buf), L.D, 4 * g.V, h->stream));
    LGF_CK(h, launch_fft_xy<float>(g, L.plan, L.D, L.tw, L.pos, sign, 4, h->stream));
    LGF_CK(h, launch_fft_zt<float>(g, L.plan, L.D, L.tw, L.pos, L.K, sign, 4, h->stream));
    LGF_CK(h, launch_c2_f32_to_f64(L.D, reinterpret_cast<double2*>(buf), 4 * g.V, h->stream));
  }
  s = copy_out(h, buf, data, n, where);
  if (s != LGF_OK) return s;
  // the transform used the divergence buffer: restore it from the links
  if (h->have_links) {
    s = measure_current(h);
    if (s != LGF_OK) return s;
    s = sync_state(h);
  }
  return s;
}

lgf_status lgf_set_timing(lgf_handle h, int32_t enable) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  TimingRing& T = h->timing;
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  if (enable && !T.ev[0][0]) {
    for (int i = 0; i < TimingRing::kSlots; ++i)
      for (int k = 0; k <= TimingRing::kMaxK; ++k) LGF_CK(h, cudaEventCreate(&T.ev[i][k]));
  }
  for (int i = 0; i < TimingRing::kSlots; ++i) T.pending[i] = false;
  for (int k = 0; k < TimingRing::kCat; ++k) T.sum_ms[k] = 0.0;
  T.steps = 0;
  T.next = 0;
  T.enabled = enable != 0;
  return LGF_OK;
}

lgf_status lgf_get_timing(lgf_handle h, double* ms, int32_t nkernels, int32_t* nsteps) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!ms || nkernels < 1 || nkernels > TimingRing::kCat) return fail(h, LGF_E_ARG, "bad timing arguments");
  TimingRing& T = h->timing;
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < TimingRing::kSlots; ++i) LGF_CK(h, timing_collect(T, i));
  for (int k = 0; k < nkernels; ++k) ms[k] = T.steps ? T.sum_ms[k] / (double)T.steps : 0.0;
  if (nsteps) *nsteps = (int32_t)T.steps;
  return LGF_OK;
}

lgf_status lgf_load_preconditioner(lgf_handle h, const uint16_t* w, size_t n_w, int where) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!w || n_w != (size_t)MLP_NPARAM || (where != LGF_HOST && where != LGF_DEVICE))
    return fail(h, LGF_E_ARG, "expected LGF_MLP_NPARAM BF16 parameters");
  if (!h->mlp_w) LGF_CK(h, h->mem.get(&h->mlp_w, (size_t)MLP_NPARAM));
  LGF_CK(h, cudaMemcpyAsync(h->mlp_w, w, (size_t)MLP_NPARAM * 2,
                            where == LGF_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, h->stream));
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  return LGF_OK;
}

lgf_status lgf_get_fallbacks(lgf_handle h, int32_t* n) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!n) return fail(h, LGF_E_ARG, "null pointer");
  if ((s = sync_state(h)) != LGF_OK) return s;
  *n = h->st_host->n_fallback;
  return LGF_OK;
}

lgf_status lgf_set_mode_log(lgf_handle h, int32_t enable) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  h->logging = false;
  h->log_primed = false;
  if (!enable) return LGF_OK;
  const int64_t V = h->geom.V;
  const int64_t nclass = h->phase == 64 ? h->d.mg.nclass : h->f.mg.nclass;
  if (!h->stats) LGF_CK(h, h->mem.get(&h->stats, (size_t)MLP_NBUCKET * nclass * MLP_NSTAT));
  if (!h->ls) LGF_CK(h, h->mem.get(&h->ls, 1));
  if (h->phase == 64 && !h->d.Dlog) {
    LGF_CK(h, h->mem.get(&h->d.Dlog, (size_t)4 * V));
    LGF_CK(h, h->mem.get(&h->d.Dprev, (size_t)4 * V));
    LGF_CK(h, h->mem.get(&h->d.Dprev2, (size_t)4 * V));
  }
  if (h->phase == 32 && !h->f.Dlog) {
    LGF_CK(h, h->mem.get(&h->f.Dlog, (size_t)4 * V));
    LGF_CK(h, h->mem.get(&h->f.Dprev, (size_t)4 * V));
    LGF_CK(h, h->mem.get(&h->f.Dprev2, (size_t)4 * V));
  }
  LGF_CK(h, cudaMemsetAsync(h->stats, 0, sizeof(double) * MLP_NBUCKET * nclass * MLP_NSTAT, h->stream));
  LGF_CK(h, cudaMemsetAsync(h->ls, 0, sizeof(LogState), h->stream));
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  h->logging = true;
  return LGF_OK;
}

lgf_status lgf_get_mode_log(lgf_handle h, double* out, int64_t n) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  const int64_t nclass = h->phase == 64 ? h->d.mg.nclass : h->f.mg.nclass;
  if (!out || !h->stats || n != (int64_t)MLP_NBUCKET * nclass * MLP_NSTAT)
    return fail(h, LGF_E_ARG, "mode log not enabled or wrong size");
  LGF_CK(h, cudaMemcpyAsync(out, h->stats, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  return LGF_OK;
}

lgf_status lgf_mlp_eval(const uint16_t* P, const float* X, int64_t n, float* m, void* cuda_stream) {
  if (!P || !X || !m || n < 0) return LGF_E_ARG;
  if (n == 0) return LGF_OK;
  return launch_mlp_eval(P, X, n, m, (cudaStream_t)cuda_stream) == cudaSuccess ? LGF_OK : LGF_E_CUDA;
}


lgf_status lgf_mlp_loss_grad(const float* P, const float* X, const float* Y, const float* W, int64_t n, float* grad,
                             double* loss, void* cuda_stream) {
  if (!P || !X || !Y || !W || !grad || n <= 0) return LGF_E_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  MlpScratch sc;
  const int nb = (int)std::min<int64_t>((n + 63) / 64, 304);
  cudaError_t e = sc.alloc(nb, 1, s);
  if (e == cudaSuccess)
    e = launch_mlp_grad(P, X, Y, W, n, 0, 0, 0, 1.f / (float)n, sc.part_g, sc.part_l, nb, grad, sc.loss, s);
  double l = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l, sc.loss, sizeof(double), cudaMemcpyDeviceToHost, s);
  sc.release(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LGF_E_NOMEM : LGF_E_CUDA;
  if (loss) *loss = l;
  return LGF_OK;
}

lgf_status lgf_mlp_train(float* P, float* adam, const float* X, const float* Y, const float* W, int64_t n,
                         int32_t batch, int32_t steps, float lr, uint64_t seed, int32_t t0, double* loss_hist,
                         void* cuda_stream) {
  if (!P || !adam || !X || !Y || !W || n <= 0 || batch <= 0 || steps < 0 || !(lr > 0.f) || t0 < 0) return LGF_E_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  MlpScratch sc;
  const int nb = (int)std::min<int64_t>((batch + 63) / 64, 304);
  cudaError_t e = sc.alloc(nb, steps, s);
  for (int i = 0; i < steps && e == cudaSuccess; ++i) {
    e = launch_mlp_grad(P, X, Y, W, n, batch, seed, t0 + i, 1.f / (float)batch, sc.part_g, sc.part_l, nb, sc.grad,
                        sc.loss + i, s);
    if (e == cudaSuccess) e = launch_adam(P, adam, adam + MLP_NPARAM, sc.grad, lr, t0 + i + 1, s);
  }
  if (e == cudaSuccess && loss_hist && steps > 0)
    e = cudaMemcpyAsync(loss_hist, sc.loss, sizeof(double) * steps, cudaMemcpyDeviceToHost, s);
  sc.release(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? LGF_E_NOMEM : LGF_E_CUDA;
  return LGF_OK;
}

lgf_status lgf_mlp_to_bf16(const float* P, uint16_t* out, void* cuda_stream) {
  if (!P || !out) return LGF_E_ARG;
  return launch_f32_to_bf16(P, out, MLP_NPARAM, (cudaStream_t)cuda_stream) == cudaSuccess ? LGF_OK : LGF_E_CUDA;
}

lgf_status lgf_set_learned_theta(lgf_handle h, double theta) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (!h->learned) return fail(h, LGF_E_STATE, "not an LGF_LEARNED handle");
  if (!(theta >= 0.0)) return fail(h, LGF_E_ARG, "the learned level must be >= 0 (or +inf)");
  // the level is a kernel argument of the captured loop bodies: capture again
  h->d.mg.theta_on = theta;
  drop_graph(h->d);
  h->f.mg.theta_on = theta;
  drop_graph(h->f);
  return LGF_OK;
}

lgf_status lgf_set_switch_theta(lgf_handle h, double theta) {
  if (!h) return LGF_E_ARG;
  if (!(theta >= 1e-10 && theta <= 1e-6)) return fail(h, LGF_E_ARG, "switch level must lie in [1e-10, 1e-6]");
  h->switch_theta = theta;
  return LGF_OK;
}

}  // extern "C"

namespace {

const char* decomp_name(int d) { return d == FFT_1D4 ? "1d4" : d == FFT_3D1D ? "3d1d" : "2d2d"; }

// Device time (ms, best of 3 after a warm-up) of the transform and g of one
// step under the lane's current plan and decomposition.
template <typename R> cudaError_t time_transform(lgf_ctx* h, Lane<R>& L, float* ms_out) {
  int ks[TimingRing::kMaxK];
  int nk = 0;
  if (L.decomp == FFT_1D4) {
    for (int k : {K_F1X, K_F1Y, K_F1Z, K_T1, K_I1Z, K_I1Y, K_I1X, K_GD}) ks[nk++] = k;
  } else if (L.decomp == FFT_3D1D) {
    for (int k : {K_F3, K_T1, K_I3, K_GD}) ks[nk++] = k;
  } else {
    for (int k : {K_A, K_B, K_C}) ks[nk++] = k;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, h->stream);
    for (int i = 0; i < nk && e == cudaSuccess; ++i) e = enqueue_kernel<R>(h, L, ks[i], 0, 0, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  *ms_out = best;
  return e;
}

// Times every tile plan of the 2D + 2D passes and the other decompositions
// (not with LGF_LEARNED), keeps the fastest and appends a JSON report.
template <typename R> lgf_status tune_lane(lgf_ctx* h, Lane<R>& L, std::string& rep) {
  lgf_status s = ensure_filter<R>(h, L, std::isnan(L.alpha) ? 0.08 : L.alpha);
  if (s != LGF_OK) return s;
  std::vector<FFTPlan> cand;
  fft_plan_candidates(h->geom.L, (int)sizeof(R), cand);
  struct Trial { int decomp; FFTPlan plan; float ms; };
  std::vector<Trial> trials;
  for (const FFTPlan& p : cand) trials.push_back({FFT_2D2D, p, 0.f});
  // 1D x 4 with every tile of its passes: 8, 16 or 32 x-lines per CTA in
  // the x pass, 4 to 32 x columns per CTA in the y, z, t passes
  for (int nl : {8, 16, 32})
    for (int xc : {4, 8, 16, 32}) {
      FFTPlan p = L.plan;
      if (set_line_tiles(h->geom.L, (int)sizeof(R), nl, xc, &p)) trials.push_back({FFT_1D4, p, 0.f});
    }
  if (L.plan.fit_xyz) trials.push_back({FFT_3D1D, L.plan, 0.f});
  // a choice recorded in the LGF_AUTOTUNE_CACHE file is reused without timing
  cudaDeviceProp prop;
  LGF_CK(h, cudaGetDeviceProperties(&prop, h->device));
  char kb[256];
  std::snprintf(kb, sizeof(kb), "single,%d,%d,%d,%d,%s,rows=%d,learned=%d,%s", h->geom.L[0], h->geom.L[1],
                h->geom.L[2], h->geom.L[3], sizeof(R) == 8 ? "fp64" : "fp32", L.rows, h->learned ? 1 : 0, prop.name);
  std::string key = kb;
  for (char& c : key)
    if (c == ' ') c = '_';
  TuneChoice tc;
  if (std::getenv("LGF_AUTOTUNE_CACHE") && tune_cache_get(key, &tc)) {
    for (size_t i = 0; i < trials.size(); ++i)
      if (trials[i].decomp == tc.decomp && tune_choice_matches(trials[i].plan, tc)) {
        drop_graph(L);
        L.plan = trials[i].plan;
        L.decomp = trials[i].decomp;
        char item[256];
        std::snprintf(item, sizeof(item),
                      "{\"cached\":true,\"chosen\":0,\"candidates\":[{\"decomposition\":\"%s\","
                      "\"fields_per_cta_xy\":%d,\"x_columns_zt\":%d,\"threads\":[%d,%d,%d],\"lines_x\":%d,"
                      "\"x_columns_line\":%d,\"ms\":null}]}",
                      decomp_name(L.decomp), L.plan.fpb_xy, L.plan.xc, L.plan.threads_xy, L.plan.threads_zt,
                      L.plan.threads_c, L.plan.nl_x, L.plan.xc_line);
        rep += item;
        return LGF_OK;
      }
  }
  int best = -1;
  for (size_t i = 0; i < trials.size(); ++i) {
    L.plan = trials[i].plan;
    L.decomp = trials[i].decomp;
    LGF_CK(h, time_transform<R>(h, L, &trials[i].ms));
    if (best < 0 || trials[i].ms < trials[best].ms) best = (int)i;
  }
  drop_graph(L);
  L.plan = trials[best].plan;
  L.decomp = trials[best].decomp;
  if (std::getenv("LGF_AUTOTUNE_CACHE")) tune_cache_put(key, tune_choice_of(L.plan, L.decomp));
  char item[256];
  rep += "{\"cached\":false,\"chosen\":" + std::to_string(best) + ",\"candidates\":[";
  for (size_t i = 0; i < trials.size(); ++i) {
    const Trial& t = trials[i];
    std::snprintf(item, sizeof(item),
                  "%s{\"decomposition\":\"%s\",\"fields_per_cta_xy\":%d,\"x_columns_zt\":%d,"
                  "\"threads\":[%d,%d,%d],\"lines_x\":%d,\"x_columns_line\":%d,\"ms\":%.5f}",
                  i ? "," : "", decomp_name(t.decomp), t.plan.fpb_xy, t.plan.xc, t.plan.threads_xy,
                  t.plan.threads_zt, t.plan.threads_c, t.plan.nl_x, t.plan.xc_line, t.ms);
    rep += item;
  }
  rep += "]}";
  return LGF_OK;
}

}  // namespace

extern "C" {

lgf_status lgf_autotune(lgf_handle h, char* report, size_t len) {
  NvtxRange nvtx_("lgf_autotune");
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  std::string rep = "{";
  if (h->d.active) {
    rep += "\"fp64\":";
    if ((s = tune_lane<double>(h, h->d, rep)) != LGF_OK) return s;
  }
  if (h->f.active) {
    rep += h->d.active ? ",\"fp32\":" : "\"fp32\":";
    if ((s = tune_lane<float>(h, h->f, rep)) != LGF_OK) return s;
  }
  rep += "}";
  // the trials overwrote the divergence, g and the divergence snapshots of a
  // learned handle: restore the measurement, forget the snapshots
  h->have_g = false;
  LGF_CK(h, cudaMemsetAsync(&h->st->snaps, 0, sizeof(int), h->stream));
  if (h->have_links) {
    if ((s = measure_current(h)) != LGF_OK) return s;
    if ((s = sync_state(h)) != LGF_OK) return s;
  } else {
    LGF_CK(h, cudaStreamSynchronize(h->stream));
  }
  if (report && len) {
    std::snprintf(report, len, "%s", rep.c_str());
    if (rep.size() >= len) return fail(h, LGF_E_ARG, "report buffer too small");
  }
  return LGF_OK;
}

lgf_status lgf_set_fused_update(lgf_handle h, int32_t enable) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  Lane<float>& L = h->f;
  if (!L.active) return LGF_OK;  // FP64 handles never fuse
  if (enable && !L.U2) return fail(h, LGF_E_UNSUPPORTED, "the FP32 lane has no second link buffer");
  if ((enable != 0) == L.fused) return LGF_OK;
  if ((s = sync_state(h)) != LGF_OK) return s;
  if (!enable && h->st_host->ubuf) {
    // the unfused update works in place on U: move the current links there
    LGF_CK(h, cudaMemcpyAsync(L.U, L.U2, sizeof(float2) * 4 * L.rows * 3 * h->geom.V, cudaMemcpyDeviceToDevice,
                              h->stream));
    LGF_CK(h, cudaMemsetAsync(&h->st->ubuf, 0, sizeof(int), h->stream));
    LGF_CK(h, cudaStreamSynchronize(h->stream));
  }
  drop_graph(L);
  L.fused = enable != 0;
  return LGF_OK;
}

lgf_status lgf_set_fft_decomposition(lgf_handle h, int32_t decomposition) {
  lgf_status s = check_handle(h);
  if (s != LGF_OK) return s;
  if (decomposition != LGF_FFT_2D2D && decomposition != LGF_FFT_1D4 && decomposition != LGF_FFT_3D1D)
    return fail(h, LGF_E_ARG, "unknown decomposition");
  if (decomposition == LGF_FFT_3D1D && ((h->d.active && !h->d.plan.fit_xyz) || (h->f.active && !h->f.plan.fit_xyz)))
    return fail(h, LGF_E_UNSUPPORTED, "the (x, y, z) slab does not fit in shared memory");
  LGF_CK(h, cudaStreamSynchronize(h->stream));
  // the loop graphs hold the old body: rebuild them on the next fix
  set_decomp(h->d, decomposition);
  set_decomp(h->f, decomposition);
  return LGF_OK;
}

lgf_status lgf_get_phase(lgf_handle h, int32_t* bits) {
  if (!h || !bits) return LGF_E_ARG;
  *bits = h->phase;
  return LGF_OK;
}

}  // extern "C"
