// Internal interface between the lgf C-ABI layer (lgf_api.cu) and the
// kernel translation units.  Not installed; no torch types anywhere.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lgf_common.cuh"

namespace lgf {

// Controller state kept in device memory.  Written by the last CTA of the
// measurement kernel; read by the host after a fix and by the graph's WHILE
// condition.
struct DevState {
  double F;          // gauge functional of the current links
  double theta;      // stopping quantity of the current links
  double F_prev;     // F before the last step
  double theta_prev; // theta before the last step (0 before the first)
  double tol;        // loop runs while theta >= tol
  int iter;          // link updates performed since the counter was reset
  int max_iter;      // loop stops when iter reaches it
  int status;        // 0 ok, 1 non-finite F or theta, 2 timeout
  unsigned int ticket;  // CTA completion counter of the measurement reduction
  int hist_cap;      // capacity of the history buffers (0 = none)
  int done;          // batch mode: this configuration has retired (theta < tol or iter >= max_iter)
  int use_m;         // the running step multiplies the filter by the learned table
  int revert;        // the last learned step lowered F: undo it and redo it with the plain filter
  int n_fallback;    // learned steps rejected since the counter was reset
  int ubuf;          // fused lanes: which of the two link buffers holds the current links
  double* F_hist;    // F after measurement number i (i = iter) if i < hist_cap
  double* theta_hist;
  double defect;       // largest unitarity defect of the sampled links (last measurement)
  double defect_bound; // > 0: a measurement whose defect exceeds it ends the loop with ST_DEFECT
  int redo;            // the running step redoes a rejected learned step with the plain filter
  int repaired;        // the links were reunitarised since the last counted measurement
  int* flag_hist;      // flags of measurement number i (TRACE_* bits) if i < hist_cap
  double* defect_hist; // defect of measurement number i if i < hist_cap
  int snaps;           // learned handles: steps whose Fourier-space divergence snapshot is kept
};

enum { ST_OK = 0, ST_NONFINITE = 1, ST_DEFECT = 3 };

// Per-measurement trace flags (the LGF_TRACE_* bits of include/lgf.h).
enum { TRACE_FP64 = 1, TRACE_LEARNED = 2, TRACE_REDO = 4, TRACE_REPAIRED = 8, TRACE_REJECTED = 16 };

// Measurement CTAs keep three partials each: the F sum, the theta sum and
// the largest sampled link defect.
constexpr int MEASURE_PARTIALS = 3;

// Batch dimension of a launch: blockIdx.z selects one of n configurations of
// the same lattice shape, whose buffers are the given strides (in elements)
// apart.  In batch mode (st != nullptr) st[z] is the configuration's
// controller state and retired configurations (st[z].done) are skipped.
struct Batch {
  int n = 1;
  int64_t s_links = 0, s_delta = 0, s_g = 0, s_G = 0, s_part = 0;
  DevState* st = nullptr;
};

__device__ __forceinline__ bool batch_skip(const Batch& b) { return b.st != nullptr && b.st[blockIdx.z].done; }

constexpr int MEASURE_THREADS = 256;

inline int64_t measure_blocks(int64_t V) { return (V + MEASURE_THREADS - 1) / MEASURE_THREADS; }

// ---- lgf_site.cu -------------------------------------------------------
// Delta, F and theta of the current links (Sec. 2; kernel k2 of Sec. 3.2).
// count_iter > 0: this measurement follows count_iter link updates (iter += count_iter):
// one step of Algorithm 1, or count_iter overrelaxation sweeps.
// use_cond != 0: set the graph conditional to (theta >= tol && iter < max_iter).
// count_iter = -1: this measurement follows the undo of a rejected step (iter -= 1).
// only_if_revert != 0: do nothing unless an undo is pending (st->revert).
// After a counted step that used the learned table (st->use_m) and lowered F,
// st->revert is set and the WHILE condition stays true so that the next
// body undoes the step and redoes it with the plain filter.
// In batch mode (B->st set) each configuration's state is B->st[z] and its
// last CTA sets that state's `done` instead of a graph condition.
// links_alt (fused lanes): the second link buffer, read instead of links when st->ubuf is set.
// cond_undo (use_cond only): handle of the graph's IF node around the undo
// pair, set by a counted measurement to whether its step was rejected.
template <typename R, int ROWS>
cudaError_t launch_measure(const Geom& g, const C2<R>* links, C2<R>* delta, double* partials, DevState* st,
                           int count_iter, unsigned long long cond_handle, int use_cond, cudaStream_t s,
                           int only_if_revert = 0, const Batch& B = Batch(), const C2<R>* links_alt = nullptr,
                           unsigned long long cond_undo = 0);

// Link update fused with the measurement that follows it: the links are read
// from buffer st->ubuf of {U0, U1} and the updated links written to the other
// buffer; the updated backward links U'_mu(x - mu^) = g(x - mu^) U_mu(x - mu^)
// g^dag(x) are recomputed in registers instead of being read back, then
// Delta, F and theta are formed and reduced as by launch_measure with
// count_iter = 1, and the last CTA flips st->ubuf.  The result is
// bit-identical to launch_update followed by launch_measure.
template <typename R, int LROWS, int GROWS>
cudaError_t launch_update_measure(const Geom& g, C2<R>* U0, C2<R>* U1, const C2<R>* gfield, C2<R>* delta,
                                  double* partials, DevState* st, unsigned long long cond, int use_cond,
                                  cudaStream_t s, unsigned long long cond_undo = 0);

// Undo of the last update when st->revert is set: U_mu(x) <- g^dag(x) U_mu(x)
// g(x + mu^) and, when G is given (3 rows, precision R), G <- g^dag G.
// links_alt (fused lanes): the second link buffer, used instead of links when st->ubuf is set.
template <typename R, int LROWS, int GROWS>
cudaError_t launch_revert(const Geom& g, C2<R>* links, const C2<R>* gfield, C2<R>* Gacc, const DevState* st,
                          cudaStream_t s, C2<R>* links_alt = nullptr);

// U_mu(x) <- g(x) U_mu(x) g^dagger(x + mu^) in place (Sec. 2 eq. 2; kernel k6).
// Links in precision R with LROWS stored rows; g in precision R with GROWS rows.
template <typename R, int LROWS, int GROWS>
cudaError_t launch_update(const Geom& g, C2<R>* links, const C2<R>* gfield, cudaStream_t s, const Batch& B = Batch());

// Graph condition of a batch: true while any of the n configurations is active.
cudaError_t launch_batch_condition(const DevState* st, int n, unsigned long long cond, cudaStream_t s);

// AoS FP64 user layout [mu][t][z][y][x][3][3][2] -> SoA links of precision R.
template <typename R, int ROWS>
cudaError_t launch_links_from_aos(const Geom& g, const double* aos, C2<R>* links, cudaStream_t s);
template <typename R, int ROWS>
cudaError_t launch_links_to_aos(const Geom& g, const C2<R>* links, double* aos, cudaStream_t s);
// Site matrix field (nmat = 1) SoA <-> AoS, FP64 user layout [t][z][y][x][3][3][2].
template <typename R, int ROWS>
cudaError_t launch_sites_to_aos(const Geom& g, const C2<R>* field, double* aos, cudaStream_t s);
template <typename R, int ROWS>
cudaError_t launch_sites_from_aos(const Geom& g, const double* aos, C2<R>* field, cudaStream_t s);
// Packed divergence fields -> 3x3 anti-Hermitian matrices in the site AoS layout.
template <typename R>
cudaError_t launch_delta_to_aos(const Geom& g, const C2<R>* delta, double* aos, cudaStream_t s);

// Largest SU(3) defect max(|U U^dag - 1|, |det U - 1|) of an AoS link array,
// as the bit pattern of a non-negative double (NaN maps to +inf bits).
// reset = 0: fold into the maximum already in *out_bits (checks of pieces).
cudaError_t launch_su3_defect(const double* aos, int64_t nmat, unsigned long long* out_bits, cudaStream_t s,
                              int reset = 1);

// Loop parameters of the controller state (tol, max_iter, history);
// reset_iter != 0 also zeroes the iteration counter and the status word.
cudaError_t launch_set_state(DevState* st, double tol, int max_iter, int reset_iter, int hist_cap, double* F_hist,
                             double* theta_hist, cudaStream_t s, int* flag_hist = nullptr,
                             double* defect_hist = nullptr, double defect_bound = 0.0, int flags0 = 0);

// Gram-Schmidt reunitarisation of every link in place (rows 1-2 orthonormal
// in the link precision, row 3 = (a x b)^* when stored), after a measured
// defect passed the bound; marks st->repaired and clears ST_DEFECT.
template <typename R, int ROWS>
cudaError_t launch_reunitarize_links(const Geom& g, C2<R>* links, DevState* st, cudaStream_t s);

// Complex array precision conversion (n elements).
cudaError_t launch_c2_f64_to_f32(const double2* in, float2* out, int64_t n, cudaStream_t s);
cudaError_t launch_c2_f32_to_f64(const float2* in, double2* out, int64_t n, cudaStream_t s);

// G64 = reunitarize(G32) in FP64 (3-row FP32 site field -> 3-row FP64 site field).
cudaError_t launch_project_sites_f32_to_f64(const Geom& g, const float2* G32, double2* G64, cudaStream_t s);

// Site field G <- 1.
template <typename R, int ROWS>
cudaError_t launch_set_identity(const Geom& g, C2<R>* field, cudaStream_t s);

// Momentum filter table K(k) = alpha * p2max / p2(k) / V with K(0) = 0, stored
// [kt][kz][ky][kx] in precision R (kernel k1 of Sec. 3.2).
template <typename R>
cudaError_t launch_filter_table(const Geom& g, const double* sin2 /* 4 x Lmax: 4 sin^2(pi k/L) */, int lmax,
                                double alpha, double p2max, int plain_sd, R* K, cudaStream_t s);

// ---- lgf_or.cu ----------------------------------------------------------
// One colour of an overrelaxation sweep (the local maximisation of F named in
// Sec. 3.2, Cabibbo-Marinari subgroups, Mandula-Ogilvie overrelaxation):
// every site x with (x + y + z + t) % 2 == parity gets g(x), and
// U_mu(x) <- g(x) U_mu(x), U_mu(x - mu^) <- U_mu(x - mu^) g^dag(x), in place.
// Links of precision R with ROWS stored rows; U1 != nullptr (fused lanes):
// the current links are U1 when st->ubuf is set, else U0.  G != nullptr:
// G(x) <- g(x) G(x) (3 rows, precision R).  Every extent must be even.
template <typename R, int ROWS>
cudaError_t launch_or_half_sweep(const Geom& g, C2<R>* U0, C2<R>* U1, const DevState* st, C2<R>* G, int parity,
                                 double omega, cudaStream_t s);

// ---- lgf_fft.cu ---------------------------------------------------------
// Radix schedule of one lattice direction.
struct FFTDir {
  int N;
  int nst;
  int radix[8];
  FastDiv ns[8];  // divisors by the span Ns = radix[0] ... radix[st-1] of each stage
};

struct FFTPlan {
  FFTDir d[4];
  int xc;          // consecutive x columns per CTA in the (z,t) pass
  int fpb_xy;      // fields per CTA in the (x,y) passes (1, 2 or 4)
  int threads_xy;
  int threads_zt;
  int threads_c;
  size_t smem_xy;
  size_t smem_zt;
  size_t smem_c;   // pass C (needs all 4 fields when fused with g)
  int fuse_g;      // pass C computes g directly (4 fields fit in shared memory)
  // alternative decompositions (1D x 4 and 3D + 1D)
  int nl_x;        // x-lines per CTA of the 1D x pass
  int xc_line;     // x columns per CTA of the 1D y, z, t passes
  int threads_line[4];
  size_t smem_line[4];
  int fit_xyz;     // the (x, y, z) slab of one field fits in shared memory
  int threads_xyz;
  size_t smem_xyz;
};

// Decomposition of the 4D transform of one step.
enum FFTDecomp { FFT_2D2D = 0, FFT_1D4 = 1, FFT_3D1D = 2 };

// Twiddle tables W_N^m = exp(-2 pi i m / N), m < N, for the four directions,
// concatenated at offsets 0, Lx, Lx+Ly, Lx+Ly+Lz (FP64 and FP32 copies).
// pos: digit-reversal position tables of the four directions (fft_positions).
template <typename R>
cudaError_t launch_fft_xy(const Geom& g, const FFTPlan& p, C2<R>* data, const C2<R>* tw, const short* pos, int sign,
                          int nfields, cudaStream_t s, const Batch& B = Batch());
// mode 0: forward (z,t) DFT, multiply by K, inverse (z,t) DFT (pass B);
// mode -1 / +1: forward / inverse (z,t) DFT only (K unused).
// lio (mode 0 only): with lio.mtab the learned multiplier per momentum class
// is applied when st->use_m != 0; with lio.snap the transformed divergence is
// stored before the filter.
// Learned handles' extras of the pass that carries the filter: the multiplier
// table of step k is mtab + (k & 1) * nclass and the Fourier-space divergence
// (before the filter) is stored in snap + (k & 1) * 4 V, with k = st->iter
// read on the device.  A snapshot entry is one complex value as two BF16
// halves (real part in the low 16 bits): the class contraction it feeds is a
// network input, which the tensor cores read in BF16 anyway.
struct LearnedIO {
  const float* mtab = nullptr;   // [2][nclass]
  uint32_t* snap = nullptr;      // [2][4][V]
  const DevState* st = nullptr;  // st->use_m, st->iter
  int64_t nclass = 0;
};

// BF16 bits of x by truncation of its FP32 value.
__device__ __forceinline__ uint32_t bf16_trunc_bits(float x) { return __float_as_uint(x) >> 16; }
// BF16 bits of an FP64 value by truncation, on the integer pipe (no FP64
// instruction): sign, exponent rebiased from 1023 to 127, top 7 mantissa bits;
// values below the FP32 range flush to zero, values above it become infinite.
__device__ __forceinline__ uint32_t bf16_trunc_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 48) & 0x8000u;
  const int e = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return sign;
  if (e >= 255) return sign | 0x7f80u;
  return sign | ((uint32_t)e << 7) | ((uint32_t)(b >> 45) & 0x7fu);
}
template <typename R> __device__ __forceinline__ uint32_t bf16x2_of(C2<R> v) {
  return bf16_trunc_bits(v.x) | (bf16_trunc_bits(v.y) << 16);
}
__device__ __forceinline__ float bf16x2_re(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf16x2_im(uint32_t p) { return __uint_as_float(p & 0xffff0000u); }

template <typename R>
cudaError_t launch_fft_zt(const Geom& g, const FFTPlan& p, C2<R>* data, const C2<R>* tw, const short* pos,
                          const R* K, int mode, int nfields, cudaStream_t s, const LearnedIO& lio = LearnedIO(),
                          const Batch& B = Batch());
// Inverse (x,y) transform fused with g(x) = reunitarize(1 + Delta'(x)) in FP64
// (exact_exp != 0: g(x) = reunitarize(exp(Delta'(x)))); g stored with GROWS
// rows in precision RG; optional G <- g G (precision RG with 3 rows).
template <typename R, typename RG, int GROWS>
cudaError_t launch_fft_xy_inv_gauge(const Geom& g, const FFTPlan& p, C2<R>* data, const C2<R>* tw, const short* pos,
                                    C2<RG>* gfield, C2<RG>* Gfield, cudaStream_t s, const Batch& B = Batch(),
                                    int exact_exp = 0);

// 1D pass along mu (0..3) over nfields fields: mode -1 forward, +1 inverse,
// 0 forward, multiply by K (and by the learned table when lio.mtab is given
// and st->use_m != 0; snapshot of the transform when lio.snap is given),
// inverse.
template <typename R>
cudaError_t launch_fft_line(const Geom& g, const FFTPlan& p, int mu, C2<R>* data, const C2<R>* tw, const short* pos,
                            const R* K, int mode, int nfields, cudaStream_t s, const Batch& B = Batch(),
                            const LearnedIO& lio = LearnedIO());
// 3D DFT over every (x, y, z) slab (requires p.fit_xyz); sign -1 / +1.
template <typename R>
cudaError_t launch_fft_xyz(const Geom& g, const FFTPlan& p, C2<R>* data, const C2<R>* tw, const short* pos, int sign,
                           int nfields, cudaStream_t s, const Batch& B = Batch());
// g(x) from the filtered field in natural order (after an inverse transform
// that is not fused with g); same storage conventions as launch_fft_xy_inv_gauge.
template <typename R, typename RG, int GROWS>
cudaError_t launch_gauge_from_delta(const Geom& g, const C2<R>* data, C2<RG>* gfield, C2<RG>* Gfield, cudaStream_t s,
                                    const Batch& B = Batch(), int exact_exp = 0);

cudaError_t configure_fft_plan(const int L[4], int real_bytes, FFTPlan* p);

// An autotuner's choice: the decomposition and the tile fields of the plan.
struct TuneChoice {
  int decomp, fpb_xy, xc, threads_xy, threads_zt, threads_c, nl_x, xc_line;
};
// Tiles of the 1D passes (nl x-lines per CTA, xc x columns in the strided
// passes); false if they do not divide the lattice or fit shared memory.
bool set_line_tiles(const int L[4], int real_bytes, int nl, int xc, FFTPlan* p);
TuneChoice tune_choice_of(const FFTPlan& p, int decomp);
bool tune_choice_matches(const FFTPlan& p, const TuneChoice& c);  // same tile fields
// Autotune cache, kept for the process and, when the environment variable
// LGF_AUTOTUNE_CACHE names a file, read from it on first use and appended to
// (one "key decomposition fpb xc threads_xy threads_zt threads_c nl_x xc_line"
// line per choice).
bool tune_cache_get(const std::string& key, TuneChoice* c);
void tune_cache_put(const std::string& key, const TuneChoice& c);
// All plans the autotuner may choose among for a lattice shape.
void fft_plan_candidates(const int L[4], int real_bytes, std::vector<FFTPlan>& out);
// Digit-reversal position tables of the four directions, concatenated
// (Lx + Ly + Lz + Lt entries).
void fft_positions(const FFTPlan& p, short* out);

}  // namespace lgf
