// Site-local kernels of FA steepest-descent Landau gauge fixing:
//   * measure  : Delta(x), F and theta with a deterministic FP64 reduction
//                (arXiv:1206.0675 Sec. 2 and kernel k2 of Sec. 3.2),
//   * update   : U_mu(x) -> g(x) U_mu(x) g^dagger(x + mu^) (Sec. 2 eq. 2, kernel k6),
//   * layout conversion, SU(3) validation, the momentum filter table (k1).
// One thread per lattice site; link arrays are structure-of-arrays so that a
// warp touches 32 consecutive sites of one matrix element per load.
#include <algorithm>
#include <cmath>

#include "lgf_internal.h"

namespace lgf {

// ---------------------------------------------------------------------------
// measure: Delta, F, theta
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of two sums (FP64, fixed order) and a maximum (FP32: the
// link defect is compared with bounds far above FP32 resolution, and FP32
// max and shuffles keep the FP64 pipe free); result valid in thread 0.
__device__ __forceinline__ void block_reduce3(double& a, double& b, float& m) {
  __shared__ double sa[32], sb[32];
  __shared__ float sm[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if (lane == 0) { sa[warp] = a; sb[warp] = b; sm[warp] = m; }
  __syncthreads();
  if (warp == 0) {
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    m = lane < nw ? sm[lane] : 0.f;
    a = warp_sum(a);
    b = warp_sum(b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  }
  __syncthreads();
}

// Unitarity defect of a link from its rows 1-2 (row 3 is always rebuilt as
// (a x b)^* or stored from that rebuild): the largest of | |a|^2 - 1 |,
// | |b|^2 - 1 | and the components of <a, b>, in the link precision.
template <typename R> __device__ __forceinline__ float rows_defect(const C2<R> a[3], const C2<R> b[3]) {
  const R na = cnorm2<R>(a[0]) + cnorm2<R>(a[1]) + cnorm2<R>(a[2]);
  const R nb = cnorm2<R>(b[0]) + cnorm2<R>(b[1]) + cnorm2<R>(b[2]);
  C2<R> ip = cconjmul<R>(a[0], b[0]);
  ip = cadd<R>(ip, cconjmul<R>(a[1], b[1]));
  ip = cadd<R>(ip, cconjmul<R>(a[2], b[2]));
  // the four deviations, each taken to FP32 before the maximum
  return fmaxf(fmaxf(fabsf((float)(na - (R)1)), fabsf((float)(nb - (R)1))),
               fmaxf(fabsf((float)ip.x), fabsf((float)ip.y)));
}

// The links whose defect a measurement samples: every sixteenth warp of the
// grid (warp index w with w % 16 == 0) takes direction (w / 16) % 4 of its 32
// sites, i.e. one link in 64, spread over all directions (the drift the
// guard watches is slow and lattice-wide).  The choice is uniform within a
// warp, so the other warps skip the work entirely.
__device__ __forceinline__ int defect_sample_mu() {
  const unsigned w = (unsigned)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  return (w & 15u) == 0 ? (int)((w >> 4) & 3u) : -1;
}

// Reduction of the per-thread F and theta sums and the sampled link defect
// and, in the last CTA to finish, the controller update: F, theta and the
// defect, the iteration count, the history and its flags, the status word,
// the batch retirement flag or the graph's WHILE condition; flip_ubuf != 0
// also flips st->ubuf (after every CTA has read it); fp64 != 0 marks the
// measurement as one of FP64 links in the trace flags.
// fsum and tsum are one site's sums, already in FP64; every sum above a
// site (warp, CTA, grid) is FP64 in a fixed order.
__device__ __forceinline__ void measure_tail(const Geom& g, double fsum, double tsum, float dmax,
                                             double* __restrict__ partials, DevState* __restrict__ st, int count_iter,
                                             unsigned long long cond, int use_cond, bool batch, int flip_ubuf,
                                             int fp64, unsigned long long cond_undo) {
  double fb = fsum, tb = tsum;
  float db = dmax;
  block_reduce3(fb, tb, db);
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    partials[MEASURE_PARTIALS * blockIdx.x] = fb;
    partials[MEASURE_PARTIALS * blockIdx.x + 1] = tb;
    partials[MEASURE_PARTIALS * blockIdx.x + 2] = (double)db;
    __threadfence();
    const unsigned int t = atomicAdd(&st->ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  // Final sum over the per-CTA partials in a fixed order (independent of
  // which CTA finished last), so the result is bit-reproducible.
  double f = 0.0, t = 0.0;
  float d = 0.f;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    f += __ldcg(&partials[MEASURE_PARTIALS * i]);
    t += __ldcg(&partials[MEASURE_PARTIALS * i + 1]);
    d = fmaxf(d, (float)__ldcg(&partials[MEASURE_PARTIALS * i + 2]));
  }
  block_reduce3(f, t, d);
  if (threadIdx.x == 0) {
    const double Vd = (double)g.V;
    const double F = f / (12.0 * Vd);
    const double th = 4.0 * t / (3.0 * Vd);
    int it = st->iter;
    int revert = 0;
    int flags = fp64 ? TRACE_FP64 : 0;
    if (count_iter > 0) {
      it += count_iter;  // one FA step, or count_iter overrelaxation sweeps
      st->iter = it;
      st->F_prev = st->F;
      st->theta_prev = st->theta;
      // a learned step that lowered F is undone and redone with the plain filter
      if (st->use_m && F < st->F) {
        revert = 1;
        st->n_fallback += 1;
      }
      st->revert = revert;
      if (st->use_m) flags |= TRACE_LEARNED;
      if (st->redo) flags |= TRACE_REDO;
      if (st->repaired) flags |= TRACE_REPAIRED;
      st->redo = 0;
      st->repaired = 0;
    } else if (count_iter < 0) {
      it -= 1;
      st->iter = it;
    }
    st->snaps += count_iter;  // a rejected step's snapshot is replaced by its redo
    st->F = F;
    st->theta = th;
    st->defect = d;
    // The re-measurement after an undo repeats an entry already written; a
    // measurement without an update (after a precision switch or a repair)
    // refreshes F, theta and the defect of the current entry but keeps the
    // flags of the update that produced it.
    if (it < st->hist_cap && count_iter >= 0) {
      st->F_hist[it] = F;
      st->theta_hist[it] = th;
      if (st->flag_hist && count_iter > 0) st->flag_hist[it] = flags;
      if (st->defect_hist) st->defect_hist[it] = d;
    }
    const bool finite = isfinite(F) && isfinite(th);
    const bool sound = !(st->defect_bound > 0.0 && d > st->defect_bound);
    if (!finite) st->status = ST_NONFINITE;
    else if (!sound) st->status = ST_DEFECT;
    if (flip_ubuf) st->ubuf ^= 1;
    st->ticket = 0u;
    if (batch) st->done = !(finite && th >= st->tol && it < st->max_iter);
    if (use_cond) {
      cudaGraphConditionalHandle h = (cudaGraphConditionalHandle)cond;
      cudaGraphSetConditional(h, (finite && sound && ((th >= st->tol && it < st->max_iter) || revert)) ? 1u : 0u);
      if (cond_undo != 0 && count_iter > 0)
        cudaGraphSetConditional((cudaGraphConditionalHandle)cond_undo, revert ? 1u : 0u);
    }
  }
}

// ||Delta_A||_F^2 of the packed components, as an explicit FMA chain (the
// same rounding in every kernel that forms it).
template <typename R>
__device__ __forceinline__ R delta_norm2(R a0, R a1, R a2, C2<R> d01, C2<R> d02, C2<R> d12) {
  R off = d01.x * d01.x;
  off = fma(d01.y, d01.y, off);
  off = fma(d02.x, d02.x, off);
  off = fma(d02.y, d02.y, off);
  off = fma(d12.x, d12.x, off);
  off = fma(d12.y, d12.y, off);
  R dia = a0 * a0;
  dia = fma(a1, a1, dia);
  dia = fma(a2, a2, dia);
  return fma((R)2, off, dia);
}

template <typename R, int ROWS>
__global__ void __launch_bounds__(MEASURE_THREADS)
measure_kernel(Geom g, MatField<R, ROWS> U, const C2<R>* __restrict__ links_alt, C2<R>* __restrict__ delta,
               double* __restrict__ partials, DevState* __restrict__ st, int count_iter, unsigned long long cond,
               int use_cond, int only_if_revert, Batch B, unsigned long long cond_undo) {
  if (batch_skip(B)) return;
  const bool batch = B.st != nullptr;
  if (batch) {
    const int cfg = blockIdx.z;
    st = B.st + cfg;
    U.p += cfg * B.s_links;
    delta += cfg * B.s_delta;
    partials += cfg * B.s_part;
  }
  if (only_if_revert && !st->revert) return;
  if (links_alt != nullptr && st->ubuf) U.p = const_cast<C2<R>*>(links_alt);  // ping-pong links of a fused lane
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // Re Tr of one link in the link precision; every sum above one link (the
  // site's F and theta terms, warp, CTA and grid sums) in FP64
  double fsum = 0, tsum = 0;
  if (s < g.V) {
    int c[4];
    site_coords(g, s, c);
    // W = sum_mu [U_mu(x - mu^) - U_mu(x)]; only the entries that enter its
    // traceless anti-Hermitian part are accumulated.
    R im0 = 0, im1 = 0, im2 = 0;           // Im W_ii
    C2<R> w01 = mkc<R>(0, 0), w02 = mkc<R>(0, 0), w12 = mkc<R>(0, 0);  // W_ij - conj(W_ji)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      M3<R> u;
      U.load_ro(mu, s, u);
      fsum += (double)(u.e[0][0].x + u.e[1][1].x + u.e[2][2].x);
      im0 -= u.e[0][0].y; im1 -= u.e[1][1].y; im2 -= u.e[2][2].y;
      w01 = csub<R>(w01, csub<R>(u.e[0][1], cconj<R>(u.e[1][0])));
      w02 = csub<R>(w02, csub<R>(u.e[0][2], cconj<R>(u.e[2][0])));
      w12 = csub<R>(w12, csub<R>(u.e[1][2], cconj<R>(u.e[2][1])));
      M3<R> b;
      U.load_ro(mu, site_back(g, s, c, mu), b);
      im0 += b.e[0][0].y; im1 += b.e[1][1].y; im2 += b.e[2][2].y;
      w01 = cadd<R>(w01, csub<R>(b.e[0][1], cconj<R>(b.e[1][0])));
      w02 = cadd<R>(w02, csub<R>(b.e[0][2], cconj<R>(b.e[2][0])));
      w12 = cadd<R>(w12, csub<R>(b.e[1][2], cconj<R>(b.e[2][1])));
    }
    const R tr = (im0 + im1 + im2) * (R)(1.0 / 3.0);
    const R a0 = im0 - tr, a1 = im1 - tr, a2 = im2 - tr;
    const C2<R> d01 = cscale<R>(w01, (R)0.5), d02 = cscale<R>(w02, (R)0.5), d12 = cscale<R>(w12, (R)0.5);
    delta[s] = mkc<R>(a0, a1);
    delta[g.V + s] = d01;
    delta[2 * g.V + s] = d02;
    delta[3 * g.V + s] = d12;
    // ||Delta_A||_F^2
    tsum = (double)delta_norm2<R>(a0, a1, a2, d01, d02, d12);
  }
  float dmax = 0.f;
  const int dmu = defect_sample_mu();
  if (dmu >= 0 && s < g.V) {
    C2<R> rows[2][3];
    U.load_rows01_ro(dmu, s, rows);
    dmax = rows_defect<R>(rows[0], rows[1]);
  }
  measure_tail(g, fsum, tsum, dmax, partials, st, count_iter, cond, use_cond, batch, 0, sizeof(R) == 8, cond_undo);
}

template <typename R, int ROWS>
cudaError_t launch_measure(const Geom& g, const C2<R>* links, C2<R>* delta, double* partials, DevState* st,
                           int count_iter, unsigned long long cond_handle, int use_cond, cudaStream_t s,
                           int only_if_revert, const Batch& B, const C2<R>* links_alt,
                           unsigned long long cond_undo) {
  MatField<R, ROWS> U{const_cast<C2<R>*>(links), g.V};
  const int64_t nb = measure_blocks(g.V);
  measure_kernel<R, ROWS><<<dim3((unsigned)nb, 1, (unsigned)B.n), MEASURE_THREADS, 0, s>>>(
      g, U, links_alt, delta, partials, st, count_iter, cond_handle, use_cond, only_if_revert, B, cond_undo);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fused update + measure (ping-pong links, backward neighbours recomputed)
// ---------------------------------------------------------------------------

// o = g u h^dagger: rows 0, 1 by products, row 2 = (row0 x row1)^* -- the
// same arithmetic as update_kernel, so that a recomputed neighbour link is
// bit-identical to the one its own thread stores.
template <typename R>
__device__ __forceinline__ void gauge_product(const M3<R>& gl, const M3<R>& u, const M3<R>& h, M3<R>& o) {
  C2<R> T[2][3];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C2<R> acc = cmul_fx<R>(gl.e[i][0], u.e[0][j]);
      acc = cfma<R>(gl.e[i][1], u.e[1][j], acc);
      T[i][j] = cfma<R>(gl.e[i][2], u.e[2][j], acc);
    }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C2<R> acc = cmulc_fx<R>(T[i][0], h.e[j][0]);
      acc = cfmac<R>(T[i][1], h.e[j][1], acc);
      o.e[i][j] = cfmac<R>(T[i][2], h.e[j][2], acc);
    }
  su3_third_row<R>(o.e[0], o.e[1], o.e[2]);
}

// Contribution of one link M to W = sum_mu [U_mu(x - mu^) - U_mu(x)]: the
// entries that enter its traceless anti-Hermitian part, with sign sg.
template <typename R>
__device__ __forceinline__ void add_antiherm(const M3<R>& m, R sg, R& im0, R& im1, R& im2, C2<R>& w01, C2<R>& w02,
                                             C2<R>& w12) {
  im0 += sg * m.e[0][0].y;
  im1 += sg * m.e[1][1].y;
  im2 += sg * m.e[2][2].y;
  const C2<R> a = csub<R>(m.e[0][1], cconj<R>(m.e[1][0]));
  const C2<R> b = csub<R>(m.e[0][2], cconj<R>(m.e[2][0]));
  const C2<R> c = csub<R>(m.e[1][2], cconj<R>(m.e[2][1]));
  w01 = mkc<R>(w01.x + sg * a.x, w01.y + sg * a.y);
  w02 = mkc<R>(w02.x + sg * b.x, w02.y + sg * b.y);
  w12 = mkc<R>(w12.x + sg * c.x, w12.y + sg * c.y);
}

template <typename R, int LROWS, int GROWS>
__global__ void __launch_bounds__(MEASURE_THREADS, 3)
update_measure_kernel(Geom g, C2<R>* __restrict__ U0, C2<R>* __restrict__ U1, MatField<R, GROWS> Gf,
                      C2<R>* __restrict__ delta, double* __restrict__ partials, DevState* __restrict__ st,
                      unsigned long long cond, int use_cond, unsigned long long cond_undo) {
  const int cur = st->ubuf;
  const MatField<R, LROWS> Us{cur ? U1 : U0, g.V}, Ud{cur ? U0 : U1, g.V};
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double fsum = 0, tsum = 0;  // as in measure_kernel: FP64 above one link
  float dmax = 0.f;
  const int dmu = defect_sample_mu();
  if (s < g.V) {
    int c[4];
    site_coords(g, s, c);
    M3<R> gx;
    Gf.load_ro(0, s, gx);
    R im0 = 0, im1 = 0, im2 = 0;
    C2<R> w01 = mkc<R>(0, 0), w02 = mkc<R>(0, 0), w12 = mkc<R>(0, 0);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      M3<R> u, h, o;
      Us.load_ro(mu, s, u);
      Gf.load_ro(0, site_fwd(g, s, c, mu), h);
      gauge_product<R>(gx, u, h, o);
      Ud.store(mu, s, o);
      fsum += (double)(o.e[0][0].x + o.e[1][1].x + o.e[2][2].x);
      add_antiherm<R>(o, (R)-1, im0, im1, im2, w01, w02, w12);
      const int64_t sb = site_back(g, s, c, mu);
      M3<R> b, gb, ob;
      Us.load_ro(mu, sb, b);
      Gf.load_ro(0, sb, gb);
      gauge_product<R>(gb, b, gx, ob);
      add_antiherm<R>(ob, (R)1, im0, im1, im2, w01, w02, w12);
    }
    const R tr = (im0 + im1 + im2) * (R)(1.0 / 3.0);
    const R a0 = im0 - tr, a1 = im1 - tr, a2 = im2 - tr;
    const C2<R> d01 = cscale<R>(w01, (R)0.5), d02 = cscale<R>(w02, (R)0.5), d12 = cscale<R>(w12, (R)0.5);
    delta[s] = mkc<R>(a0, a1);
    delta[g.V + s] = d01;
    delta[2 * g.V + s] = d02;
    delta[3 * g.V + s] = d12;
    tsum = (double)delta_norm2<R>(a0, a1, a2, d01, d02, d12);
    if (dmu >= 0) {
      // the sampled link as this thread stored it above (plain loads see the
      // thread's own stores; keeping the rows in registers instead spilled)
      C2<R> rows[2][3];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) rows[r][c] = Ud.p[Ud.off(dmu, r, c, s)];
      dmax = rows_defect<R>(rows[0], rows[1]);
    }
  }
  measure_tail(g, fsum, tsum, dmax, partials, st, 1, cond, use_cond, false, 1, sizeof(R) == 8, cond_undo);
}

template <typename R, int LROWS, int GROWS>
cudaError_t launch_update_measure(const Geom& g, C2<R>* U0, C2<R>* U1, const C2<R>* gfield, C2<R>* delta,
                                  double* partials, DevState* st, unsigned long long cond, int use_cond,
                                  cudaStream_t s, unsigned long long cond_undo) {
  MatField<R, GROWS> Gf{const_cast<C2<R>*>(gfield), g.V};
  const int64_t nb = measure_blocks(g.V);
  update_measure_kernel<R, LROWS, GROWS><<<(unsigned)nb, MEASURE_THREADS, 0, s>>>(g, U0, U1, Gf, delta, partials,
                                                                                  st, cond, use_cond, cond_undo);
  return cudaGetLastError();
}

__global__ void batch_condition_kernel(const DevState* __restrict__ st, int n, unsigned long long cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    if (!st[i].done) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, any ? 1u : 0u);
}

cudaError_t launch_batch_condition(const DevState* st, int n, unsigned long long cond, cudaStream_t s) {
  batch_condition_kernel<<<1, 256, 0, s>>>(st, n, cond);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// update: U_mu(x) <- g(x) U_mu(x) g^dagger(x + mu^)
// ---------------------------------------------------------------------------

constexpr int UPDATE_THREADS = 128;

template <typename R, int LROWS, int GROWS>
__global__ void __launch_bounds__(UPDATE_THREADS)
update_kernel(Geom g, MatField<R, LROWS> U, MatField<R, GROWS> Gf, Batch B) {
  if (batch_skip(B)) return;
  U.p += blockIdx.z * B.s_links;
  Gf.p += blockIdx.z * B.s_g;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  C2<R> gx[2][3];
  Gf.load_rows01_ro(0, s, gx);  // rows 1-2 of g(x) are all the product needs
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    M3<R> u;
    U.load(mu, s, u);
    M3<R> h;
    int64_t sf, sb;
    site_nbrs_sel(g, s, c, mu, sf, sb);  // selects: no local-memory copy of c[] in the loop
    Gf.load_ro(0, sf, h);
    // T = g(x)[rows 0,1] * U
    C2<R> T[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        C2<R> acc = cmul_fx<R>(gx[i][0], u.e[0][j]);
        acc = cfma<R>(gx[i][1], u.e[1][j], acc);
        T[i][j] = cfma<R>(gx[i][2], u.e[2][j], acc);
      }
    // rows 0,1 of T h^dagger; row 2 = (row0 x row1)^* (the result is in SU(3))
    M3<R> o;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        C2<R> acc = cmulc_fx<R>(T[i][0], h.e[j][0]);
        acc = cfmac<R>(T[i][1], h.e[j][1], acc);
        o.e[i][j] = cfmac<R>(T[i][2], h.e[j][2], acc);
      }
    if (LROWS == 3) su3_third_row<R>(o.e[0], o.e[1], o.e[2]);
    U.store(mu, s, o);
  }
}

template <typename R, int LROWS, int GROWS>
cudaError_t launch_update(const Geom& g, C2<R>* links, const C2<R>* gfield, cudaStream_t s, const Batch& B) {
  MatField<R, LROWS> U{links, g.V};
  MatField<R, GROWS> Gf{const_cast<C2<R>*>(gfield), g.V};
  const int64_t nb = (g.V + UPDATE_THREADS - 1) / UPDATE_THREADS;
  update_kernel<R, LROWS, GROWS><<<dim3((unsigned)nb, 1, (unsigned)B.n), UPDATE_THREADS, 0, s>>>(g, U, Gf, B);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// undo of a rejected step: U_mu(x) <- g^dag(x) U_mu(x) g(x + mu^), G <- g^dag G
// ---------------------------------------------------------------------------

template <typename R, int LROWS, int GROWS>
__global__ void __launch_bounds__(UPDATE_THREADS)
revert_kernel(Geom g, MatField<R, LROWS> U, MatField<R, GROWS> Gf, MatField<R, 3> Gacc, const DevState* st,
              C2<R>* links_alt) {
  if (!st->revert) return;
  if (links_alt != nullptr && st->ubuf) U.p = links_alt;  // the current buffer of a fused lane
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  M3<R> gx;
  Gf.load_ro(0, s, gx);
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    M3<R> u, h;
    U.load(mu, s, u);
    Gf.load_ro(0, site_fwd(g, s, c, mu), h);
    // T = (g^dag U)[rows 0,1]: T_ij = sum_k conj(g_ki) U_kj
    C2<R> T[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        C2<R> acc = cconjmul<R>(gx.e[0][i], u.e[0][j]);
        acc = cadd<R>(acc, cconjmul<R>(gx.e[1][i], u.e[1][j]));
        T[i][j] = cadd<R>(acc, cconjmul<R>(gx.e[2][i], u.e[2][j]));
      }
    M3<R> o;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        C2<R> acc = cmul<R>(T[i][0], h.e[0][j]);
        acc = cfma<R>(T[i][1], h.e[1][j], acc);
        o.e[i][j] = cfma<R>(T[i][2], h.e[2][j], acc);
      }
    su3_third_row<R>(o.e[0], o.e[1], o.e[2]);
    U.store(mu, s, o);
  }
  if (Gacc.p != nullptr) {
    M3<R> G0, G1;
    Gacc.load(0, s, G0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        C2<R> acc = cconjmul<R>(gx.e[0][i], G0.e[0][j]);
        acc = cadd<R>(acc, cconjmul<R>(gx.e[1][i], G0.e[1][j]));
        G1.e[i][j] = cadd<R>(acc, cconjmul<R>(gx.e[2][i], G0.e[2][j]));
      }
    Gacc.store(0, s, G1);
  }
}

template <typename R, int LROWS, int GROWS>
cudaError_t launch_revert(const Geom& g, C2<R>* links, const C2<R>* gfield, C2<R>* Gacc, const DevState* st,
                          cudaStream_t s, C2<R>* links_alt) {
  MatField<R, LROWS> U{links, g.V};
  MatField<R, GROWS> Gf{const_cast<C2<R>*>(gfield), g.V};
  MatField<R, 3> Ga{Gacc, g.V};
  const int64_t nb = (g.V + UPDATE_THREADS - 1) / UPDATE_THREADS;
  revert_kernel<R, LROWS, GROWS><<<(unsigned)nb, UPDATE_THREADS, 0, s>>>(g, U, Gf, Ga, st, links_alt);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// layout conversion
// ---------------------------------------------------------------------------

constexpr int CONV_THREADS = 256;

// nmat matrices per site field: links use nmat = 4 (mu), site fields nmat = 1.
template <typename R, int ROWS>
__global__ void from_aos_kernel(int64_t V, int nmat, const double2* __restrict__ aos, MatField<R, ROWS> F) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * nmat) return;
  const int m = (int)(i / V);
  const int64_t s = i - (int64_t)m * V;
  const double2* src = aos + i * 9;
#pragma unroll
  for (int r = 0; r < ROWS; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double2 v = __ldg(&src[r * 3 + c]);
      F.p[F.off(m, r, c, s)] = mkc<R>((R)v.x, (R)v.y);
    }
}

template <typename R, int ROWS>
__global__ void to_aos_kernel(int64_t V, int nmat, MatField<R, ROWS> F, double2* __restrict__ aos) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= V * nmat) return;
  const int m = (int)(i / V);
  const int64_t s = i - (int64_t)m * V;
  M3<R> M;
  F.load_ro(m, s, M);
  double2* dst = aos + i * 9;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) dst[r * 3 + c] = make_double2((double)M.e[r][c].x, (double)M.e[r][c].y);
}

template <typename R, int ROWS>
cudaError_t launch_links_from_aos(const Geom& g, const double* aos, C2<R>* links, cudaStream_t s) {
  MatField<R, ROWS> F{links, g.V};
  const int64_t n = 4 * g.V;
  from_aos_kernel<R, ROWS><<<(unsigned)((n + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(
      g.V, 4, reinterpret_cast<const double2*>(aos), F);
  return cudaGetLastError();
}

template <typename R, int ROWS>
cudaError_t launch_links_to_aos(const Geom& g, const C2<R>* links, double* aos, cudaStream_t s) {
  MatField<R, ROWS> F{const_cast<C2<R>*>(links), g.V};
  const int64_t n = 4 * g.V;
  to_aos_kernel<R, ROWS><<<(unsigned)((n + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(
      g.V, 4, F, reinterpret_cast<double2*>(aos));
  return cudaGetLastError();
}

template <typename R, int ROWS>
cudaError_t launch_sites_to_aos(const Geom& g, const C2<R>* field, double* aos, cudaStream_t s) {
  MatField<R, ROWS> F{const_cast<C2<R>*>(field), g.V};
  to_aos_kernel<R, ROWS><<<(unsigned)((g.V + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(
      g.V, 1, F, reinterpret_cast<double2*>(aos));
  return cudaGetLastError();
}

template <typename R, int ROWS>
cudaError_t launch_sites_from_aos(const Geom& g, const double* aos, C2<R>* field, cudaStream_t s) {
  MatField<R, ROWS> F{field, g.V};
  from_aos_kernel<R, ROWS><<<(unsigned)((g.V + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(
      g.V, 1, reinterpret_cast<const double2*>(aos), F);
  return cudaGetLastError();
}

template <typename R>
__global__ void delta_to_aos_kernel(int64_t V, const C2<R>* __restrict__ d, double2* __restrict__ aos) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  const C2<R> f0 = d[s], f1 = d[V + s], f2 = d[2 * V + s], f3 = d[3 * V + s];
  const double a0 = f0.x, a1 = f0.y, a2 = -(a0 + a1);
  double2* o = aos + s * 9;
  o[0] = make_double2(0.0, a0);
  o[1] = make_double2(f1.x, f1.y);
  o[2] = make_double2(f2.x, f2.y);
  o[3] = make_double2(-(double)f1.x, (double)f1.y);
  o[4] = make_double2(0.0, a1);
  o[5] = make_double2(f3.x, f3.y);
  o[6] = make_double2(-(double)f2.x, (double)f2.y);
  o[7] = make_double2(-(double)f3.x, (double)f3.y);
  o[8] = make_double2(0.0, a2);
}

template <typename R>
cudaError_t launch_delta_to_aos(const Geom& g, const C2<R>* delta, double* aos, cudaStream_t s) {
  delta_to_aos_kernel<R><<<(unsigned)((g.V + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(
      g.V, delta, reinterpret_cast<double2*>(aos));
  return cudaGetLastError();
}

template <typename R, int ROWS>
__global__ void identity_kernel(int64_t V, MatField<R, ROWS> F) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
#pragma unroll
  for (int r = 0; r < ROWS; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) F.p[F.off(0, r, c, s)] = mkc<R>(r == c ? (R)1 : (R)0, (R)0);
}

template <typename R, int ROWS>
cudaError_t launch_set_identity(const Geom& g, C2<R>* field, cudaStream_t s) {
  MatField<R, ROWS> F{field, g.V};
  identity_kernel<R, ROWS><<<(unsigned)((g.V + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(g.V, F);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SU(3) validation of user links
// ---------------------------------------------------------------------------

__device__ __forceinline__ double su3_defect_of(const double2* __restrict__ mat) {
  double2 m[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) m[r][c] = __ldg(&mat[r * 3 + c]);
  double d = 0.0;
  // U U^dag is Hermitian: its upper triangle holds every distinct entry
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = r; c < 3; ++c) {
      double2 acc = mkc<double>(0.0, 0.0);
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = cfmac<double>(m[r][k], m[c][k], acc);
      if (r == c) acc.x -= 1.0;
      d = fmax(d, fmax(fabs(acc.x), fabs(acc.y)));
    }
  double2 cr[3];
  su3_third_row<double>(m[0], m[1], cr);  // conj(r0 x r1)
  // det = r2 . (r0 x r1) = sum_j r2_j conj(cr_j)
  double2 det = mkc<double>(0.0, 0.0);
#pragma unroll
  for (int j = 0; j < 3; ++j) det = cfmac<double>(m[2][j], cr[j], det);
  d = fmax(d, sqrt((det.x - 1.0) * (det.x - 1.0) + det.y * det.y));
  bool finite = true;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) finite = finite && isfinite(m[r][c].x) && isfinite(m[r][c].y);
  return (!finite || !isfinite(d)) ? INFINITY : d;
}

// Grid-stride over the matrices; the maximum of a CTA goes to *out by one
// atomic (a few thousand in all, instead of one per warp on one address).
__global__ void su3_defect_kernel(const double2* __restrict__ aos, int64_t nmat, unsigned long long* out) {
  double d = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nmat; i += (int64_t)gridDim.x * blockDim.x)
    d = fmax(d, su3_defect_of(aos + i * 9));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
  __shared__ double wm[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) wm[warp] = d;
  __syncthreads();
  if (warp == 0) {
    d = lane < nw ? wm[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(d));
  }
}

cudaError_t launch_su3_defect(const double* aos, int64_t nmat, unsigned long long* out_bits, cudaStream_t s,
                              int reset) {
  if (reset) {
    cudaError_t e = cudaMemsetAsync(out_bits, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = std::min<int64_t>((nmat + CONV_THREADS - 1) / CONV_THREADS, 152 * 8);
  su3_defect_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), CONV_THREADS, 0, s>>>(
      reinterpret_cast<const double2*>(aos), nmat, out_bits);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// momentum filter table (kernel k1 of Sec. 3.2)
// ---------------------------------------------------------------------------

template <typename R>
__global__ void filter_table_kernel(Geom g, const double* __restrict__ sin2, int lmax, double alpha, double p2max,
                                    int plain_sd, R* __restrict__ K) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  const double p2 = sin2[3 * lmax + c[3]] + sin2[2 * lmax + c[2]] + sin2[lmax + c[1]] + sin2[c[0]];
  double k = 0.0;
  if (s != 0) k = plain_sd ? alpha / (double)g.V : alpha * p2max / (p2 * (double)g.V);
  K[s] = (R)k;
}

template <typename R>
cudaError_t launch_filter_table(const Geom& g, const double* sin2, int lmax, double alpha, double p2max, int plain_sd,
                                R* K, cudaStream_t s) {
  filter_table_kernel<R><<<(unsigned)((g.V + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(
      g, sin2, lmax, alpha, p2max, plain_sd, K);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// controller state, precision conversion, FP64 projection of G
// ---------------------------------------------------------------------------

__global__ void set_state_kernel(DevState* st, double tol, int max_iter, int reset_iter, int hist_cap, double* Fh,
                                 double* Th, int* flh, double* dfh, double defect_bound, int flags0) {
  st->tol = tol;
  st->max_iter = max_iter;
  if (reset_iter) {
    st->iter = 0;
    st->theta_prev = 0.0;
    st->status = ST_OK;
    st->revert = 0;
    st->use_m = 0;
    st->n_fallback = 0;
    st->redo = 0;
    st->repaired = 0;
    st->snaps = 0;
  }
  st->hist_cap = hist_cap;
  st->F_hist = Fh;
  st->theta_hist = Th;
  st->flag_hist = flh;
  st->defect_hist = dfh;
  st->defect_bound = defect_bound;
  if (hist_cap > 0 && reset_iter) {
    Fh[0] = st->F;
    Th[0] = st->theta;
    if (flh) flh[0] = flags0;
    if (dfh) dfh[0] = st->defect;
  }
}

cudaError_t launch_set_state(DevState* st, double tol, int max_iter, int reset_iter, int hist_cap, double* F_hist,
                             double* theta_hist, cudaStream_t s, int* flag_hist, double* defect_hist,
                             double defect_bound, int flags0) {
  set_state_kernel<<<1, 1, 0, s>>>(st, tol, max_iter, reset_iter, hist_cap, F_hist, theta_hist, flag_hist,
                                   defect_hist, defect_bound, flags0);
  return cudaGetLastError();
}

// Gram-Schmidt on rows 1-2 of every link, row 3 = (a x b)^* when stored.
template <typename R, int ROWS>
__global__ void reunitarize_links_kernel(int64_t n, MatField<R, ROWS> U) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m = (int)(i / U.V);
  const int64_t s = i - (int64_t)m * U.V;
  M3<R> M;
  U.load(m, s, M);
  C2<R>* a = M.e[0];
  C2<R>* b = M.e[1];
  const R ia = (R)1 / sqrt(cnorm2<R>(a[0]) + cnorm2<R>(a[1]) + cnorm2<R>(a[2]));
#pragma unroll
  for (int j = 0; j < 3; ++j) a[j] = cscale<R>(a[j], ia);
  C2<R> ip = cconjmul<R>(a[0], b[0]);
  ip = cadd<R>(ip, cconjmul<R>(a[1], b[1]));
  ip = cadd<R>(ip, cconjmul<R>(a[2], b[2]));
  const C2<R> nip = mkc<R>(-ip.x, -ip.y);
#pragma unroll
  for (int j = 0; j < 3; ++j) b[j] = cfma<R>(nip, a[j], b[j]);
  const R ib = (R)1 / sqrt(cnorm2<R>(b[0]) + cnorm2<R>(b[1]) + cnorm2<R>(b[2]));
#pragma unroll
  for (int j = 0; j < 3; ++j) b[j] = cscale<R>(b[j], ib);
  su3_third_row<R>(M.e[0], M.e[1], M.e[2]);
  U.store(m, s, M);
}

__global__ void mark_repaired_kernel(DevState* st) {
  st->repaired = 1;
  if (st->status == ST_DEFECT) st->status = ST_OK;
}

template <typename R, int ROWS>
cudaError_t launch_reunitarize_links(const Geom& g, C2<R>* links, DevState* st, cudaStream_t s) {
  MatField<R, ROWS> U{links, g.V};
  const int64_t n = 4 * g.V;
  reunitarize_links_kernel<R, ROWS><<<(unsigned)((n + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(n, U);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  mark_repaired_kernel<<<1, 1, 0, s>>>(st);
  return cudaGetLastError();
}

__global__ void c2_f64_to_f32_kernel(const double2* __restrict__ in, float2* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

__global__ void c2_f32_to_f64_kernel(const float2* __restrict__ in, double2* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

cudaError_t launch_c2_f64_to_f32(const double2* in, float2* out, int64_t n, cudaStream_t s) {
  c2_f64_to_f32_kernel<<<(unsigned)((n + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_c2_f32_to_f64(const float2* in, double2* out, int64_t n, cudaStream_t s) {
  c2_f32_to_f64_kernel<<<(unsigned)((n + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

// Gram-Schmidt projection of rows 1-2 to SU(3) in FP64, row 3 = (a x b)^*.
__global__ void project_sites_kernel(int64_t V, const float2* __restrict__ in, double2* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= V) return;
  double2 a[3], b[3], c[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float2 x = in[(0 * 3 + j) * V + s], y = in[(1 * 3 + j) * V + s];
    a[j] = make_double2(x.x, x.y);
    b[j] = make_double2(y.x, y.y);
  }
  const double ia = rsqrt(cnorm2<double>(a[0]) + cnorm2<double>(a[1]) + cnorm2<double>(a[2]));
#pragma unroll
  for (int j = 0; j < 3; ++j) a[j] = cscale<double>(a[j], ia);
  double2 ip = cconjmul<double>(a[0], b[0]);
  ip = cadd<double>(ip, cconjmul<double>(a[1], b[1]));
  ip = cadd<double>(ip, cconjmul<double>(a[2], b[2]));
  const double2 nip = make_double2(-ip.x, -ip.y);
#pragma unroll
  for (int j = 0; j < 3; ++j) b[j] = cfma<double>(nip, a[j], b[j]);
  const double ib = rsqrt(cnorm2<double>(b[0]) + cnorm2<double>(b[1]) + cnorm2<double>(b[2]));
#pragma unroll
  for (int j = 0; j < 3; ++j) b[j] = cscale<double>(b[j], ib);
  su3_third_row<double>(a, b, c);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    out[(0 * 3 + j) * V + s] = a[j];
    out[(1 * 3 + j) * V + s] = b[j];
    out[(2 * 3 + j) * V + s] = c[j];
  }
}

cudaError_t launch_project_sites_f32_to_f64(const Geom& g, const float2* G32, double2* G64, cudaStream_t s) {
  project_sites_kernel<<<(unsigned)((g.V + CONV_THREADS - 1) / CONV_THREADS), CONV_THREADS, 0, s>>>(g.V, G32, G64);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// explicit instantiations
// ---------------------------------------------------------------------------

#define LGF_INST_R_ROWS(R, ROWS)                                                                                     \
  template cudaError_t launch_measure<R, ROWS>(const Geom&, const C2<R>*, C2<R>*, double*, DevState*, int,           \
                                               unsigned long long, int, cudaStream_t, int, const Batch&,            \
                                               const C2<R>*, unsigned long long);                                   \
  template cudaError_t launch_links_from_aos<R, ROWS>(const Geom&, const double*, C2<R>*, cudaStream_t);            \
  template cudaError_t launch_links_to_aos<R, ROWS>(const Geom&, const C2<R>*, double*, cudaStream_t);              \
  template cudaError_t launch_sites_to_aos<R, ROWS>(const Geom&, const C2<R>*, double*, cudaStream_t);              \
  template cudaError_t launch_sites_from_aos<R, ROWS>(const Geom&, const double*, C2<R>*, cudaStream_t);            \
  template cudaError_t launch_set_identity<R, ROWS>(const Geom&, C2<R>*, cudaStream_t);                        \
  template cudaError_t launch_reunitarize_links<R, ROWS>(const Geom&, C2<R>*, DevState*, cudaStream_t);

LGF_INST_R_ROWS(double, 3)
LGF_INST_R_ROWS(double, 2)
LGF_INST_R_ROWS(float, 3)
LGF_INST_R_ROWS(float, 2)

template cudaError_t launch_revert<double, 3, 3>(const Geom&, C2<double>*, const C2<double>*, C2<double>*,
                                                 const DevState*, cudaStream_t, C2<double>*);
template cudaError_t launch_revert<double, 2, 3>(const Geom&, C2<double>*, const C2<double>*, C2<double>*,
                                                 const DevState*, cudaStream_t, C2<double>*);
template cudaError_t launch_revert<float, 2, 2>(const Geom&, C2<float>*, const C2<float>*, C2<float>*,
                                                 const DevState*, cudaStream_t, C2<float>*);
template cudaError_t launch_revert<float, 3, 3>(const Geom&, C2<float>*, const C2<float>*, C2<float>*,
                                                 const DevState*, cudaStream_t, C2<float>*);
template cudaError_t launch_update<double, 3, 3>(const Geom&, C2<double>*, const C2<double>*, cudaStream_t, const Batch&);
template cudaError_t launch_update<double, 2, 3>(const Geom&, C2<double>*, const C2<double>*, cudaStream_t, const Batch&);
template cudaError_t launch_update<float, 2, 2>(const Geom&, C2<float>*, const C2<float>*, cudaStream_t, const Batch&);
template cudaError_t launch_update<float, 3, 3>(const Geom&, C2<float>*, const C2<float>*, cudaStream_t, const Batch&);
#define LGF_INST_UM(R, LR, GR)                                                                                     \
  template cudaError_t launch_update_measure<R, LR, GR>(const Geom&, C2<R>*, C2<R>*, const C2<R>*, C2<R>*, double*, \
                                                        DevState*, unsigned long long, int, cudaStream_t,          \
                                                        unsigned long long);
LGF_INST_UM(float, 2, 2)
LGF_INST_UM(float, 3, 3)
template cudaError_t launch_delta_to_aos<double>(const Geom&, const C2<double>*, double*, cudaStream_t);
template cudaError_t launch_delta_to_aos<float>(const Geom&, const C2<float>*, double*, cudaStream_t);
template cudaError_t launch_filter_table<double>(const Geom&, const double*, int, double, double, int, double*,
                                                 cudaStream_t);
template cudaError_t launch_filter_table<float>(const Geom&, const double*, int, double, double, int, float*,
                                                cudaStream_t);

}  // namespace lgf
