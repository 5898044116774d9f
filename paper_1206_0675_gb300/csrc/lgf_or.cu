// Overrelaxation Landau gauge fixing: one colour of a checkerboard sweep.
//
// arXiv:1206.0675 (Sec. 3.2) names overrelaxation as the gauge-fixing method
// that needs less memory than the Fourier-accelerated one; the method is the
// published one it refers to:
//   * local maximisation of F[g] = (1/(4 Nc V)) sum Re Tr g(x) U_mu(x)
//     g^dag(x + mu^) (Sec. 2) one site at a time, all sites of one
//     checkerboard colour at once (no site has a neighbour of its own colour);
//   * Cabibbo and Marinari (Phys. Lett. B 119 (1982) 387): the SU(3)
//     maximisation in the SU(2) subgroups (0,1), (0,2), (1,2) in turn;
//   * Mandula and Ogilvie (Phys. Lett. B 248 (1990) 156): each SU(2)
//     maximiser r replaced by r^omega ~ 1 + omega (r - 1), 1 <= omega < 2,
//     projected back onto SU(2).
// At a site x of the colour, w(x) = sum_mu [U_mu(x) + U_mu^dag(x - mu^)]; the
// hit gives g(x), and then U_mu(x) <- g(x) U_mu(x), U_mu(x - mu^) <-
// U_mu(x - mu^) g^dag(x) and, when the transform is tracked, G(x) <- g(x) G(x).
// Every link joins two sites of opposite colour, so within one colour each
// link is read and written by exactly one thread: the update is in place.
//
// One thread per site of the colour.  Its links are read twice (once for w,
// once for the product, the second time from L1/L2) so that only w, the
// running subgroup block and g stay in registers.  The site algebra runs in
// the link precision; rows 1-2 of every product are formed and row 3 is
// rebuilt as (a x b)^* (Sec. 3.2), as in the Fourier-accelerated update.
#include "lgf_internal.h"

namespace lgf {

constexpr int OR_THREADS = 128;

// 1/sqrt(x) in the lane precision for x > 0 (FP32: the hardware estimate and
// one Newton step).
template <typename R> __device__ __forceinline__ R or_rsqrt(R x);
template <> __device__ __forceinline__ double or_rsqrt<double>(double x) { return rsqrt_fp64(x); }
template <> __device__ __forceinline__ float or_rsqrt<float>(float x) {
  const float y = rsqrtf(x);
  return y * fmaf(-0.5f * x * y, y, 1.5f);
}

// Overrelaxed SU(2) element of one subgroup from its 2x2 block
// B = [[mii, mij], [mji, mjj]] of the running local field.  In quaternion
// form B contributes Re Tr(r B) = 2 (r0 b0 - r1 b1 - r2 b2 - r3 b3) with
// b0 = Re(B00 + B11)/2, b1 = Im(B01 + B10)/2, b2 = Re(B01 - B10)/2,
// b3 = Im(B00 - B11)/2, largest at r = (b0, -b1, -b2, -b3)/|b| (the common
// factor 1/2 drops out); r = 1 where |b|^2 is below the smallest normal
// number.  q = (1 - omega) + omega r, normalised (|q| >= 1 for omega >= 1).
// Result as the matrix [[a, b], [-conj(b), conj(a)]], a = q0 + i q3,
// b = q2 + i q1.
template <typename R>
__device__ __forceinline__ void or_subgroup(C2<R> mii, C2<R> mij, C2<R> mji, C2<R> mjj, R omega, C2<R>& a,
                                            C2<R>& b) {
  const R b0 = mii.x + mjj.x, b1 = mij.y + mji.y, b2 = mij.x - mji.x, b3 = mii.y - mjj.y;
  const R n2 = fma(b0, b0, fma(b1, b1, fma(b2, b2, b3 * b3)));
  const R tiny = sizeof(R) == sizeof(double) ? (R)2.2250738585072014e-308 : (R)1.17549435e-38f;
  R r0 = 1, r1 = 0, r2 = 0, r3 = 0;
  if (n2 >= tiny) {
    const R inv = or_rsqrt<R>(n2);
    r0 = b0 * inv;
    r1 = -b1 * inv;
    r2 = -b2 * inv;
    r3 = -b3 * inv;
  }
  const R q0 = fma(omega, r0, (R)1 - omega), q1 = omega * r1, q2 = omega * r2, q3 = omega * r3;
  const R iq = or_rsqrt<R>(fma(q0, q0, fma(q1, q1, fma(q2, q2, q3 * q3))));
  a = mkc<R>(q0 * iq, q3 * iq);
  b = mkc<R>(q2 * iq, q1 * iq);
}

// (xi, xj) <- [[a, b], [-conj(b), conj(a)]] (xi, xj): one column of the two
// rows a subgroup acts on.
template <typename R> __device__ __forceinline__ void or_rot(C2<R> a, C2<R> b, C2<R>& xi, C2<R>& xj) {
  const C2<R> ni = cfma<R>(b, xj, cmul<R>(a, xi));
  const C2<R> nj = csub<R>(cconjmul<R>(a, xj), cconjmul<R>(b, xi));
  xi = ni;
  xj = nj;
}

// g(x) of one Cabibbo-Marinari hit on the local field M (M is consumed).
template <typename R> __device__ __forceinline__ void or_site_gauge(M3<R>& M, R omega, M3<R>& gx) {
  C2<R> a, b;
  // subgroup (0, 1): g = R01 embedded; rows 0 and 1 of M rotated
  or_subgroup<R>(M.e[0][0], M.e[0][1], M.e[1][0], M.e[1][1], omega, a, b);
  gx.e[0][0] = a;
  gx.e[0][1] = b;
  gx.e[0][2] = mkc<R>(0, 0);
  gx.e[1][0] = mkc<R>(-b.x, b.y);
  gx.e[1][1] = cconj<R>(a);
  gx.e[1][2] = mkc<R>(0, 0);
  gx.e[2][0] = mkc<R>(0, 0);
  gx.e[2][1] = mkc<R>(0, 0);
  gx.e[2][2] = mkc<R>(1, 0);
#pragma unroll
  for (int c = 0; c < 3; ++c) or_rot<R>(a, b, M.e[0][c], M.e[1][c]);
  // subgroup (0, 2): rows 0 and 2 of g; of M only row 2's columns 1 and 2
  // are read again
  or_subgroup<R>(M.e[0][0], M.e[0][2], M.e[2][0], M.e[2][2], omega, a, b);
#pragma unroll
  for (int c = 0; c < 3; ++c) or_rot<R>(a, b, gx.e[0][c], gx.e[2][c]);
#pragma unroll
  for (int c = 1; c < 3; ++c) or_rot<R>(a, b, M.e[0][c], M.e[2][c]);
  // subgroup (1, 2): rows 1 and 2 of g
  or_subgroup<R>(M.e[1][1], M.e[1][2], M.e[2][1], M.e[2][2], omega, a, b);
#pragma unroll
  for (int c = 0; c < 3; ++c) or_rot<R>(a, b, gx.e[1][c], gx.e[2][c]);
}

// x - mu^ with periodic wrap, for a direction mu known only at run time:
// selects instead of indexed arrays, so that coordinates and geometry stay in
// registers (no local-memory frame in the loops over mu).
__device__ __forceinline__ int64_t or_back(const Geom& g, int64_t s, const int c[4], int mu) {
  int cm = c[0], L = g.L[0];
  int64_t st = 1;
  if (mu == 1) { cm = c[1]; L = g.L[1]; st = g.stride[1]; }
  if (mu == 2) { cm = c[2]; L = g.L[2]; st = g.stride[2]; }
  if (mu == 3) { cm = c[3]; L = g.L[3]; st = g.stride[3]; }
  return cm == 0 ? s + (int64_t)(L - 1) * st : s - st;
}

template <typename R, int ROWS>
__global__ void __launch_bounds__(OR_THREADS)
or_half_sweep_kernel(Geom g, C2<R>* __restrict__ U0, C2<R>* __restrict__ U1, const DevState* __restrict__ st,
                     C2<R>* __restrict__ G, int parity, R omega) {
  // fused FP32 lanes keep their current links in one of two buffers
  const MatField<R, ROWS> U{(U1 != nullptr && st->ubuf) ? U1 : U0, g.V};
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if ((int64_t)j >= (g.V >> 1)) return;
  // site of the colour: x = 2 xh + ((y + z + t + parity) & 1) in its (y, z, t) row
  const uint32_t hx = (uint32_t)g.L[0] >> 1;
  const uint32_t row = j / hx;
  int c[4];
  c[1] = (int)(row % (uint32_t)g.L[1]);
  const uint32_t r2 = row / (uint32_t)g.L[1];
  c[2] = (int)(r2 % (uint32_t)g.L[2]);
  c[3] = (int)(r2 / (uint32_t)g.L[2]);
  c[0] = 2 * (int)(j - row * hx) + ((c[1] + c[2] + c[3] + parity) & 1);
  const int64_t s = (int64_t)c[0] + (int64_t)g.L[0] * row;

  // w(x) = sum_mu [U_mu(x) + U_mu^dag(x - mu^)]
  M3<R> M;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k) M.e[r][k] = mkc<R>(0, 0);
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    M3<R> u;
    U.load(mu, s, u);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) M.e[r][k] = cadd<R>(M.e[r][k], u.e[r][k]);
    U.load(mu, or_back(g, s, c, mu), u);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int k = 0; k < 3; ++k) M.e[r][k] = cadd<R>(M.e[r][k], cconj<R>(u.e[k][r]));
  }

  M3<R> gx;
  or_site_gauge<R>(M, omega, gx);

#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    // U_mu(x) <- g U_mu(x): rows 0, 1 by products, row 2 = (row0 x row1)^*
    M3<R> u, o;
    U.load(mu, s, u);
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        C2<R> acc = cmul_fx<R>(gx.e[i][0], u.e[0][k]);
        acc = cfma<R>(gx.e[i][1], u.e[1][k], acc);
        o.e[i][k] = cfma<R>(gx.e[i][2], u.e[2][k], acc);
      }
    su3_third_row<R>(o.e[0], o.e[1], o.e[2]);
    U.store(mu, s, o);
    // U_mu(x - mu^) <- U_mu(x - mu^) g^dag: rows 0, 1 of the old link suffice
    const int64_t sb = or_back(g, s, c, mu);
    C2<R> v[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) v[i][k] = U.p[U.off(mu, i, k, sb)];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        C2<R> acc = cmulc_fx<R>(v[i][0], gx.e[k][0]);
        acc = cfmac<R>(v[i][1], gx.e[k][1], acc);
        o.e[i][k] = cfmac<R>(v[i][2], gx.e[k][2], acc);
      }
    su3_third_row<R>(o.e[0], o.e[1], o.e[2]);
    U.store(mu, sb, o);
  }

  if (G != nullptr) {
    // G(x) <- g(x) G(x), full 3x3
    const MatField<R, 3> Gf{G, g.V};
    M3<R> Go, Gn;
    Gf.load(0, s, Go);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        C2<R> acc = cmul<R>(gx.e[i][0], Go.e[0][k]);
        acc = cfma<R>(gx.e[i][1], Go.e[1][k], acc);
        Gn.e[i][k] = cfma<R>(gx.e[i][2], Go.e[2][k], acc);
      }
    Gf.store(0, s, Gn);
  }
}

template <typename R, int ROWS>
cudaError_t launch_or_half_sweep(const Geom& g, C2<R>* U0, C2<R>* U1, const DevState* st, C2<R>* G, int parity,
                                 double omega, cudaStream_t s) {
  const int64_t n = g.V >> 1;
  const unsigned nb = (unsigned)((n + OR_THREADS - 1) / OR_THREADS);
  or_half_sweep_kernel<R, ROWS><<<nb, OR_THREADS, 0, s>>>(g, U0, U1, st, G, parity & 1, (R)omega);
  return cudaGetLastError();
}

template cudaError_t launch_or_half_sweep<double, 3>(const Geom&, double2*, double2*, const DevState*, double2*, int,
                                                     double, cudaStream_t);
template cudaError_t launch_or_half_sweep<double, 2>(const Geom&, double2*, double2*, const DevState*, double2*, int,
                                                     double, cudaStream_t);
template cudaError_t launch_or_half_sweep<float, 3>(const Geom&, float2*, float2*, const DevState*, float2*, int,
                                                    double, cudaStream_t);
template cudaError_t launch_or_half_sweep<float, 2>(const Geom&, float2*, float2*, const DevState*, float2*, int,
                                                    double, cudaStream_t);

}  // namespace lgf
