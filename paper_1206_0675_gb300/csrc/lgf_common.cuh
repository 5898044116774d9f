// Shared device helpers of the lgf CUDA library: complex arithmetic, SU(3)
// row algebra and structure-of-arrays link access.
//
// Storage (all fields are structure-of-arrays over lattice sites, site index
// s = x + Lx*(y + Ly*(z + Lz*t))):
//   links  : [mu][row][col][s] complex (double2 or float2); ROWS = 3 keeps the
//            full matrix ("18-real"), ROWS = 2 keeps rows 1-2 ("12-real") and
//            rebuilds row 3 as (a x b)^* (Sec. 3.2 of arXiv:1206.0675).
//   g, G   : [row][col][s] complex, same convention without mu.
//   Delta  : 4 complex fields [f][s]: f0 = Im D11 + i Im D22, f1 = D12,
//            f2 = D13, f3 = D23 of the traceless anti-Hermitian divergence.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lgf {

template <typename R> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };
template <typename R> using C2 = typename cplx_of<R>::type;

template <typename R> __host__ __device__ __forceinline__ C2<R> mkc(R re, R im) {
  C2<R> z; z.x = re; z.y = im; return z;
}
template <typename R> __device__ __forceinline__ C2<R> cadd(C2<R> a, C2<R> b) { return mkc<R>(a.x + b.x, a.y + b.y); }
template <typename R> __device__ __forceinline__ C2<R> csub(C2<R> a, C2<R> b) { return mkc<R>(a.x - b.x, a.y - b.y); }
template <typename R> __device__ __forceinline__ C2<R> cconj(C2<R> a) { return mkc<R>(a.x, -a.y); }
// a * b
template <typename R> __device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
  return mkc<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename R> __device__ __forceinline__ C2<R> cmulc(C2<R> a, C2<R> b) {
  return mkc<R>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conj(a) * b
template <typename R> __device__ __forceinline__ C2<R> cconjmul(C2<R> a, C2<R> b) {
  return mkc<R>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// The same products with their rounding fixed by explicit fused
// multiply-adds, whatever the compiler's contraction choices.  The link
// update uses these, so that the fused update + measurement can recompute a
// neighbour's updated link bit for bit.
template <typename R> __device__ __forceinline__ C2<R> cmul_fx(C2<R> a, C2<R> b) {
  return mkc<R>(fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x));
}
template <typename R> __device__ __forceinline__ C2<R> cmulc_fx(C2<R> a, C2<R> b) {
  return mkc<R>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -(a.x * b.y)));
}
// acc + a * b
template <typename R> __device__ __forceinline__ C2<R> cfma(C2<R> a, C2<R> b, C2<R> acc) {
  return mkc<R>(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc + a * conj(b)
template <typename R> __device__ __forceinline__ C2<R> cfmac(C2<R> a, C2<R> b, C2<R> acc) {
  return mkc<R>(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.y, b.x, fma(-a.x, b.y, acc.y)));
}
template <typename R> __device__ __forceinline__ C2<R> cscale(C2<R> a, R s) { return mkc<R>(a.x * s, a.y * s); }
template <typename R> __device__ __forceinline__ R cnorm2(C2<R> a) { return fma(a.x, a.x, a.y * a.y); }

template <typename To, typename From> __device__ __forceinline__ C2<To> ccast(C2<From> a) {
  return mkc<To>((To)a.x, (To)a.y);
}

// 1/sqrt(x) in FP64 for finite x > 0: the hardware estimate of PTX
// rsqrt.approx.ftz.f64 refined by one third-order Householder step for
// f(y) = y^-2 - x.  With e = 1 - x y0^2 the exact value is
// y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + 5e^3/16 + ...); keeping the
// terms to e^2 leaves a relative error of (5/16) e^3, below 2^-60 for an
// estimate within 2^-20, so the result is within rounding of 1/sqrt(x).
// Five FP64 operations after the estimate.
__device__ __forceinline__ double rsqrt_fp64(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-(x * y), y, 1.0);
  return fma(y * e, fma(0.375, e, 0.5), y);
}

// 3x3 complex matrix held in registers.
template <typename R> struct M3 {
  C2<R> e[3][3];
};

// Third row of an SU(3) matrix from its first two: c = (a x b)^*
// (Sec. 3.2 of arXiv:1206.0675).  Each entry c_j = conj(a_k b_l - a_l b_k)
// is one multiply and three fused multiply-adds per real component.
template <typename R> __device__ __forceinline__ C2<R> cross_conj(C2<R> ak, C2<R> al, C2<R> bk, C2<R> bl) {
  // re(a_k b_l - a_l b_k), and minus its imaginary part
  const R re = fma(ak.x, bl.x, fma(-ak.y, bl.y, fma(-al.x, bk.x, al.y * bk.y)));
  const R nim = fma(-ak.x, bl.y, fma(-ak.y, bl.x, fma(al.x, bk.y, al.y * bk.x)));
  return mkc<R>(re, nim);
}

template <typename R> __device__ __forceinline__ void su3_third_row(const C2<R> a[3], const C2<R> b[3], C2<R> c[3]) {
  c[0] = cross_conj<R>(a[1], a[2], b[1], b[2]);
  c[1] = cross_conj<R>(a[2], a[0], b[2], b[0]);
  c[2] = cross_conj<R>(a[0], a[1], b[0], b[1]);
}

// Structure-of-arrays matrix field: element (m, r, c) of site s lives at
// p[((m * ROWS + r) * 3 + c) * V + s]; m is the direction for links, 0 otherwise.
template <typename R, int ROWS> struct MatField {
  C2<R>* p;
  int64_t V;
  __device__ __forceinline__ int64_t off(int m, int r, int c, int64_t s) const {
    return ((int64_t)((m * ROWS + r) * 3 + c)) * V + s;
  }
  __device__ __forceinline__ void load(int m, int64_t s, M3<R>& M) const {
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) M.e[r][c] = p[off(m, r, c, s)];
    if (ROWS == 2) su3_third_row<R>(M.e[0], M.e[1], M.e[2]);
  }
  __device__ __forceinline__ void load_ro(int m, int64_t s, M3<R>& M) const {
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) M.e[r][c] = __ldg(&p[off(m, r, c, s)]);
    if (ROWS == 2) su3_third_row<R>(M.e[0], M.e[1], M.e[2]);
  }
  // rows 0..1 only (never reconstructs)
  __device__ __forceinline__ void load_rows01_ro(int m, int64_t s, C2<R> rows[2][3]) const {
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) rows[r][c] = __ldg(&p[off(m, r, c, s)]);
  }
  __device__ __forceinline__ void store(int m, int64_t s, const M3<R>& M) const {
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) p[off(m, r, c, s)] = M.e[r][c];
  }
};

// Division by a run-time constant d >= 1 through a multiply-high and a shift
// (valid for 0 <= n < 2^31): q = (umulhi(n, m) + n) >> s with s = ceil(log2 d)
// and m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
  uint32_t d, m, s;
  static FastDiv make(uint32_t d) {
    uint32_t s = 0;
    while ((1ull << s) < d) ++s;
    const uint64_t m = ((1ull << 32) * ((1ull << s) - d)) / d + 1;
    return FastDiv{d, (uint32_t)m, s};
  }
  __device__ __forceinline__ uint32_t div(uint32_t n) const { return (__umulhi(n, m) + n) >> s; }
};

// Lattice geometry passed by value to every kernel.
struct Geom {
  int L[4];        // Lx, Ly, Lz, Lt
  int64_t V;       // volume
  int64_t stride[4];  // 1, Lx, Lx*Ly, Lx*Ly*Lz
};

__device__ __forceinline__ void site_coords(const Geom& g, int64_t s, int c[4]) {
  int64_t r = s;
  c[0] = (int)(r % g.L[0]); r /= g.L[0];
  c[1] = (int)(r % g.L[1]); r /= g.L[1];
  c[2] = (int)(r % g.L[2]); r /= g.L[2];
  c[3] = (int)r;
}

__device__ __forceinline__ int64_t site_back(const Geom& g, int64_t s, const int c[4], int mu) {
  return c[mu] == 0 ? s + (int64_t)(g.L[mu] - 1) * g.stride[mu] : s - g.stride[mu];
}

// x + mu^ and x - mu^ for a direction known only at run time, by selects:
// coordinates and geometry stay in registers (no local-memory copy of c[]
// or of the geometry inside a loop over mu).
__device__ __forceinline__ void site_nbrs_sel(const Geom& g, int64_t s, const int c[4], int mu, int64_t& fwd,
                                              int64_t& back) {
  int cm = c[0], L = g.L[0];
  int64_t st = 1;
  if (mu == 1) { cm = c[1]; L = g.L[1]; st = g.stride[1]; }
  if (mu == 2) { cm = c[2]; L = g.L[2]; st = g.stride[2]; }
  if (mu == 3) { cm = c[3]; L = g.L[3]; st = g.stride[3]; }
  const int64_t wrap = (int64_t)(L - 1) * st;
  fwd = cm == L - 1 ? s - wrap : s + st;
  back = cm == 0 ? s + wrap : s - st;
}

__device__ __forceinline__ int64_t site_fwd(const Geom& g, int64_t s, const int c[4], int mu) {
  return c[mu] == g.L[mu] - 1 ? s - (int64_t)(g.L[mu] - 1) * g.stride[mu] : s + g.stride[mu];
}

}  // namespace lgf
