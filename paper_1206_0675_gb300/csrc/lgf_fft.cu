// 4D Fourier transform of the packed divergence as two plane passes
// (the "2D + 2D" decomposition of arXiv:1206.0675 Sec. 3.2), written for
// shared memory instead of cuFFT plus a reorder kernel:
//
//   pass A : forward DFT over each (x, y) plane                     [k3 removed]
//   pass B : forward DFT over (z, t), multiply by the momentum filter,
//            inverse DFT over (z, t)                                [k4 fused]
//   pass C : inverse DFT over (x, y), then g(x) = reunitarize(1 + Delta'(x))
//            in FP64, optionally G <- g G                           [k5 fused]
//
// Each 1D transform is an in-place mixed-radix (2, 3, 4, 8) Cooley-Tukey FFT
// in shared memory (see ct_stage).  Consecutive threads work on neighbouring
// lines and every line stride is padded by one element, so the butterflies'
// shared-memory accesses are free of bank conflicts in every direction.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <vector>

#include "lgf_internal.h"

namespace lgf {

// ---------------------------------------------------------------------------
// radix-R DFTs in registers; SIGN = -1 forward (e^{-2 pi i nk/R}), +1 inverse
// ---------------------------------------------------------------------------

template <typename R, int SIGN> __device__ __forceinline__ C2<R> mul_i(C2<R> a) {
  // multiply by SIGN * i
  return SIGN < 0 ? mkc<R>(a.y, -a.x) : mkc<R>(-a.y, a.x);
}

template <typename R, int RAD, int SIGN> struct DFT;

template <typename R, int SIGN> struct DFT<R, 2, SIGN> {
  __device__ __forceinline__ static void run(C2<R>* v) {
    const C2<R> a = v[0], b = v[1];
    v[0] = cadd<R>(a, b);
    v[1] = csub<R>(a, b);
  }
};

template <typename R, int SIGN> struct DFT<R, 3, SIGN> {
  __device__ __forceinline__ static void run(C2<R>* v) {
    const R h = (R)0.5, s3 = (R)0.86602540378443864676372317075294;  // cos(pi/3), sin(pi/3)
    const C2<R> t1 = cadd<R>(v[1], v[2]);
    const C2<R> t2 = mkc<R>(fma(-h, t1.x, v[0].x), fma(-h, t1.y, v[0].y));
    const C2<R> d = csub<R>(v[1], v[2]);
    const C2<R> t3 = mul_i<R, SIGN>(mkc<R>(s3 * d.x, s3 * d.y));
    v[0] = cadd<R>(v[0], t1);
    v[1] = cadd<R>(t2, t3);
    v[2] = csub<R>(t2, t3);
  }
};

template <typename R, int SIGN> struct DFT<R, 4, SIGN> {
  __device__ __forceinline__ static void run(C2<R>* v) {
    const C2<R> a = cadd<R>(v[0], v[2]), b = csub<R>(v[0], v[2]);
    const C2<R> c = cadd<R>(v[1], v[3]), d = mul_i<R, SIGN>(csub<R>(v[1], v[3]));
    v[0] = cadd<R>(a, c);
    v[2] = csub<R>(a, c);
    v[1] = cadd<R>(b, d);
    v[3] = csub<R>(b, d);
  }
};

template <typename R, int SIGN> struct DFT<R, 8, SIGN> {
  __device__ __forceinline__ static void run(C2<R>* v) {
    C2<R> e[4] = {v[0], v[2], v[4], v[6]};
    C2<R> o[4] = {v[1], v[3], v[5], v[7]};
    DFT<R, 4, SIGN>::run(e);
    DFT<R, 4, SIGN>::run(o);
    const R r2 = (R)0.70710678118654752440084436210485;
    // o[k] *= W8^k, W8 = e^{SIGN 2 pi i / 8}
    {
      const C2<R> a = o[1];  // (1 + SIGN i)/sqrt2
      o[1] = SIGN < 0 ? mkc<R>(r2 * (a.x + a.y), r2 * (a.y - a.x)) : mkc<R>(r2 * (a.x - a.y), r2 * (a.y + a.x));
    }
    o[2] = mul_i<R, SIGN>(o[2]);
    {
      const C2<R> a = o[3];  // (-1 + SIGN i)/sqrt2
      o[3] = SIGN < 0 ? mkc<R>(r2 * (a.y - a.x), -r2 * (a.x + a.y)) : mkc<R>(-r2 * (a.x + a.y), r2 * (a.x - a.y));
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[k] = cadd<R>(e[k], o[k]);
      v[k + 4] = csub<R>(e[k], o[k]);
    }
  }
};

// ---------------------------------------------------------------------------
// in-place mixed-radix Cooley-Tukey stages over a set of lines of a tile
// ---------------------------------------------------------------------------
//
// With radices R_0..R_{m-1} (stage s spans Ns = R_0...R_{s-1}), a butterfly
// of stage s acts on the R_s elements  g*Ns*R_s + j + r*Ns  (r < R_s) of a
// line.  Decimation in time (DIT) multiplies input r by W_{Ns R_s}^{j r}
// before the R_s-point DFT and expects its input in mixed-radix digit-reversed
// order; decimation in frequency (DIF) runs the stages in reverse, applies
// the DFT first and the twiddles to the outputs, and leaves its output in
// digit-reversed order.  The reorder is folded into the global <-> shared
// copies through the position table pos[n] of each direction, so no
// separate reorder kernel (k3 of Sec. 3.2) exists.  A butterfly reads and
// writes only its own elements, so each thread works through its butterflies
// one at a time and stages are separated by a single __syncthreads.

// Line l starts at (l / inner) * outer_stride + (l % inner) * inner_stride and
// its elements are es apart.
struct Lines {
  int nlines, inner, inner_stride, outer_stride, es;
  FastDiv dn, di;  // divisors by nlines and inner
};

static Lines make_lines(int nlines, int inner, int inner_stride, int outer_stride, int es) {
  return Lines{nlines, inner, inner_stride, outer_stride, es, FastDiv::make(nlines), FastDiv::make(inner)};
}

template <typename R, int RAD, int SIGN, bool DIT>
__device__ __forceinline__ void ct_stage(C2<R>* __restrict__ tile, const Lines& ln, const int N, const FastDiv fns,
                                         const C2<R>* __restrict__ tw) {
  const int Ns = (int)fns.d;
  const int nbl = N / RAD;
  const int NB = ln.nlines * nbl;
  const int tws = nbl / Ns;
  for (int b = threadIdx.x; b < NB; b += blockDim.x) {
    const int q = (int)ln.dn.div((uint32_t)b), l = b - q * ln.nlines;
    const int grp = (int)fns.div((uint32_t)q), j = q - grp * Ns;
    const int lo = (int)ln.di.div((uint32_t)l), li = l - lo * ln.inner;
    const int base = lo * ln.outer_stride + li * ln.inner_stride + (grp * Ns * RAD + j) * ln.es;
    const int step = Ns * ln.es;
    C2<R> v[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[r] = tile[base + r * step];
    if (DIT && j > 0) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        const C2<R> w = tw[j * r * tws];
        v[r] = SIGN < 0 ? cmul<R>(v[r], w) : cmulc<R>(v[r], w);
      }
    }
    DFT<R, RAD, SIGN>::run(v);
    if (!DIT && j > 0) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        const C2<R> w = tw[j * r * tws];
        v[r] = SIGN < 0 ? cmul<R>(v[r], w) : cmulc<R>(v[r], w);
      }
    }
#pragma unroll
    for (int r = 0; r < RAD; ++r) tile[base + r * step] = v[r];
  }
  __syncthreads();
}

template <typename R, int SIGN, bool DIT>
__device__ __forceinline__ void ct_stage_any(C2<R>* tile, const Lines& ln, int N, const FastDiv& fns, int rad,
                                             const C2<R>* tw) {
  if (rad == 8) ct_stage<R, 8, SIGN, DIT>(tile, ln, N, fns, tw);
  else if (rad == 4) ct_stage<R, 4, SIGN, DIT>(tile, ln, N, fns, tw);
  else if (rad == 3) ct_stage<R, 3, SIGN, DIT>(tile, ln, N, fns, tw);
  else ct_stage<R, 2, SIGN, DIT>(tile, ln, N, fns, tw);
}

// DFT of every line: input digit-reversed, output natural.
template <typename R, int SIGN>
__device__ __forceinline__ void fft_lines_dit(C2<R>* tile, const Lines& ln, const FFTDir& d, const C2<R>* tw) {
  for (int st = 0; st < d.nst; ++st) ct_stage_any<R, SIGN, true>(tile, ln, d.N, d.ns[st], d.radix[st], tw);
}

// DFT of every line: input natural, output digit-reversed.
template <typename R, int SIGN>
__device__ __forceinline__ void fft_lines_dif(C2<R>* tile, const Lines& ln, const FFTDir& d, const C2<R>* tw) {
  for (int st = d.nst - 1; st >= 0; --st) ct_stage_any<R, SIGN, false>(tile, ln, d.N, d.ns[st], d.radix[st], tw);
}

// ---------------------------------------------------------------------------
// shared-memory layout helpers
// ---------------------------------------------------------------------------

// Global -> shared copy of one complex element without a register round trip
// (PTX cp.async; 8 bytes for FP32, 16 bytes for FP64, both aligned to their
// size), so that a thread keeps all of its tile's loads in flight at once
// instead of waiting for each before issuing the next.  cp_async_wait() waits
// for this thread's copies; a __syncthreads() after it publishes the tile.
template <typename R> __device__ __forceinline__ void cp_async_elem(C2<R>* dst, const C2<R>* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(C2<R>) == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Shared memory of a pass: twiddles of two directions, position tables of two
// directions, then the tile.  Returns the tile pointer.
template <typename R>
__device__ __forceinline__ C2<R>* setup_smem(unsigned char* raw, const C2<R>* __restrict__ twg,
                                             const short* __restrict__ posg, int n0, int n1, C2<R>** tw,
                                             short** pos) {
  *tw = reinterpret_cast<C2<R>*>(raw);
  const int twn = (n0 + n1 + 1) & ~1;
  *pos = reinterpret_cast<short*>(*tw + twn);
  const int posn = (n0 + n1 + 7) & ~7;  // keeps the tile 16-byte aligned
  for (int i = threadIdx.x; i < n0 + n1; i += blockDim.x) {
    (*tw)[i] = __ldg(&twg[i]);
    (*pos)[i] = __ldg(&posg[i]);
  }
  return reinterpret_cast<C2<R>*>(*pos + posn);
}

template <typename R> __host__ __device__ inline size_t smem_header_bytes(int n0, int n1) {
  return (size_t)((n0 + n1 + 1) & ~1) * sizeof(C2<R>) + (size_t)((n0 + n1 + 7) & ~7) * sizeof(short);
}

// ---------------------------------------------------------------------------
// (x, y) plane pass: one CTA per (z, t) slab and group of fpb fields;
// digit-reversed load, DIT in x and y, natural store (passes A and, for large
// planes, C).
// ---------------------------------------------------------------------------

// Divisors of the global <-> shared copies of a pass.
struct CopyDiv {
  FastDiv a, b;
};

template <typename R, int SIGN>
__global__ void __launch_bounds__(512) fft_xy_kernel(Geom g, FFTDir dx, FFTDir dy, C2<R>* __restrict__ data, const C2<R>* __restrict__ twg,
                              const short* __restrict__ posg, int fpb, Lines lx, Lines ly, CopyDiv cd, Batch B) {
  if (batch_skip(B)) return;
  data += blockIdx.z * B.s_delta;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Lx = g.L[0], Ly = g.L[1];
  C2<R>* tw;
  short* pos;
  C2<R>* tile = setup_smem<R>(smem_raw, twg, posg, Lx, Ly, &tw, &pos);
  const int RS = Lx + 1, PS = Ly * RS;
  const int64_t slab = blockIdx.x;
  const int f0 = blockIdx.y * fpb;
  const int plane = Lx * Ly;
  __syncthreads();
  for (int i = threadIdx.x; i < fpb * plane; i += blockDim.x) {
    const int f = (int)cd.a.div((uint32_t)i), r = i - f * plane, y = (int)cd.b.div((uint32_t)r), x = r - y * Lx;
    cp_async_elem<R>(&tile[f * PS + pos[Lx + y] * RS + pos[x]], &data[(int64_t)(f0 + f) * g.V + slab * plane + r]);
  }
  cp_async_wait();
  __syncthreads();
  fft_lines_dit<R, SIGN>(tile, lx, dx, tw);
  fft_lines_dit<R, SIGN>(tile, ly, dy, tw + Lx);
  for (int i = threadIdx.x; i < fpb * plane; i += blockDim.x) {
    const int f = (int)cd.a.div((uint32_t)i), r = i - f * plane, y = (int)cd.b.div((uint32_t)r), x = r - y * Lx;
    data[(int64_t)(f0 + f) * g.V + slab * plane + r] = tile[f * PS + y * RS + x];
  }
}

// ---------------------------------------------------------------------------
// (z, t) plane pass with the momentum filter: one CTA per (x-block, y, field)
// ---------------------------------------------------------------------------

// LRN: the learned handles' variant (multiplier table, divergence snapshot);
// the plain variant carries none of that code.
template <typename R, bool LRN>
__global__ void __launch_bounds__(512) fft_zt_filter_kernel(Geom g, FFTDir dz, FFTDir dt, C2<R>* __restrict__ data,
                                     const C2<R>* __restrict__ twg, const short* __restrict__ posg,
                                     const R* __restrict__ K, int xc, int mode, LearnedIO lio, int4 H, Lines lz,
                                     Lines lt, CopyDiv cd, Batch B) {
  if (batch_skip(B)) return;
  data += blockIdx.z * B.s_delta;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
  C2<R>* tw;
  short* pos;
  C2<R>* tile = setup_smem<R>(smem_raw, twg + Lx + Ly, posg + Lx + Ly, Lz, Lt, &tw, &pos);
  const int TS = Lz * xc + 1;
  const int nxb = Lx / xc;
  const int x0 = (blockIdx.x % nxb) * xc, y = blockIdx.x / nxb;
  C2<R>* fld = data + (int64_t)blockIdx.y * g.V;
  const int n = Lz * Lt * xc;
  const int64_t sxy = (int64_t)y * Lx + x0;
  const int64_t plane = (int64_t)Lx * Ly;
  __syncthreads();
#define LGF_ZT_IDX(i)                                                       \
  const int zt = (int)cd.a.div((uint32_t)(i)), xi = (i) - zt * xc;          \
  const int t = (int)cd.b.div((uint32_t)zt), z = zt - t * Lz;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    LGF_ZT_IDX(i)
    cp_async_elem<R>(&tile[pos[Lz + t] * TS + pos[z] * xc + xi], &fld[(int64_t)zt * plane + sxy + xi]);
  }
  cp_async_wait();
  __syncthreads();
  if (mode == 0) {
    fft_lines_dit<R, -1>(tile, lz, dz, tw);
    fft_lines_dit<R, -1>(tile, lt, dt, tw + Lz);
    // learned multiplier of the momentum class (f_mu = min(k_mu, L_mu - k_mu))
    // and the snapshot of the transformed divergence, both of step k
    const int kit = LRN ? lio.st->iter : 0;
    const bool learned = LRN && lio.mtab != nullptr && lio.st->use_m != 0;
    const float* mtab = lio.mtab + (int64_t)(kit & 1) * lio.nclass;
    uint32_t* snap = (LRN && lio.snap != nullptr) ? lio.snap + ((int64_t)(kit & 1) * 4 + blockIdx.y) * g.V : nullptr;
    const int fy = min(y, Ly - y);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      LGF_ZT_IDX(i)
      R k = __ldg(&K[(int64_t)zt * plane + sxy + xi]);
      if (learned) {
        const int kx = x0 + xi;
        const int fx = min(kx, Lx - kx), fz = min(z, Lz - z), ft = min(t, Lt - t);
        k *= (R)__ldg(&mtab[((ft * H.z + fz) * H.y + fy) * H.x + fx]);
      }
      C2<R>& e = tile[t * TS + z * xc + xi];
      if (LRN && snap != nullptr) snap[(int64_t)zt * plane + sxy + xi] = bf16x2_of<R>(e);
      e = mkc<R>(e.x * k, e.y * k);
    }
    __syncthreads();
    fft_lines_dif<R, +1>(tile, lt, dt, tw + Lz);
    fft_lines_dif<R, +1>(tile, lz, dz, tw);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      LGF_ZT_IDX(i)
      fld[(int64_t)zt * plane + sxy + xi] = tile[pos[Lz + t] * TS + pos[z] * xc + xi];
    }
  } else {
    if (mode < 0) {
      fft_lines_dit<R, -1>(tile, lz, dz, tw);
      fft_lines_dit<R, -1>(tile, lt, dt, tw + Lz);
    } else {
      fft_lines_dit<R, +1>(tile, lz, dz, tw);
      fft_lines_dit<R, +1>(tile, lt, dt, tw + Lz);
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      LGF_ZT_IDX(i)
      fld[(int64_t)zt * plane + sxy + xi] = tile[t * TS + z * xc + xi];
    }
  }
#undef LGF_ZT_IDX
}

// ---------------------------------------------------------------------------
// Alternative decompositions of the 4D transform (Sec. 3.2 compares 1D x 4,
// 3D + 1D and 2D + 2D on cuFFT): one pass per direction, or one pass over
// the (x, y, z) slab of each t plus a pass over t.  Both keep every line of a
// pass in shared memory with the same Cooley-Tukey stages as the plane passes.
// ---------------------------------------------------------------------------

// One 1D pass along direction mu.  Contiguous form (mu = x): each CTA takes nl
// consecutive x-lines.  Strided form (mu = y, z, t): each CTA takes xc
// consecutive x columns at fixed other coordinates, so that the global
// accesses are runs of xc elements.  Tile: line l at l * (N + 1).
struct LinePass {
  int N;            // line length L_mu
  int nl;           // lines per CTA
  int contiguous;   // 1 for mu = x
  int64_t S;        // element stride of mu in a field
  int64_t SN;       // S * N
  FastDiv dload;    // by N (contiguous) or by nl (strided)
  FastDiv dlob;     // by S / nl (strided): column blocks per (coordinate above mu)
};

// mode -1: forward DFT; +1: inverse DFT (unnormalised); 0: forward DFT,
// multiplication by K (same layout as the field), inverse DFT.
// mtab (mode 0, may be NULL): learned multiplier per momentum class, applied
// when *use_m != 0; the class of momentum k is (min(k_mu, L_mu - k_mu))_mu in
// a table of H.x * H.y * H.z * H.w classes.
template <typename R, bool LRN>
__global__ void __launch_bounds__(512) fft_line_kernel(LinePass lp, FFTDir d, Geom g, C2<R>* __restrict__ data,
                                                       const C2<R>* __restrict__ twg, const short* __restrict__ posg,
                                                       const R* __restrict__ K, int mode, Lines ln, LearnedIO lio,
                                                       int4 H, Batch B) {
  const int64_t V = g.V;
  if (batch_skip(B)) return;
  data += blockIdx.z * B.s_delta;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* tw;
  short* pos;
  C2<R>* tile = setup_smem<R>(smem_raw, twg, posg, lp.N, 0, &tw, &pos);
  C2<R>* fld = data + (int64_t)blockIdx.y * V;
  const int N = lp.N, RS = N + 1, n_el = lp.nl * N;
  int64_t s0;
  if (lp.contiguous) {
    s0 = (int64_t)blockIdx.x * n_el;
  } else {
    const uint32_t b = blockIdx.x;
    const uint32_t hi = lp.dlob.div(b), lob = b - hi * lp.dlob.d;
    s0 = (int64_t)lob * lp.nl + (int64_t)hi * lp.SN;
  }
  // element i of the CTA -> (line l, position n) and its site
#define LGF_LINE_IDX(i)                                                          \
  int l, n;                                                                      \
  if (lp.contiguous) { l = (int)lp.dload.div((uint32_t)(i)); n = (i) - l * N; }  \
  else { n = (int)lp.dload.div((uint32_t)(i)); l = (i) - n * lp.nl; }            \
  const int64_t site = lp.contiguous ? s0 + (i) : s0 + l + (int64_t)n * lp.S;
  __syncthreads();
  const bool natural_in = mode > 0;
  for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
    LGF_LINE_IDX(i)
    cp_async_elem<R>(&tile[l * RS + (natural_in ? n : pos[n])], &fld[site]);
  }
  cp_async_wait();
  __syncthreads();
  if (mode < 0) {
    fft_lines_dit<R, -1>(tile, ln, d, tw);
  } else if (mode > 0) {
    fft_lines_dif<R, +1>(tile, ln, d, tw);
  } else {
    fft_lines_dit<R, -1>(tile, ln, d, tw);
    const int kit = LRN ? lio.st->iter : 0;
    const bool learned = LRN && lio.mtab != nullptr && lio.st->use_m != 0;
    const float* mtab = lio.mtab + (int64_t)(kit & 1) * lio.nclass;
    uint32_t* snap = (LRN && lio.snap != nullptr) ? lio.snap + ((int64_t)(kit & 1) * 4 + blockIdx.y) * V : nullptr;
    for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
      LGF_LINE_IDX(i)
      R k = __ldg(&K[site]);
      if (learned) {
        int c[4];
        site_coords(g, site, c);
        const int fx = min(c[0], g.L[0] - c[0]), fy = min(c[1], g.L[1] - c[1]);
        const int fz = min(c[2], g.L[2] - c[2]), ft = min(c[3], g.L[3] - c[3]);
        k *= (R)__ldg(&mtab[((ft * H.z + fz) * H.y + fy) * H.x + fx]);
      }
      C2<R>& e = tile[l * RS + n];
      if (LRN && snap != nullptr) snap[site] = bf16x2_of<R>(e);
      e = mkc<R>(e.x * k, e.y * k);
    }
    __syncthreads();
    fft_lines_dif<R, +1>(tile, ln, d, tw);
  }
  const bool natural_out = mode < 0;
  for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
    LGF_LINE_IDX(i)
    fld[site] = tile[l * RS + (natural_out ? n : pos[n])];
  }
#undef LGF_LINE_IDX
}

// 3D DFT over the (x, y, z) slab of one t and one field (SIGN -1 forward:
// digit-reversed load, DIT, natural store; +1 inverse: natural load, DIF,
// digit-reversed read-out).  The slab must fit in shared memory.
template <typename R, int SIGN>
__global__ void __launch_bounds__(512) fft_xyz_kernel(Geom g, FFTDir dx, FFTDir dy, FFTDir dz, C2<R>* __restrict__ data,
                                                      const C2<R>* __restrict__ twg, const short* __restrict__ posg,
                                                      Lines lx, Lines ly, Lines lz, CopyDiv cd, Batch B) {
  if (batch_skip(B)) return;
  data += blockIdx.z * B.s_delta;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2];
  C2<R>* tw;
  short* pos;
  C2<R>* tile = setup_smem<R>(smem_raw, twg, posg, Lx, Ly + Lz, &tw, &pos);
  const int RS = Lx + 1, PS = Ly * RS;
  const int n_el = Lx * Ly * Lz;
  C2<R>* fld = data + (int64_t)blockIdx.y * g.V + (int64_t)blockIdx.x * n_el;
  __syncthreads();
#define LGF_XYZ_IDX(i)                                                     \
  const int z = (int)cd.a.div((uint32_t)(i)), r = (i) - z * Lx * Ly;       \
  const int y = (int)cd.b.div((uint32_t)r), x = r - y * Lx;
  for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
    LGF_XYZ_IDX(i)
    const int o = SIGN < 0 ? pos[Lx + Ly + z] * PS + pos[Lx + y] * RS + pos[x] : z * PS + y * RS + x;
    cp_async_elem<R>(&tile[o], &fld[i]);
  }
  cp_async_wait();
  __syncthreads();
  if (SIGN < 0) {
    fft_lines_dit<R, -1>(tile, lx, dx, tw);
    fft_lines_dit<R, -1>(tile, ly, dy, tw + Lx);
    fft_lines_dit<R, -1>(tile, lz, dz, tw + Lx + Ly);
  } else {
    fft_lines_dif<R, +1>(tile, lz, dz, tw + Lx + Ly);
    fft_lines_dif<R, +1>(tile, ly, dy, tw + Lx);
    fft_lines_dif<R, +1>(tile, lx, dx, tw);
  }
  for (int i = threadIdx.x; i < n_el; i += blockDim.x) {
    LGF_XYZ_IDX(i)
    const int o = SIGN < 0 ? z * PS + y * RS + x : pos[Lx + Ly + z] * PS + pos[Lx + y] * RS + pos[x];
    fld[i] = tile[o];
  }
#undef LGF_XYZ_IDX
}

// ---------------------------------------------------------------------------
// g(x) = reunitarize(1 + Delta'(x)) in FP64 (Sec. 2 first-order expansion,
// Gram-Schmidt on rows 1-2, row 3 = (a x b)^* as in Sec. 3.2)
// ---------------------------------------------------------------------------

// f0 = (Im D11, Im D22), f1 = D12, f2 = D13, f3 = D23 of the filtered field.
// Rows of 1 + X: r1 = (1 + i a, f1, f2) and r2 = (-conj f1, 1 + i d, f3)
// with a = Re f0, d = Im f0.  Gram-Schmidt: u = r1 / |r1| and
// v = w / |w| with w = r2 - <u, r2> u = r2 - (c / |r1|^2) r1, where
// c = <r1, r2> = sum_j conj(r1_j) r2_j = (a + d)(Im f1 + i Re f1) + conj(f2) f3
// (the two terms in f1 combine).  All of it in FP64.
// The FP64 Gram-Schmidt factors of 1 + X: i1 = 1/|r1|, w = r2 - k r1 and
// i2 = 1/|w|, so that u = i1 r1 and v = i2 w.
struct GSFactors {
  double i1, i2;
  double2 w[3];
};

__device__ __forceinline__ void gram_schmidt_factors(double a, double d, double2 f1, double2 f2, double2 f3,
                                                     GSFactors& o) {
  const double n1 = fma(f2.x, f2.x, fma(f2.y, f2.y, fma(f1.x, f1.x, fma(f1.y, f1.y, fma(a, a, 1.0)))));
  o.i1 = rsqrt_fp64(n1);
  const double s = a + d;
  const double q = o.i1 * o.i1;  // 1 / |r1|^2
  const double kx = q * fma(f2.x, f3.x, fma(f2.y, f3.y, s * f1.y));
  const double ky = q * fma(f2.x, f3.y, fma(-f2.y, f3.x, s * f1.x));
  // w = r2 - k r1
  o.w[0] = make_double2(fma(ky, a, -f1.x - kx), fma(-kx, a, f1.y - ky));
  o.w[1] = make_double2(fma(ky, f1.y, fma(-kx, f1.x, 1.0)), fma(-ky, f1.x, fma(-kx, f1.y, d)));
  o.w[2] = make_double2(fma(ky, f2.y, fma(-kx, f2.x, f3.x)), fma(-ky, f2.x, fma(-kx, f2.y, f3.y)));
  const double n2 = fma(o.w[2].x, o.w[2].x, fma(o.w[2].y, o.w[2].y, fma(o.w[1].x, o.w[1].x,
                    fma(o.w[1].y, o.w[1].y, fma(o.w[0].x, o.w[0].x, o.w[0].y * o.w[0].y)))));
  o.i2 = rsqrt_fp64(n2);
}

// The FP64 factors for fields stored in FP32: i1 = 1/|r1|, the projection
// coefficient k = <r1, r2>/|r1|^2 and i2 = 1/|w| with w = r2 - k r1, where
// |w|^2 = |r2|^2 - |<r1, r2>|^2/|r1|^2 (Pythagoras for the projection) is
// formed from the inputs, so that w itself is never needed in FP64: the
// FP32 field applies k in FP32.  For 1 + X with X anti-Hermitian the rows are
// nearly orthogonal (|<r1, r2>| <= |X|^2 while |r1|, |r2| >= 1), so the
// difference does not cancel.  33 FP64 operations and two estimates, against
// 43 when w is formed in FP64.
struct GSFactors32 {
  double i1, i2, kx, ky;
};

__device__ __forceinline__ void gram_schmidt_factors_f32(double a, double d, double2 f1, double2 f2, double2 f3,
                                                         GSFactors32& o) {
  const double n1 = fma(f2.x, f2.x, fma(f2.y, f2.y, fma(f1.x, f1.x, fma(f1.y, f1.y, fma(a, a, 1.0)))));
  o.i1 = rsqrt_fp64(n1);
  const double s = a + d;
  const double q = o.i1 * o.i1;  // 1 / |r1|^2
  const double cx = fma(f2.x, f3.x, fma(f2.y, f3.y, s * f1.y));
  const double cy = fma(f2.x, f3.y, fma(-f2.y, f3.x, s * f1.x));
  const double nr2 = fma(f3.x, f3.x, fma(f3.y, f3.y, fma(d, d, fma(f1.x, f1.x, fma(f1.y, f1.y, 1.0)))));
  const double n2 = fma(-q, fma(cx, cx, cy * cy), nr2);
  o.kx = q * cx;
  o.ky = q * cy;
  o.i2 = rsqrt_fp64(n2);
}

// FP32 <-> FP64 conversions on the integer pipe, written from the IEEE 754
// binary32 / binary64 layouts.  On this GPU the conversion instructions run
// on the FP64 pipe, which bounds pass C of FP32 lanes; these take sign,
// rebiased exponent and mantissa apart with integer operations instead.
// Zero and subnormal inputs give zero; FP64 -> FP32 rounds to nearest with
// ties away from zero (IEEE rounds ties to even: the two differ only on exact
// ties) and overflows to infinity.  Non-finite values are not expected here.
__device__ __forceinline__ double f32_to_f64_int(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xffu;
  const uint64_t body = ((uint64_t)(e + (1023u - 127u)) << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
  return __longlong_as_double((long long)(sign | (e == 0u ? 0ull : body)));
}
__device__ __forceinline__ float f64_to_f32_int(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int64_t r = (int64_t)(b & 0x7fffffffffffffffull) - ((int64_t)(1023 - 127) << 52) + (1ll << 28);
  uint32_t f = r <= (1ll << 28) ? 0u : (uint32_t)(r >> 29);
  if (r > (1ll << 28) && f >= 0x7f800000u) f = 0x7f800000u;
  return __uint_as_float(sign | f);
}
__device__ __forceinline__ double2 c_f32_to_f64_int(float2 v) { return make_double2(f32_to_f64_int(v.x), f32_to_f64_int(v.y)); }
__device__ __forceinline__ float2 c_f64_to_f32_int(double2 v) { return make_float2(f64_to_f32_int(v.x), f64_to_f32_int(v.y)); }

// Rows u, v of g = reunitarize(1 + X) in the field precision R; the
// Gram-Schmidt factors are FP64 in both.  FP64 fields take u = i1 r1 and
// v = i2 w in FP64.  FP32 fields, whose rows are stored in FP32, apply the
// FP64 factors in FP32: u = fl(i1) r1 with r1 the FP32 entries of the
// filtered field itself, v = fl(i2) fl(w) -- within one FP32 rounding of the
// FP64 product, without the FP64 multiplies -- and take their values to and
// from FP64 on the integer pipe.
template <typename R>
__device__ __forceinline__ void gauge_rows(C2<R> f0, C2<R> f1, C2<R> f2, C2<R> f3, C2<R> u[3], C2<R> v[3]) {
  if constexpr (sizeof(R) == sizeof(double)) {
    GSFactors o;
    gram_schmidt_factors(f0.x, f0.y, f1, f2, f3, o);
    u[0] = mkc<R>(o.i1, f0.x * o.i1);
    u[1] = cscale<R>(f1, o.i1);
    u[2] = cscale<R>(f2, o.i1);
#pragma unroll
    for (int j = 0; j < 3; ++j) v[j] = cscale<double>(o.w[j], o.i2);
  } else {
    GSFactors32 o32;
    gram_schmidt_factors_f32(f32_to_f64_int(f0.x), f32_to_f64_int(f0.y), c_f32_to_f64_int(f1), c_f32_to_f64_int(f2),
                             c_f32_to_f64_int(f3), o32);
    const float i1 = f64_to_f32_int(o32.i1), i2 = f64_to_f32_int(o32.i2);
    const float kx = f64_to_f32_int(o32.kx), ky = f64_to_f32_int(o32.ky);
    const float a = f0.x, d = f0.y;
    u[0] = mkc<R>(i1, a * i1);
    u[1] = cscale<R>(f1, i1);
    u[2] = cscale<R>(f2, i1);
    // w = r2 - k r1 in FP32, normalised by the FP64 factor
    const C2<R> w0 = mkc<R>(fmaf(ky, a, -f1.x - kx), fmaf(-kx, a, f1.y - ky));
    const C2<R> w1 = mkc<R>(fmaf(ky, f1.y, fmaf(-kx, f1.x, 1.f)), fmaf(-ky, f1.x, fmaf(-kx, f1.y, d)));
    const C2<R> w2 = mkc<R>(fmaf(ky, f2.y, fmaf(-kx, f2.x, f3.x)), fmaf(-ky, f2.x, fmaf(-kx, f2.y, f3.y)));
    v[0] = cscale<R>(w0, i2);
    v[1] = cscale<R>(w1, i2);
    v[2] = cscale<R>(w2, i2);
  }
}

// Rows 1 and 2 of g = exp(X) (the exponential of Eq. (eq:gx) evaluated
// exactly instead of to first order), for X traceless anti-Hermitian packed
// as above, followed by the same Gram-Schmidt projection.
//
// With X = iQ (Q Hermitian, traceless) the Cayley-Hamilton theorem gives
// Q^3 = u Q + w 1, u = tr(Q^2)/2, w = det Q, so exp(iQ) = c0 1 + c1 Q + c2 Q^2.
// Scaling and squaring (Moler and Van Loan, "Nineteen dubious ways to compute
// the exponential of a matrix", 1978): Z = Q / 2^s with |Z|_F <= 1/4, the
// Taylor series of exp(iZ) to order 12 (remainder below 3e-18) reduced to
// c0 + c1 Z + c2 Z^2 through Z^3 = uz Z + wz 1, then s squarings carried out on
// the three coefficients with the same reduction.
__device__ __forceinline__ void gauge_exp_from_packed(double2 f0, double2 f1, double2 f2, double2 f3, double2 u[3],
                                                      double2 v[3]) {
  const double a = f0.x, d = f0.y, q33 = -(a + d);
  // Q = -iX: off-diagonal entries q12, q13, q23; Q_ji = conj(Q_ij)
  const double2 q12 = make_double2(f1.y, -f1.x), q13 = make_double2(f2.y, -f2.x), q23 = make_double2(f3.y, -f3.x);
  const double n12 = cnorm2<double>(q12), n13 = cnorm2<double>(q13), n23 = cnorm2<double>(q23);
  const double uq = 0.5 * (a * a + d * d + q33 * q33) + n12 + n13 + n23;
  const double2 t = cconjmul<double>(q13, cmul<double>(q12, q23));  // q12 q23 conj(q13)
  const double wq = a * d * q33 + 2.0 * t.x - a * n23 - d * n13 - q33 * n12;
  int s = 0;
  double n2 = 2.0 * uq, uz = uq, wz = wq;
  while (n2 > 0.0625 && s < 64) {
    n2 *= 0.25;
    uz *= 0.25;
    wz *= 0.125;
    ++s;
  }
  // Z^n / n! = al 1 + be Z + ga Z^2 (real); exp(iZ) = sum_n i^n Z^n / n!
  double al = 1.0, be = 0.0, ga = 0.0;
  double2 c0 = make_double2(1.0, 0.0), c1 = make_double2(0.0, 0.0), c2 = make_double2(0.0, 0.0);
#pragma unroll
  for (int n = 1; n <= 12; ++n) {
    const double inv = 1.0 / (double)n;
    const double al2 = ga * wz * inv, be2 = fma(ga, uz, al) * inv, ga2 = be * inv;
    al = al2;
    be = be2;
    ga = ga2;
    const double sg = ((n & 3) < 2) ? 1.0 : -1.0;
    if (n & 1) {
      c0.y = fma(sg, al, c0.y);
      c1.y = fma(sg, be, c1.y);
      c2.y = fma(sg, ga, c2.y);
    } else {
      c0.x = fma(sg, al, c0.x);
      c1.x = fma(sg, be, c1.x);
      c2.x = fma(sg, ga, c2.x);
    }
  }
  double h1 = 1.0;
  for (int k = 0; k < s; ++k) {
    const double2 p00 = cmul<double>(c0, c0), p12 = cmul<double>(c1, c2), p01 = cmul<double>(c0, c1);
    const double2 p22 = cmul<double>(c2, c2), p02 = cmul<double>(c0, c2), p11 = cmul<double>(c1, c1);
    c0 = make_double2(fma(2.0 * wz, p12.x, p00.x), fma(2.0 * wz, p12.y, p00.y));
    c1 = make_double2(fma(wz, p22.x, fma(2.0 * uz, p12.x, 2.0 * p01.x)),
                      fma(wz, p22.y, fma(2.0 * uz, p12.y, 2.0 * p01.y)));
    c2 = make_double2(fma(uz, p22.x, fma(2.0, p02.x, p11.x)), fma(uz, p22.y, fma(2.0, p02.y, p11.y)));
    h1 *= 0.5;
  }
  c1 = cscale<double>(c1, h1);       // coefficient of Q
  c2 = cscale<double>(c2, h1 * h1);  // coefficient of Q^2
  // rows 1 and 2 of Q^2
  const double s11 = a * a + n12 + n13, s22 = n12 + d * d + n23;
  const double2 s12 = cadd<double>(cscale<double>(q12, a + d), cmulc<double>(q13, q23));  // + q13 conj(q23)
  const double2 s13 = cadd<double>(cscale<double>(q13, -d), cmul<double>(q12, q23));
  const double2 s23 = cadd<double>(cconjmul<double>(q12, q13), cscale<double>(q23, -a));  // conj(q12) q13 - a q23
  const double2 s21 = make_double2(s12.x, -s12.y);
  const double2 q21 = make_double2(q12.x, -q12.y);
  double2 r1[3], r2[3];
  r1[0] = cadd<double>(cadd<double>(c0, cscale<double>(c1, a)), cscale<double>(c2, s11));
  r1[1] = cadd<double>(cmul<double>(c1, q12), cmul<double>(c2, s12));
  r1[2] = cadd<double>(cmul<double>(c1, q13), cmul<double>(c2, s13));
  r2[0] = cadd<double>(cmul<double>(c1, q21), cmul<double>(c2, s21));
  r2[1] = cadd<double>(cadd<double>(c0, cscale<double>(c1, d)), cscale<double>(c2, s22));
  r2[2] = cadd<double>(cmul<double>(c1, q23), cmul<double>(c2, s23));
  // Gram-Schmidt: u = r1/|r1|, v = (r2 - <u,r2> u)/|.|
  const double i1 = rsqrt(cnorm2<double>(r1[0]) + cnorm2<double>(r1[1]) + cnorm2<double>(r1[2]));
#pragma unroll
  for (int j = 0; j < 3; ++j) u[j] = cscale<double>(r1[j], i1);
  double2 ip = cconjmul<double>(u[0], r2[0]);
  ip = cadd<double>(ip, cconjmul<double>(u[1], r2[1]));
  ip = cadd<double>(ip, cconjmul<double>(u[2], r2[2]));
  const double2 nip = make_double2(-ip.x, -ip.y);
#pragma unroll
  for (int j = 0; j < 3; ++j) v[j] = cfma<double>(nip, u[j], r2[j]);
  const double i2 = rsqrt(cnorm2<double>(v[0]) + cnorm2<double>(v[1]) + cnorm2<double>(v[2]));
#pragma unroll
  for (int j = 0; j < 3; ++j) v[j] = cscale<double>(v[j], i2);
}

// Stores rows u, v (precision RG) and, where needed, row 3 = (u x v)^*.
template <typename RG, int GROWS>
__device__ __forceinline__ void store_gauge_rows(int64_t V, int64_t s, const C2<RG> a[3], const C2<RG> b[3],
                                                 C2<RG>* __restrict__ gf, C2<RG>* __restrict__ Gf) {
  C2<RG> c[3];
  const bool need_c = (GROWS == 3) || (Gf != nullptr);
  if (need_c) su3_third_row<RG>(a, b, c);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    gf[(0 * 3 + j) * V + s] = a[j];
    gf[(1 * 3 + j) * V + s] = b[j];
    if (GROWS == 3) gf[(2 * 3 + j) * V + s] = c[j];
  }
  if (Gf != nullptr) {
    // G <- g G (full 3x3, precision RG)
    C2<RG> Go[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int col = 0; col < 3; ++col) Go[r][col] = Gf[(r * 3 + col) * V + s];
    const C2<RG>* rows[3] = {a, b, c};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int col = 0; col < 3; ++col) {
        C2<RG> acc = cmul<RG>(rows[r][0], Go[0][col]);
        acc = cfma<RG>(rows[r][1], Go[1][col], acc);
        acc = cfma<RG>(rows[r][2], Go[2][col], acc);
        Gf[(r * 3 + col) * V + s] = acc;
      }
  }
}

// g(x) of one site from its packed filtered field and its store (and G <- g G).
template <typename R, typename RG, int GROWS, bool EXPG>
__device__ __forceinline__ void gauge_site(C2<R> f0, C2<R> f1, C2<R> f2, C2<R> f3, int64_t V, int64_t s,
                                           C2<RG>* __restrict__ gf, C2<RG>* __restrict__ Gf) {
  static_assert(sizeof(R) == sizeof(RG), "g is stored in the precision of the divergence");
  C2<RG> a[3], b[3];
  if constexpr (EXPG) {
    double2 u[3], v[3];
    gauge_exp_from_packed(ccast<double, R>(f0), ccast<double, R>(f1), ccast<double, R>(f2), ccast<double, R>(f3),
                          u, v);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      a[j] = ccast<RG, double>(u[j]);
      b[j] = ccast<RG, double>(v[j]);
    }
  } else {
    gauge_rows<RG>(f0, f1, f2, f3, a, b);
  }
  store_gauge_rows<RG, GROWS>(V, s, a, b, gf, Gf);
}

template <typename R, typename RG, int GROWS, bool EXPG>
__global__ void __launch_bounds__(512) fft_xy_inv_gauge_kernel(Geom g, FFTDir dx, FFTDir dy, const C2<R>* __restrict__ data,
                                        const C2<R>* __restrict__ twg, const short* __restrict__ posg,
                                        C2<RG>* __restrict__ gf, C2<RG>* __restrict__ Gf, Lines lx, Lines ly,
                                        CopyDiv cd, Batch B) {
  if (batch_skip(B)) return;
  data += blockIdx.z * B.s_delta;
  gf += blockIdx.z * B.s_g;
  if (Gf != nullptr) Gf += blockIdx.z * B.s_G;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Lx = g.L[0], Ly = g.L[1];
  C2<R>* tw;
  short* pos;
  C2<R>* tile = setup_smem<R>(smem_raw, twg, posg, Lx, Ly, &tw, &pos);
  const int RS = Lx + 1, PS = Ly * RS;
  const int64_t slab = blockIdx.x;
  const int plane = Lx * Ly;
  for (int i = threadIdx.x; i < 4 * plane; i += blockDim.x) {
    const int f = (int)cd.a.div((uint32_t)i), r = i - f * plane, y = (int)cd.b.div((uint32_t)r), x = r - y * Lx;
    cp_async_elem<R>(&tile[f * PS + y * RS + x], &data[(int64_t)f * g.V + slab * plane + r]);
  }
  cp_async_wait();
  __syncthreads();
  fft_lines_dif<R, +1>(tile, lx, dx, tw);
  fft_lines_dif<R, +1>(tile, ly, dy, tw + Lx);
  for (int i = threadIdx.x; i < plane; i += blockDim.x) {
    const int y = (int)cd.b.div((uint32_t)i), x = i - y * Lx;
    const int o = pos[Lx + y] * RS + pos[x];
    gauge_site<R, RG, GROWS, EXPG>(tile[o], tile[PS + o], tile[2 * PS + o], tile[3 * PS + o], g.V, slab * plane + i, gf,
                                   Gf);
  }
}

// Unfused variant for planes whose four fields do not fit in shared memory:
// the inverse (x, y) transform has already been applied to data.
template <typename R, typename RG, int GROWS, bool EXPG>
__global__ void gauge_from_delta_kernel(Geom g, const C2<R>* __restrict__ data, C2<RG>* __restrict__ gf,
                                        C2<RG>* __restrict__ Gf, Batch B) {
  if (batch_skip(B)) return;
  data += blockIdx.z * B.s_delta;
  gf += blockIdx.z * B.s_g;
  if (Gf != nullptr) Gf += blockIdx.z * B.s_G;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  gauge_site<R, RG, GROWS, EXPG>(data[s], data[g.V + s], data[2 * g.V + s], data[3 * g.V + s], g.V, s, gf, Gf);
}

// ---------------------------------------------------------------------------
// plan and launchers
// ---------------------------------------------------------------------------

static int radix_schedule(int N, int* radix) {
  int a = 0, b = 0, n = N;
  while (n % 2 == 0) { n /= 2; ++a; }
  while (n % 3 == 0) { n /= 3; ++b; }
  if (n != 1 || N < 2) return -1;
  int k = 0;
  while (a >= 3) { radix[k++] = 8; a -= 3; }
  if (a == 2) radix[k++] = 4;
  if (a == 1) radix[k++] = 2;
  while (b-- > 0) radix[k++] = 3;
  return k;
}

// Position of natural index n in the digit-reversed order that the DIT
// stages expect (and the DIF stages produce) for the given radix sequence.
static void digit_positions(int N, const int* radix, int nst, short* pos) {
  if (nst == 0) { pos[0] = 0; return; }
  const int Rl = radix[nst - 1], Ns = N / Rl;
  std::vector<short> sub(Ns);
  digit_positions(Ns, radix, nst - 1, sub.data());
  for (int n = 0; n < N; ++n) pos[n] = (short)((n % Rl) * Ns + sub[n / Rl]);
}

void fft_positions(const FFTPlan& p, short* out) {
  int off = 0;
  for (int mu = 0; mu < 4; ++mu) {
    digit_positions(p.d[mu].N, p.d[mu].radix, p.d[mu].nst, out + off);
    off += p.d[mu].N;
  }
}

static int threads_for(int points) {
  int t = (points + 7) / 8;
  t = ((t + 31) / 32) * 32;
  return std::max(64, std::min(512, t));
}

// Tiles of the 1D x 4 and 3D + 1D decompositions: up to 32 x-lines per CTA
// in the x pass, up to 16 x columns in the y, z, t passes (runs of 16
// elements), and the whole (x, y, z) slab of one field in the 3D pass when
// it fits.
// Tiles of the 1D passes: nl x-lines per CTA in the x pass, xc x columns in
// the y, z, t passes.  False when they do not divide the lattice.
bool set_line_tiles(const int L[4], int real_bytes, int nl, int xc, FFTPlan* p) {
  const size_t cb = 2 * (size_t)real_bytes;
  const int64_t xlines = (int64_t)L[1] * L[2] * L[3];
  if (nl < 1 || xc < 1 || xlines % nl || L[0] % xc) return false;
  p->nl_x = nl;
  p->xc_line = xc;
  for (int mu = 0; mu < 4; ++mu) {
    const int lines = mu == 0 ? nl : xc;
    const size_t hdr = (size_t)((L[mu] + 1) & ~1) * cb + (size_t)((L[mu] + 7) & ~7) * 2;
    p->smem_line[mu] = hdr + (size_t)lines * (L[mu] + 1) * cb;
    p->threads_line[mu] = threads_for(lines * L[mu]);
    if (p->smem_line[mu] > 220 * 1024) return false;
  }
  return true;
}

static void configure_alt_passes(const int L[4], int real_bytes, FFTPlan* p) {
  const size_t cb = 2 * (size_t)real_bytes, maxsm = 220 * 1024;
  const int64_t V = (int64_t)L[0] * L[1] * L[2] * L[3];
  const int64_t xlines = V / L[0];
  int nl = 32;
  while (nl > 1 && (xlines % nl || smem_header_bytes<double>(L[0], 0) + (size_t)nl * (L[0] + 1) * cb > 64 * 1024))
    --nl;
  int xc = 16;
  while (xc > 1 && L[0] % xc) --xc;
  set_line_tiles(L, real_bytes, nl, xc, p);
  const size_t hxyz = (size_t)((L[0] + L[1] + L[2] + 1) & ~1) * cb + (size_t)((L[0] + L[1] + L[2] + 7) & ~7) * 2;
  p->smem_xyz = hxyz + (size_t)L[2] * L[1] * (L[0] + 1) * cb;
  p->fit_xyz = p->smem_xyz <= maxsm ? 1 : 0;
  p->threads_xyz = threads_for(L[0] * L[1] * L[2]);
}

cudaError_t configure_fft_plan(const int L[4], int real_bytes, FFTPlan* p) {
  const size_t cb = 2 * (size_t)real_bytes;  // bytes per complex element
  for (int mu = 0; mu < 4; ++mu) {
    p->d[mu].N = L[mu];
    p->d[mu].nst = radix_schedule(L[mu], p->d[mu].radix);
    if (p->d[mu].nst < 0) return cudaErrorInvalidValue;
    int Ns = 1;
    for (int st = 0; st < p->d[mu].nst; ++st) {
      p->d[mu].ns[st] = FastDiv::make((uint32_t)Ns);
      Ns *= p->d[mu].radix[st];
    }
  }
  const int Lx = L[0], Ly = L[1], Lz = L[2], Lt = L[3];
  const size_t hxy = (size_t)((Lx + Ly + 1) & ~1) * cb + (size_t)((Lx + Ly + 7) & ~7) * 2;
  const size_t hzt = (size_t)((Lz + Lt + 1) & ~1) * cb + (size_t)((Lz + Lt + 7) & ~7) * 2;
  const size_t plane_xy = (size_t)Ly * (Lx + 1) * cb;
  const size_t budget = 100 * 1024, maxsm = 220 * 1024;
  p->fpb_xy = 4;
  while (p->fpb_xy > 1 && p->fpb_xy * plane_xy > budget) p->fpb_xy /= 2;
  if (plane_xy * p->fpb_xy + hxy > maxsm) return cudaErrorInvalidValue;
  p->smem_xy = hxy + p->fpb_xy * plane_xy;
  p->fuse_g = (4 * plane_xy + hxy <= maxsm) ? 1 : 0;
  p->smem_c = hxy + 4 * plane_xy;
  int xc = 1;
  for (int c = 8; c >= 1; c /= 2) {
    if (Lx % c) continue;
    if (hzt + (size_t)Lt * (Lz * c + 1) * cb <= budget) { xc = c; break; }
  }
  if (xc == 1 && Lx % 2 == 0 && hzt + (size_t)Lt * (Lz * 2 + 1) * cb <= maxsm) xc = 2;
  p->xc = xc;
  p->smem_zt = hzt + (size_t)Lt * (Lz * xc + 1) * cb;
  if (p->smem_zt > maxsm) return cudaErrorInvalidValue;
  p->threads_xy = threads_for(p->fpb_xy * Lx * Ly);
  p->threads_zt = threads_for(Lz * Lt * xc);
  p->threads_c = threads_for(4 * Lx * Ly);
  configure_alt_passes(L, real_bytes, p);
  return cudaSuccess;
}

// Candidate plans for the autotuner: every fields-per-CTA count of the (x,y)
// passes, every x-column count of the (z,t) pass that fits shared memory,
// and three CTA sizes (8, 16 or 32 elements per thread) for each.
void fft_plan_candidates(const int L[4], int real_bytes, std::vector<FFTPlan>& out) {
  FFTPlan base;
  out.clear();
  if (configure_fft_plan(L, real_bytes, &base) != cudaSuccess) return;
  const size_t cb = 2 * (size_t)real_bytes, maxsm = 220 * 1024;
  const int Lx = L[0], Ly = L[1], Lz = L[2], Lt = L[3];
  const size_t hxy = (size_t)((Lx + Ly + 1) & ~1) * cb + (size_t)((Lx + Ly + 7) & ~7) * 2;
  const size_t hzt = (size_t)((Lz + Lt + 1) & ~1) * cb + (size_t)((Lz + Lt + 7) & ~7) * 2;
  const size_t plane_xy = (size_t)Ly * (Lx + 1) * cb;
  for (int fpb = 1; fpb <= 4; fpb *= 2) {
    if (hxy + fpb * plane_xy > maxsm) continue;
    for (int xc = 1; xc <= 8; xc *= 2) {
      if (Lx % xc || hzt + (size_t)Lt * (Lz * xc + 1) * cb > maxsm) continue;
      for (int tdiv = 8; tdiv <= 32; tdiv *= 2) {
        FFTPlan p = base;
        p.fpb_xy = fpb;
        p.smem_xy = hxy + fpb * plane_xy;
        p.xc = xc;
        p.smem_zt = hzt + (size_t)Lt * (Lz * xc + 1) * cb;
        auto thr = [&](int points) {
          int t = (points + tdiv - 1) / tdiv;
          t = ((t + 31) / 32) * 32;
          return std::max(64, std::min(512, t));
        };
        p.threads_xy = thr(fpb * Lx * Ly);
        p.threads_zt = thr(Lz * Lt * xc);
        p.threads_c = thr(4 * Lx * Ly);
        out.push_back(p);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// autotune cache
// ---------------------------------------------------------------------------

static std::mutex g_tune_mutex;
static std::map<std::string, TuneChoice> g_tune_cache;
static bool g_tune_loaded = false;

TuneChoice tune_choice_of(const FFTPlan& p, int decomp) {
  return TuneChoice{decomp, p.fpb_xy, p.xc, p.threads_xy, p.threads_zt, p.threads_c, p.nl_x, p.xc_line};
}

bool tune_choice_matches(const FFTPlan& p, const TuneChoice& c) {
  return p.fpb_xy == c.fpb_xy && p.xc == c.xc && p.threads_xy == c.threads_xy && p.threads_zt == c.threads_zt &&
         p.threads_c == c.threads_c && p.nl_x == c.nl_x && p.xc_line == c.xc_line;
}

bool tune_cache_get(const std::string& key, TuneChoice* c) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  if (!g_tune_loaded) {
    g_tune_loaded = true;
    const char* path = std::getenv("LGF_AUTOTUNE_CACHE");
    FILE* f = path ? std::fopen(path, "r") : nullptr;
    if (f) {
      char k[256];
      TuneChoice t{};
      while (std::fscanf(f, "%255s %d %d %d %d %d %d %d %d", k, &t.decomp, &t.fpb_xy, &t.xc, &t.threads_xy,
                         &t.threads_zt, &t.threads_c, &t.nl_x, &t.xc_line) == 9)
        g_tune_cache[k] = t;
      std::fclose(f);
    }
  }
  auto it = g_tune_cache.find(key);
  if (it == g_tune_cache.end()) return false;
  *c = it->second;
  return true;
}

void tune_cache_put(const std::string& key, const TuneChoice& c) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[key] = c;
  const char* path = std::getenv("LGF_AUTOTUNE_CACHE");
  FILE* f = path ? std::fopen(path, "a") : nullptr;
  if (!f) return;
  std::fprintf(f, "%s %d %d %d %d %d %d %d %d\n", key.c_str(), c.decomp, c.fpb_xy, c.xc, c.threads_xy, c.threads_zt,
               c.threads_c, c.nl_x, c.xc_line);
  std::fclose(f);
}

template <typename K> static cudaError_t allow_smem(K kernel, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R>
cudaError_t launch_fft_xy(const Geom& g, const FFTPlan& p, C2<R>* data, const C2<R>* tw, const short* pos, int sign,
                          int nfields, cudaStream_t s, const Batch& B) {
  int fpb = std::min(p.fpb_xy, nfields);
  while (nfields % fpb) fpb /= 2;
  const int thr = fpb == p.fpb_xy ? p.threads_xy : threads_for(fpb * g.L[0] * g.L[1]);
  const size_t smem = smem_header_bytes<R>(g.L[0], g.L[1]) + (size_t)fpb * g.L[1] * (g.L[0] + 1) * sizeof(C2<R>);
  dim3 grid((unsigned)(g.L[2] * g.L[3]), (unsigned)(nfields / fpb), (unsigned)B.n);
  const int Lx = g.L[0], Ly = g.L[1], RS = Lx + 1, PS = Ly * RS;
  const Lines lx = make_lines(fpb * Ly, fpb * Ly, RS, 0, 1), ly = make_lines(fpb * Lx, Lx, 1, PS, RS);
  const CopyDiv cd{FastDiv::make((uint32_t)(Lx * Ly)), FastDiv::make((uint32_t)Lx)};
  cudaError_t e;
  if (sign < 0) {
    if ((e = allow_smem(fft_xy_kernel<R, -1>, smem)) != cudaSuccess) return e;
    fft_xy_kernel<R, -1><<<grid, thr, smem, s>>>(g, p.d[0], p.d[1], data, tw, pos, fpb, lx, ly, cd, B);
  } else {
    if ((e = allow_smem(fft_xy_kernel<R, +1>, smem)) != cudaSuccess) return e;
    fft_xy_kernel<R, +1><<<grid, thr, smem, s>>>(g, p.d[0], p.d[1], data, tw, pos, fpb, lx, ly, cd, B);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_zt(const Geom& g, const FFTPlan& p, C2<R>* data, const C2<R>* tw, const short* pos,
                          const R* K, int mode, int nfields, cudaStream_t s, const LearnedIO& lio, const Batch& B) {
  const size_t smem = p.smem_zt;
  dim3 grid((unsigned)(g.L[0] / p.xc * g.L[1]), (unsigned)nfields, (unsigned)B.n);
  const bool lrn = mode == 0 && (lio.mtab != nullptr || lio.snap != nullptr);
  cudaError_t e = lrn ? allow_smem(fft_zt_filter_kernel<R, true>, smem) : allow_smem(fft_zt_filter_kernel<R, false>, smem);
  if (e != cudaSuccess) return e;
  const int4 H = make_int4(g.L[0] / 2 + 1, g.L[1] / 2 + 1, g.L[2] / 2 + 1, g.L[3] / 2 + 1);
  const int xc = p.xc, Lz = g.L[2], Lt = g.L[3], TS = Lz * xc + 1;
  const Lines lz = make_lines(Lt * xc, xc, 1, TS, xc), lt = make_lines(Lz * xc, Lz * xc, 1, 0, TS);
  const CopyDiv cd{FastDiv::make((uint32_t)xc), FastDiv::make((uint32_t)Lz)};
  if (lrn)
    fft_zt_filter_kernel<R, true><<<grid, p.threads_zt, smem, s>>>(g, p.d[2], p.d[3], data, tw, pos, K, p.xc, mode, lio,
                                                                   H, lz, lt, cd, B);
  else
    fft_zt_filter_kernel<R, false><<<grid, p.threads_zt, smem, s>>>(g, p.d[2], p.d[3], data, tw, pos, K, p.xc, mode,
                                                                    lio, H, lz, lt, cd, B);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_line(const Geom& g, const FFTPlan& p, int mu, C2<R>* data, const C2<R>* tw, const short* pos,
                            const R* K, int mode, int nfields, cudaStream_t s, const Batch& B, const LearnedIO& lio) {
  const int N = g.L[mu];
  LinePass lp;
  lp.N = N;
  lp.contiguous = mu == 0;
  lp.nl = mu == 0 ? p.nl_x : p.xc_line;
  lp.S = g.stride[mu];
  lp.SN = lp.S * N;
  lp.dload = FastDiv::make((uint32_t)(lp.contiguous ? N : lp.nl));
  lp.dlob = FastDiv::make((uint32_t)(lp.contiguous ? 1 : lp.S / lp.nl));
  const int64_t blocks = g.V / ((int64_t)N * lp.nl);
  const size_t smem = p.smem_line[mu];
  const bool lrn = mode == 0 && (lio.mtab != nullptr || lio.snap != nullptr);
  cudaError_t e = lrn ? allow_smem(fft_line_kernel<R, true>, smem) : allow_smem(fft_line_kernel<R, false>, smem);
  if (e != cudaSuccess) return e;
  const int off = mu == 0 ? 0 : mu == 1 ? g.L[0] : mu == 2 ? g.L[0] + g.L[1] : g.L[0] + g.L[1] + g.L[2];
  const Lines ln = make_lines(lp.nl, lp.nl, N + 1, 0, 1);
  const int4 H = make_int4(g.L[0] / 2 + 1, g.L[1] / 2 + 1, g.L[2] / 2 + 1, g.L[3] / 2 + 1);
  const dim3 grid((unsigned)blocks, (unsigned)nfields, (unsigned)B.n);
  if (lrn)
    fft_line_kernel<R, true><<<grid, p.threads_line[mu], smem, s>>>(lp, p.d[mu], g, data, tw + off, pos + off, K, mode,
                                                                    ln, lio, H, B);
  else
    fft_line_kernel<R, false><<<grid, p.threads_line[mu], smem, s>>>(lp, p.d[mu], g, data, tw + off, pos + off, K,
                                                                     mode, ln, lio, H, B);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_xyz(const Geom& g, const FFTPlan& p, C2<R>* data, const C2<R>* tw, const short* pos, int sign,
                           int nfields, cudaStream_t s, const Batch& B) {
  if (!p.fit_xyz) return cudaErrorInvalidConfiguration;
  const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], RS = Lx + 1, PS = Ly * RS;
  const Lines lx = make_lines(Ly * Lz, Ly * Lz, RS, 0, 1);
  const Lines ly = make_lines(Lx * Lz, Lx, 1, PS, RS);
  const Lines lz = make_lines(Lx * Ly, Lx, 1, RS, PS);
  const CopyDiv cd{FastDiv::make((uint32_t)(Lx * Ly)), FastDiv::make((uint32_t)Lx)};
  const dim3 grid((unsigned)g.L[3], (unsigned)nfields, (unsigned)B.n);
  cudaError_t e;
  if (sign < 0) {
    if ((e = allow_smem(fft_xyz_kernel<R, -1>, p.smem_xyz)) != cudaSuccess) return e;
    fft_xyz_kernel<R, -1><<<grid, p.threads_xyz, p.smem_xyz, s>>>(g, p.d[0], p.d[1], p.d[2], data, tw, pos, lx, ly, lz,
                                                                  cd, B);
  } else {
    if ((e = allow_smem(fft_xyz_kernel<R, +1>, p.smem_xyz)) != cudaSuccess) return e;
    fft_xyz_kernel<R, +1><<<grid, p.threads_xyz, p.smem_xyz, s>>>(g, p.d[0], p.d[1], p.d[2], data, tw, pos, lx, ly, lz,
                                                                  cd, B);
  }
  return cudaGetLastError();
}

template <typename R, typename RG, int GROWS>
cudaError_t launch_gauge_from_delta(const Geom& g, const C2<R>* data, C2<RG>* gfield, C2<RG>* Gfield, cudaStream_t s,
                                    const Batch& B, int exact_exp) {
  const dim3 grid((unsigned)((g.V + 127) / 128), 1, (unsigned)B.n);
  if (exact_exp)
    gauge_from_delta_kernel<R, RG, GROWS, true><<<grid, 128, 0, s>>>(g, data, gfield, Gfield, B);
  else
    gauge_from_delta_kernel<R, RG, GROWS, false><<<grid, 128, 0, s>>>(g, data, gfield, Gfield, B);
  return cudaGetLastError();
}

template <typename R, typename RG, int GROWS, bool EXPG>
static cudaError_t launch_pass_c(const Geom& g, const FFTPlan& p, C2<R>* data, const C2<R>* tw, const short* pos,
                                 C2<RG>* gfield, C2<RG>* Gfield, cudaStream_t s, const Batch& B) {
  cudaError_t e;
  if (!p.fuse_g) {
    if ((e = launch_fft_xy<R>(g, p, data, tw, pos, +1, 4, s, B)) != cudaSuccess) return e;
    gauge_from_delta_kernel<R, RG, GROWS, EXPG><<<dim3((unsigned)((g.V + 127) / 128), 1, (unsigned)B.n), 128, 0, s>>>(
        g, data, gfield, Gfield, B);
    return cudaGetLastError();
  }
  const size_t smem = p.smem_c;
  if ((e = allow_smem(fft_xy_inv_gauge_kernel<R, RG, GROWS, EXPG>, smem)) != cudaSuccess) return e;
  const int Lx = g.L[0], Ly = g.L[1], RS = Lx + 1, PS = Ly * RS;
  const Lines lx = make_lines(4 * Ly, 4 * Ly, RS, 0, 1), ly = make_lines(4 * Lx, Lx, 1, PS, RS);
  const CopyDiv cd{FastDiv::make((uint32_t)(Lx * Ly)), FastDiv::make((uint32_t)Lx)};
  fft_xy_inv_gauge_kernel<R, RG, GROWS, EXPG>
      <<<dim3((unsigned)(g.L[2] * g.L[3]), 1, (unsigned)B.n), p.threads_c, smem, s>>>(g, p.d[0], p.d[1], data, tw, pos,
                                                                                    gfield, Gfield, lx, ly, cd, B);
  return cudaGetLastError();
}

template <typename R, typename RG, int GROWS>
cudaError_t launch_fft_xy_inv_gauge(const Geom& g, const FFTPlan& p, C2<R>* data, const C2<R>* tw, const short* pos,
                                    C2<RG>* gfield, C2<RG>* Gfield, cudaStream_t s, const Batch& B, int exact_exp) {
  return exact_exp ? launch_pass_c<R, RG, GROWS, true>(g, p, data, tw, pos, gfield, Gfield, s, B)
                   : launch_pass_c<R, RG, GROWS, false>(g, p, data, tw, pos, gfield, Gfield, s, B);
}

template cudaError_t launch_fft_xy<double>(const Geom&, const FFTPlan&, C2<double>*, const C2<double>*, const short*,
                                           int, int, cudaStream_t, const Batch&);
template cudaError_t launch_fft_xy<float>(const Geom&, const FFTPlan&, C2<float>*, const C2<float>*, const short*,
                                          int, int, cudaStream_t, const Batch&);
template cudaError_t launch_fft_zt<double>(const Geom&, const FFTPlan&, C2<double>*, const C2<double>*, const short*,
                                           const double*, int, int, cudaStream_t, const LearnedIO&, const Batch&);
template cudaError_t launch_fft_zt<float>(const Geom&, const FFTPlan&, C2<float>*, const C2<float>*, const short*,
                                          const float*, int, int, cudaStream_t, const LearnedIO&, const Batch&);
#define LGF_INST_C(R, RG, GR)                                                                                    \
  template cudaError_t launch_fft_xy_inv_gauge<R, RG, GR>(const Geom&, const FFTPlan&, C2<R>*, const C2<R>*,      \
                                                          const short*, C2<RG>*, C2<RG>*, cudaStream_t, const Batch&, \
                                                          int);
LGF_INST_C(double, double, 3)
LGF_INST_C(double, double, 2)
LGF_INST_C(float, float, 2)
LGF_INST_C(float, float, 3)
#define LGF_INST_G(R, RG, GR)                                                                                   \
  template cudaError_t launch_gauge_from_delta<R, RG, GR>(const Geom&, const C2<R>*, C2<RG>*, C2<RG>*,         \
                                                          cudaStream_t, const Batch&, int);
LGF_INST_G(double, double, 3)
LGF_INST_G(double, double, 2)
LGF_INST_G(float, float, 2)
LGF_INST_G(float, float, 3)
#define LGF_INST_ALT(R)                                                                                         \
  template cudaError_t launch_fft_line<R>(const Geom&, const FFTPlan&, int, C2<R>*, const C2<R>*, const short*, \
                                          const R*, int, int, cudaStream_t, const Batch&, const LearnedIO&);   \
  template cudaError_t launch_fft_xyz<R>(const Geom&, const FFTPlan&, C2<R>*, const C2<R>*, const short*, int,  \
                                         int, cudaStream_t, const Batch&);
LGF_INST_ALT(double)
LGF_INST_ALT(float)

}  // namespace lgf
