// Learned momentum-space multiplier m(k) (not in arXiv:1206.0675; an
// addition on top of the filter alpha p2max/p2(k) of its Eq. (eq:gx)).
//
//   * inference: MLP 8 -> 64 -> 64 -> 64 -> 1 with BF16 weights and FP32
//     accumulation on the tensor cores (mma.sync m16n8k16), one warp per 16
//     feature rows, hidden activations kept in registers between layers;
//     evaluated once per iteration for the distinct momentum classes
//     (identical per-direction p2 tuples) and gathered by pass B;
//   * training: forward and backward in FP32 (CTA-chunked, deterministic
//     fixed-order gradient reduction) and an Adam update;
//   * logging: per (theta bucket, momentum class) statistics of consecutive
//     Fourier-space divergences of a plain trajectory, the training data.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "lgf_internal.h"
#include "lgf_mlp.h"

namespace lgf {

// ---------------------------------------------------------------------------
// tensor-core inference
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory copy of the network: weight rows padded so that the B
// fragment loads of a warp hit 32 distinct banks.
constexpr int W1S = 24;  // 16 inputs (6 used) + 8 pad, bf16
constexpr int WHS = 72;  // 64 + 8 pad, bf16

struct MlpSmem {
  __nv_bfloat16 W1[MLP_NH * W1S];
  __nv_bfloat16 W2[MLP_NH * WHS];
  __nv_bfloat16 W3[MLP_NH * WHS];
  float b1[MLP_NH], b2[MLP_NH], b3[MLP_NH], w4[MLP_NH];
  float b4;
};

__device__ void mlp_load_smem(MlpSmem& S, const __nv_bfloat16* __restrict__ P) {
  for (int i = threadIdx.x; i < MLP_NH * 16; i += blockDim.x) {
    const int n = i / 16, k = i % 16;
    S.W1[n * W1S + k] = k < MLP_NIN ? P[MLP_OFF_W1 + n * MLP_NIN + k] : __float2bfloat16(0.f);
  }
  for (int i = threadIdx.x; i < MLP_NH * MLP_NH; i += blockDim.x) {
    const int n = i / MLP_NH, k = i % MLP_NH;
    S.W2[n * WHS + k] = P[MLP_OFF_W2 + i];
    S.W3[n * WHS + k] = P[MLP_OFF_W3 + i];
  }
  for (int i = threadIdx.x; i < MLP_NH; i += blockDim.x) {
    S.b1[i] = __bfloat162float(P[MLP_OFF_B1 + i]);
    S.b2[i] = __bfloat162float(P[MLP_OFF_B2 + i]);
    S.b3[i] = __bfloat162float(P[MLP_OFF_B3 + i]);
    S.w4[i] = __bfloat162float(P[MLP_OFF_W4 + i]);
  }
  if (threadIdx.x == 0) S.b4 = __bfloat162float(P[MLP_OFF_B4]);
}

// One hidden layer 64 -> 64 from A fragments (4 k-blocks) into accumulators.
__device__ __forceinline__ void mlp_hidden(const MlpSmem& S, const __nv_bfloat16* W, const float* bias,
                                           const uint32_t a[4][4], float acc[8][4], int g, int tig) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float bl = bias[8 * j + 2 * tig], bh = bias[8 * j + 2 * tig + 1];
    acc[j][0] = bl; acc[j][1] = bh; acc[j][2] = bl; acc[j][3] = bh;
    const __nv_bfloat16* row = W + (8 * j + g) * WHS;
#pragma unroll
    for (int kb = 0; kb < 4; ++kb) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row + 16 * kb + 2 * tig);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 16 * kb + 8 + 2 * tig);
      mma_16816(acc[j], a[kb], b0, b1);
    }
  }
}

// ReLU of the accumulators, repacked as BF16 A fragments of the next layer.
__device__ __forceinline__ void relu_to_frags(float acc[8][4], uint32_t a[4][4]) {
#pragma unroll
  for (int j = 0; j < 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[j][e] = fmaxf(acc[j][e], 0.f);
#pragma unroll
  for (int kb = 0; kb < 4; ++kb) {
    a[kb][0] = pack_bf16(acc[2 * kb][0], acc[2 * kb][1]);
    a[kb][1] = pack_bf16(acc[2 * kb][2], acc[2 * kb][3]);
    a[kb][2] = pack_bf16(acc[2 * kb + 1][0], acc[2 * kb + 1][1]);
    a[kb][3] = pack_bf16(acc[2 * kb + 1][2], acc[2 * kb + 1][3]);
  }
}

// z for the 16 rows of a warp tile.  xr0 / xr1: the 6 features of rows
// g and g + 8 (g = lane / 4).  Returns z of rows g (lane's tig == 0 holds
// the reduced value in all four lanes of the group) and g + 8.
__device__ __forceinline__ void mlp_tile(const MlpSmem& S, const float xr0[MLP_NIN], const float xr1[MLP_NIN],
                                         float& z0, float& z1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  uint32_t a1[4];
  const int c0 = 2 * tig;
  a1[0] = pack_bf16(c0 < MLP_NIN ? xr0[c0] : 0.f, c0 + 1 < MLP_NIN ? xr0[c0 + 1] : 0.f);
  a1[1] = pack_bf16(c0 < MLP_NIN ? xr1[c0] : 0.f, c0 + 1 < MLP_NIN ? xr1[c0 + 1] : 0.f);
  a1[2] = 0u;
  a1[3] = 0u;
  float acc[8][4];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float bl = S.b1[8 * j + 2 * tig], bh = S.b1[8 * j + 2 * tig + 1];
    acc[j][0] = bl; acc[j][1] = bh; acc[j][2] = bl; acc[j][3] = bh;
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(S.W1 + (8 * j + g) * W1S + 2 * tig);
    const uint32_t b1 = *reinterpret_cast<const uint32_t*>(S.W1 + (8 * j + g) * W1S + 8 + 2 * tig);
    mma_16816(acc[j], a1, b0, b1);
  }
  uint32_t a[4][4];
  relu_to_frags(acc, a);
  mlp_hidden(S, S.W2, S.b2, a, acc, g, tig);
  relu_to_frags(acc, a);
  mlp_hidden(S, S.W3, S.b3, a, acc, g, tig);
  float s0 = 0.f, s1 = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float wl = S.w4[8 * j + 2 * tig], wh = S.w4[8 * j + 2 * tig + 1];
    s0 = fmaf(fmaxf(acc[j][0], 0.f), wl, fmaf(fmaxf(acc[j][1], 0.f), wh, s0));
    s1 = fmaf(fmaxf(acc[j][2], 0.f), wl, fmaf(fmaxf(acc[j][3], 0.f), wh, s1));
  }
  s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
  s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
  s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
  z0 = s0 + S.b4;
  z1 = s1 + S.b4;
}

__device__ __forceinline__ float softplusf(float z) { return z > 20.f ? z : log1pf(expf(z)); }

// m = softplus(z) for arbitrary feature rows X[n][6] (used to check the
// tensor-core network against the CPU oracle).
__global__ void __launch_bounds__(128) mlp_eval_kernel(const __nv_bfloat16* __restrict__ P,
                                                       const float* __restrict__ X, int64_t n,
                                                       float* __restrict__ out) {
  __shared__ MlpSmem S;
  mlp_load_smem(S, P);
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = wid * 16; base < n; base += nw * 16) {
    float x0[MLP_NIN], x1[MLP_NIN];
    const int64_t r0 = base + g, r1 = base + g + 8;
#pragma unroll
    for (int k = 0; k < MLP_NIN; ++k) {
      x0[k] = r0 < n ? X[r0 * MLP_NIN + k] : 0.f;
      x1[k] = r1 < n ? X[r1 * MLP_NIN + k] : 0.f;
    }
    float z0, z1;
    mlp_tile(S, x0, x1, z0, z1);
    if ((lane & 3) == 0) {
      if (r0 < n) out[r0] = softplusf(z0);
      if (r1 < n) out[r1] = softplusf(z1);
    }
  }
}

// Multiplier of every momentum class of the lattice for the step that starts
// from the current links (iteration k): class c = ((ft Hz + fz) Hy + fy) Hx + fx
// with f = min(k, L - k) and H = L/2 + 1.  Features: p2 = 4 sin^2(pi f / L)
// per direction, the theta bucket, the iteration fraction, the contraction
// of theta over the last step, and the class's own contraction over the last
// step whose two divergences are stored:
//   r = 1 - (1 - r_obs) / m,  r_obs = sum Re<D^_{k-1}, D^_{k-2}> / sum |D^_{k-2}|^2
// over the modes and packed fields of the class, m the multiplier that step
// k - 2 applied to the class (the table of step k - 2, which this kernel then
// overwrites), so that r is the contraction the plain filter would have given.
// The four lanes that share a feature row gather one packed field each, in a
// fixed order, and add their sums by shuffles (deterministic).  A step that
// redoes a rejected one runs the plain filter: its table is all ones.
// Block 0 also decides whether the step uses the table.
__global__ void __launch_bounds__(128) mlp_multiplier_kernel(const __nv_bfloat16* __restrict__ P, MlpGeom mg,
                                                             Geom geo, const float* __restrict__ p2, DevState* st,
                                                             float* __restrict__ mtab_base,
                                                             const uint32_t* __restrict__ snap) {
  __shared__ MlpSmem S;
  __shared__ float sf[3];  // the features shared by every class, formed once per CTA
  mlp_load_smem(S, P);
  const int iter = st->iter;
  const int redo = st->revert;  // the measurement after the step assigns revert afresh
  const bool have_rate = snap != nullptr && st->snaps >= 2;
  if (threadIdx.x == 0) {
    // FP64 logarithms: one thread per CTA, not every thread (they would
    // occupy the FP64 pipe for most of the kernel)
    const double theta = st->theta, theta_prev = st->theta_prev;
    const float fb = theta > 0.0 ? (float)(floor(2.0 * log10(theta)) * 0.5) : -20.f;
    sf[0] = -fb / 16.f;
    sf[1] = fminf((float)iter / MLP_ITER_SCALE, 1.f);
    sf[2] = iter > 0 ? mlp_rate_feature(theta, theta_prev) : 0.f;
  }
  __syncthreads();
  // the plain filter: a redo of a rejected step, or a step from links whose
  // theta is not yet below the level where the table is applied
  const bool plain = redo || !(st->theta < mg.theta_on);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->use_m = plain ? 0 : 1;
    st->redo = redo;
  }
  float* mtab = mtab_base + (int64_t)(iter & 1) * mg.nclass;
  const int64_t V = geo.V;
  const uint32_t* sa = snap + (int64_t)((iter + 1) & 1) * 4 * V;  // divergence k - 1
  const uint32_t* sb = snap + (int64_t)(iter & 1) * 4 * V;        // divergence k - 2
  const float f4 = sf[0], f5 = sf[1], f6 = sf[2];
  const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t n = mg.nclass;
  for (int64_t base = wid * 16; base < n; base += nw * 16) {
    if (plain) {
      if (tig == 0) {
        if (base + g < n) mtab[base + g] = 1.f;
        if (base + g + 8 < n) mtab[base + g + 8] = 1.f;
      }
      continue;
    }
    float x[2][MLP_NIN];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int64_t c = base + g + 8 * h;
      if (c >= n) c = n - 1;
      const int64_t cls = c;
      int f[4];
      f[0] = (int)(c % mg.H[0]); c /= mg.H[0];
      f[1] = (int)(c % mg.H[1]); c /= mg.H[1];
      f[2] = (int)(c % mg.H[2]); c /= mg.H[2];
      f[3] = (int)c;
      x[h][0] = 0.25f * p2[f[0]];
      x[h][1] = 0.25f * p2[mg.off[1] + f[1]];
      x[h][2] = 0.25f * p2[mg.off[2] + f[2]];
      x[h][3] = 0.25f * p2[mg.off[3] + f[3]];
      x[h][4] = f4;
      x[h][5] = f5;
      x[h][6] = f6;
      float r = 0.f;
      if (have_rate) {
        // the modes k_mu in {f_mu, L_mu - f_mu} of the class (one value where
        // f_mu = 0 or 2 f_mu = L_mu); this lane takes packed field tig.  All
        // sixteen candidate loads are issued before any is used (predicated,
        // fully unrolled): a loop that waited on each load left the kernel
        // bound by load latency.
        int64_t off[4][2];
        bool two[4];
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
          two[mu] = f[mu] != 0 && 2 * f[mu] != geo.L[mu];
          off[mu][0] = geo.stride[mu] * f[mu];
          off[mu][1] = geo.stride[mu] * (geo.L[mu] - f[mu]);
        }
        const int64_t fbase = (int64_t)tig * V;
        uint32_t pa[16], pb[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const int bx = m & 1, by = (m >> 1) & 1, bz = (m >> 2) & 1, bt = (m >> 3) & 1;
          const bool ok = (!bx || two[0]) && (!by || two[1]) && (!bz || two[2]) && (!bt || two[3]);
          const int64_t sidx = fbase + off[0][bx] + off[1][by] + off[2][bz] + off[3][bt];
          pa[m] = ok ? __ldg(&sa[sidx]) : 0u;
          pb[m] = ok ? __ldg(&sb[sidx]) : 0u;
        }
        float ip = 0.f, nb = 0.f;
#pragma unroll
        for (int m = 0; m < 16; ++m) {
          const float are = bf16x2_re(pa[m]), aim = bf16x2_im(pa[m]), bre = bf16x2_re(pb[m]), bim = bf16x2_im(pb[m]);
          ip = fmaf(are, bre, fmaf(aim, bim, ip));
          nb = fmaf(bre, bre, fmaf(bim, bim, nb));
        }
        ip += __shfl_xor_sync(0xffffffffu, ip, 1);
        nb += __shfl_xor_sync(0xffffffffu, nb, 1);
        ip += __shfl_xor_sync(0xffffffffu, ip, 2);
        nb += __shfl_xor_sync(0xffffffffu, nb, 2);
        if (nb > 0.f) {
          const float m_prev = mtab[cls];
          r = 1.f - (1.f - ip / nb) / m_prev;
          r = fminf(fmaxf(r, -1.f), 1.f);
        }
      }
      x[h][7] = r;
    }
    float z0, z1;
    mlp_tile(S, x[0], x[1], z0, z1);
    if (tig == 0) {
      const int64_t r0 = base + g, r1 = base + g + 8;
      if (r0 < n) mtab[r0] = fminf(fmaxf(softplusf(z0), mg.m_lo), mg.m_hi);
      if (r1 < n) mtab[r1] = fminf(fmaxf(softplusf(z1), mg.m_lo), mg.m_hi);
    }
  }
}

cudaError_t launch_mlp_eval(const uint16_t* P, const float* X, int64_t n, float* out, cudaStream_t s) {
  const int64_t warps = (n + 15) / 16;
  const unsigned blocks = (unsigned)std::min<int64_t>((warps + 3) / 4, 152 * 8);
  mlp_eval_kernel<<<blocks > 0 ? blocks : 1, 128, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(P), X, n, out);
  return cudaGetLastError();
}

cudaError_t launch_mlp_multiplier(const uint16_t* P, const MlpGeom& mg, const Geom& g, const float* p2, DevState* st,
                                  float* mtab, const uint32_t* snap, cudaStream_t s) {
  // one 16-row tile per warp up to 16 CTAs per SM: the gathers of the class
  // contraction need many warps in flight
  const int64_t warps = (mg.nclass + 15) / 16;
  const unsigned blocks = (unsigned)std::min<int64_t>((warps + 3) / 4, 152 * 16);
  mlp_multiplier_kernel<<<blocks > 0 ? blocks : 1, 128, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(P), mg, g, p2,
                                                               st, mtab, snap);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// training: FP32 forward + backward over chunks of samples
// ---------------------------------------------------------------------------

constexpr int TCH = 64;   // samples per chunk
constexpr int TTH = 256;  // threads per CTA

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

struct TrainSmem {
  float P[MLP_NPARAM + 3];
  float G[MLP_NPARAM + 3];
  float X[TCH * MLP_NIN];
  float H1[TCH * MLP_NH], H2[TCH * MLP_NH], H3[TCH * MLP_NH], D[TCH * MLP_NH];
  float dz[TCH];
  int idx[TCH];
};

// out[s][n] = act(sum_k in[s][k] W[n][k] + b[n]) for a chunk; W row-major [n][K].
__device__ __forceinline__ void dense_fwd(const float* in, int K, const float* W, const float* b, float* out) {
  for (int e = threadIdx.x; e < TCH * MLP_NH; e += blockDim.x) {
    const int s = e / MLP_NH, n = e % MLP_NH;
    float a = b[n];
    const float* x = in + s * K;
    const float* w = W + n * K;
    for (int k = 0; k < K; ++k) a = fmaf(x[k], w[k], a);
    out[e] = fmaxf(a, 0.f);
  }
}

// Loss and gradient of the weighted MSE of log m against y, summed over the
// samples of this CTA's chunks; partial gradient and loss of the CTA are
// written to part_g[blockIdx] and part_l[blockIdx] (reduced later in order).
// Samples: idx = hash(seed, step, j) mod n for j < batch when batch > 0,
// otherwise every sample once in order.
__global__ void __launch_bounds__(TTH) mlp_grad_kernel(const float* __restrict__ Pg, const float* __restrict__ X,
                                                       const float* __restrict__ Y, const float* __restrict__ Wt,
                                                       int64_t n, int64_t batch, uint64_t seed, int step,
                                                       float inv_sw, float* __restrict__ part_g,
                                                       double* __restrict__ part_l) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) {
    S.P[i] = Pg[i];
    S.G[i] = 0.f;
  }
  const float* W1 = S.P + MLP_OFF_W1;
  const float* b1 = S.P + MLP_OFF_B1;
  const float* W2 = S.P + MLP_OFF_W2;
  const float* b2 = S.P + MLP_OFF_B2;
  const float* W3 = S.P + MLP_OFF_W3;
  const float* b3 = S.P + MLP_OFF_B3;
  const float* w4 = S.P + MLP_OFF_W4;
  const int64_t total = batch > 0 ? batch : n;
  const int64_t nchunks = (total + TCH - 1) / TCH;
  double lsum = 0.0;
  __syncthreads();
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    for (int s = threadIdx.x; s < TCH; s += blockDim.x) {
      const int64_t j = ch * TCH + s;
      int64_t i = -1;
      if (j < total) i = batch > 0 ? (int64_t)(splitmix64(seed ^ splitmix64(((uint64_t)step << 32) + j)) % n) : j;
      S.idx[s] = (int)i;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TCH * MLP_NIN; e += blockDim.x) {
      const int i = S.idx[e / MLP_NIN];
      S.X[e] = i >= 0 ? X[(int64_t)i * MLP_NIN + e % MLP_NIN] : 0.f;
    }
    __syncthreads();
    dense_fwd(S.X, MLP_NIN, W1, b1, S.H1);
    __syncthreads();
    dense_fwd(S.H1, MLP_NH, W2, b2, S.H2);
    __syncthreads();
    dense_fwd(S.H2, MLP_NH, W3, b3, S.H3);
    __syncthreads();
    // output, loss and dL/dz
    for (int s = threadIdx.x; s < TCH; s += blockDim.x) {
      const int i = S.idx[s];
      float dz = 0.f;
      if (i >= 0) {
        float z = S.P[MLP_OFF_B4];
        for (int k = 0; k < MLP_NH; ++k) z = fmaf(S.H3[s * MLP_NH + k], w4[k], z);
        const float m = softplusf(z);
        const float e = logf(m) - Y[i];
        const float w = Wt[i] * inv_sw;
        lsum += (double)w * e * e;
        const float sig = 1.f / (1.f + expf(-z));
        dz = 2.f * w * e * sig / m;
      }
      S.dz[s] = dz;
    }
    __syncthreads();
    // dA3 = dz w4 (H3 > 0), in place of H3 after its use for gw4
    for (int k = threadIdx.x; k < MLP_NH; k += blockDim.x) {
      float gw = 0.f;
      for (int s = 0; s < TCH; ++s) gw = fmaf(S.dz[s], S.H3[s * MLP_NH + k], gw);
      S.G[MLP_OFF_W4 + k] += gw;
    }
    if (threadIdx.x == 0) {
      float gb = 0.f;
      for (int s = 0; s < TCH; ++s) gb += S.dz[s];
      S.G[MLP_OFF_B4] += gb;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TCH * MLP_NH; e += blockDim.x) {
      const int s = e / MLP_NH, k = e % MLP_NH;
      S.H3[e] = S.H3[e] > 0.f ? S.dz[s] * w4[k] : 0.f;
    }
    __syncthreads();
    // layer 3 gradients and dH2 = dA3 W3 (into D), then dA2 = dH2 (H2 > 0)
    for (int e = threadIdx.x; e < MLP_NH * MLP_NH; e += blockDim.x) {
      const int nn = e / MLP_NH, k = e % MLP_NH;
      float gw = 0.f;
      for (int s = 0; s < TCH; ++s) gw = fmaf(S.H3[s * MLP_NH + nn], S.H2[s * MLP_NH + k], gw);
      S.G[MLP_OFF_W3 + e] += gw;
    }
    for (int nn = threadIdx.x; nn < MLP_NH; nn += blockDim.x) {
      float gb = 0.f;
      for (int s = 0; s < TCH; ++s) gb += S.H3[s * MLP_NH + nn];
      S.G[MLP_OFF_B3 + nn] += gb;
    }
    for (int e = threadIdx.x; e < TCH * MLP_NH; e += blockDim.x) {
      const int s = e / MLP_NH, k = e % MLP_NH;
      float d = 0.f;
      for (int nn = 0; nn < MLP_NH; ++nn) d = fmaf(S.H3[s * MLP_NH + nn], W3[nn * MLP_NH + k], d);
      S.D[e] = S.H2[e] > 0.f ? d : 0.f;
    }
    __syncthreads();
    // layer 2 gradients and dH1 = dA2 W2 (into H3), then dA1 = dH1 (H1 > 0)
    for (int e = threadIdx.x; e < MLP_NH * MLP_NH; e += blockDim.x) {
      const int nn = e / MLP_NH, k = e % MLP_NH;
      float gw = 0.f;
      for (int s = 0; s < TCH; ++s) gw = fmaf(S.D[s * MLP_NH + nn], S.H1[s * MLP_NH + k], gw);
      S.G[MLP_OFF_W2 + e] += gw;
    }
    for (int nn = threadIdx.x; nn < MLP_NH; nn += blockDim.x) {
      float gb = 0.f;
      for (int s = 0; s < TCH; ++s) gb += S.D[s * MLP_NH + nn];
      S.G[MLP_OFF_B2 + nn] += gb;
    }
    for (int e = threadIdx.x; e < TCH * MLP_NH; e += blockDim.x) {
      const int s = e / MLP_NH, k = e % MLP_NH;
      float d = 0.f;
      for (int nn = 0; nn < MLP_NH; ++nn) d = fmaf(S.D[s * MLP_NH + nn], W2[nn * MLP_NH + k], d);
      S.H3[e] = S.H1[e] > 0.f ? d : 0.f;
    }
    __syncthreads();
    // layer 1 gradients
    for (int e = threadIdx.x; e < MLP_NH * MLP_NIN; e += blockDim.x) {
      const int nn = e / MLP_NIN, k = e % MLP_NIN;
      float gw = 0.f;
      for (int s = 0; s < TCH; ++s) gw = fmaf(S.H3[s * MLP_NH + nn], S.X[s * MLP_NIN + k], gw);
      S.G[MLP_OFF_W1 + e] += gw;
    }
    for (int nn = threadIdx.x; nn < MLP_NH; nn += blockDim.x) {
      float gb = 0.f;
      for (int s = 0; s < TCH; ++s) gb += S.H3[s * MLP_NH + nn];
      S.G[MLP_OFF_B1 + nn] += gb;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) part_g[(int64_t)blockIdx.x * MLP_NPARAM + i] = S.G[i];
  // loss partial of the CTA (fixed order: per-thread sums, then thread order)
  __shared__ double ls[TTH];
  ls[threadIdx.x] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += ls[i];
    part_l[blockIdx.x] = t;
  }
}

__global__ void mlp_reduce_kernel(const float* __restrict__ part_g, const double* __restrict__ part_l, int nb,
                                  float* __restrict__ grad, double* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < MLP_NPARAM) {
    float s = 0.f;
    for (int b = 0; b < nb; ++b) s += part_g[(int64_t)b * MLP_NPARAM + i];
    grad[i] = s;
  }
  if (i == 0 && loss) {
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part_l[b];
    *loss = t;
  }
}

__global__ void adam_kernel(float* __restrict__ P, float* __restrict__ mom, float* __restrict__ vel,
                            const float* __restrict__ grad, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= MLP_NPARAM) return;
  const float g = grad[i];
  const float m = b1 * mom[i] + (1.f - b1) * g;
  const float v = b2 * vel[i] + (1.f - b2) * g * g;
  mom[i] = m;
  vel[i] = v;
  P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

size_t mlp_train_smem() { return sizeof(TrainSmem); }

cudaError_t launch_mlp_grad(const float* P, const float* X, const float* Y, const float* Wt, int64_t n, int64_t batch,
                            uint64_t seed, int step, float inv_sw, float* part_g, double* part_l, int nblocks,
                            float* grad, double* loss, cudaStream_t s) {
  const size_t smem = sizeof(TrainSmem);
  cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  mlp_grad_kernel<<<nblocks, TTH, smem, s>>>(P, X, Y, Wt, n, batch, seed, step, inv_sw, part_g, part_l);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  mlp_reduce_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(part_g, part_l, nblocks, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* P, float* mom, float* vel, const float* grad, float lr, int t, cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(P, mom, vel, grad, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

__global__ void f32_to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

cudaError_t launch_f32_to_bf16(const float* in, uint16_t* out, int n, cudaStream_t s) {
  f32_to_bf16_kernel<<<(n + 255) / 256, 256, 0, s>>>(in, reinterpret_cast<__nv_bfloat16*>(out), n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// logging: per (theta bucket, class) statistics of consecutive D^
// ---------------------------------------------------------------------------

// stats[(b * nclass + c) * 5 + {0..4}] += {Re<cur, prev>, |prev|^2, 1, iter_frac, rate}
// for every mode k of the four packed fields; b, iter_frac and the contraction
// rate feature belong to the links of prev.
template <typename R>
__global__ void mode_log_kernel(Geom g, MlpGeom mg, const C2<R>* __restrict__ cur, const C2<R>* __restrict__ prev,
                                const C2<R>* __restrict__ prev2, const LogState* __restrict__ ls,
                                double* __restrict__ stats) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V || !ls->have_prev) return;
  const int bucket = mlp_bucket_index(ls->theta_prev);
  const float iter_frac = fminf((float)ls->iter_prev / MLP_ITER_SCALE, 1.f);
  const float rate = mlp_rate_feature(ls->theta_prev, ls->theta_prev2);
  int c[4];
  site_coords(g, s, c);
  int64_t cls = 0;
  for (int mu = 3; mu >= 0; --mu) {
    const int f = min(c[mu], g.L[mu] - c[mu]);
    cls = cls * mg.H[mu] + f;
  }
  double num = 0.0, den = 0.0, num_lag = 0.0, den_lag = 0.0;
  const bool lag = ls->have_prev2 != 0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const C2<R> a = cur[f * g.V + s], b = prev[f * g.V + s];
    num += (double)a.x * b.x + (double)a.y * b.y;
    den += (double)b.x * b.x + (double)b.y * b.y;
    if (lag) {
      const C2<R> c = prev2[f * g.V + s];
      num_lag += (double)b.x * c.x + (double)b.y * c.y;
      den_lag += (double)c.x * c.x + (double)c.y * c.y;
    }
  }
  double* row = stats + ((int64_t)bucket * mg.nclass + cls) * MLP_NSTAT;
  atomicAdd(row, num);
  atomicAdd(row + 1, den);
  atomicAdd(row + 2, 1.0);
  atomicAdd(row + 3, (double)iter_frac);
  atomicAdd(row + 4, (double)rate);
  if (lag) {
    atomicAdd(row + 5, num_lag);
    atomicAdd(row + 6, den_lag);
  }
}

template <typename R>
cudaError_t launch_mode_log(const Geom& g, const MlpGeom& mg, const C2<R>* cur, const C2<R>* prev,
                            const C2<R>* prev2, const LogState* ls, double* stats, cudaStream_t s) {
  mode_log_kernel<R><<<(unsigned)((g.V + 255) / 256), 256, 0, s>>>(g, mg, cur, prev, prev2, ls, stats);
  return cudaGetLastError();
}

__global__ void log_state_update_kernel(LogState* ls, const DevState* st) {
  ls->have_prev2 = ls->have_prev;
  ls->theta_prev2 = ls->have_prev ? ls->theta_prev : 0.0;
  ls->theta_prev = st->theta;
  ls->iter_prev = st->iter;
  ls->have_prev = 1;
}

cudaError_t launch_log_state_update(LogState* ls, const DevState* st, cudaStream_t s) {
  log_state_update_kernel<<<1, 1, 0, s>>>(ls, st);
  return cudaGetLastError();
}

template cudaError_t launch_mode_log<double>(const Geom&, const MlpGeom&, const C2<double>*, const C2<double>*,
                                             const C2<double>*, const LogState*, double*, cudaStream_t);
template cudaError_t launch_mode_log<float>(const Geom&, const MlpGeom&, const C2<float>*, const C2<float>*,
                                            const C2<float>*, const LogState*, double*, cudaStream_t);

}  // namespace lgf
