// lgf_measure_static: the measurement of Delta, F and theta for callers that
// cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc/cudaFree at the point where
// it measures a configuration -- for example a host framework whose device
// memory is entirely owned by its own pool allocator (a library-side
// cudaMalloc could fail or fragment that budget), or monitoring code placed
// between the steps of a time-critical loop (cudaMalloc and cudaFree can
// synchronise the whole device).  The handle-based lgf_create path allocates
// its workspace; this entry point allocates nothing: the caller passes the
// input links and the output buffers, and the only scratch (per-CTA partial
// sums and the completion ticket of the reduction) lives in one file-scope
// device array of fixed size, shared by every call on a device.
#include <cmath>
#include <mutex>

#include "../../include/lgf.h"
#include "lgf_common.cuh"

namespace {

using namespace lgf;

constexpr int kThreads = 256;                                   // sites per CTA
constexpr int64_t kMaxBlocks = LGF_STATIC_MAX_SITES / kThreads;  // one partial pair per CTA
constexpr int kTicketDoubles = 32;                               // first 256 bytes: ticket
constexpr int kMaxDevices = 64;

// Scratch of every lgf_measure_static call on a device: [0, 256 B) holds the
// reduction ticket, then 2 doubles (F and theta partial sums) per CTA.
// In host code `g_scratch` is only a stand-in for the symbol; its device
// address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_scratch[kTicketDoubles + 2 * kMaxBlocks];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) { sa[warp] = a; sb[warp] = b; }
  __syncthreads();
  if (warp == 0) {
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
  __syncthreads();
}

// The same arithmetic as the handle path's measurement, reading the FP64
// user layout U[mu][t][z][y][x][3][3][2] directly and writing Delta_A in the
// site layout D[t][z][y][x][3][3][2].
__global__ void __launch_bounds__(kThreads)
measure_aos_kernel(Geom g, const double2* __restrict__ U, double2* __restrict__ D, double* __restrict__ out,
                   double* __restrict__ scratch) {
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch);
  double* partials = scratch + kTicketDoubles;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double fsum = 0.0, tsum = 0.0;
  if (s < g.V) {
    int c[4];
    site_coords(g, s, c);
    double im0 = 0, im1 = 0, im2 = 0;
    double2 w01 = make_double2(0, 0), w02 = make_double2(0, 0), w12 = make_double2(0, 0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const double2* u = U + ((int64_t)mu * g.V + s) * 9;
      const double2* b = U + ((int64_t)mu * g.V + site_back(g, s, c, mu)) * 9;
      double2 m[9], n[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) {
        m[e] = __ldg(&u[e]);
        n[e] = __ldg(&b[e]);
      }
      fsum += m[0].x + m[4].x + m[8].x;
      im0 -= m[0].y; im1 -= m[4].y; im2 -= m[8].y;
      w01 = csub<double>(w01, csub<double>(m[1], cconj<double>(m[3])));
      w02 = csub<double>(w02, csub<double>(m[2], cconj<double>(m[6])));
      w12 = csub<double>(w12, csub<double>(m[5], cconj<double>(m[7])));
      im0 += n[0].y; im1 += n[4].y; im2 += n[8].y;
      w01 = cadd<double>(w01, csub<double>(n[1], cconj<double>(n[3])));
      w02 = cadd<double>(w02, csub<double>(n[2], cconj<double>(n[6])));
      w12 = cadd<double>(w12, csub<double>(n[5], cconj<double>(n[7])));
    }
    const double tr = (im0 + im1 + im2) * (1.0 / 3.0);
    const double a0 = im0 - tr, a1 = im1 - tr, a2 = im2 - tr;
    const double2 d01 = cscale<double>(w01, 0.5), d02 = cscale<double>(w02, 0.5), d12 = cscale<double>(w12, 0.5);
    if (D != nullptr) {
      double2* o = D + s * 9;
      o[0] = make_double2(0.0, a0);
      o[1] = d01;
      o[2] = d02;
      o[3] = make_double2(-d01.x, d01.y);
      o[4] = make_double2(0.0, a1);
      o[5] = d12;
      o[6] = make_double2(-d02.x, d02.y);
      o[7] = make_double2(-d12.x, d12.y);
      o[8] = make_double2(0.0, a2);
    }
    tsum = a0 * a0 + a1 * a1 + a2 * a2 +
           2.0 * (d01.x * d01.x + d01.y * d01.y + d02.x * d02.x + d02.y * d02.y + d12.x * d12.x + d12.y * d12.y);
  }
  block_sum2(fsum, tsum);
  __shared__ int is_last;
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = fsum;
    partials[2 * blockIdx.x + 1] = tsum;
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  double f = 0.0, t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    f += __ldcg(&partials[2 * i]);
    t += __ldcg(&partials[2 * i + 1]);
  }
  block_sum2(f, t);
  if (threadIdx.x == 0) {
    const double Vd = (double)g.V;
    out[0] = f / (12.0 * Vd);
    out[1] = 4.0 * t / (3.0 * Vd);
    *ticket = 0u;
  }
}

bool extent_ok(int L) {
  if (L < 2 || L > 128) return false;
  while (L % 2 == 0) L /= 2;
  while (L % 3 == 0) L /= 3;
  return L == 1;
}

}  // namespace

extern "C" lgf_status lgf_measure_static(const int32_t extents[4], const double* U, double* D, double* F_theta,
                                         void* cuda_stream) {
  if (!extents || !U || !F_theta) return LGF_E_ARG;
  Geom g{};
  g.V = 1;
  for (int mu = 0; mu < 4; ++mu) {
    if (!extent_ok(extents[mu])) return LGF_E_UNSUPPORTED;
    g.L[mu] = extents[mu];
    g.stride[mu] = g.V;
    g.V *= extents[mu];
  }
  if (g.V > LGF_STATIC_MAX_SITES) return LGF_E_UNSUPPORTED;  // scratch holds one partial pair per 256 sites
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LGF_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return LGF_E_UNSUPPORTED;
  void* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the array
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return LGF_E_CUDA;
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the ticket must start at zero whatever an earlier call left behind
  if (cudaMemsetAsync(scratch, 0, kTicketDoubles * sizeof(double), s) != cudaSuccess) return LGF_E_CUDA;
  const unsigned nb = (unsigned)((g.V + kThreads - 1) / kThreads);
  measure_aos_kernel<<<nb, kThreads, 0, s>>>(g, reinterpret_cast<const double2*>(U), reinterpret_cast<double2*>(D),
                                             F_theta, static_cast<double*>(scratch));
  return cudaGetLastError() == cudaSuccess ? LGF_OK : LGF_E_CUDA;
}
