// Batched gauge fixing of many configurations of uneven lattice shapes on one
// GPU (an addition; arXiv:1206.0675 fixes one configuration at a time).
//
// Configurations are grouped by lattice shape.  Each shape class keeps its
// configurations' buffers contiguous, and every kernel of Algorithm 1's body
// runs once per class over all of its configurations (blockIdx.z); a
// configuration whose theta fell below tol retires: its controller state
// marks it done and every later kernel skips it.  The whole fix is one CUDA
// graph launch: WHILE(any configuration active) { for each class, in
// parallel branches: pass A, pass B, pass C, update, measure; then one kernel
// sets the loop condition }.  There is no inter-CTA waiting anywhere.
//
// The FFT tile shapes of every class (fields per CTA of the (x,y) passes,
// x columns per CTA of the (z,t) pass, CTA sizes) are chosen by timing every
// candidate on the class's own buffers when the batch is created; results
// are cached per process and, when LGF_AUTOTUNE_CACHE names a file, on disk.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/lgf.h"
#include "lgf_internal.h"
#include "lgf_mem.h"

using namespace lgf;

namespace {

struct ClassLane {
  Geom geom{};
  FFTPlan plan{};
  int n = 0;       // configurations of this shape
  int off = 0;     // index of its first state in the batch's state array
  double2* U = nullptr;
  double2* D = nullptr;
  double2* g = nullptr;
  double* K = nullptr;
  double2* tw = nullptr;
  short* pos = nullptr;
  double* partials = nullptr;
  double* sin2 = nullptr;
  int lmax = 0;
  double p2max = 0;
  double alpha = NAN;
  float tuned_ms = 0.f;
  Batch B;
  int64_t nb = 0;  // measurement CTAs per configuration
};

}  // namespace

struct lgf_batch_ctx {
  DeviceMemory mem;  // every device buffer of the batch (stream-ordered on `stream`)
  int n = 0;
  std::vector<int> cls_of, slot_of;
  std::vector<ClassLane> cls;
  DevState* st = nullptr;
  DevState* st_host = nullptr;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> ev;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double* stage = nullptr;
  unsigned long long* defect = nullptr;
  unsigned long long* defect_host = nullptr;
  int device = 0;
  bool broken = false;
  std::string err;
};

namespace {

lgf_status bfail(lgf_batch_ctx* b, lgf_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

lgf_status bfail_cuda(lgf_batch_ctx* b, cudaError_t e, const char* what) {
  if (b) {
    b->broken = true;
    b->err = std::string(what) + ": " + cudaGetErrorString(e);
  }
  return e == cudaErrorMemoryAllocation ? LGF_E_NOMEM : LGF_E_CUDA;
}

#define LGF_BCK(b, call)                                    \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return bfail_cuda(b, e_, #call); \
  } while (0)

bool extent_ok(int L) {
  if (L < 2 || L > 128) return false;
  while (L % 2 == 0) L /= 2;
  while (L % 3 == 0) L /= 3;
  return L == 1;
}


// ---- autotune cache key ----------------------------------------------------

std::string tune_key(const Geom& g, int n, const char* dev) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%d,%d,%d,%d,fp64,n=%d,%s", g.L[0], g.L[1], g.L[2], g.L[3], n, dev);
  std::string k = buf;
  for (char& c : k)
    if (c == ' ') c = '_';
  return k;
}

// Device time of passes A, B and C of a class under a plan (best of 3).
cudaError_t time_plan(ClassLane& C, const FFTPlan& p, cudaStream_t s, float* ms_out) {
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) return e;
  Batch B = C.B;
  B.st = nullptr;  // time every configuration
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_fft_xy<double>(C.geom, p, C.D, C.tw, C.pos, -1, 4, s, B);
    if (e == cudaSuccess) e = launch_fft_zt<double>(C.geom, p, C.D, C.tw, C.pos, C.K, 0, 4, s, LearnedIO(), B);
    if (e == cudaSuccess)
      e = launch_fft_xy_inv_gauge<double, double, 3>(C.geom, p, C.D, C.tw, C.pos, C.g, nullptr, s, B);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);  // the first run warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = best;
  return e;
}

lgf_status autotune(lgf_batch_ctx* b, ClassLane& C) {
  std::vector<FFTPlan> cand;
  fft_plan_candidates(C.geom.L, 8, cand);
  if (cand.empty()) return bfail(b, LGF_E_UNSUPPORTED, "lattice planes do not fit the shared-memory FFT passes");
  cudaDeviceProp prop;
  LGF_BCK(b, cudaGetDeviceProperties(&prop, b->device));
  const std::string key = tune_key(C.geom, C.n, prop.name);
  TuneChoice tc;
  if (tune_cache_get(key, &tc))
    for (const FFTPlan& p : cand)
      if (tc.decomp == FFT_2D2D && p.fpb_xy == tc.fpb_xy && p.xc == tc.xc && p.threads_xy == tc.threads_xy &&
          p.threads_zt == tc.threads_zt && p.threads_c == tc.threads_c) {
        C.plan = p;
        return LGF_OK;
      }
  LGF_BCK(b, cudaMemsetAsync(C.D, 0, sizeof(double2) * 4 * C.geom.V * C.n, b->stream));
  float best = 1e30f;
  for (const FFTPlan& p : cand) {
    float ms;
    LGF_BCK(b, time_plan(C, p, b->stream, &ms));
    if (ms < best) {
      best = ms;
      C.plan = p;
    }
  }
  C.tuned_ms = best;
  tune_cache_put(key, tune_choice_of(C.plan, FFT_2D2D));
  return LGF_OK;
}

// ---- per-class set-up ------------------------------------------------------

lgf_status setup_class(lgf_batch_ctx* b, ClassLane& C) {
  const Geom& g = C.geom;
  const int64_t V = g.V;
  C.nb = measure_blocks(V);
  LGF_BCK(b, b->mem.get(&C.U, (size_t)C.n * 36 * V));
  LGF_BCK(b, b->mem.get(&C.D, (size_t)C.n * 4 * V));
  LGF_BCK(b, b->mem.get(&C.g, (size_t)C.n * 9 * V));
  LGF_BCK(b, b->mem.get(&C.K, (size_t)V));
  LGF_BCK(b, b->mem.get(&C.partials, (size_t)C.n * MEASURE_PARTIALS * C.nb));
  const int nt = g.L[0] + g.L[1] + g.L[2] + g.L[3];
  LGF_BCK(b, b->mem.get(&C.tw, (size_t)nt));
  LGF_BCK(b, b->mem.get(&C.pos, (size_t)nt));
  if (configure_fft_plan(g.L, 8, &C.plan) != cudaSuccess)
    return bfail(b, LGF_E_UNSUPPORTED, "lattice planes do not fit the shared-memory FFT passes");
  std::vector<double2> tw(nt);
  std::vector<short> pos(nt);
  int off = 0;
  for (int mu = 0; mu < 4; ++mu) {
    for (int m = 0; m < g.L[mu]; ++m) {
      const double a = -2.0 * M_PI * (double)m / (double)g.L[mu];
      tw[off + m] = make_double2(std::cos(a), std::sin(a));
    }
    off += g.L[mu];
  }
  fft_positions(C.plan, pos.data());
  LGF_BCK(b, cudaMemcpyAsync(C.tw, tw.data(), nt * sizeof(double2), cudaMemcpyHostToDevice, b->stream));
  LGF_BCK(b, cudaMemcpyAsync(C.pos, pos.data(), nt * sizeof(short), cudaMemcpyHostToDevice, b->stream));
  C.lmax = 0;
  for (int mu = 0; mu < 4; ++mu) C.lmax = std::max(C.lmax, g.L[mu]);
  std::vector<double> sin2((size_t)4 * C.lmax, 0.0);
  C.p2max = 0;
  for (int mu = 0; mu < 4; ++mu) {
    for (int k = 0; k < g.L[mu]; ++k) {
      const double sv = std::sin(M_PI * (double)k / (double)g.L[mu]);
      sin2[(size_t)mu * C.lmax + k] = 4.0 * sv * sv;
    }
    const double sm = std::sin(M_PI * (double)(g.L[mu] / 2) / (double)g.L[mu]);
    C.p2max += 4.0 * sm * sm;
  }
  LGF_BCK(b, b->mem.get(&C.sin2, sin2.size()));
  LGF_BCK(b, cudaMemcpyAsync(C.sin2, sin2.data(), sin2.size() * 8, cudaMemcpyHostToDevice, b->stream));
  C.B.n = C.n;
  C.B.s_links = 36 * V;
  C.B.s_delta = 4 * V;
  C.B.s_g = 9 * V;
  C.B.s_G = 0;
  C.B.s_part = MEASURE_PARTIALS * C.nb;
  C.B.st = b->st + C.off;
  LGF_BCK(b, launch_filter_table<double>(g, C.sin2, C.lmax, 0.08, C.p2max, 0, C.K, b->stream));
  C.alpha = 0.08;
  return autotune(b, C);
}



cudaError_t enqueue_class_body(ClassLane& C, cudaStream_t s) {
  cudaError_t e;
  if ((e = launch_fft_xy<double>(C.geom, C.plan, C.D, C.tw, C.pos, -1, 4, s, C.B)) != cudaSuccess) return e;
  if ((e = launch_fft_zt<double>(C.geom, C.plan, C.D, C.tw, C.pos, C.K, 0, 4, s, LearnedIO(), C.B)) != cudaSuccess)
    return e;
  if ((e = launch_fft_xy_inv_gauge<double, double, 3>(C.geom, C.plan, C.D, C.tw, C.pos, C.g, nullptr, s, C.B)) !=
      cudaSuccess)
    return e;
  if ((e = launch_update<double, 3, 3>(C.geom, C.U, C.g, s, C.B)) != cudaSuccess) return e;
  return launch_measure<double, 3>(C.geom, C.U, C.D, C.partials, nullptr, 1, 0, 0, s, 0, C.B);
}

lgf_status ensure_batch_graph(lgf_batch_ctx* b) {
  if (b->exec) return LGF_OK;
  cudaGraph_t graph;
  LGF_BCK(b, cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle cond;
  LGF_BCK(b, cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  LGF_BCK(b, cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  LGF_BCK(b, cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  cudaError_t e = cudaEventRecord(b->ev[0], b->cap);
  // one branch per shape class, joined before the loop condition
  for (size_t c = 0; c < b->cls.size() && e == cudaSuccess; ++c) {
    cudaStream_t s = b->branch[c];
    e = cudaStreamWaitEvent(s, b->ev[0], 0);
    if (e == cudaSuccess) e = enqueue_class_body(b->cls[c], s);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev[1 + c], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->ev[1 + c], 0);
  }
  if (e == cudaSuccess) e = launch_batch_condition(b->st, b->n, (unsigned long long)cond, b->cap);
  cudaGraph_t captured = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->cap, &captured);
  if (e != cudaSuccess) return bfail_cuda(b, e, "capture of the batch body");
  if (e2 != cudaSuccess) return bfail_cuda(b, e2, "cudaStreamEndCapture");
  LGF_BCK(b, cudaGraphInstantiate(&b->exec, graph, 0));
  b->graph = graph;
  return LGF_OK;
}

__global__ void batch_state_kernel(DevState* st, int n, double tol, int max_iter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  DevState& s = st[i];
  s.tol = tol;
  s.max_iter = max_iter;
  s.iter = 0;
  s.status = ST_OK;
  s.hist_cap = 0;
  s.revert = 0;
  s.use_m = 0;
  s.done = !(isfinite(s.F) && isfinite(s.theta) && s.theta >= tol && max_iter > 0);
}

lgf_status check_batch(lgf_batch_ctx* b) {
  if (!b) return LGF_E_ARG;
  if (b->broken) return LGF_E_CUDA;
  if (cudaSetDevice(b->device) != cudaSuccess) return bfail_cuda(b, cudaErrorInvalidDevice, "cudaSetDevice");
  return LGF_OK;
}

}  // namespace

extern "C" {

lgf_status lgf_batch_destroy(lgf_batch b) {
  if (!b) return LGF_OK;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->mem.put_all();
  for (cudaStream_t s : b->branch) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  cudaStreamSynchronize(b->stream);
  if (b->st_host) cudaFreeHost(b->st_host);
  if (b->defect_host) cudaFreeHost(b->defect_host);
  delete b;
  return LGF_OK;
}

lgf_status lgf_batch_create(int32_t n, const int32_t* extents, lgf_precision prec, uint32_t flags, void* cuda_stream,
                            lgf_batch* out) {
  if (!out || !extents || n <= 0) return LGF_E_ARG;
  *out = nullptr;
  if (prec != LGF_FP64 || flags != 0) return LGF_E_UNSUPPORTED;
  for (int i = 0; i < 4 * n; ++i)
    if (!extent_ok(extents[i])) return LGF_E_UNSUPPORTED;
  lgf_batch_ctx* b = new (std::nothrow) lgf_batch_ctx();
  if (!b) return LGF_E_NOMEM;
  try {
    b->n = n;
    b->stream = (cudaStream_t)cuda_stream;
    b->mem.stream = b->stream;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
      delete b;
      return LGF_E_CUDA;
    }
    // group by shape, in order of first appearance
    b->cls_of.resize(n);
    b->slot_of.resize(n);
    for (int i = 0; i < n; ++i) {
      const int32_t* L = extents + 4 * i;
      int c = 0;
      for (; c < (int)b->cls.size(); ++c) {
        const int* M = b->cls[c].geom.L;
        if (M[0] == L[0] && M[1] == L[1] && M[2] == L[2] && M[3] == L[3]) break;
      }
      if (c == (int)b->cls.size()) {
        ClassLane C;
        C.geom.V = 1;
        for (int mu = 0; mu < 4; ++mu) {
          C.geom.L[mu] = L[mu];
          C.geom.stride[mu] = C.geom.V;
          C.geom.V *= L[mu];
        }
        b->cls.push_back(C);
      }
      b->cls_of[i] = c;
      b->slot_of[i] = b->cls[c].n++;
    }
    int off = 0;
    int64_t vmax = 0;
    for (ClassLane& C : b->cls) {
      C.off = off;
      off += C.n;
      vmax = std::max(vmax, C.geom.V);
    }
    lgf_status s = LGF_OK;
    cudaError_t e = b->mem.get(&b->st, (size_t)n);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->st, 0, sizeof(DevState) * n, b->stream);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->st_host, sizeof(DevState) * n);
    if (e == cudaSuccess) e = b->mem.get(&b->stage, (size_t)72 * vmax);
    if (e == cudaSuccess) e = b->mem.get(&b->defect, 1);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->defect_host, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (size_t c = 0; c < b->cls.size() && e == cudaSuccess; ++c) {
      cudaStream_t st;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->branch.push_back(st);
    }
    for (size_t c = 0; c <= b->cls.size() && e == cudaSuccess; ++c) {
      cudaEvent_t ev;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) b->ev.push_back(ev);
    }
    if (e != cudaSuccess) s = bfail_cuda(b, e, "lgf_batch_create allocation");
    for (size_t c = 0; c < b->cls.size() && s == LGF_OK; ++c) s = setup_class(b, b->cls[c]);
    if (s == LGF_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) s = LGF_E_CUDA;
    if (s != LGF_OK) {
      lgf_batch_destroy(b);
      return s;
    }
    *out = b;
    return LGF_OK;
  } catch (...) {
    lgf_batch_destroy(b);
    return LGF_E_NOMEM;
  }
}

lgf_status lgf_batch_set_links(lgf_batch b, int32_t i, const double* U, int where) {
  lgf_status s = check_batch(b);
  if (s != LGF_OK) return s;
  if (i < 0 || i >= b->n || !U || (where != LGF_HOST && where != LGF_DEVICE))
    return bfail(b, LGF_E_ARG, "bad index, pointer or location");
  ClassLane& C = b->cls[b->cls_of[i]];
  const int j = b->slot_of[i];
  const Geom& g = C.geom;
  const size_t nd = (size_t)72 * g.V;
  const double* src = U;
  if (where == LGF_HOST) {
    LGF_BCK(b, cudaMemcpyAsync(b->stage, U, nd * 8, cudaMemcpyHostToDevice, b->stream));
    src = b->stage;
  }
  LGF_BCK(b, launch_su3_defect(src, 4 * g.V, b->defect, b->stream));
  LGF_BCK(b, cudaMemcpyAsync(b->defect_host, b->defect, 8, cudaMemcpyDeviceToHost, b->stream));
  LGF_BCK(b, cudaStreamSynchronize(b->stream));
  double defect;
  std::memcpy(&defect, b->defect_host, 8);
  if (!std::isfinite(defect)) return bfail(b, LGF_E_NONFINITE, "input links contain non-finite values");
  if (defect > 1e-10) return bfail(b, LGF_E_ARG, "input links are not in SU(3)");
  LGF_BCK(b, (launch_links_from_aos<double, 3>(g, src, C.U + j * C.B.s_links, b->stream)));
  DevState* st = b->st + C.off + j;
  LGF_BCK(b, launch_set_state(st, 0.0, 0, 1, 0, nullptr, nullptr, b->stream));
  LGF_BCK(b, (launch_measure<double, 3>(g, C.U + j * C.B.s_links, C.D + j * C.B.s_delta, C.partials + j * C.B.s_part,
                                        st, 0, 0, 0, b->stream)));
  LGF_BCK(b, cudaStreamSynchronize(b->stream));
  return LGF_OK;
}

lgf_status lgf_batch_get_links(lgf_batch b, int32_t i, double* U, int where) {
  lgf_status s = check_batch(b);
  if (s != LGF_OK) return s;
  if (i < 0 || i >= b->n || !U || (where != LGF_HOST && where != LGF_DEVICE))
    return bfail(b, LGF_E_ARG, "bad index, pointer or location");
  ClassLane& C = b->cls[b->cls_of[i]];
  const int j = b->slot_of[i];
  double* dst = where == LGF_DEVICE ? U : b->stage;
  LGF_BCK(b, (launch_links_to_aos<double, 3>(C.geom, C.U + j * C.B.s_links, dst, b->stream)));
  if (where == LGF_HOST)
    LGF_BCK(b, cudaMemcpyAsync(U, dst, sizeof(double) * 72 * C.geom.V, cudaMemcpyDeviceToHost, b->stream));
  LGF_BCK(b, cudaStreamSynchronize(b->stream));
  return LGF_OK;
}

lgf_status lgf_batch_fix(lgf_batch b, double theta_tol, int32_t max_iter, double alpha, int32_t* iters, double* F,
                         double* theta) {
  lgf_status s = check_batch(b);
  if (s != LGF_OK) return s;
  if (!(theta_tol >= 0.0) || max_iter < 0 || !std::isfinite(alpha)) return bfail(b, LGF_E_ARG, "bad fix arguments");
  for (ClassLane& C : b->cls)
    if (C.alpha != alpha) {
      LGF_BCK(b, launch_filter_table<double>(C.geom, C.sin2, C.lmax, alpha, C.p2max, 0, C.K, b->stream));
      C.alpha = alpha;
    }
  batch_state_kernel<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->st, b->n, theta_tol, max_iter);
  LGF_BCK(b, cudaGetLastError());
  LGF_BCK(b, cudaMemcpyAsync(b->st_host, b->st, sizeof(DevState) * b->n, cudaMemcpyDeviceToHost, b->stream));
  LGF_BCK(b, cudaStreamSynchronize(b->stream));
  bool any = false;
  for (int i = 0; i < b->n; ++i) any = any || !b->st_host[i].done;
  if (any) {
    if ((s = ensure_batch_graph(b)) != LGF_OK) return s;
    LGF_BCK(b, cudaGraphLaunch(b->exec, b->stream));
    LGF_BCK(b, cudaMemcpyAsync(b->st_host, b->st, sizeof(DevState) * b->n, cudaMemcpyDeviceToHost, b->stream));
    LGF_BCK(b, cudaStreamSynchronize(b->stream));
  }
  bool all_conv = true, finite = true;
  for (int i = 0; i < b->n; ++i) {
    const DevState& S = b->st_host[b->cls[b->cls_of[i]].off + b->slot_of[i]];
    if (iters) iters[i] = S.iter;
    if (F) F[i] = S.F;
    if (theta) theta[i] = S.theta;
    finite = finite && std::isfinite(S.F) && std::isfinite(S.theta);
    all_conv = all_conv && S.theta < theta_tol;
  }
  if (!finite) return bfail(b, LGF_E_NONFINITE, "F or theta became non-finite");
  if (!all_conv) return bfail(b, LGF_E_NOTCONV, "some configurations reached max_iter");
  return LGF_OK;
}

lgf_status lgf_batch_describe(lgf_batch b, char* buf, size_t len) {
  if (!b || !buf || len == 0) return LGF_E_ARG;
  std::string s = "[";
  for (size_t c = 0; c < b->cls.size(); ++c) {
    const ClassLane& C = b->cls[c];
    char item[320];
    std::snprintf(item, sizeof(item),
                  "%s{\"extents\":[%d,%d,%d,%d],\"n\":%d,\"fields_per_cta_xy\":%d,\"x_columns_zt\":%d,"
                  "\"threads\":[%d,%d,%d],\"tuned_ms\":%.4f}",
                  c ? "," : "", C.geom.L[0], C.geom.L[1], C.geom.L[2], C.geom.L[3], C.n, C.plan.fpb_xy, C.plan.xc,
                  C.plan.threads_xy, C.plan.threads_zt, C.plan.threads_c, C.tuned_ms);
    s += item;
  }
  s += "]";
  std::snprintf(buf, len, "%s", s.c_str());
  return s.size() < len ? LGF_OK : LGF_E_ARG;
}

const char* lgf_batch_last_error(lgf_batch b) {
  if (!b) return "null handle";
  return b->err.c_str();
}

}  // extern "C"
