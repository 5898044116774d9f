// Device memory of one lgf handle or batch.  Every buffer comes from the
// caller's allocator when one was given (lgf_create_with_allocator), and
// otherwise from CUDA's stream-ordered allocator (cudaMallocAsync /
// cudaFreeAsync on the handle's stream).  Each buffer is remembered with its
// size so that it goes back the way it came.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "../../include/lgf.h"

namespace lgf {

struct DeviceMemory {
  lgf_allocator user{};            // user.alloc == nullptr: stream-ordered allocation
  cudaStream_t stream = nullptr;
  std::vector<std::pair<void*, size_t>> live;
  bool misaligned = false;         // the caller's allocator returned memory not 256-byte aligned

  cudaError_t get_bytes(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    if (user.alloc) {
      void* q = user.alloc(bytes, (void*)stream, user.ctx);
      if (!q) return cudaErrorMemoryAllocation;
      if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
        user.free(q, bytes, (void*)stream, user.ctx);
        misaligned = true;
        return cudaErrorInvalidValue;
      }
      *p = q;
    } else {
      cudaError_t e = cudaMallocAsync(p, bytes, stream);
      if (e != cudaSuccess) return e;
    }
    try {
      live.emplace_back(*p, bytes);
    } catch (...) {
      put(*p);
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    return cudaSuccess;
  }

  template <typename T> cudaError_t get(T** p, size_t n) {
    void* q = nullptr;
    cudaError_t e = get_bytes(&q, n * sizeof(T));
    *p = static_cast<T*>(q);
    return e;
  }

  // Return one buffer (nullptr and unknown pointers are ignored).
  void put(void* p) {
    if (!p) return;
    for (size_t i = 0; i < live.size(); ++i) {
      if (live[i].first != p) continue;
      if (user.free) user.free(p, live[i].second, (void*)stream, user.ctx);
      else cudaFreeAsync(p, stream);
      live[i] = live.back();
      live.pop_back();
      return;
    }
  }

  void put_all() {
    while (!live.empty()) put(live.back().first);
  }
};

}  // namespace lgf
