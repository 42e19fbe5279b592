// Internal helpers shared by the DF-J/K CUDA sources: status handling, launch
// accounting, Cartesian component tables.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/dfjk.h"

namespace dfjk {

// ---- status ---------------------------------------------------------------

void set_error(const std::string &msg);
std::atomic<uint64_t> &launch_counter();

struct Error {
  int code;
  std::string msg;
};

#define DFJK_CUDA_CHECK(call)                                                   \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      throw ::dfjk::Error{e_ == cudaErrorMemoryAllocation ? DFJK_ERR_OOM        \
                                                          : DFJK_ERR_CUDA,      \
                          std::string(#call) + ": " + cudaGetErrorString(e_)};  \
  } while (0)

// Call after every kernel launch: counts it and surfaces launch errors.
#define DFJK_LAUNCHED()                                                         \
  do {                                                                          \
    ::dfjk::launch_counter().fetch_add(1, std::memory_order_relaxed);           \
    DFJK_CUDA_CHECK(cudaGetLastError());                                        \
  } while (0)

// Phase timer: a CUDA event pair per phase instance on the launching stream.
struct PhaseScope {
  int phase;
  cudaStream_t st;
  void *ev0 = nullptr;
  PhaseScope(int phase, cudaStream_t st);
  ~PhaseScope();
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Device status word bits (written by kernels, read by the host).
enum : int { STATUS_NOT_PD = 1, STATUS_TIMEOUT = 2, STATUS_BOUNDS = 4 };

// ---- Cartesian components ---------------------------------------------------

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }

// Powers of component c of angular momentum l (order: descending x, then y).
__host__ __device__ constexpr int cart_x(int l, int c) {
  return l == 0 ? 0 : l == 1 ? (c == 0 ? 1 : 0) : (c == 0 ? 2 : c <= 2 ? 1 : 0);
}
__host__ __device__ constexpr int cart_y(int l, int c) {
  return l == 0 ? 0
         : l == 1 ? (c == 1 ? 1 : 0)
                  : (c == 1 ? 1 : c == 3 ? 2 : c == 4 ? 1 : 0);
}
__host__ __device__ constexpr int cart_z(int l, int c) {
  return l - cart_x(l, c) - cart_y(l, c);
}
// 1 / sqrt((2i-1)!!(2j-1)!!(2k-1)!!): only (2,0,0)-type components get 1/sqrt(3).
__host__ __device__ constexpr double comp_factor(int l, int c) {
  return (cart_x(l, c) == 2 || cart_y(l, c) == 2 || cart_z(l, c) == 2)
             ? 0.57735026918962576451
             : 1.0;
}

}  // namespace dfjk
