// Arithmetic-rate probe: the FP64 and FP32 fused multiply-add throughput of
// the current GPU, measured with independent FMA chains (no memory traffic).
// The integral kernels are bound by these pipes, so their roofline is stated
// against this measured rate rather than a data-sheet figure.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace dfjk {
namespace {

constexpr int PROBE_THREADS = 256;

// x <- x b + c per chain; with b < 1 every chain converges to c / (1 - b),
// so no value overflows or becomes subnormal whatever the iteration count.
template <typename Real, int PROBE_CHAINS>
__global__ void __launch_bounds__(PROBE_THREADS) fma_chain_kernel(long long iters, Real b, Real c, Real *out) {
  Real x[PROBE_CHAINS];
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) x[j] = Real(threadIdx.x + j);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) x[j] = fma(x[j], b, c);
  }
  Real s = 0;
#pragma unroll
  for (int j = 0; j < PROBE_CHAINS; ++j) s += x[j];
  out[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;
}

// One configuration: `chains` independent FMA chains per thread, `per_sm`
// blocks of 256 threads per SM; calibrated towards ~40 ms per launch.
template <typename Real, int CHAINS>
double run_config(int per_sm, cudaStream_t st) {
  int dev = 0, nsm = 0;
  DFJK_CUDA_CHECK(cudaGetDevice(&dev));
  DFJK_CUDA_CHECK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * per_sm;
  Real *out = nullptr;
  DFJK_CUDA_CHECK(cudaMalloc(&out, sizeof(Real) * (size_t)blocks * PROBE_THREADS));
  cudaEvent_t e0, e1;
  DFJK_CUDA_CHECK(cudaEventCreate(&e0));
  DFJK_CUDA_CHECK(cudaEventCreate(&e1));
  double tflops = 0.0;
  long long iters = 1024;
  for (int pass = 0; pass < 4; ++pass) {  // the last pass is the measurement
    DFJK_CUDA_CHECK(cudaEventRecord(e0, st));
    fma_chain_kernel<Real, CHAINS><<<blocks, PROBE_THREADS, 0, st>>>(iters, Real(0.999999), Real(1e-6), out);
    DFJK_LAUNCHED();
    DFJK_CUDA_CHECK(cudaEventRecord(e1, st));
    DFJK_CUDA_CHECK(cudaEventSynchronize(e1));
    float ms = 0.f;
    DFJK_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    tflops = 2.0 * CHAINS * (double)iters * blocks * PROBE_THREADS / (ms * 1e-3) / 1e12;
    if (pass < 3) iters = std::max<long long>(1024, (long long)(iters * 40.0 / std::max(ms, 0.01f)));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  return tflops;
}

// The best of a few occupancy / instruction-level-parallelism shapes.
template <typename Real>
double run_probe(cudaStream_t st) {
  double best = 0.0;
  best = std::max(best, run_config<Real, 8>(4, st));
  best = std::max(best, run_config<Real, 4>(8, st));
  best = std::max(best, run_config<Real, 16>(2, st));
  best = std::max(best, run_config<Real, 8>(1, st));
  return best;
}

}  // namespace
}  // namespace dfjk

extern "C" int dfjk_fma_rate(int32_t bits, double *tflops, void *stream) {
  try {
    if (!tflops || (bits != 32 && bits != 64)) throw dfjk::Error{DFJK_ERR_ARG, "fma_rate: bits must be 32 or 64"};
    cudaStream_t st = (cudaStream_t)stream;
    *tflops = bits == 64 ? dfjk::run_probe<double>(st) : dfjk::run_probe<float>(st);
    return DFJK_OK;
  } catch (const dfjk::Error &e) {
    dfjk::set_error(e.msg);
    return e.code;
  }
}
