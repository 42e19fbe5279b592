// Energies E_J = Tr(D J)/2 and E_K = Tr(D K)/2 without any device allocation.
//
// Some callers cannot call cudaMalloc: an application whose memory pool has
// already reserved the device memory (a serving process that claims its HBM
// budget at start-up and forbids allocations outside it), or code whose latency
// path cannot absorb the device-wide synchronisation that cudaMalloc/cudaFree
// imply.  For them this entry point keeps its scratch (one pair of partial sums
// per thread block) in a file-scope device array that every GPU loading this
// library holds until the process exits.  The paper has no counterpart.
#include <map>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_BLOCK = NA_THREADS * 16;  // matrix elements reduced by one block
constexpr int NA_MAX_BLOCKS = 16384;           // n*n <= 16384 * 4096, i.e. n <= 8192
constexpr int NA_MAX_N = 8192;

// Partial sums of Tr(D J) and Tr(D K), two doubles per block (256 KB).  In host
// code this name is only a stand-in: the device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) double g_energy_scratch[2 * NA_MAX_BLOCKS];

__global__ void __launch_bounds__(NA_THREADS) na_partial_kernel(const double *__restrict__ D,
                                                                const double *__restrict__ J,
                                                                const double *__restrict__ K,
                                                                long long n2, double *scratch) {
  __shared__ double sj[NA_THREADS], sk[NA_THREADS];
  const long long b0 = (long long)blockIdx.x * NA_PER_BLOCK;
  const long long b1 = min(n2, b0 + NA_PER_BLOCK);
  double aj = 0.0, ak = 0.0;
  for (long long e = b0 + threadIdx.x; e < b1; e += NA_THREADS) {
    aj = fma(D[e], J[e], aj);
    ak = fma(D[e], K[e], ak);
  }
  sj[threadIdx.x] = aj;
  sk[threadIdx.x] = ak;
  __syncthreads();
  for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sj[threadIdx.x] += sj[threadIdx.x + s];
      sk[threadIdx.x] += sk[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // every slot the final kernel reads is written here first
    scratch[2 * blockIdx.x] = sj[0];
    scratch[2 * blockIdx.x + 1] = sk[0];
  }
}

__global__ void __launch_bounds__(NA_THREADS) na_final_kernel(const double *__restrict__ scratch,
                                                              int nblk, double *E) {
  __shared__ double sj[NA_THREADS], sk[NA_THREADS];
  double aj = 0.0, ak = 0.0;
  for (int b = threadIdx.x; b < nblk; b += NA_THREADS) {
    aj += scratch[2 * b];
    ak += scratch[2 * b + 1];
  }
  sj[threadIdx.x] = aj;
  sk[threadIdx.x] = ak;
  __syncthreads();
  for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sj[threadIdx.x] += sj[threadIdx.x + s];
      sk[threadIdx.x] += sk[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    E[0] = 0.5 * sj[0];
    E[1] = 0.5 * sk[0];
  }
}

// Device address of g_energy_scratch for the current device, looked up once per
// device (the first call on each device does this set-up).
double *scratch_for_current_device() {
  static std::mutex mu;
  static std::map<int, double *> addr;
  int dev = -1;
  DFJK_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto it = addr.find(dev);
  if (it != addr.end()) return it->second;
  double *p = nullptr;
  DFJK_CUDA_CHECK(cudaGetSymbolAddress((void **)&p, g_energy_scratch));
  if (!p) throw dfjk::Error{DFJK_ERR_CUDA, "cudaGetSymbolAddress returned a null address"};
  addr[dev] = p;
  return p;
}

}  // namespace

extern "C" int dfjk_energies_noalloc(int32_t n, const double *D, const double *J, const double *K,
                                     double *E, void *stream) {
  try {
    if (n < 1 || !D || !J || !K || !E) throw dfjk::Error{DFJK_ERR_ARG, "energies_noalloc: null pointer or n < 1"};
    if (n > NA_MAX_N)
      throw dfjk::Error{DFJK_ERR_ARG, "energies_noalloc: n = " + std::to_string(n) +
                                          " exceeds the maximum of 8192 set by the static scratch"};
    const long long n2 = (long long)n * n;
    const int nblk = (int)((n2 + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
    double *scratch = scratch_for_current_device();
    cudaStream_t st = (cudaStream_t)stream;
    na_partial_kernel<<<nblk, NA_THREADS, 0, st>>>(D, J, K, n2, scratch);
    DFJK_LAUNCHED();
    na_final_kernel<<<1, NA_THREADS, 0, st>>>(scratch, nblk, E);
    DFJK_LAUNCHED();
    return DFJK_OK;
  } catch (const dfjk::Error &e) {
    dfjk::set_error(e.msg);
    return e.code;
  }
}
