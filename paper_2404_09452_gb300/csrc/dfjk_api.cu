// C ABI of the DF-J/K build: handle lifetime, setup (integrals, metric,
// Cholesky, whitening) and build (X, K, rho, J, energies) orchestration, diagnostic accessors and error plumbing.
// Paper: Introduction, contribution 1 (density fitting: 3-centre integrals,
// then tensor contractions) and Sec. "Dataset and Performance" (intermediates
// of small and medium molecules kept resident in GPU memory).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "boys.cuh"
#include "common.cuh"
#include "grad.cuh"
#include "integrals.cuh"
#include "linalg.cuh"
#include "ozaki.cuh"
#include "pool.cuh"

namespace dfjk {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }
std::atomic<uint64_t> &launch_counter() {
  static std::atomic<uint64_t> c{0};
  return c;
}

// ---- phase timing ----------------------------------------------------------------

struct PhaseRec {
  int phase;
  cudaEvent_t a, b;
};
static std::mutex g_timing_mu;
static bool g_timing = false;
static std::vector<PhaseRec> g_phase_recs;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  DFJK_CUDA_CHECK(cudaEventCreate(&e));
  return e;
}

PhaseScope::PhaseScope(int ph, cudaStream_t s) : phase(ph), st(s) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  if (!g_timing) return;
  cudaEvent_t e = take_event();
  DFJK_CUDA_CHECK(cudaEventRecord(e, st));
  ev0 = (void *)e;
}

PhaseScope::~PhaseScope() {
  if (!ev0) return;
  std::lock_guard<std::mutex> lk(g_timing_mu);
  cudaEvent_t e1;
  if (!g_event_pool.empty()) {
    e1 = g_event_pool.back();
    g_event_pool.pop_back();
  } else if (cudaEventCreate(&e1) != cudaSuccess) {
    return;
  }
  if (cudaEventRecord(e1, st) != cudaSuccess) return;
  g_phase_recs.push_back(PhaseRec{phase, (cudaEvent_t)ev0, e1});
}

// ---- device buffers -------------------------------------------------------------

template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    p = (T *)pool_alloc(count * sizeof(T));
    n = count;
  }
  void upload(const std::vector<T> &v, cudaStream_t st) {
    alloc(v.size());
    if (!v.empty()) DFJK_CUDA_CHECK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  }
  void release() {
    if (p) pool_free(p, n * sizeof(T));
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
  ~DBuf() { release(); }
};

// B: device memory from the cache, or pinned host memory mapped into the device
// address space, read and written by the kernels in place (NVLink-C2C on a
// Grace-Blackwell node) so that molecules whose B does not fit next to the
// build's work buffers still run.
struct BStore {
  double *p = nullptr;   // device-usable address
  void *hp = nullptr;    // host allocation (host-resident only)
  size_t n = 0;
  bool host = false;
  void alloc(size_t count, bool on_host) {
    release();
    if (on_host) {
      if (cudaHostAlloc(&hp, std::max<size_t>(count, 1) * sizeof(double), cudaHostAllocMapped) != cudaSuccess) {
        cudaGetLastError();
        hp = nullptr;
        throw Error{DFJK_ERR_OOM, "pinned host memory for B (" + std::to_string(count * 8) + " bytes)"};
      }
      void *d = nullptr;
      DFJK_CUDA_CHECK(cudaHostGetDevicePointer(&d, hp, 0));
      p = (double *)d;
    } else {
      p = (double *)pool_alloc(std::max<size_t>(count, 1) * sizeof(double));
    }
    host = on_host;
    n = count;
  }
  void release() {
    if (host && hp) cudaFreeHost(hp);
    if (!host && p) pool_free(p, std::max<size_t>(n, 1) * sizeof(double));
    p = nullptr;
    hp = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(double); }
  size_t device_bytes() const { return host ? 0 : bytes(); }
  ~BStore() { release(); }
};

// ---- Boys table per device ---------------------------------------------------------

const double *boys_table_device() {
  static std::mutex mu;
  static std::map<int, double *> tabs;
  int dev = 0;
  DFJK_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto it = tabs.find(dev);
  if (it != tabs.end()) return it->second;
  std::vector<double> h((size_t)BOYS_NPT * (BOYS_NCOL + 1));
  boys_table_host(h.data());
  double *d = nullptr;
  DFJK_CUDA_CHECK(cudaMalloc(&d, h.size() * sizeof(double)));
  DFJK_CUDA_CHECK(cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  tabs[dev] = d;
  return d;
}

const float *boys_table_device_f32() {
  static std::mutex mu;
  static std::map<int, float *> tabs;
  int dev = 0;
  DFJK_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto it = tabs.find(dev);
  if (it != tabs.end()) return it->second;
  std::vector<double> h((size_t)BOYS_NPT * (BOYS_NCOL + 1));
  boys_table_host(h.data());
  std::vector<float> f(h.begin(), h.end());
  float *d = nullptr;
  DFJK_CUDA_CHECK(cudaMalloc(&d, f.size() * sizeof(float)));
  DFJK_CUDA_CHECK(cudaMemcpy(d, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
  tabs[dev] = d;
  return d;
}

// ---- host-side basis ---------------------------------------------------------------

struct HostBasis {
  int nshell = 0, nfunc = 0;
  std::vector<int> l, nprim, prim_off, func_off, atom;
  std::vector<double> exps, coefs_raw, coefs, center;  // coefs: normalised radial
};

static void read_basis(const dfjk_basis *b, int natom, const double *coords, HostBasis &hb,
                       const char *what) {
  if (!b || b->nshell < 0 || (b->nshell > 0 && !b->shells))
    throw Error{DFJK_ERR_ARG, std::string(what) + ": null basis"};
  hb = HostBasis();
  hb.nshell = b->nshell;
  for (int s = 0; s < b->nshell; ++s) {
    const dfjk_shell &sh = b->shells[s];
    if (sh.l < 0 || sh.l > 2) throw Error{DFJK_ERR_UNSUPPORTED, std::string(what) + ": l must be 0..2"};
    if (sh.nprim < 1 || sh.nprim > 8)
      throw Error{DFJK_ERR_UNSUPPORTED, std::string(what) + ": nprim must be 1..8"};
    if (sh.atom < 0 || sh.atom >= natom) throw Error{DFJK_ERR_ARG, std::string(what) + ": atom index"};
    if (!sh.exps || !sh.coefs) throw Error{DFJK_ERR_ARG, std::string(what) + ": null exps/coefs"};
    hb.l.push_back(sh.l);
    hb.atom.push_back(sh.atom);
    hb.nprim.push_back(sh.nprim);
    hb.prim_off.push_back((int)hb.exps.size());
    hb.func_off.push_back(hb.nfunc);
    hb.nfunc += ncart(sh.l);
    for (int d = 0; d < 3; ++d) {
      const double x = coords[3 * sh.atom + d];
      if (!std::isfinite(x)) throw Error{DFJK_ERR_ARG, "non-finite coordinate"};
      hb.center.push_back(x);
    }
    // <chi|chi> with per-component normalised primitives:
    // sum_kl d_k d_l (2 sqrt(a_k a_l)/(a_k + a_l))^(l + 3/2)
    double ss = 0.0;
    for (int k = 0; k < sh.nprim; ++k) {
      if (!(sh.exps[k] > 0.0) || !std::isfinite(sh.exps[k]) || !std::isfinite(sh.coefs[k]))
        throw Error{DFJK_ERR_ARG, std::string(what) + ": exponents must be positive and finite"};
      for (int q = 0; q < sh.nprim; ++q) {
        const double a = sh.exps[k], c = sh.exps[q];
        ss += sh.coefs[k] * sh.coefs[q] * std::pow(2.0 * std::sqrt(a * c) / (a + c), sh.l + 1.5);
      }
    }
    if (!(ss > 0.0)) throw Error{DFJK_ERR_ARG, std::string(what) + ": contraction has zero norm"};
    const double scale = 1.0 / std::sqrt(ss);
    for (int k = 0; k < sh.nprim; ++k) {
      const double a = sh.exps[k];
      hb.exps.push_back(a);
      hb.coefs_raw.push_back(sh.coefs[k]);
      hb.coefs.push_back(sh.coefs[k] * scale * std::pow(2.0 * a / M_PI, 0.75) * std::pow(4.0 * a, 0.5 * sh.l));
    }
  }
}

// Launch-shape choices that do not change what is computed, only how fast:
// rows per block of the slicing kernels, the K GEMM's split-K range and the
// mixed build's work-buffer cap (which sets the aux-row chunk).  0 = the
// built-in default (or the corresponding environment variable).
struct Tuning {
  int slice_rows = 0;   // DFJK_SLICE_ROWS: 8, 16, 32
  int pslice_rows = 0;  // DFJK_PSLICE_ROWS: 4, 8, 16 (default 4)
  int k_range_mb = 0;   // DFJK_K_RANGE_MB
  int build_ws_mb = 0;  // DFJK_BUILD_WS_MB
};

// A tuning table: text lines "nao_lo nao_hi slice_rows pslice_rows k_range_mb
// build_ws_mb [anything]" ('#' starts a comment); the first line with
// nao_lo <= nao < nao_hi applies.  Tables are parsed once per path.
static bool lookup_tuning(const char *path, int nao, Tuning &t) {
  if (!path || !*path) return false;
  static std::mutex mu;
  static std::map<std::string, std::vector<std::vector<long>>> tables;
  std::lock_guard<std::mutex> lk(mu);
  auto it = tables.find(path);
  if (it == tables.end()) {
    std::vector<std::vector<long>> rows;
    FILE *f = std::fopen(path, "r");
    if (!f) throw Error{DFJK_ERR_ARG, std::string("tuning table not readable: ") + path};
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
      if (char *c = std::strchr(line, '#')) *c = 0;
      long v[6];
      if (std::sscanf(line, "%ld %ld %ld %ld %ld %ld", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 6)
        rows.push_back(std::vector<long>(v, v + 6));
    }
    std::fclose(f);
    it = tables.emplace(path, rows).first;
  }
  for (const auto &r : it->second)
    if (r[0] <= nao && nao < r[1]) {
      t.slice_rows = (int)r[2];
      t.pslice_rows = (int)r[3];
      t.k_range_mb = (int)r[4];
      t.build_ws_mb = (int)r[5];
      return true;
    }
  return false;
}

}  // namespace dfjk

using namespace dfjk;

struct dfjk_ctx {
  int device = 0;
  dfjk_options opt{};
  int natom = 0;
  std::vector<double> coords;
  HostBasis orb, aux;
  int nao = 0, naux = 0, naux_pad = 0;
  bool resident = false;

  // device: bases
  DBuf<double> o_center, o_exps, o_coefs, a_center, a_exps, a_cdiv, a_g1;
  DBuf<int> o_prim_off, o_nprim, o_func_off, a_prim_off, a_nprim, a_func_off;
  DBuf<int> aux_cls[3];
  std::vector<int> aux_cls_n = std::vector<int>(3, 0);
  // shell pairs (global ids in class order)
  std::vector<int> cls_begin;  // 7 entries: ss ps pp ds dp dd
  std::vector<int> pa_h, pb_h, npp_h;
  DBuf<int> pair_a, pair_b, pair_npp, pair_keep, kept;
  DBuf<long long> pair_rec_off, pair_col;
  DBuf<double> rec, q, scal;
  std::vector<int> kept_h;
  std::vector<long long> pair_col_h;
  std::vector<int> kept_cls_begin;  // 7 entries into kept list
  long long ncol = 0;
  int npair_kept = 0;
  std::vector<int> kept32_begin;  // per class: first kept index evaluated in FP32
  long long prim_pairs64[6] = {0, 0, 0, 0, 0, 0}, prim_pairs32[6] = {0, 0, 0, 0, 0, 0};
  int npair_fp32 = 0;
  double fp32_thresh = 0.0;
  int nslab = 0;  // T column slabs of the last setup (one whitening launch each)
  DBuf<int> colmu, colnu;
  // metric
  DBuf<double> V, L, Linv, Dinv;
  DBuf<int> status;
  DBuf<int> tctr;  // tile counter of the tensor-core GEMM launches (stream-ordered)
  DBuf<int> kseq;  // split counters of the ordered split-K GEMM
  // whitened tensor B, P contiguous: DFJK_FP64 keeps both triangles,
  // B[(mu nao + nu) ldb + P]; DFJK_MIXED keeps one row per kept column m (the
  // whitening's output order), B[m ldb + P], found through rowmap, and slices
  // it per build, chunk by chunk of rows P (Bchunk: batch mu, rows P of the
  // chunk, K nu), just before X = B C of that chunk
  BStore B;
  long long ldb = 0;
  bool lean = false;    // B of the kept pairs only (the mixed path)
  SlicedOp Bchunk;
  int chunk_rows = 0;   // rows P per build chunk (mixed path)
  DBuf<int> Bexpo;      // slice exponents of B's slices, [mu][expo_rows][nkb]
  int expo_rows = 0;    // rows P of Bexpo (naux_pad rounded up to 128)
  Tuning tune;          // launch-shape choices (tuning table entry or defaults)
  // build workspace
  int ws_nocc = -1;
  DBuf<double> D, rho, rho_work, X, Kpart, en_work, e;
  DBuf<int> rowmap;  // DFJK_MIXED: row of B for AO pair (mu, nu), -1 if screened
  int ksplit = 1;
  SlicedOp Csl, Xsl;  // DFJK_MIXED build operands
  DBuf<double> uks_D, uks_J;  // spin-unrestricted build: D_a + D_b and J[D_b]
  cudaStream_t side = nullptr;  // setup: Cholesky + inverse beside the integrals
  cudaStream_t side2 = nullptr;  // the Cholesky's bulk trailing updates (look-ahead)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_panel = nullptr, ev_bulk = nullptr;
  ~dfjk_ctx() {
    oz_free(Bchunk);
    oz_free(Csl);
    oz_free(Xsl);
    for (cudaStream_t s : {side, side2})
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    for (cudaEvent_t e : {ev_fork, ev_join, ev_panel, ev_bulk})
      if (e) cudaEventDestroy(e);
  }
};

// Waits for a stream on scope exit (error paths included), so that buffers the
// stream still uses are not returned to the cache under it.
struct StreamDrain {
  cudaStream_t s;
  ~StreamDrain() {
    if (s) cudaStreamSynchronize(s);
  }
};

namespace {

cudaStream_t S(void *s) { return (cudaStream_t)s; }

int fail(const Error &e) {
  set_error(e.msg);
  return e.code;
}

// Orbital shell pairs (l_a >= l_b; equal l: a >= b), grouped by class.
void enumerate_pairs(dfjk_ctx *h) {
  static const int cls[6][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}};
  h->cls_begin.assign(7, 0);
  h->pa_h.clear();
  h->pb_h.clear();
  h->npp_h.clear();
  std::vector<int> by_l[3];  // orbital shells of each l, ascending
  for (int a = 0; a < h->orb.nshell; ++a) by_l[h->orb.l[a]].push_back(a);
  for (int c = 0; c < 6; ++c) {
    h->cls_begin[c] = (int)h->pa_h.size();
    for (int a : by_l[cls[c][0]])
      for (int b : by_l[cls[c][1]]) {
        if (cls[c][0] == cls[c][1] && b > a) break;
        h->pa_h.push_back(a);
        h->pb_h.push_back(b);
        h->npp_h.push_back(h->orb.nprim[a] * h->orb.nprim[b]);
      }
  }
  h->cls_begin[6] = (int)h->pa_h.size();
}

// Device bytes of a handle's resident data: B (none when B is in host
// memory) and the metric, its Cholesky factor and inverse.  Before screening:
// the mixed path's B holds one row per kept AO pair, at most the
// nao (nao + 1) / 2 of the triangle (the bound used here); the FP64 path's
// holds both triangles of every pair.
size_t resident_estimate(const dfjk_ctx *h) {
  const size_t np2 = (size_t)h->naux_pad * h->naux_pad;
  const bool mixed = h->opt.precision == DFJK_MIXED;
  const size_t rows = mixed ? (size_t)h->nao * (h->nao + 1) / 2 : (size_t)h->nao * h->nao;
  const size_t b = h->opt.b_on_host ? 0 : rows * h->naux_pad * sizeof(double);
  return b + 3 * np2 * sizeof(double);
}

void upload_bases(dfjk_ctx *h, cudaStream_t st) {
  h->o_center.upload(h->orb.center, st);
  h->o_exps.upload(h->orb.exps, st);
  h->o_coefs.upload(h->orb.coefs, st);
  h->o_prim_off.upload(h->orb.prim_off, st);
  h->o_nprim.upload(h->orb.nprim, st);
  h->o_func_off.upload(h->orb.func_off, st);
  std::vector<double> cdiv(h->aux.exps.size()), g1(h->aux.exps.size());
  for (size_t k = 0; k < h->aux.exps.size(); ++k) {
    cdiv[k] = h->aux.coefs[k] / h->aux.exps[k];
    g1[k] = 0.5 / h->aux.exps[k];
  }
  h->a_center.upload(h->aux.center, st);
  h->a_exps.upload(h->aux.exps, st);
  h->a_cdiv.upload(cdiv, st);
  h->a_g1.upload(g1, st);
  h->a_prim_off.upload(h->aux.prim_off, st);
  h->a_nprim.upload(h->aux.nprim, st);
  h->a_func_off.upload(h->aux.func_off, st);
  for (int c = 0; c < 3; ++c) {
    std::vector<int> lst;
    for (int s = 0; s < h->aux.nshell; ++s)
      if (h->aux.l[s] == c) lst.push_back(s);
    h->aux_cls_n[c] = (int)lst.size();
    h->aux_cls[c].upload(lst, st);
  }
}

OrbArgs orb_args(dfjk_ctx *h) {
  return OrbArgs{h->o_center.p, h->o_prim_off.p, h->o_nprim.p, h->o_exps.p, h->o_coefs.p, h->o_func_off.p};
}
AuxArgs aux_args(dfjk_ctx *h) {
  return AuxArgs{h->a_center.p, h->a_prim_off.p, h->a_nprim.p, h->a_exps.p,
                 h->a_cdiv.p,   h->a_g1.p,       h->a_func_off.p};
}

__global__ void pad_identity_kernel(double *V, int n, int npad, int ld) {
  const int i = n + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < npad) V[(long long)i * ld + i] = 1.0;
}

__global__ void zero_upper_kernel(double *A, int n, int ld) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n * n) return;
  const int i = (int)(e / n), j = (int)(e % n);
  if (j > i) A[(long long)i * ld + j] = 0.0;
}

// Metric (P|Q) into V (naux_pad^2, identity on the padding).
void compute_metric(dfjk_ctx *h, const double *tab, cudaStream_t st) {
  const int np = h->naux_pad;
  h->V.alloc((size_t)np * np);
  DFJK_CUDA_CHECK(cudaMemsetAsync(h->V.p, 0, h->V.bytes(), st));
  if (np > h->naux) {
    pad_identity_kernel<<<ceil_div(np - h->naux, 64), 64, 0, st>>>(h->V.p, h->naux, np, np);
    DFJK_LAUNCHED();
  }
  static const int cls[6][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}};
  std::vector<int> by_l[3];  // aux shells of each l, ascending
  for (int p = 0; p < h->aux.nshell; ++p) by_l[h->aux.l[p]].push_back(p);
  for (int c = 0; c < 6; ++c) {
    std::vector<int> sp, sq;
    for (int p : by_l[cls[c][0]])
      for (int q : by_l[cls[c][1]]) {
        if (cls[c][0] == cls[c][1] && q > p) break;
        sp.push_back(p);
        sq.push_back(q);
      }
    if (sp.empty()) continue;
    DBuf<int> dp, dq;
    dp.upload(sp, st);
    dq.upload(sq, st);
    MetricArgs a{(int)sp.size(), dp.p, dq.p, h->V.p, np};
    launch_metric(cls[c][0], cls[c][1], a, aux_args(h), tab, st);
    DFJK_CUDA_CHECK(cudaStreamSynchronize(st));  // dp/dq go out of scope
  }
}

// The setup on the device: shell pairs and screening, metric, Cholesky and
// inverse, 3-centre integrals, whitening.
void make_resident(dfjk_ctx *h, cudaStream_t st) {
  const double *tab = boys_table_device();
  const float *tab32 = boys_table_device_f32();
  const int np = h->naux_pad;
  if (h->opt.hbm_budget_bytes > 0 && resident_estimate(h) > h->opt.hbm_budget_bytes)
    throw Error{DFJK_ERR_BUDGET, "resident data (" + std::to_string(resident_estimate(h)) +
                                     " bytes) exceeds hbm_budget_bytes"};
  PhaseScope span(12, st);
  upload_bases(h, st);
  h->status.alloc(1);
  if (!h->tctr.p) h->tctr.alloc(1);
  DFJK_CUDA_CHECK(cudaMemsetAsync(h->status.p, 0, sizeof(int), st));

  PhaseScope *ph0 = new PhaseScope(0, st);
  // a2: metric
  compute_metric(h, tab, st);

  // a3: Cholesky and inverse of the metric, on a side stream: they depend on
  // the metric alone, so they run beside the shell-pair kernels, the host's
  // pair bookkeeping and the 3-centre integrals; the first whitening waits
  // for them
  const bool mixed = h->opt.precision == DFJK_MIXED;
  if (!h->side) {
    // highest priority: the Cholesky chain is a sequence of small launches on
    // the critical path, its blocks go first whenever the integrals free an SM
    int lo = 0, hi = 0;
    DFJK_CUDA_CHECK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    DFJK_CUDA_CHECK(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, hi));
    DFJK_CUDA_CHECK(cudaStreamCreateWithPriority(&h->side2, cudaStreamNonBlocking, hi));
    DFJK_CUDA_CHECK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    DFJK_CUDA_CHECK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    DFJK_CUDA_CHECK(cudaEventCreateWithFlags(&h->ev_panel, cudaEventDisableTiming));
    DFJK_CUDA_CHECK(cudaEventCreateWithFlags(&h->ev_bulk, cudaEventDisableTiming));
  }
  const cudaStream_t s2 = h->side;
  DFJK_CUDA_CHECK(cudaEventRecord(h->ev_fork, st));
  DFJK_CUDA_CHECK(cudaStreamWaitEvent(s2, h->ev_fork, 0));
  struct OzLocal {  // slice buffers that live only during setup
    SlicedOp op;
    ~OzLocal() { oz_free(op); }
  } linv8_, t8_;
  SlicedOp &Linv8 = linv8_.op, &T8 = t8_.op;
  DBuf<double> inv_work;
  StreamDrain drain_side{s2};  // destroyed before the buffers above
  {
    PhaseScope ph1(1, s2);
    h->L.alloc((size_t)np * np);
    DFJK_CUDA_CHECK(cudaMemcpyAsync(h->L.p, h->V.p, h->V.bytes(), cudaMemcpyDeviceToDevice, s2));
    h->Dinv.alloc((size_t)(np / CHOL_NB) * CHOL_NB * CHOL_NB);
    // look-ahead on a second stream (DFJK_CHOL_AHEAD=0: one stream)
    static const bool ahead = [] {
      const char *e = std::getenv("DFJK_CHOL_AHEAD");
      return !(e && e[0] == '0');
    }();
    if (ahead) cholesky_f64(h->L.p, np, np, h->Dinv.p, h->status.p, nullptr, s2, h->side2, h->ev_panel, h->ev_bulk);
    else cholesky_f64(h->L.p, np, np, h->Dinv.p, h->status.p, nullptr, s2);
    zero_upper_kernel<<<(unsigned)(((long long)np * np + 255) / 256), 256, 0, s2>>>(h->L.p, np, np);
    DFJK_LAUNCHED();
    h->Linv.alloc((size_t)np * np);
    inv_work.alloc((size_t)np * np);
    tri_inverse_f64(h->L.p, np, np, h->Dinv.p, h->Linv.p, inv_work.p, s2);
  }
  if (mixed) {  // L^-1 as the B operand of the whitening (rows P, K Q), 8 slices
    PhaseScope ph3(3, s2);
    oz_alloc(Linv8, 1, 8, np, np, OZ_BN);
    oz_slice_f64(h->Linv.p, 0, np, 1, Linv8, s2);
  }
  DFJK_CUDA_CHECK(cudaEventRecord(h->ev_join, s2));


  // a0: shell pairs, primitive-pair records, Schwarz factors
  enumerate_pairs(h);
  const int npair = h->cls_begin[6];
  std::vector<long long> rec_off(npair);
  long long tot = 0;
  static const int cls[6][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}};
  for (int c = 0; c < 6; ++c)
    for (int i = h->cls_begin[c]; i < h->cls_begin[c + 1]; ++i) {
      rec_off[i] = tot;
      tot += (long long)h->npp_h[i] * pair_record_len(cls[c][0], cls[c][1]);
    }
  h->pair_a.upload(h->pa_h, st);
  h->pair_b.upload(h->pb_h, st);
  h->pair_npp.upload(h->npp_h, st);
  h->pair_rec_off.upload(rec_off, st);
  h->rec.alloc((size_t)std::max<long long>(tot, 1));
  h->q.alloc(std::max(npair, 1));
  for (int c = 0; c < 6; ++c) {
    const int b0 = h->cls_begin[c], n = h->cls_begin[c + 1] - b0;
    PairClassArgs a{n, h->pair_a.p + b0, h->pair_b.p + b0, h->pair_rec_off.p + b0, h->rec.p, h->q.p + b0,
                    h->pair_npp.p + b0};
    launch_pair_kernel(cls[c][0], cls[c][1], a, orb_args(h), tab, st);
    launch_schwarz(cls[c][0], cls[c][1], a, tab, tab32, h->opt.precision == DFJK_MIXED, st);
  }
  h->scal.alloc(1);
  max_sqrt_diag(h->V.p, h->naux, np, h->scal.p, st);
  h->pair_keep.alloc(std::max(npair, 1));
  screen_pairs(h->q.p, npair, h->scal.p, h->opt.schwarz_thresh, h->pair_keep.p, st);
  delete ph0;
  std::vector<int> keep(npair);
  std::vector<double> qh(npair);
  double scal = 0.0;
  if (npair) {
    DFJK_CUDA_CHECK(cudaMemcpyAsync(keep.data(), h->pair_keep.p, npair * sizeof(int), cudaMemcpyDeviceToHost, st));
    DFJK_CUDA_CHECK(cudaMemcpyAsync(qh.data(), h->q.p, npair * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  DFJK_CUDA_CHECK(cudaMemcpyAsync(&scal, h->scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
  // Schwarz-guided precision: kept pairs with bound below thr32 go to the FP32
  // kernels; within each class the FP64 pairs come first
  const double thr32 = h->opt.fp32_pair_thresh >= 0.0 ? h->opt.fp32_pair_thresh
                       : (h->opt.precision == DFJK_MIXED ? 1e-5 : 0.0);
  h->fp32_thresh = thr32;

  // kept list, columns, column -> (mu, nu) map (host bookkeeping)
  h->kept_h.clear();
  h->kept_cls_begin.assign(7, 0);
  h->pair_col_h.assign(npair, -1);
  std::vector<int> cmu, cnu;
  long long col = 0;
  h->kept32_begin.assign(6, 0);
  h->npair_fp32 = 0;
  for (int c = 0; c < 6; ++c) {
    h->kept_cls_begin[c] = (int)h->kept_h.size();
    const int na = ncart(cls[c][0]), nb = ncart(cls[c][1]);
    std::vector<int> order;
    for (int i = h->cls_begin[c]; i < h->cls_begin[c + 1]; ++i)
      if (keep[i] && !(qh[i] * scal < thr32)) order.push_back(i);
    h->kept32_begin[c] = h->kept_cls_begin[c] + (int)order.size();
    for (int i = h->cls_begin[c]; i < h->cls_begin[c + 1]; ++i)
      if (keep[i] && qh[i] * scal < thr32) order.push_back(i);
    h->npair_fp32 += h->kept_cls_begin[c] + (int)order.size() - h->kept32_begin[c];
    for (int i : order) {
      h->kept_h.push_back(i);
      h->pair_col_h[i] = col;
      const int sa = h->pa_h[i], sb = h->pb_h[i];
      for (int ca = 0; ca < na; ++ca)
        for (int cb = 0; cb < nb; ++cb) {
          const bool dup = (sa == sb) && (ca < cb);
          cmu.push_back(dup ? -1 : h->orb.func_off[sa] + ca);
          cnu.push_back(dup ? -1 : h->orb.func_off[sb] + cb);
        }
      col += na * nb;
    }
  }
  h->kept_cls_begin[6] = (int)h->kept_h.size();
  for (int c = 0; c < 6; ++c) {  // primitive pairs per class and precision
    h->prim_pairs64[c] = h->prim_pairs32[c] = 0;
    for (int i = h->kept_cls_begin[c]; i < h->kept_cls_begin[c + 1]; ++i)
      (i < h->kept32_begin[c] ? h->prim_pairs64 : h->prim_pairs32)[c] += h->npp_h[h->kept_h[i]];
  }
  h->npair_kept = (int)h->kept_h.size();
  h->ncol = col;
  h->kept.upload(h->kept_h, st);
  h->pair_col.upload(h->pair_col_h, st);
  h->colmu.upload(cmu, st);
  h->colnu.upload(cnu, st);
  if (mixed) {
    h->rowmap.alloc((size_t)h->nao * h->nao);
    build_rowmap(h->colmu.p, h->colnu.p, h->ncol, h->nao, h->rowmap.p, st);
  }

  bool joined = false;

  // a4 + a5: 3-centre integrals in column slabs, whitened into B
  // mixed: one row per kept column (the whitening writes every row); FP64:
  // both triangles of every AO pair, zero for the screened ones
  h->ldb = np;
  h->lean = mixed;
  h->B.alloc((h->lean ? (size_t)std::max<long long>(h->ncol, 1) : (size_t)h->nao * h->nao) * np,
             h->opt.b_on_host != 0);
  if (!h->lean) DFJK_CUDA_CHECK(cudaMemsetAsync(h->B.p, 0, h->B.bytes(), st));
  // bytes of one T slab: 4 GiB, or 2 GiB in the mixed path, whose slab also
  // has an 8-slice copy (twice the bytes) during the whitening
  const long long slab_budget = mixed ? (2LL << 30) : (4LL << 30);
  long long slab_cols = std::max<long long>(36, slab_budget / ((long long)np * 8));
  slab_cols = std::min<long long>(slab_cols, std::max<long long>(h->ncol, 1));
  DBuf<double> T;
  T.alloc((size_t)slab_cols * np);
  DFJK_CUDA_CHECK(cudaMemsetAsync(T.p, 0, T.bytes(), st));
  int r0 = 0;
  h->nslab = 0;
  while (r0 < h->npair_kept) {
    ++h->nslab;
    const long long c0 = h->pair_col_h[h->kept_h[r0]];
    int r1 = r0;
    while (r1 < h->npair_kept) {
      const int g = h->kept_h[r1];
      const int c = [&] { int k = 0; while (g >= h->cls_begin[k + 1]) ++k; return k; }();
      const long long cend = h->pair_col_h[g] + ncart(cls[c][0]) * ncart(cls[c][1]);
      if (cend - c0 > slab_cols) break;
      ++r1;
    }
    const long long c1 = (r1 < h->npair_kept) ? h->pair_col_h[h->kept_h[r1]] : h->ncol;
    // the FP64 pairs of every class, then the FP32 ones (phase timers 2 and 11)
    for (int prec32 = 0; prec32 < 2; ++prec32) {
      PhaseScope ph2(prec32 ? 11 : 2, st);
      for (int c = 0; c < 6; ++c) {
        const int lo = std::max(r0, h->kept_cls_begin[c]), hi = std::min(r1, h->kept_cls_begin[c + 1]);
        if (hi <= lo) continue;
        const int mid = std::min(std::max(lo, h->kept32_begin[c]), hi);  // [lo, mid) FP64, [mid, hi) FP32
        for (int lc = 0; lc < 3; ++lc) {
          Eri3cArgs a{h->kept.p + (prec32 ? mid : lo), prec32 ? hi - mid : mid - lo, h->pair_rec_off.p,
                      h->pair_npp.p, h->pair_col.p, h->rec.p, h->aux_cls[lc].p, h->aux_cls_n[lc], T.p, c0, np};
          if (prec32) launch_eri3c32(cls[c][0], cls[c][1], lc, a, aux_args(h), tab32, st);
          else launch_eri3c(cls[c][0], cls[c][1], lc, a, aux_args(h), tab, st);
        }
      }
    }
    PhaseScope ph3(3, st);
    const int ncols = (int)(c1 - c0);
    if (mixed) {  // slices of T need only T: taken before waiting for L^-1
      if (!T8.data || T8.rows_pad < ncols) oz_alloc(T8, 1, 8, (int)slab_cols, np, OZ_BM);
      T8.rows = ncols;
      oz_slice_f64(T.p, 0, np, 1, T8, st, h->tune.slice_rows);
    }
    if (!joined) {  // L^-1 (and its slices) ready
      DFJK_CUDA_CHECK(cudaStreamWaitEvent(st, h->ev_join, 0));
      joined = true;
    }
    if (!mixed) {
      GemmArgs g;  // B[(mu,nu)][P] = sum_Q T[col][Q] Linv[P][Q]
      g.M = (int)(c1 - c0); g.N = np; g.K = np;
      g.A = T.p; g.sAm = np; g.sAk = 1;
      g.B = h->Linv.p; g.sBn = np; g.sBk = 1;
      g.k_upto_n = 1;
      g.colmu = h->colmu.p + c0; g.colnu = h->colnu.p + c0;
      g.nao = h->nao; g.ldo = h->ldb; g.out = h->B.p;
      gemm_f64(g, st);
    } else {  // the same product on the tensor cores, 8 slices per operand
      OzGemmArgs g;  // B row c0 + m = whitened column c0 + m
      g.M = ncols; g.N = np; g.K = np; g.k_upto_n = 1;
      g.mode = 0; g.out = h->B.p + c0 * h->ldb; g.ldo = h->ldb;
      g.status = h->status.p; g.timeout = h->opt.timeout_iters;
      g.tile_ctr = h->tctr.p;
      g.phase = 8;
      oz_gemm(T8, Linv8, g, st);
    }
    r0 = r1;
  }
  if (!joined) DFJK_CUDA_CHECK(cudaStreamWaitEvent(st, h->ev_join, 0));
  if (mixed) {
    DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
    oz_free(T8);
    oz_free(Linv8);
    // the slice exponents of B (per mu, P and 1024-block of nu) do not change
    // between builds: computed once here, each build's slicing reads B once
    PhaseScope ph(3, st);
    h->expo_rows = (np + OZ_BM - 1) / OZ_BM * OZ_BM;
    h->Bexpo.alloc((size_t)h->nao * h->expo_rows * ((h->nao + OZ_KB - 1) / OZ_KB));
    oz_expo_packed(h->B.p, h->ldb, h->rowmap.p, h->nao, np, h->expo_rows, h->Bexpo.p, st);
  }
  int status = 0;
  DFJK_CUDA_CHECK(cudaMemcpyAsync(&status, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
  if (status & STATUS_NOT_PD)
    throw Error{DFJK_ERR_NOT_PD, "(P|Q) metric is not positive definite (non-positive Cholesky pivot)"};
  if (status & STATUS_TIMEOUT) throw Error{DFJK_ERR_TIMEOUT, "a bounded device wait expired during setup"};
  h->resident = true;
}

void release_device(dfjk_ctx *h) {
  h->B.release();
  h->Bexpo.release();
  h->rowmap.release();
  oz_free(h->Bchunk);
  h->V.release();
  h->L.release();
  h->Linv.release();
  h->Dinv.release();
  h->rec.release();
  h->q.release();
  h->colmu.release();
  h->colnu.release();
  h->D.release();
  h->rho.release();
  h->rho_work.release();
  h->X.release();
  h->Kpart.release();
  h->en_work.release();
  h->e.release();
  oz_free(h->Csl);
  oz_free(h->Xsl);
  h->chunk_rows = 0;
  h->uks_D.release();
  h->uks_J.release();
  h->ws_nocc = -1;
  h->resident = false;
}

// Rows P per chunk of the mixed build: the largest multiple of 128 whose work
// buffers (X in FP64 and its 6 slices, the 6 slices of B for the chunk) stay
// within DFJK_BUILD_WS_MB megabytes (default 8192), at least 128, at most the
// whole (padded) aux range.
int build_chunk_rows(int nao, int np, int nocc, int ws_mb = 0) {
  static const size_t cap_env = [] {
    const char *e = std::getenv("DFJK_BUILD_WS_MB");
    const long v = e ? std::atol(e) : 0;
    return (size_t)(v > 0 ? v : 8192) << 20;
  }();
  const size_t cap = ws_mb > 0 ? (size_t)ws_mb << 20 : cap_env;
  const size_t kp = ((size_t)nao + OZ_BK - 1) / OZ_BK * OZ_BK;
  const size_t per_row = (size_t)nao * ((size_t)nocc * 8 + (size_t)nocc * 12 + 12 * kp);
  size_t rows = std::max<size_t>(128, cap / per_row / 128 * 128);
  return (int)std::min<size_t>(rows, (size_t)np);
}

// Build buffers, sized on the first build at a given nocc and reused after.
void ensure_workspace(dfjk_ctx *h, int nocc, int nset) {
  const size_t nao2 = (size_t)h->nao * h->nao;
  const bool mixed = h->opt.precision == DFJK_MIXED;
  if (h->ws_nocc < nocc || !h->D.p) {
    h->D.alloc(nao2);
    h->rho.alloc(h->naux_pad);
    if (mixed) {
      const int pc = build_chunk_rows(h->nao, h->naux_pad, nocc, h->tune.build_ws_mb);
      h->chunk_rows = pc;
      h->X.alloc((size_t)h->nao * pc * nocc);
      h->rho_work.alloc((size_t)h->nao * pc);
      oz_alloc(h->Xsl, 1, 6, h->nao, pc * nocc, OZ_BM);
      oz_alloc(h->Bchunk, h->nao, 6, pc, h->nao, OZ_BM);
    } else {
      h->rho_work.alloc(std::max((size_t)128 * ceil_div(h->naux_pad, 256) * 256, (size_t)h->nao * h->naux_pad));
      h->X.alloc((size_t)h->nao * h->naux_pad * nocc);
      const int t = ceil_div(h->nao, 64);
      const int tiles = t * (t + 1) / 2;
      h->ksplit = std::max(1, std::min(64, ceil_div(4 * 152, tiles)));
      h->Kpart.alloc(nao2 * h->ksplit);
    }
    h->en_work.alloc(2 * 256);
    h->ws_nocc = nocc;
  }
  if (!h->e.p || h->e.n < (size_t)(2 * nset)) h->e.alloc(2 * nset);
}

__global__ void split_energies_kernel(const double *e, int nset, double *EJ, double *EK) {
  const int s = threadIdx.x + blockIdx.x * blockDim.x;
  if (s < nset) {
    EJ[s] = e[2 * s];
    EK[s] = e[2 * s + 1];
  }
}

// y += x over n doubles (the sum of the two spin densities and of their J).
__global__ void add_inplace_kernel(double *__restrict__ y, const double *__restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] += x[i];
}

void add_inplace(double *y, const double *x, long long n, cudaStream_t st) {
  add_inplace_kernel<<<(unsigned)std::min<long long>(ceil_div(n, 256), 152 * 8), 256, 0, st>>>(y, x, n);
  DFJK_LAUNCHED();
}

// K (lower triangle) += Xs Xs^T for one chunk of the reduction range (K
// dimension kt = rows P of the chunk x nocc), on the tensor cores.  Split-K
// ranges of about 64 MB of operand slices (all rows): the tiles in flight
// (work is handed out split-major, a few ranges at a time) then reuse their
// operands from L2.  The persistent kernel adds the splits of a tile into K in
// split order (deterministic, no partial buffers; `add` makes the first split
// add onto the previous chunks' sum as well); the one-tile-per-CTA kernel
// writes partials (capped at 4 GiB) and reduces them in the same order.
void k_gemm_sliced(dfjk_ctx *h, const SlicedOp &xs, int nao, long long kt, double *Kout, bool add,
                   cudaStream_t st) {
  const int mt = ceil_div(nao, OZ_BM), nt = ceil_div(nao, OZ_BN);
  int tiles = 0;
  for (int i = 0; i < mt; ++i)
    for (int j = 0; j < nt; ++j)
      if (j * OZ_BN <= i * OZ_BM + OZ_BM - 1) ++tiles;
  static const size_t range_env = [] {
    const char *e = std::getenv("DFJK_K_RANGE_MB");
    const long v = e ? std::atol(e) : 0;
    return (size_t)(v > 0 ? v : 64) << 20;
  }();
  const size_t range_bytes = h->tune.k_range_mb > 0 ? (size_t)h->tune.k_range_mb << 20 : range_env;
  const int nkb = xs.nkb;
  const size_t chunk_kb_bytes = (size_t)xs.rows_pad * 6 * 2 * OZ_KB;
  int per = (int)std::max<size_t>(1, range_bytes / chunk_kb_bytes);
  const bool ordered = !oz_simple_mode();
  const int max_split = ordered ? nkb : (int)std::max<size_t>(1, ((size_t)4 << 30) / ((size_t)nao * nao * 8));
  int nsplit = std::min(ceil_div(nkb, per), max_split);
  nsplit = std::max(nsplit, std::min(nkb, (2 * 152 + tiles - 1) / tiles));
  per = ceil_div(nkb, nsplit);
  nsplit = ceil_div(nkb, per);
  OzGemmArgs k;
  k.M = nao; k.N = nao; k.K = (int)kt; k.nz = nsplit; k.kb_per_split = per; k.lower_only = 1;
  k.status = h->status.p; k.timeout = h->opt.timeout_iters;
  k.tile_ctr = h->tctr.p;
  k.phase = 10;
  if (ordered) {
    const size_t nseq = oz_tile_seq_count(nao, nao);
    if (h->kseq.n < nseq) h->kseq.alloc(nseq);
    k.mode = 2; k.out = Kout; k.ldo = nao; k.tile_seq = h->kseq.p; k.accumulate = add ? 1 : 0;
    oz_gemm(xs, xs, k, st);
  } else {
    if (h->Kpart.n < (size_t)nsplit * nao * nao) h->Kpart.alloc((size_t)nsplit * nao * nao);
    k.mode = 0; k.out = h->Kpart.p; k.ldo = nao; k.out_bs = (long long)nao * nao;
    oz_gemm(xs, xs, k, st);
    reduce_sym_f64(h->Kpart.p, nsplit, nao, Kout, st, add ? 1 : 0);
  }
}

// The build for one occupied set.  DFJK_FP64 runs X = B C and K on the
// FP64 pipe; DFJK_MIXED runs both on the tensor cores as exact sliced
// products (6 slices); D, rho, J and the energies are FP64 in both.
void build_one(dfjk_ctx *h, int nocc, const double *C, double *J, double *Kout, double *e,
               cudaStream_t st) {
  const int nao = h->nao, np = h->naux_pad;
  const bool mixed = h->opt.precision == DFJK_MIXED;
  GemmArgs d;  // D = C C^T
  d.M = nao; d.N = nao; d.K = nocc;
  d.A = C; d.sAm = nocc; d.sAk = 1;
  d.B = C; d.sBn = nocc; d.sBk = 1;
  d.C = h->D.p; d.sCm = nao; d.sCn = 1;
  {
    PhaseScope ph(6, st);
    gemm_f64(d, st);
  }
  const long long kt = (long long)np * nocc;
  if (!mixed) {
    GemmArgs x;  // X[mu][P][i] = sum_nu B[(mu,nu)][P] C[nu][i]
    x.M = np; x.N = nocc; x.K = nao; x.batch = nao;
    x.A = h->B.p; x.sAm = 1; x.sAk = h->ldb; x.sAb = (long long)nao * h->ldb;
    x.B = C; x.sBn = 1; x.sBk = nocc; x.sBb = 0;
    x.C = h->X.p; x.sCm = nocc; x.sCn = 1; x.sCb = (long long)np * nocc;
    {
      PhaseScope ph(4, st);
      gemm_f64(x, st);
    }
    {  // rho from X (5x smaller than B), then J over B
      PhaseScope ph(6, st);
      rho_from_x_f64(h->X.p, C, nao, np, nocc, h->rho.p, h->rho_work.p, st);
      j_gemv_f64(h->B.p, h->ldb, nao, np, h->rho.p, J, h->lean ? h->rowmap.p : nullptr, st);
    }
    GemmArgs k;  // K[mu][nu] = sum_(P,i) X[mu][(P,i)] X[nu][(P,i)]
    k.M = nao; k.N = nao; k.K = (int)kt;
    k.A = h->X.p; k.sAm = kt; k.sAk = 1;
    k.B = h->X.p; k.sBn = kt; k.sBk = 1;
    k.C = h->Kpart.p; k.sCm = nao; k.sCn = 1; k.sCb = (long long)nao * nao;
    k.k_split = (int)((kt + h->ksplit - 1) / h->ksplit);
    k.k_split = ((k.k_split + 15) / 16) * 16;
    k.lower_only = 1;
    PhaseScope ph(5, st);
    gemm_f64(k, st);
    reduce_sym_f64(h->Kpart.p, ceil_div(kt, k.k_split), nao, Kout, st);
  } else {
    // The mixed path keeps B for the kept AO pairs (FP64) and works
    // through the aux index in chunks of rows P: per chunk, the 6 slices of
    // B[mu][nu][P in chunk] (all mu, nu), X_P = B_P C for P in the chunk,
    // rho of the chunk from X, the slices of X and its contribution to K
    // (added in chunk order).  One chunk holds the whole aux range unless the
    // build's work buffers would exceed the workspace cap.
    {
      PhaseScope ph(4, st);
      if (!h->Csl.data || h->Csl.rows != nocc) oz_alloc(h->Csl, 1, 6, nocc, nao, OZ_BN);
      oz_slice_f64(C, 0, 1, nocc, h->Csl, st, h->tune.slice_rows);  // rows i, K nu
    }
    const int pc_max = h->chunk_rows;
    const int nchunk = ceil_div(np, pc_max);
    const cudaStream_t sj = h->side ? h->side : st;
    for (int c = 0; c < nchunk; ++c) {
      const int p0 = c * pc_max, pc = std::min(pc_max, np - p0);
      const long long kt = (long long)pc * nocc;  // K of the K GEMM: (P, i) of the chunk, P-major
      double *Xc = h->X.p;                        // X[mu][p][i] of this chunk
      {
        PhaseScope ph(4, st);
        SlicedOp bv = oz_view(h->Bchunk, pc, nao);  // batch mu, rows P of the chunk, K nu
        oz_slice_f64_packed_pre(h->B.p, h->ldb, h->rowmap.p, h->Bexpo.p, h->expo_rows, p0, bv, st, h->tune.pslice_rows);
        OzGemmArgs x;
        x.M = pc; x.N = nocc; x.K = nao; x.nz = nao; x.a_batched = 1;
        x.mode = 0; x.out = Xc; x.ldo = nocc; x.out_bs = kt;
        x.status = h->status.p; x.timeout = h->opt.timeout_iters;
        x.tile_ctr = h->tctr.p;
        x.phase = 9;
        oz_gemm(bv, h->Csl, x, st);
      }
      {
        PhaseScope ph(6, st);
        rho_from_x_f64(Xc, C, nao, pc, nocc, h->rho.p + p0, h->rho_work.p, st);
      }
      if (c == nchunk - 1) {
        // J = B^T rho over the kept rows of B, on the handle's side stream beside the
        // last K GEMM: both only read finished data, and the HBM-bound GEMV
        // fits next to the tensor-bound GEMM on the SMs
        if (h->side) {
          DFJK_CUDA_CHECK(cudaEventRecord(h->ev_fork, st));
          DFJK_CUDA_CHECK(cudaStreamWaitEvent(sj, h->ev_fork, 0));
        }
        PhaseScope ph(6, sj);
        j_gemv_f64(h->B.p, h->ldb, nao, np, h->rho.p, J, h->rowmap.p, sj);
        if (h->side) DFJK_CUDA_CHECK(cudaEventRecord(h->ev_join, sj));
      }
      PhaseScope ph(5, st);
      SlicedOp xs = oz_view(h->Xsl, nao, (int)kt);  // rows mu, K (p, i)
      oz_slice_f64(Xc, 0, kt, 1, xs, st);
      k_gemm_sliced(h, xs, nao, kt, Kout, c > 0, st);
    }
    mirror_lower_f64(Kout, nao, st);
    if (h->side) DFJK_CUDA_CHECK(cudaStreamWaitEvent(st, h->ev_join, 0));  // J ready
  }
  PhaseScope ph(7, st);
  energies_f64(h->D.p, J, Kout, nao, e, h->en_work.p, st);
}

}  // namespace

extern "C" {

void dfjk_default_options(dfjk_options *opt) {
  if (!opt) return;
  opt->precision = DFJK_FP64;
  opt->schwarz_thresh = 1e-12;
  opt->hbm_budget_bytes = 0;
  opt->timeout_iters = 1LL << 26;
  opt->energies_on_host = 1;
  opt->fp32_pair_thresh = -1.0;
  opt->b_on_host = 0;
  opt->tune_table = nullptr;
}

const char *dfjk_status_string(int code) {
  switch (code) {
    case DFJK_OK: return "ok";
    case DFJK_ERR_ARG: return "invalid argument";
    case DFJK_ERR_UNSUPPORTED: return "unsupported input";
    case DFJK_ERR_NOT_PD: return "metric not positive definite";
    case DFJK_ERR_OOM: return "out of device memory";
    case DFJK_ERR_BUDGET: return "HBM budget exceeded";
    case DFJK_ERR_TIMEOUT: return "bounded device wait expired";
    case DFJK_ERR_CUDA: return "CUDA error";
    case DFJK_ERR_STATE: return "invalid handle state";
    default: return "unknown status";
  }
}

const char *dfjk_last_error(void) { return g_last_error.c_str(); }

uint64_t dfjk_launch_count(void) { return launch_counter().load(); }

int dfjk_set_timing(int32_t enable) {
  std::lock_guard<std::mutex> lk(g_timing_mu);
  g_timing = enable != 0;
  return DFJK_OK;
}

int dfjk_phase_times(double *ms, int32_t n) {
  if (!ms || n < 0) return fail(Error{DFJK_ERR_ARG, "phase_times arguments"});
  std::lock_guard<std::mutex> lk(g_timing_mu);
  for (int i = 0; i < n; ++i) ms[i] = 0.0;
  int rc = DFJK_OK;
  for (auto &r : g_phase_recs) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      if (r.phase >= 0 && r.phase < n) ms[r.phase] += t;
    } else {
      rc = DFJK_ERR_CUDA;
    }
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_phase_recs.clear();
  if (rc) set_error("event timing failed");
  return rc;
}

int dfjk_setup(const dfjk_basis *orb, const dfjk_basis *aux, int32_t natom, const double *coords,
               const dfjk_options *opt, void *stream, dfjk_handle *out) {
  if (!out) return fail(Error{DFJK_ERR_ARG, "out is null"});
  *out = nullptr;
  dfjk_ctx *h = nullptr;
  try {
    if (natom <= 0 || !coords) throw Error{DFJK_ERR_ARG, "natom/coords"};
    h = new dfjk_ctx();
    DFJK_CUDA_CHECK(cudaGetDevice(&h->device));
    if (opt) h->opt = *opt;
    else dfjk_default_options(&h->opt);
    if (h->opt.precision != DFJK_FP64 && h->opt.precision != DFJK_MIXED)
      throw Error{DFJK_ERR_UNSUPPORTED, "precision"};
    if (!(h->opt.schwarz_thresh >= 0.0)) throw Error{DFJK_ERR_ARG, "schwarz_thresh"};
    h->natom = natom;
    h->coords.assign(coords, coords + 3 * (size_t)natom);
    read_basis(orb, natom, coords, h->orb, "orbital basis");
    read_basis(aux, natom, coords, h->aux, "aux basis");
    h->nao = h->orb.nfunc;
    h->naux = h->aux.nfunc;
    if (h->nao == 0 || h->naux == 0) throw Error{DFJK_ERR_ARG, "empty basis"};
    h->naux_pad = ((h->naux + 63) / 64) * 64;
    const char *tab = h->opt.tune_table ? h->opt.tune_table : std::getenv("DFJK_TUNE_TABLE");
    lookup_tuning(tab, h->nao, h->tune);
    h->opt.tune_table = nullptr;  // the caller's string is not kept
    make_resident(h, S(stream));
    *out = h;
    return DFJK_OK;
  } catch (const Error &e) {
    delete h;
    return fail(e);
  } catch (const std::exception &e) {
    delete h;
    return fail(Error{DFJK_ERR_CUDA, e.what()});
  }
}

int dfjk_query(dfjk_handle h, int32_t *nao, int32_t *naux, int32_t *npair_kept, size_t *bytes) {
  if (!h) return fail(Error{DFJK_ERR_ARG, "null handle"});
  if (nao) *nao = h->nao;
  if (naux) *naux = h->naux;
  if (npair_kept) *npair_kept = h->npair_kept;
  if (bytes) *bytes = h->B.device_bytes() + h->Bexpo.bytes() + h->rowmap.bytes() + h->V.bytes() +
                      h->L.bytes() + h->Linv.bytes() + h->rec.bytes();
  return DFJK_OK;
}

int dfjk_query_precision(dfjk_handle h, int32_t *npair_fp32, double *fp32_thresh) {
  if (!h) return fail(Error{DFJK_ERR_ARG, "null handle"});
  if (npair_fp32) *npair_fp32 = h->npair_fp32;
  if (fp32_thresh) *fp32_thresh = h->fp32_thresh;
  return DFJK_OK;
}

int dfjk_estimate_bytes(int32_t nao, int32_t naux, int32_t nocc, int32_t precision, size_t *resident,
                        size_t *build_ws, size_t *setup_ws) {
  if (nao < 1 || naux < 1 || nocc < 1 || nocc > nao || (precision != DFJK_FP64 && precision != DFJK_MIXED))
    return fail(Error{DFJK_ERR_ARG, "estimate_bytes arguments"});
  const size_t np = ((size_t)naux + 63) / 64 * 64, n = (size_t)nao, no = (size_t)nocc;
  const bool mixed = precision == DFJK_MIXED;
  const size_t npack = n * (n + 1) / 2;
  const size_t b = (mixed ? npack : n * n) * np * 8;
  auto rup0 = [](size_t x, size_t m) { return (x + m - 1) / m * m; };
  const size_t r = b + 3 * np * np * 8 + (mixed ? n * rup0(np, OZ_BM) * ((n + OZ_KB - 1) / OZ_KB) * 4 : 0);
  auto rup = [](size_t x, size_t m) { return (x + m - 1) / m * m; };
  size_t ws = n * n * 8 + np * 8 * 2;  // D, rho
  if (mixed) {
    const size_t pc = (size_t)build_chunk_rows(nao, (int)np, nocc);
    const size_t kt = pc * no, nkb = (kt + OZ_KB - 1) / OZ_KB;
    const size_t kpx = nkb > 4 ? nkb * OZ_KB : rup(kt, OZ_BK);
    ws += n * pc * no * 8 + n * pc * 8;                       // X of a chunk, rho partials
    ws += 6 * rup(n, OZ_BM) * kpx * 2 + rup(n, OZ_BM) * nkb * 4;  // X slices
    ws += n * 6 * rup(pc, OZ_BM) * rup(n, OZ_BK) * 2 + n * rup(pc, OZ_BM) * 4;  // B slices
    ws += 6 * rup(no, OZ_BN) * rup(n, OZ_BK) * 2;            // C slices
  } else {
    const size_t t = (n + 63) / 64, ksplit = std::max<size_t>(1, std::min<size_t>(64, (4 * 152 + t * (t + 1) / 2 - 1) / (t * (t + 1) / 2)));
    ws += n * np * no * 8 + n * n * ksplit * 8 + n * np * 8;  // X, K partials, rho partials
  }
  // setup: one T slab of at most 4 GiB (2 GiB plus its 8 slices in the mixed path),
  // L^-1 and a work copy (plus L^-1's 8 slices in the mixed path)
  const size_t slab = std::min<size_t>((size_t)(mixed ? 2 : 4) << 30, npack * np * 8);
  size_t sw = slab * (mixed ? 3 : 1) + 2 * np * np * 8 + (mixed ? np * np * 16 : 0);
  if (resident) *resident = r;
  if (build_ws) *build_ws = ws;
  if (setup_ws) *setup_ws = sw;
  return DFJK_OK;
}

int dfjk_query_pair_classes(dfjk_handle h, int64_t *prim_pairs_fp64, int64_t *prim_pairs_fp32) {
  if (!h) return fail(Error{DFJK_ERR_ARG, "null handle"});
  for (int c = 0; c < 6; ++c) {
    if (prim_pairs_fp64) prim_pairs_fp64[c] = h->prim_pairs64[c];
    if (prim_pairs_fp32) prim_pairs_fp32[c] = h->prim_pairs32[c];
  }
  return DFJK_OK;
}

int dfjk_query_tuning(dfjk_handle h, int32_t *vals) {
  if (!h || !vals) return fail(Error{DFJK_ERR_ARG, "null argument"});
  vals[0] = h->tune.slice_rows;
  vals[1] = h->tune.pslice_rows;
  vals[2] = h->tune.k_range_mb;
  vals[3] = h->tune.build_ws_mb;
  return DFJK_OK;
}

int dfjk_query_setup(dfjk_handle h, int32_t *nslab, int32_t *lean) {
  if (!h) return fail(Error{DFJK_ERR_ARG, "null handle"});
  if (nslab) *nslab = h->nslab;
  if (lean) *lean = h->lean ? 1 : 0;
  return DFJK_OK;
}

int dfjk_query_build(dfjk_handle h, int32_t *chunk_rows, int32_t *nchunk) {
  if (!h) return fail(Error{DFJK_ERR_ARG, "null handle"});
  const bool mixed = h->opt.precision == DFJK_MIXED && h->chunk_rows > 0;
  if (chunk_rows) *chunk_rows = mixed ? h->chunk_rows : 0;
  if (nchunk) *nchunk = mixed ? ceil_div(h->naux_pad, h->chunk_rows) : 0;
  return DFJK_OK;
}

int dfjk_build(dfjk_handle h, int32_t nset, int32_t nocc, const double *C, double *J, double *K,
               double *EJ, double *EK, void *stream) {
  try {
    if (!h) throw Error{DFJK_ERR_ARG, "null handle"};
    if (nset < 1 || nocc < 1 || !C || !J || !K || !EJ || !EK) throw Error{DFJK_ERR_ARG, "build arguments"};
    cudaStream_t st = S(stream);
    DFJK_CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->resident) make_resident(h, st);
    ensure_workspace(h, nocc, nset);
    const size_t nao2 = (size_t)h->nao * h->nao;
    {
      PhaseScope span(13, st);
      for (int s = 0; s < nset; ++s) {
        const double *Cs = C + (size_t)s * h->nao * nocc;
        build_one(h, nocc, Cs, J + s * nao2, K + s * nao2, h->e.p + 2 * s, st);
      }
    }
    // energies go to host or device memory as the pointers are (detected per call)
    cudaPointerAttributes pa{}, pb{};
    DFJK_CUDA_CHECK(cudaPointerGetAttributes(&pa, EJ));
    DFJK_CUDA_CHECK(cudaPointerGetAttributes(&pb, EK));
    const bool dev_j = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
    const bool dev_k = pb.type == cudaMemoryTypeDevice || pb.type == cudaMemoryTypeManaged;
    if (dev_j != dev_k) throw Error{DFJK_ERR_ARG, "E_J and E_K must both be host or both device memory"};
    if (!dev_j) {
      std::vector<double> e(2 * nset);
      DFJK_CUDA_CHECK(cudaMemcpyAsync(e.data(), h->e.p, e.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
      for (int s = 0; s < nset; ++s) {
        EJ[s] = e[2 * s];
        EK[s] = e[2 * s + 1];
      }
      int status = 0;  // the stream is synchronised here: surface device status
      DFJK_CUDA_CHECK(cudaMemcpy(&status, h->status.p, sizeof(int), cudaMemcpyDeviceToHost));
      if (status & STATUS_TIMEOUT) {
        DFJK_CUDA_CHECK(cudaMemset(h->status.p, 0, sizeof(int)));
        throw Error{DFJK_ERR_TIMEOUT, "a bounded device wait expired during the build"};
      }
    } else {
      split_energies_kernel<<<ceil_div(nset, 64), 64, 0, st>>>(h->e.p, nset, EJ, EK);
      DFJK_LAUNCHED();
    }
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_build_uks(dfjk_handle h, int32_t nocc_a, const double *C_a, int32_t nocc_b, const double *C_b,
                   double *J, double *K_a, double *K_b, double *E, void *stream) {
  try {
    if (!h) throw Error{DFJK_ERR_ARG, "null handle"};
    if (nocc_a < 1 || nocc_b < 0 || nocc_b > nocc_a || !C_a || (nocc_b > 0 && !C_b) || !J || !K_a || !K_b || !E)
      throw Error{DFJK_ERR_ARG, "build_uks arguments"};
    cudaStream_t st = S(stream);
    DFJK_CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->resident) make_resident(h, st);
    ensure_workspace(h, nocc_a, 3);
    const size_t nao2 = (size_t)h->nao * h->nao;
    if (!h->uks_D.p) h->uks_D.alloc(nao2);
    if (!h->uks_J.p) h->uks_J.alloc(nao2);
    double *e = h->e.p;  // [E_J a, E_K a, E_J b, E_K b, E_J total, -]
    build_one(h, nocc_a, C_a, J, K_a, e, st);
    DFJK_CUDA_CHECK(cudaMemcpyAsync(h->uks_D.p, h->D.p, nao2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (nocc_b > 0) {
      build_one(h, nocc_b, C_b, h->uks_J.p, K_b, e + 2, st);
      add_inplace(h->uks_D.p, h->D.p, (long long)nao2, st);
      add_inplace(J, h->uks_J.p, (long long)nao2, st);
    } else {
      DFJK_CUDA_CHECK(cudaMemsetAsync(K_b, 0, nao2 * sizeof(double), st));
      DFJK_CUDA_CHECK(cudaMemsetAsync(e + 2, 0, 2 * sizeof(double), st));
    }
    {
      PhaseScope ph(7, st);
      energies_f64(h->uks_D.p, J, K_a, h->nao, e + 4, h->en_work.p, st);
    }
    // E = {E_J of the total density, E_K alpha, E_K beta}
    cudaPointerAttributes pa{};
    DFJK_CUDA_CHECK(cudaPointerGetAttributes(&pa, E));
    const bool dev = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
    if (dev) {  // E[0] = e[4], E[1] = e[1], E[2] = e[3], stream-ordered
      DFJK_CUDA_CHECK(cudaMemcpyAsync(E, e + 4, sizeof(double), cudaMemcpyDeviceToDevice, st));
      DFJK_CUDA_CHECK(cudaMemcpyAsync(E + 1, e + 1, sizeof(double), cudaMemcpyDeviceToDevice, st));
      DFJK_CUDA_CHECK(cudaMemcpyAsync(E + 2, e + 3, sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      double host[6];
      DFJK_CUDA_CHECK(cudaMemcpyAsync(host, e, sizeof(host), cudaMemcpyDeviceToHost, st));
      DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
      E[0] = host[4];
      E[1] = host[1];
      E[2] = host[3];
      int status = 0;
      DFJK_CUDA_CHECK(cudaMemcpy(&status, h->status.p, sizeof(int), cudaMemcpyDeviceToHost));
      if (status & STATUS_TIMEOUT) {
        DFJK_CUDA_CHECK(cudaMemset(h->status.p, 0, sizeof(int)));
        throw Error{DFJK_ERR_TIMEOUT, "a bounded device wait expired during the build"};
      }
    }
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_build_density(dfjk_handle h, int32_t nset, const double *D, double *J, double *K, double *EJ,
                       double *EK, void *stream) {
  try {
    if (!h) throw Error{DFJK_ERR_ARG, "null handle"};
    if (nset < 1 || !D || !J || !K || !EJ || !EK) throw Error{DFJK_ERR_ARG, "build_density arguments"};
    cudaStream_t st = S(stream);
    DFJK_CUDA_CHECK(cudaSetDevice(h->device));
    if (!h->resident) make_resident(h, st);
    const int nao = h->nao, np = h->naux_pad;
    const size_t nao2 = (size_t)nao * nao;
    ensure_workspace(h, 1, nset);
    if (!h->Kpart.p || h->ksplit < 1) {  // the FP64 split-K partials (mixed handles have none yet)
      const int t = ceil_div(nao, 64);
      h->ksplit = std::max(1, std::min(64, ceil_div(4 * 152, t * (t + 1) / 2)));
      h->Kpart.alloc(nao2 * h->ksplit);
    }
    if (!h->rho_work.p || h->rho_work.n < (size_t)128 * ceil_div(np, 256) * 256)
      h->rho_work.alloc((size_t)128 * ceil_div(np, 256) * 256);
    // the GEMMs below take B in both triangles of every pair: a B of kept
    // rows only is expanded into a temporary copy for the duration of the call
    DBuf<double> Bfull;
    const double *Bf = h->B.p;
    if (h->lean) {
      Bfull.alloc(nao2 * h->ldb);
      unpack_rows_f64(h->B.p, h->ldb, nao, h->rowmap.p, Bfull.p, st);
      Bf = Bfull.p;
    }
    DBuf<double> W;  // W[mu][sigma][P] = sum_lambda D[sigma][lambda] B[mu][lambda][P]
    W.alloc(nao2 * h->ldb);
    const long long kt = (long long)nao * h->ldb;
    for (int s = 0; s < nset; ++s) {
      const double *Ds = D + s * nao2;
      double *Js = J + s * nao2, *Ks = K + s * nao2;
      {  // J = B^T (B vec D)
        PhaseScope ph(6, st);
        rho_gemv_f64(Bf, h->ldb, nao, np, Ds, h->rho.p, h->rho_work.p, 128, st);
        j_gemv_f64(Bf, h->ldb, nao, np, h->rho.p, Js, 0, st);
      }
      {
        PhaseScope ph(4, st);
        GemmArgs w;  // batch mu: W_mu (sigma x P) = D (sigma x lambda) B_mu (lambda x P)
        w.M = nao; w.N = np; w.K = nao; w.batch = nao;
        w.A = Ds; w.sAm = nao; w.sAk = 1; w.sAb = 0;
        w.B = Bf; w.sBn = 1; w.sBk = h->ldb; w.sBb = (long long)nao * h->ldb;
        w.C = W.p; w.sCm = h->ldb; w.sCn = 1; w.sCb = (long long)nao * h->ldb;
        gemm_f64(w, st);
      }
      PhaseScope ph(5, st);
      GemmArgs k;  // K[mu][nu] = sum_(sigma,P) W[mu][(sigma,P)] B[nu][(sigma,P)]
      k.M = nao; k.N = nao; k.K = (int)kt;
      k.A = W.p; k.sAm = kt; k.sAk = 1;
      k.B = Bf; k.sBn = kt; k.sBk = 1;
      k.C = h->Kpart.p; k.sCm = nao; k.sCn = 1; k.sCb = (long long)nao2;
      k.k_split = (int)((kt + h->ksplit - 1) / h->ksplit);
      k.k_split = ((k.k_split + 15) / 16) * 16;
      k.lower_only = 1;
      gemm_f64(k, st);
      reduce_sym_f64(h->Kpart.p, ceil_div(kt, k.k_split), nao, Ks, st);
      PhaseScope pe(7, st);
      energies_f64(Ds, Js, Ks, nao, h->e.p + 2 * s, h->en_work.p, st);
    }
    cudaPointerAttributes pa{}, pb{};
    DFJK_CUDA_CHECK(cudaPointerGetAttributes(&pa, EJ));
    DFJK_CUDA_CHECK(cudaPointerGetAttributes(&pb, EK));
    const bool dev_j = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
    const bool dev_k = pb.type == cudaMemoryTypeDevice || pb.type == cudaMemoryTypeManaged;
    if (dev_j != dev_k) throw Error{DFJK_ERR_ARG, "E_J and E_K must both be host or both device memory"};
    if (dev_j) {
      split_energies_kernel<<<ceil_div(nset, 64), 64, 0, st>>>(h->e.p, nset, EJ, EK);
      DFJK_LAUNCHED();
      DFJK_CUDA_CHECK(cudaStreamSynchronize(st));  // W is released on return
    } else {
      std::vector<double> e(2 * nset);
      DFJK_CUDA_CHECK(cudaMemcpyAsync(e.data(), h->e.p, e.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
      for (int s = 0; s < nset; ++s) {
        EJ[s] = e[2 * s];
        EK[s] = e[2 * s + 1];
      }
    }
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

// d(cj E_J + ck E_K)/dR at fixed D = C C^T (or the given D when ck = 0).
// E = sum_PQ (V^-1)_PQ M_PQ / 2 for both energies, M_PQ = u_P u_Q (J) or
// Tr(D T_P D T_Q) (K), so dE/dR = sum_P Tr(Gam_P dT_P/dR) - Tr(Wt dV/dR) / 2
// with Gam_P = (V^-1 M-side)_P: d_P D for J and D (L^-T B)_P D = C Z_P C^T for
// K, Z_P = sum_Q (L^-1)_QP C^T B_Q C; Wt = d d^T for J and Z Z^T for K.
static void jk_gradient(dfjk_ctx *h, const double *Din, int nocc, const double *C, double cj, double ck,
                 double *grad, cudaStream_t st) {
  DFJK_CUDA_CHECK(cudaSetDevice(h->device));
  if (!h->resident) make_resident(h, st);
  const int nao = h->nao, np = h->naux_pad;
  const double *tab = boys_table_device();
  DBuf<double> Dl;
  const double *D = Din;
  if (!D) {  // D = C C^T
    Dl.alloc((size_t)nao * nao);
    GemmArgs dd;
    dd.M = nao; dd.N = nao; dd.K = nocc;
    dd.A = C; dd.sAm = nocc; dd.sAk = 1;
    dd.B = C; dd.sBn = nocc; dd.sBk = 1;
    dd.C = Dl.p; dd.sCm = nao; dd.sCn = 1;
    gemm_f64(dd, st);
    D = Dl.p;
  }
  // rho = B vec D (= L^-1 u), then the fitted coefficients d = L^-T rho = V^-1 u
  DBuf<double> rho, work, d;
  rho.alloc(np);
  work.alloc(std::max<size_t>((size_t)128 * ceil_div(np, 256) * 256, (size_t)16 * np));
  d.alloc(np);
  DFJK_CUDA_CHECK(cudaMemsetAsync(d.p, 0, d.bytes(), st));
  rho_gemv_f64(h->B.p, h->ldb, nao, np, D, rho.p, work.p, 128, st, h->lean ? h->rowmap.p : nullptr);
  fitted_coefficients(h->Linv.p, h->naux, np, rho.p, work.p, d.p, st);
  DBuf<double> gam, W;
  std::deque<SlicedOp> ops;  // slices of the tensor-core GEMMs, freed after the final sync
  struct OpsFree {
    std::deque<SlicedOp> &v;
    ~OpsFree() {
      for (SlicedOp &o : v) oz_free(o);
    }
  } ops_free{ops};
  // view x(z, r, k) = p[z sz + r sr + k sk] in sliced form (6 slices)
  auto slice = [&](const double *p, long long sz, long long sr, long long sk, int batch, int rows, int K,
                   int tile) -> SlicedOp & {
    ops.emplace_back();
    SlicedOp &o = ops.back();
    oz_alloc(o, batch, 6, rows, K, tile);
    oz_slice_f64(p, sz, sr, sk, o, st);
    return o;
  };
  // out[z][m][n] = sum_k A(z, m, k) B(n, k) on the tensor cores (A batched when nz > 1)
  auto tc_gemm = [&](const SlicedOp &A, const SlicedOp &Bo, int M, int N, int K, int nz, double *out,
                     long long ldo, long long obs, int lower) {
    OzGemmArgs o;
    o.M = M; o.N = N; o.K = K; o.nz = nz; o.a_batched = nz > 1 ? 1 : 0;
    o.lower_only = lower; o.mode = 0; o.out = out; o.ldo = ldo; o.out_bs = obs;
    o.status = h->status.p; o.timeout = h->opt.timeout_iters; o.tile_ctr = h->tctr.p;
    oz_gemm(A, Bo, o, st);
  };
  if (ck != 0.0) {
    // exact sliced tensor-core GEMMs when the handle is mixed (B of the kept pairs),
    // FP64 CUDA-core GEMMs otherwise (B in both triangles)
    const bool tc = h->opt.precision == DFJK_MIXED;
    const long long no2 = (long long)nocc * nocc;
    DBuf<double> X, Xt, Z;
    X.alloc((size_t)nao * np * nocc);
    Xt.alloc((size_t)np * no2);
    Z.alloc((size_t)np * no2);
    W.alloc((size_t)np * np);
    gam.alloc((size_t)np * nao * nao);
    if (tc) {
      const SlicedOp &csl = slice(C, 0, 1, nocc, 1, nocc, nao, OZ_BN);  // rows i, K nu
      const SlicedOp &cn = slice(C, 0, nocc, 1, 1, nao, nocc, OZ_BN);   // rows mu, K i
      // X[mu][P][i] = sum_nu B[(mu,nu)][P] C[nu][i], slicing B chunk
      // by chunk of rows P as the build does
      const int pcm = build_chunk_rows(nao, np, nocc, h->tune.build_ws_mb);
      ops.emplace_back();
      SlicedOp &bck = ops.back();
      oz_alloc(bck, nao, 6, pcm, nao, OZ_BM);
      for (int p0 = 0; p0 < np; p0 += pcm) {
        const int pc = std::min(pcm, np - p0);
        SlicedOp bv = oz_view(bck, pc, nao);
        oz_slice_f64_packed_pre(h->B.p, h->ldb, h->rowmap.p, h->Bexpo.p, h->expo_rows, p0, bv, st, h->tune.pslice_rows);
        tc_gemm(bv, csl, pc, nocc, nao, nao, X.p + (size_t)p0 * nocc, nocc, (long long)np * nocc, 0);
      }
      // Xt[P][j][i] = sum_mu X[mu][P][j] C[mu][i]  (symmetric in i, j)
      const SlicedOp &xs = slice(X.p, nocc, 1, (long long)np * nocc, np, nocc, nao, OZ_BM);
      tc_gemm(xs, csl, nocc, nocc, nao, np, Xt.p, nocc, no2, 0);
      // Z[P][ij] = sum_Q Linv[Q][P] Xt[Q][ij]
      const SlicedOp &lt = slice(h->Linv.p, 0, 1, np, 1, np, np, OZ_BM);
      const SlicedOp &xts = slice(Xt.p, 0, 1, no2, 1, (int)no2, np, OZ_BN);
      tc_gemm(lt, xts, np, (int)no2, np, 1, Z.p, no2, 0, 0);
      // W = Z Z^T, lower triangle, then mirrored
      const SlicedOp &zs = slice(Z.p, 0, no2, 1, 1, np, (int)no2, OZ_BM);
      tc_gemm(zs, zs, np, np, (int)no2, 1, W.p, np, 0, 1);
      mirror_lower_f64(W.p, np, st);
      // Yt[P][j][mu] = sum_i Z[P][i][j] C[mu][i]   (Yt reuses X)
      const SlicedOp &zb = slice(Z.p, no2, 1, nocc, np, nocc, nocc, OZ_BM);
      tc_gemm(zb, cn, nocc, nao, nocc, np, X.p, nao, (long long)nao * nocc, 0);
      // Gam[P][mu][nu] = sum_j Yt[P][j][mu] C[nu][j]
      const SlicedOp &ys = slice(X.p, (long long)nao * nocc, 1, nao, np, nao, nocc, OZ_BM);
      tc_gemm(ys, cn, nao, nao, nocc, np, gam.p, nao, (long long)nao * nao, 0);
    } else {
      GemmArgs x;  // X[mu][P][i] = sum_nu B[(mu,nu)][P] C[nu][i]
      x.M = np; x.N = nocc; x.K = nao; x.batch = nao;
      x.A = h->B.p; x.sAm = 1; x.sAk = h->ldb; x.sAb = (long long)nao * h->ldb;
      x.B = C; x.sBn = 1; x.sBk = nocc; x.sBb = 0;
      x.C = X.p; x.sCm = nocc; x.sCn = 1; x.sCb = (long long)np * nocc;
      gemm_f64(x, st);
      GemmArgs t;  // Xt[P][i][j] = sum_mu C[mu][i] X[mu][P][j]
      t.M = nocc; t.N = nocc; t.K = nao; t.batch = np;
      t.A = C; t.sAm = 1; t.sAk = nocc; t.sAb = 0;
      t.B = X.p; t.sBn = 1; t.sBk = (long long)np * nocc; t.sBb = nocc;
      t.C = Xt.p; t.sCm = nocc; t.sCn = 1; t.sCb = no2;
      gemm_f64(t, st);
      GemmArgs z;  // Z[P][ij] = sum_{Q >= P} Linv[Q][P] Xt[Q][ij]
      z.M = np; z.N = (int)no2; z.K = np;
      z.A = h->Linv.p; z.sAm = 1; z.sAk = np; z.k_from_m = 1;
      z.B = Xt.p; z.sBn = 1; z.sBk = no2;
      z.C = Z.p; z.sCm = no2; z.sCn = 1;
      gemm_f64(z, st);
      GemmArgs w;  // W = Z Z^T, lower triangle, then mirrored
      w.M = np; w.N = np; w.K = (int)no2;
      w.A = Z.p; w.sAm = no2; w.sAk = 1;
      w.B = Z.p; w.sBn = no2; w.sBk = 1;
      w.C = W.p; w.sCm = np; w.sCn = 1;
      w.lower_only = 1;
      gemm_f64(w, st);
      mirror_lower_f64(W.p, np, st);
      GemmArgs y;  // Y[P][mu][j] = sum_i C[mu][i] Z[P][i][j]   (Y reuses X)
      y.M = nao; y.N = nocc; y.K = nocc; y.batch = np;
      y.A = C; y.sAm = nocc; y.sAk = 1; y.sAb = 0;
      y.B = Z.p; y.sBn = 1; y.sBk = nocc; y.sBb = no2;
      y.C = X.p; y.sCm = nocc; y.sCn = 1; y.sCb = (long long)nao * nocc;
      gemm_f64(y, st);
      GemmArgs gm;  // Gam[P][mu][nu] = sum_j Y[P][mu][j] C[nu][j]
      gm.M = nao; gm.N = nao; gm.K = nocc; gm.batch = np;
      gm.A = X.p; gm.sAm = nocc; gm.sAk = 1; gm.sAb = (long long)nao * nocc;
      gm.B = C; gm.sBn = nocc; gm.sBk = 1; gm.sBb = 0;
      gm.C = gam.p; gm.sCm = nao; gm.sCn = 1; gm.sCb = (long long)nao * nao;
      gemm_f64(gm, st);
    }
    DFJK_CUDA_CHECK(cudaStreamSynchronize(st));  // X, Xt, Z are released here
  }
  DBuf<int> oat, aat, al;
  oat.upload(h->orb.atom, st);
  aat.upload(h->aux.atom, st);
  al.upload(h->aux.l, st);
  DFJK_CUDA_CHECK(cudaMemsetAsync(grad, 0, sizeof(double) * 3 * (size_t)h->natom, st));
  GradArgs g{};
  g.pair_a = h->pair_a.p;
  g.pair_b = h->pair_b.p;
  g.pair_chunk = 1;  // one pair per block: the classes with few pairs still fill the GPU
  g.d = d.p;
  g.D = D;
  g.nao = nao;
  g.cj = cj;
  g.gam = gam.p;
  g.W = W.p;
  g.ldw = np;
  g.ck = ck;
  g.orb_atom = oat.p;
  g.aux_atom = aat.p;
  g.grad = grad;
  static const int cls[6][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}};
  // Coulomb-only gradients of a mixed handle take the build's precision split:
  // the kept pairs it evaluates in FP32 (Schwarz bound below fp32_pair_thresh)
  // get FP32 derivative weights, the others FP64
  const bool split32 = ck == 0.0 && h->opt.precision == DFJK_MIXED;
  const float *tab32 = boys_table_device_f32();
  for (int c = 0; c < 6; ++c) {
    const int lo = h->kept_cls_begin[c], hi = h->kept_cls_begin[c + 1];
    if (hi <= lo) continue;
    const int mid = split32 ? std::min(std::max(lo, h->kept32_begin[c]), hi) : hi;
    for (int lc = 0; lc < 3; ++lc) {
      g.aux_shells = h->aux_cls[lc].p;
      g.naux_shells = h->aux_cls_n[lc];
      g.pairs = h->kept.p + lo;
      g.npairs = mid - lo;
      launch_grad3c(cls[c][0], cls[c][1], lc, g, orb_args(h), aux_args(h), tab, tab32, false, st);
      g.pairs = h->kept.p + mid;
      g.npairs = hi - mid;
      launch_grad3c(cls[c][0], cls[c][1], lc, g, orb_args(h), aux_args(h), tab, tab32, true, st);
    }
  }
  launch_grad2c(g, aux_args(h), al.p, h->aux.nshell, tab, st);
  DFJK_CUDA_CHECK(cudaStreamSynchronize(st));  // local buffers are released on return
  int status = 0;
  DFJK_CUDA_CHECK(cudaMemcpy(&status, h->status.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (status & STATUS_TIMEOUT) {
    DFJK_CUDA_CHECK(cudaMemset(h->status.p, 0, sizeof(int)));
    throw Error{DFJK_ERR_TIMEOUT, "a bounded device wait expired during the gradient"};
  }
}

int dfjk_coulomb_gradient(dfjk_handle h, const double *D, double *grad, void *stream) {
  try {
    if (!h || !D || !grad) throw Error{DFJK_ERR_ARG, "coulomb_gradient arguments"};
    jk_gradient(h, D, 0, nullptr, 1.0, 0.0, grad, S(stream));
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_jk_gradient(dfjk_handle h, int32_t nocc, const double *C_occ, double c_j, double c_k, double *grad,
                     void *stream) {
  try {
    if (!h || !C_occ || !grad || nocc < 1 || nocc > h->nao || !std::isfinite(c_j) || !std::isfinite(c_k))
      throw Error{DFJK_ERR_ARG, "jk_gradient arguments"};
    jk_gradient(h, nullptr, nocc, C_occ, c_j, c_k, grad, S(stream));
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_build_batch(int32_t nmol, const dfjk_handle *hs, const int32_t *nocc, const double *const *C,
                     double *const *J, double *const *K, double *EJ, double *EK, int32_t nstreams,
                     void *stream) {
  try {
    if (nmol < 0 || (nmol > 0 && (!hs || !nocc || !C || !J || !K || !EJ || !EK)))
      throw Error{DFJK_ERR_ARG, "build_batch arguments"};
    if (nmol == 0) return DFJK_OK;
    nstreams = std::max(1, std::min(nstreams, 32));
    cudaStream_t st = S(stream);
    for (int i = 0; i < nmol; ++i) {
      if (!hs[i] || nocc[i] < 1 || !C[i] || !J[i] || !K[i]) throw Error{DFJK_ERR_ARG, "build_batch entry"};
      if (!hs[i]->resident) throw Error{DFJK_ERR_STATE, "build_batch: handle evicted"};
      for (int j = 0; j < i; ++j)
        if (hs[j] == hs[i]) throw Error{DFJK_ERR_ARG, "build_batch: a handle appears twice"};
    }
    // internal streams and events, created once per device
    struct Fork {
      std::vector<cudaStream_t> streams;
      std::vector<cudaEvent_t> done;
      cudaEvent_t start;
    };
    static std::mutex mu;
    static std::map<int, Fork> forks;
    int dev = 0;
    DFJK_CUDA_CHECK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    Fork &f = forks[dev];
    if (f.streams.empty()) DFJK_CUDA_CHECK(cudaEventCreateWithFlags(&f.start, cudaEventDisableTiming));
    while ((int)f.streams.size() < nstreams) {
      cudaStream_t s2;
      cudaEvent_t e2;
      DFJK_CUDA_CHECK(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
      DFJK_CUDA_CHECK(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
      f.streams.push_back(s2);
      f.done.push_back(e2);
    }
    DFJK_CUDA_CHECK(cudaEventRecord(f.start, st));
    for (int k = 0; k < nstreams; ++k) DFJK_CUDA_CHECK(cudaStreamWaitEvent(f.streams[k], f.start, 0));
    for (int i = 0; i < nmol; ++i) {
      dfjk_ctx *h = hs[i];
      cudaStream_t s2 = f.streams[i % nstreams];
      ensure_workspace(h, nocc[i], 1);
      build_one(h, nocc[i], C[i], J[i], K[i], h->e.p, s2);
      split_energies_kernel<<<1, 64, 0, s2>>>(h->e.p, 1, EJ + i, EK + i);
      DFJK_LAUNCHED();
    }
    for (int k = 0; k < nstreams; ++k) {
      DFJK_CUDA_CHECK(cudaEventRecord(f.done[k], f.streams[k]));
      DFJK_CUDA_CHECK(cudaStreamWaitEvent(st, f.done[k], 0));
    }
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_overlap(dfjk_handle h, double *Sout, void *stream) {
  try {
    if (!h || !Sout) throw Error{DFJK_ERR_ARG, "overlap arguments"};
    cudaStream_t st = S(stream);
    if (!h->o_center.p) upload_bases(h, st);
    static const int cls[6][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}};
    for (int c = 0; c < 6; ++c) {
      std::vector<int> sa, sb;
      for (int a = 0; a < h->orb.nshell; ++a)
        for (int b = 0; b < h->orb.nshell; ++b)
          if (h->orb.l[a] == cls[c][0] && h->orb.l[b] == cls[c][1] && (cls[c][0] != cls[c][1] || b <= a)) {
            sa.push_back(a);
            sb.push_back(b);
          }
      if (sa.empty()) continue;
      DBuf<int> da, db;
      da.upload(sa, st);
      db.upload(sb, st);
      OverlapArgs a{(int)sa.size(), da.p, db.p, Sout, h->nao};
      launch_overlap(cls[c][0], cls[c][1], a, orb_args(h), st);
      DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
    }
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_overlap_matrix(const dfjk_basis *orb, int32_t natom, const double *coords, double *Sout,
                        void *stream) {
  dfjk_ctx *h = nullptr;
  try {
    if (natom <= 0 || !coords || !Sout) throw Error{DFJK_ERR_ARG, "overlap_matrix arguments"};
    h = new dfjk_ctx();
    DFJK_CUDA_CHECK(cudaGetDevice(&h->device));
    h->natom = natom;
    read_basis(orb, natom, coords, h->orb, "orbital basis");
    h->nao = h->orb.nfunc;
    const int rc = dfjk_overlap(h, Sout, stream);
    delete h;
    return rc;
  } catch (const Error &e) {
    delete h;
    return fail(e);
  }
}

int dfjk_evict(dfjk_handle h) {
  if (!h) return fail(Error{DFJK_ERR_ARG, "null handle"});
  try {
    DFJK_CUDA_CHECK(cudaSetDevice(h->device));
    DFJK_CUDA_CHECK(cudaDeviceSynchronize());
    release_device(h);
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_destroy(dfjk_handle h) {
  if (!h) return DFJK_OK;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  delete h;
  return DFJK_OK;
}

int dfjk_boys(int32_t mmax, int32_t n, const double *T, double *F, void *stream) {
  try {
    if (n < 0 || (n > 0 && (!T || !F))) throw Error{DFJK_ERR_ARG, "boys arguments"};
    launch_boys(mmax, n, T, F, boys_table_device(), S(stream));
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_get_metric(dfjk_handle h, double *Vout, void *stream) {
  try {
    if (!h || !Vout) throw Error{DFJK_ERR_ARG, "null argument"};
    if (!h->resident) throw Error{DFJK_ERR_STATE, "handle evicted"};
    DFJK_CUDA_CHECK(cudaMemcpy2DAsync(Vout, h->naux * 8, h->V.p, h->naux_pad * 8, h->naux * 8, h->naux,
                                      cudaMemcpyDeviceToDevice, S(stream)));
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_get_cholesky(dfjk_handle h, double *Lout, void *stream) {
  try {
    if (!h || !Lout) throw Error{DFJK_ERR_ARG, "null argument"};
    if (!h->resident) throw Error{DFJK_ERR_STATE, "handle evicted"};
    DFJK_CUDA_CHECK(cudaMemcpy2DAsync(Lout, h->naux * 8, h->L.p, h->naux_pad * 8, h->naux * 8, h->naux,
                                      cudaMemcpyDeviceToDevice, S(stream)));
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_get_B(dfjk_handle h, double *Bout, void *stream) {
  try {
    if (!h || !Bout) throw Error{DFJK_ERR_ARG, "null argument"};
    if (!h->resident) throw Error{DFJK_ERR_STATE, "handle evicted"};
    cudaStream_t st = S(stream);
    std::vector<int> ident(h->naux);
    for (int i = 0; i < h->naux; ++i) ident[i] = i;
    DBuf<int> perm;
    perm.upload(ident, st);
    gather_B_f64(h->B.p, h->ldb, h->nao, perm.p, h->naux, Bout, h->lean ? h->rowmap.p : nullptr, st);
    DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_get_B_columns(dfjk_handle h, int32_t ncol, const int32_t *mu, const int32_t *nu, double *out,
                       void *stream) {
  try {
    if (!h || ncol < 0 || (ncol > 0 && (!mu || !nu || !out))) throw Error{DFJK_ERR_ARG, "null argument"};
    if (!h->resident) throw Error{DFJK_ERR_STATE, "handle evicted"};
    if (ncol == 0) return DFJK_OK;
    cudaStream_t st = S(stream);
    std::vector<int> rows(ncol), ident(h->naux), map;
    if (h->lean) {  // rows of the kept pairs (-1: screened, zero)
      map.resize((size_t)h->nao * h->nao);
      DFJK_CUDA_CHECK(cudaMemcpyAsync(map.data(), h->rowmap.p, map.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
      DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
    }
    for (int c = 0; c < ncol; ++c) {
      if (mu[c] < 0 || mu[c] >= h->nao || nu[c] < 0 || nu[c] >= h->nao) throw Error{DFJK_ERR_ARG, "AO index"};
      const long long e = (long long)mu[c] * h->nao + nu[c];
      rows[c] = h->lean ? map[e] : (int)e;
    }
    for (int i = 0; i < h->naux; ++i) ident[i] = i;
    DBuf<int> r, p;
    r.upload(rows, st);
    p.upload(ident, st);
    gather2d_f64(h->B.p, h->ldb, r.p, p.p, ncol, h->naux, out, h->naux, st);
    DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

int dfjk_get_pair_mask(dfjk_handle h, int32_t *keep, void *stream) {
  try {
    if (!h || !keep) throw Error{DFJK_ERR_ARG, "null argument"};
    const int ns = h->orb.nshell;
    std::vector<int> m((size_t)ns * ns, 0);
    for (int i = 0; i < (int)h->pa_h.size(); ++i)
      if (h->pair_col_h[i] >= 0) {
        m[(size_t)h->pa_h[i] * ns + h->pb_h[i]] = 1;
        m[(size_t)h->pb_h[i] * ns + h->pa_h[i]] = 1;
      }
    DFJK_CUDA_CHECK(cudaMemcpyAsync(keep, m.data(), m.size() * sizeof(int), cudaMemcpyHostToDevice, S(stream)));
    DFJK_CUDA_CHECK(cudaStreamSynchronize(S(stream)));
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}

}  // extern "C"

namespace {
__global__ void scatter_T_kernel(const double *T, int ldT, long long ncol, int naux, const int *colmu,
                                 const int *colnu, int nao, double *out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncol * naux) return;
  const long long c = e / naux;
  const int P = (int)(e % naux);
  const int mu = colmu[c], nu = colnu[c];
  if (mu < 0) return;
  const double v = T[c * ldT + P];
  const long long n2 = (long long)nao * nao;
  out[P * n2 + (long long)mu * nao + nu] = v;
  out[P * n2 + (long long)nu * nao + mu] = v;
}
}  // namespace

extern "C" int dfjk_get_three_center(dfjk_handle h, double *Tout, void *stream) {
  try {
    if (!h || !Tout) throw Error{DFJK_ERR_ARG, "null argument"};
    if (!h->resident) throw Error{DFJK_ERR_STATE, "handle evicted"};
    cudaStream_t st = S(stream);
    const int np = h->naux_pad;
    const double *tab = boys_table_device();
    DBuf<double> T;
    T.alloc((size_t)std::max<long long>(h->ncol, 1) * np);
    DFJK_CUDA_CHECK(cudaMemsetAsync(T.p, 0, T.bytes(), st));
    DFJK_CUDA_CHECK(cudaMemsetAsync(Tout, 0, sizeof(double) * (size_t)h->naux * h->nao * h->nao, st));
    static const int cls[6][2] = {{0, 0}, {1, 0}, {1, 1}, {2, 0}, {2, 1}, {2, 2}};
    const float *tab32 = boys_table_device_f32();
    for (int c = 0; c < 6; ++c) {  // the same FP64 / FP32 split as the setup
      const int lo = h->kept_cls_begin[c], hi = h->kept_cls_begin[c + 1];
      if (hi <= lo) continue;
      const int mid = std::min(std::max(lo, h->kept32_begin[c]), hi);
      for (int lc = 0; lc < 3; ++lc) {
        Eri3cArgs a{h->kept.p + lo, mid - lo, h->pair_rec_off.p, h->pair_npp.p, h->pair_col.p, h->rec.p,
                    h->aux_cls[lc].p, h->aux_cls_n[lc], T.p, 0, np};
        launch_eri3c(cls[c][0], cls[c][1], lc, a, aux_args(h), tab, st);
        Eri3cArgs a32 = a;
        a32.pairs = h->kept.p + mid;
        a32.npairs = hi - mid;
        launch_eri3c32(cls[c][0], cls[c][1], lc, a32, aux_args(h), tab32, st);
      }
    }
    const long long n = h->ncol * h->naux;
    if (n > 0) {
      scatter_T_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(T.p, np, h->ncol, h->naux, h->colmu.p,
                                                                     h->colnu.p, h->nao, Tout);
      DFJK_LAUNCHED();
    }
    DFJK_CUDA_CHECK(cudaStreamSynchronize(st));
    return DFJK_OK;
  } catch (const Error &e) {
    return fail(e);
  }
}
