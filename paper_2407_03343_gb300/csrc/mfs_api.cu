// C ABI of libmfs: context, build (discretisation + one-body factorisation), GMRES drivers.
//
// Solve (Sec. 2.2): GMRES on G_hat mu = W b (eq. resistance) with the three-step apply
//   step 1  lambda_hat_k = V_k (Sigma_k^+ (U_k^T mu_k))      batched GEMV, eq. transform
//   step 2+3  out = mu + W sum_{k' != k} G^(kk') lambda_hat   pairs kernel, eq. uAll
// then lambda = B^+ mu and forces/torques (Sec. 2.3 remark).
// MFS_FP64 runs GMRES in FP64 with the native FP64 pair kernel.  MFS_MIXED runs the same
// FP64 GMRES but evaluates the pair sums (about 90% of the work) in double-float arithmetic
// on the FP32 pipes, because FP64 throughput on this GPU is 1/74 of FP32, while plain FP32
// pair sums cannot carry the cancellation in G B^+ mu (B^+ truncated at 5e-12 amplifies by
// up to ~1e11).  MFS_FP32 runs FP32 inner GMRES on an all-FP32 operator with FP64 iterative
// refinement; it converges only when the one-body blocks are moderately conditioned.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <string>
#include <vector>

#include <cublas_v2.h>
#include <cusolverDn.h>

#include "mfs_internal.h"

using namespace mfs;

namespace {

constexpr int kTileTargets = 512;  // 128 threads x 4 nodes, must match the pairs kernel
constexpr double kPi = 3.14159265358979323846;

inline int pad4(int x) { return (x + 3) & ~3; }

// FP32-pipe flops of the compensated double-float pair evaluation (counted from the kernel's
// operations, FMA = 2): a Stokeslet pair's geometry (differences, distance, 1/r, 1/r^2) and its
// per-right-hand-side part; an image triple's geometry (with 1/r^3) and its S + R + D part
constexpr double kDwPairGeomFlops = 99.0, kDwPairRhsFlops = 149.0;
// Each GMRES pass of a refined solve stops at kInnerTol x tol / (current relative residual); the
// accurate residual then decides whether another pass is needed.  0.8 measured fastest on the
// gap sweep (0.5 and 1.0 took 2.5 % and 3 % longer; tighter factors cost more iterations).
constexpr double kInnerTol = 0.8;
constexpr double kDwTripleGeomFlops = 106.0, kDwTripleRhsFlops = 438.0;

struct Factor {
  int m = 0, ncol = 0, rank = 0, ldA = 0, ldV = 0;
  double* A64 = nullptr;  // rank x ldA  (Sigma^+ U^T)
  double* V64 = nullptr;  // ncol x ldV  (V)
  float* A32 = nullptr;
  float* V32 = nullptr;
  float2* A2 = nullptr;   // (hi, lo) float pairs of A64 and V64 for the double-float GEMV
  float2* V2 = nullptr;
  float* Q32 = nullptr;   // far field: 3 n_eq x ldQ (row-major), collocation data -> equivalent strengths
  int ldQ = 0;
};

// keep[i] is the SVD column index of the i-th retained singular triplet
__device__ __forceinline__ float2 split2(double v) {
  float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

__global__ void pack_A_kernel(int r, int m, int ld, const double* __restrict__ U, const double* __restrict__ S,
                              const int* __restrict__ keep, double* __restrict__ A64, float* __restrict__ A32,
                              float2* __restrict__ A2) {
  long long tot = (long long)r * ld;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    int i = (int)(id / ld), j = (int)(id % ld);
    int col = keep[i];
    double v = j < m ? U[(long long)col * m + j] / S[col] : 0.0;
    A64[id] = v;
    A32[id] = (float)v;
    A2[id] = split2(v);
  }
}

// R (n x n, leading dimension n) = the upper triangle of the QR-factored B (leading dimension ldb)
__global__ void upper_copy_kernel(int n, const double* __restrict__ B, int ldb, double* __restrict__ R) {
  const long long tot = (long long)n * n;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % n), j = (int)(id / n);
    R[id] = i <= j ? B[(long long)j * ldb + i] : 0.0;
  }
}

// VT is the column-major ncol x ncol matrix V^T returned by the SVD: V(row, i) = VT[row * ncol + i]
__global__ void pack_V_kernel(int ncol, int r, int ld, const double* __restrict__ VT, const int* __restrict__ keep,
                              double* __restrict__ V64, float* __restrict__ V32, float2* __restrict__ V2) {
  long long tot = (long long)ncol * ld;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < tot; id += (long long)gridDim.x * blockDim.x) {
    int row = (int)(id / ld), i = (int)(id % ld);
    double v = i < r ? VT[(long long)row * ncol + keep[i]] : 0.0;
    V64[id] = v;
    V32[id] = (float)v;
    V2[id] = split2(v);
  }
}

// A one-body factor of a sphere without images, held by every context on the device whose
// spheres have the same self block: equal spheres share one truncated pseudo-inverse across
// contexts as they do within one (Sec. 4: a single SVD serves equal spheres).  The key holds
// every input of the factorisation; the entry is freed with the last context that holds it.
struct SharedFactor {
  int device = 0;
  std::vector<double> key;
  Factor F;
  std::vector<void*> mem;
  unsigned long long bytes = 0;  // the factor's device memory
  int q_rows = 0;                // rows of the far-field Q (3 n_eq), 0 without a far field
  // bf16 slices of Sigma^+ U^T and of Q for the tensor-core step 1, made on first use
  std::mutex tc_mtx;
  int tc_ldk = 0;
  void* as[3] = {nullptr, nullptr, nullptr};
  void* qs[3] = {nullptr, nullptr, nullptr};
  unsigned long long tc_bytes = 0;
  void* alloc(size_t n) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(n, 16)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    mem.push_back(q);
    return q;
  }
  ~SharedFactor() {
    int d0 = 0;
    const bool had = cudaGetDevice(&d0) == cudaSuccess;
    cudaSetDevice(device);
    for (void* q : mem) cudaFree(q);
    if (had) cudaSetDevice(d0);
    cudaGetLastError();
  }
};

std::mutex g_store_mtx;
std::vector<std::weak_ptr<SharedFactor>> g_store;

std::shared_ptr<SharedFactor> store_find(int device, const std::vector<double>& key) {
  std::lock_guard<std::mutex> g(g_store_mtx);
  std::shared_ptr<SharedFactor> hit;
  size_t w = 0;
  for (size_t i = 0; i < g_store.size(); ++i) {
    std::shared_ptr<SharedFactor> e = g_store[i].lock();
    if (!e) continue;  // expired: dropped from the list
    g_store[w++] = g_store[i];
    if (!hit && e->device == device && e->key == key) hit = e;
  }
  g_store.resize(w);
  return hit;
}

void store_add(const std::shared_ptr<SharedFactor>& e) {
  std::lock_guard<std::mutex> g(g_store_mtx);
  g_store.push_back(e);
}

}  // namespace

struct mfs_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  int state = 0;        // 0 empty, 1 spheres set, 2 built
  bool have_bc = false;
  bool solved = false;
  bool dw_pairs = false;  // FP64 operator uses the double-float pair kernel and factors
  bool dw_fast_a = false; // with dw_pairs: Sigma^+ U^T read from its FP32 copy (inner MIXED solves)
  bool ff_pass = false;   // with dw_pairs: far spheres through their equivalent sources (inner MIXED solves)
  bool factored = false;  // one-body pseudo-inverses available
  int mode = 0;           // 0: resistance (velocities given), 1: mobility (forces/torques given)
  int n_sys = 0;          // GMRES system size: n, or n + 6P for the bordered mobility system
  double* d_border = nullptr;  // mobility: scaled prescribed (F_k, T_k), 6 per sphere
  double* d_pparts = nullptr;  // partial sums of the source-split pair kernel, kPairMaxParts * n
  double* d_zero = nullptr;    // 3P zeros
  // measurement
  bool prof = false;
  mfs_timing_t tm{};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pair, ev_gemv, ev_krylov, ev_far, ev_pool;
  std::vector<int> ev_pair_kind;  // precision of each pair launch in ev_pair
  long long pairs_per_apply = 0, proxy_per_apply = 0, image_per_apply = 0;
  // with the far field: near pairs of one apply and the equivalent-source pairs replacing the rest
  long long near_pairs_per_apply = 0, near_proxy_per_apply = 0, near_image_per_apply = 0, far_pairs_per_apply = 0;
  long long build_id = 0;
  struct BatchPlan* batch = nullptr;  // cached lockstep-batch workspace (owned when this is the first context)
  double gemv_bytes32 = 0, gemv_bytes64 = 0, gemv_bytes_fast = 0;  // factor bytes per step 1
  int P = 0;
  double a = 1.0;
  std::vector<double> centres;
  std::vector<double> bg = std::vector<double>(15, 0.0);
  HostDisc hd;
  cusolverDnHandle_t solver = nullptr;

  // device memory owned by the current build, with its size for the memory cap
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;
  unsigned long long mem_limit = 0;  // 0: no cap
  unsigned long long mem_used = 0;
  TargetSet tg;
  SourceSet src;
  double* d_colloc_abs = nullptr;
  int* d_owner = nullptr;
  double* d_sqrtw = nullptr;
  std::vector<Factor> factors;
  // factors of spheres without images, held in the process-wide store with every context that
  // has the same self block (counted in mem_used by each holder)
  std::vector<std::shared_ptr<SharedFactor>> shared;
  int factors_reused = 0;  // of those, taken from the store instead of computed by this build
  FarField ff;             // n_eq == 0: no far field
  float* d_q = nullptr;    // equivalent strengths, 3 n_eq per sphere
  GemvBatch<float> gQ;     // q = Q_f mu_k for every sphere
  // tensor-core step 1 of the passes for the spheres that share the basic factor
  int tc_ncols = 0;        // such spheres on the tensor path (0: off)
  TcGemm tcA, tcQ;         // Sigma^+ U^T and Q of the shared factor, bf16 slices
  long long *d_tc_xoff = nullptr, *d_tc_yA = nullptr, *d_tc_yQ = nullptr;
  float* d_tc_partial = nullptr;
  int* d_tc_err = nullptr;
  GemvBatch<float> gA32_rest, gQ_rest;  // the GEMV jobs of every other sphere
  // tile shapes of the pair kernels (default: by rule; mfs_tune_pairs measures and sets them)
  PairShape shape_all, shape_near, shape_far;
  GemvBatch<float> gA32, gV32;
  GemvBatch<double> gA64, gV64;
  long long tmp_len = 0;
  int n = 0;              // operator size 3 * n_colloc
  long long n_unk = 0;
  double *d_v = nullptr, *d_om = nullptr, *d_wb = nullptr, *d_mu = nullptr, *d_r = nullptr, *d_w64 = nullptr;
  double *d_tmp64 = nullptr, *d_lh64 = nullptr, *d_lam = nullptr, *d_F = nullptr, *d_T = nullptr;
  float *d_tmp32 = nullptr, *d_lh32 = nullptr, *d_in32 = nullptr, *d_out32 = nullptr, *d_mu32 = nullptr;
  float2 *d_x2 = nullptr, *d_t2 = nullptr;  // double-float staging of step 1
  // Krylov workspace (lazily sized)
  void* d_basis = nullptr;
  size_t basis_bytes = 0;
  double* d_partial = nullptr;
  double* d_h = nullptr;
  int nblk = 1;

  mfs_status fail(mfs_status s, const std::string& m) {
    err = m;
    return s;
  }
  template <typename T>
  T* dalloc(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    const size_t bytes = count * sizeof(T);
    if (mem_limit && mem_used + bytes > mem_limit) return nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    allocs.push_back(p);
    alloc_bytes.push_back(bytes);
    mem_used += bytes;
    return static_cast<T*>(p);
  }
  // frees one allocation made by dalloc
  void dfree(void* p) {
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i] == p) {
        cudaFree(p);
        mem_used -= alloc_bytes[i];
        allocs.erase(allocs.begin() + i);
        alloc_bytes.erase(alloc_bytes.begin() + i);
        return;
      }
  }
  void free_build() {
    for (void* p : allocs) cudaFree(p);
    allocs.clear();
    alloc_bytes.clear();
    mem_used = 0;
    factors.clear();
    shared.clear();
    factors_reused = 0;
    ff = FarField();
    d_q = nullptr;
    gQ = GemvBatch<float>();
    tc_ncols = 0;
    shape_all = shape_near = shape_far = PairShape();
    tcA = TcGemm();
    tcQ = TcGemm();
    gA32_rest = gQ_rest = GemvBatch<float>();
    tg = TargetSet();
    src = SourceSet();
    d_basis = nullptr;
    basis_bytes = 0;
    solved = false;
    factored = false;
  }
};

#define CUDA_TRY(ctx, x)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess) return (ctx)->fail(MFS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define CUSOLVER_TRY(ctx, x)                                                              \
  do {                                                                                    \
    cusolverStatus_t s_ = (x);                                                            \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                                    \
      return (ctx)->fail(MFS_ERR_CUDA, std::string(#x) + ": cusolver status " + std::to_string((int)s_)); \
  } while (0)
#define ALLOC_TRY(ctx, ptr, T, count)                                                     \
  do {                                                                                    \
    (ptr) = (ctx)->dalloc<T>(count);                                                      \
    if (!(ptr)) return (ctx)->fail(MFS_ERR_OOM, "device allocation failed: " #ptr);      \
  } while (0)
#define CHECK_LAUNCH(ctx) CUDA_TRY(ctx, cudaGetLastError())

namespace {

template <typename T>
mfs_status upload(mfs_ctx* c, T*& dst, const std::vector<T>& v) {
  ALLOC_TRY(c, dst, T, v.size());
  if (!v.empty()) CUDA_TRY(c, cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  return MFS_OK;
}

// ------------------------------------------------------------------ operator pieces
template <typename T> struct Ops;
template <> struct Ops<float> {
  static const GemvBatch<float>& A(mfs_ctx* c) { return c->gA32; }
  static const GemvBatch<float>& V(mfs_ctx* c) { return c->gV32; }
  static float* tmp(mfs_ctx* c) { return c->d_tmp32; }
  static float* lh(mfs_ctx* c) { return c->d_lh32; }
};
template <> struct Ops<double> {
  static const GemvBatch<double>& A(mfs_ctx* c) { return c->gA64; }
  static const GemvBatch<double>& V(mfs_ctx* c) { return c->gV64; }
  static double* tmp(mfs_ctx* c) { return c->d_tmp64; }
  static double* lh(mfs_ctx* c) { return c->d_lh64; }
};

// CUDA-event bracket around a launch when profiling is on
std::pair<cudaEvent_t, cudaEvent_t> take_events(mfs_ctx* c) {
  if (!c->ev_pool.empty()) {
    auto e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  std::pair<cudaEvent_t, cudaEvent_t> e{nullptr, nullptr};
  cudaEventCreate(&e.first);
  cudaEventCreate(&e.second);
  return e;
}
template <typename F>
void timed(mfs_ctx* c, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& list, F&& launch) {
  if (!c->prof) {
    launch();
    return;
  }
  auto e = take_events(c);
  cudaEventRecord(e.first, c->stream);
  launch();
  cudaEventRecord(e.second, c->stream);
  list.push_back(e);
}
// folds finished event pairs into the counters (call after a stream synchronisation)
void collect_events(mfs_ctx* c) {
  for (size_t i = 0; i < c->ev_pair.size(); ++i) {
    auto& e = c->ev_pair[i];
    float ms = 0;
    if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) {
      c->tm.pair_ms += ms;
      int kind = i < c->ev_pair_kind.size() ? c->ev_pair_kind[i] : 0;
      if (kind >= 0 && kind < 3) c->tm.by_kind_ms[kind] += ms;
    }
    c->ev_pool.push_back(e);
  }
  c->ev_pair.clear();
  c->ev_pair_kind.clear();
  for (auto& e : c->ev_gemv) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) c->tm.gemv_ms += ms;
    c->ev_pool.push_back(e);
  }
  c->ev_gemv.clear();
  for (auto& e : c->ev_krylov) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) c->tm.krylov_ms += ms;
    c->ev_pool.push_back(e);
  }
  c->ev_krylov.clear();
  for (auto& e : c->ev_far) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) c->tm.far_ms += ms;
    c->ev_pool.push_back(e);
  }
  c->ev_far.clear();
  cudaGetLastError();
}

// step 1: lambda_hat = B^+ mu (two factors in turn, eq. transform); in the mixed mode the FP64
// factors are applied in double-float arithmetic from their (hi, lo) float copies
template <typename T>
void precond(mfs_ctx* c, const T* mu, T* lam_hat) {
  timed(c, c->ev_gemv, [&] {
    if constexpr (sizeof(T) == 8) {
      if (c->dw_pairs) {
        launch_split_dw(c->n, mu, c->d_x2, c->stream);
        if (c->dw_fast_a && c->tc_ncols > 0) {
          // the spheres sharing the basic factor as one product on the tensor cores
          launch_gemv_f32_dw(c->gA32_rest, c->d_x2, c->d_t2, c->stream);
          launch_tc_gemm(c->tcA, c->tc_ncols, mu, c->d_tc_xoff, c->d_tc_yA, nullptr, c->d_t2, c->d_tc_partial,
                         c->d_tc_err, true, c->stream);
          c->tm.tc_launches += 1;
          c->tm.tc_columns += c->tc_ncols;
        } else if (c->dw_fast_a) {
          launch_gemv_f32_dw(c->gA32, c->d_x2, c->d_t2, c->stream);
        } else {
          launch_gemv_dw(Ops<T>::A(c), c->d_x2, c->d_t2, nullptr, c->stream);
        }
        launch_gemv_dw(Ops<T>::V(c), c->d_t2, nullptr, lam_hat, c->stream);
        return;
      }
    }
    launch_gemv<T>(Ops<T>::A(c), mu, Ops<T>::tmp(c), c->stream);
    launch_gemv<T>(Ops<T>::V(c), Ops<T>::tmp(c), lam_hat, c->stream);
  });
  c->tm.gemv_launches += 2;
  c->tm.gemv_bytes += sizeof(T) == 8 ? (c->dw_pairs && c->dw_fast_a ? c->gemv_bytes_fast : c->gemv_bytes64)
                                     : c->gemv_bytes32;
}

// steps 2+3 with the pair kernel of the current precision
template <typename T>
void pairs_step(mfs_ctx* c, const T* lam_hat, const T* mu, T* out) {
  if constexpr (sizeof(T) == 8) {
    if (c->dw_pairs && c->ff_pass && c->ff.n_eq > 0) {
      // near spheres directly in double-float, the far ones through their equivalent sources,
      // whose strengths q = Q mu are formed from this apply's mu
      timed(c, c->ev_pair, [&] {
        launch_pairs_dw_near(c->tg, c->src, c->ff, lam_hat, mu, out, c->hd.prm.visc, c->d_pparts, kPairMaxParts,
                             c->stream, c->shape_near);
      });
      timed(c, c->ev_far, [&] {
        launch_convert<double, float>(c->n, mu, 1.0, c->d_mu32, c->stream);
        if (c->tc_ncols > 0) {
          launch_gemv<float>(c->gQ_rest, c->d_mu32, c->d_q, c->stream);
          launch_tc_gemm(c->tcQ, c->tc_ncols, mu, c->d_tc_xoff, c->d_tc_yQ, c->d_q, nullptr, c->d_tc_partial,
                         c->d_tc_err, true, c->stream);
          c->tm.tc_launches += 1;
          c->tm.tc_columns += c->tc_ncols;
        } else {
          launch_gemv<float>(c->gQ, c->d_mu32, c->d_q, c->stream);
        }
        launch_pairs_far(c->tg, c->src, c->ff, out, c->hd.prm.visc, c->d_pparts, kPairMaxParts, c->stream,
                         c->shape_far);
      });
      c->tm.pair_launches += 1;
      c->tm.pair_interactions += c->near_pairs_per_apply;
      c->tm.pair_issued_flops += (double)c->near_proxy_per_apply * (kDwPairGeomFlops + kDwPairRhsFlops) +
                                 (double)c->near_image_per_apply * (kDwTripleGeomFlops + kDwTripleRhsFlops);
      c->tm.pair_proxy += c->near_proxy_per_apply;
      c->tm.pair_image_nodes += c->near_image_per_apply;
      c->tm.pair_kind = MFS_MIXED;
      c->tm.by_kind_launches[MFS_MIXED] += 1;
      c->tm.by_kind_proxy[MFS_MIXED] += c->near_proxy_per_apply;
      c->tm.by_kind_image_nodes[MFS_MIXED] += c->near_image_per_apply;
      c->tm.far_launches += 1;
      c->tm.far_pairs += c->far_pairs_per_apply;
      if (c->prof) c->ev_pair_kind.push_back(MFS_MIXED);
      return;
    }
  }
  timed(c, c->ev_pair, [&] {
    if constexpr (sizeof(T) == 8) {
      if (c->dw_pairs) {
        launch_pairs_dw(c->tg, c->src, lam_hat, mu, out, c->hd.prm.visc, c->d_pparts, kPairMaxParts, c->stream,
                        c->shape_all);
        return;
      }
    }
    launch_pairs<T>(c->tg, c->src, lam_hat, mu, out, c->hd.prm.visc, c->stream);
  });
  c->tm.pair_launches += 1;
  c->tm.pair_interactions += c->pairs_per_apply;
  if (sizeof(T) == 8 && c->dw_pairs)
    c->tm.pair_issued_flops += (double)c->proxy_per_apply * (kDwPairGeomFlops + kDwPairRhsFlops) +
                               (double)c->image_per_apply * (kDwTripleGeomFlops + kDwTripleRhsFlops);
  c->tm.pair_proxy += c->proxy_per_apply;
  c->tm.pair_image_nodes += c->image_per_apply;
  c->tm.pair_kind = sizeof(T) == 4 ? MFS_FP32 : (c->dw_pairs ? MFS_MIXED : MFS_FP64);
  const int kind = c->tm.pair_kind;
  c->tm.by_kind_launches[kind] += 1;
  c->tm.by_kind_proxy[kind] += c->proxy_per_apply;
  c->tm.by_kind_image_nodes[kind] += c->image_per_apply;
  if (c->prof) c->ev_pair_kind.push_back(kind);
}

// out = G_hat mu
template <typename T>
void apply_op(mfs_ctx* c, const T* mu, T* out) {
  precond<T>(c, mu, Ops<T>::lh(c));
  pairs_step<T>(c, Ops<T>::lh(c), mu, out);
}

// The GMRES operator: G_hat (resistance), or the bordered mobility operator
//   [mu; U] -> [G_hat mu - W (V_k + Omega_k x (x - c_k)); s_F F_k(B^+ mu), s_T T_k(B^+ mu)]
// (forces/torques of lambda_hat = B^+ mu by the Sec. 2.3 remark, s_F = 1/(6 pi mu a),
// s_T = 1/(8 pi mu a^3)).
template <typename T>
void sys_apply(mfs_ctx* c, const T* in, T* out) {
  apply_op<T>(c, in, out);
  if constexpr (sizeof(T) == 8) {
    if (c->mode == 1) {
      const double a = c->a, mu = c->hd.prm.visc;
      launch_rigid_sub(c->tg.n, c->d_owner, c->tg.pos64, in + c->n, out, c->stream);
      launch_forces_torques_scaled(c->src, Ops<T>::lh(c), out + c->n, out + c->n + 3, 6, 1.0 / (6.0 * kPi * mu * a),
                                   1.0 / (8.0 * kPi * mu * a * a * a), c->stream);
    }
  }
}

template <typename T>
mfs_status ensure_krylov(mfs_ctx* c, int restart) {
  size_t need = (size_t)(restart + 1) * (size_t)c->n_sys * sizeof(T);
  if (c->basis_bytes < need) {
    if (c->d_basis) {
      c->dfree(c->d_basis);
      c->d_basis = nullptr;
    }
    c->d_basis = c->dalloc<char>(need);
    if (!c->d_basis) return c->fail(MFS_ERR_OOM, "device allocation failed: Krylov basis");
    c->basis_bytes = need;
  }
  return MFS_OK;
}

// dot products of w with V[0..nvec) (FP64 partials) -> host h
template <typename T>
mfs_status dots(mfs_ctx* c, int nvec, const T* V, const T* w, double* h_dev) {
  launch_multidot<T>(c->n_sys, nvec, V, c->n_sys, w, c->d_partial, c->nblk, c->stream);
  launch_reduce_partials(nvec, c->nblk, c->d_partial, h_dev, c->stream);
  CHECK_LAUNCH(c);
  return MFS_OK;
}

// Restarted GMRES(m) with CGS2 Arnoldi (classical Gram-Schmidt applied twice), Givens
// rotations and the small least-squares problem on the host in FP64 (Saad, Iterative
// Methods for Sparse Linear Systems, Alg. 6.9).  Solves op x = b from x0 = 0 and stops at
// ||b - op x|| <= tol ||b|| (the GMRES estimate; restarts use the true residual).
template <typename T>
mfs_status gmres(mfs_ctx* c, const T* b, T* x, double tol, int restart, int max_iter, int& iters, double& rel) {
  mfs_status s = ensure_krylov<T>(c, restart);
  if (s != MFS_OK) return s;
  const int n = c->n_sys;
  const int ldh = restart + 1;
  T* V = static_cast<T*>(c->d_basis);
  std::vector<double> H((size_t)ldh * restart), cs(restart), sn(restart), g(ldh), hb(2 * ldh + 1), y(restart);
  double* h1 = c->d_h;
  double* h2 = c->d_h + ldh;
  double* hn = c->d_h + 2 * ldh;
  double* coef = c->d_h + 3 * ldh;
  CUDA_TRY(c, cudaMemsetAsync(x, 0, sizeof(T) * n, c->stream));
  iters = 0;
  rel = 0.0;
  if ((s = dots<T>(c, 1, b, b, hn)) != MFS_OK) return s;
  double bn2 = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&bn2, hn, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  const double bnorm = std::sqrt(bn2);
  if (!std::isfinite(bnorm)) return c->fail(MFS_ERR_NUMERIC, "right-hand side is not finite");
  if (bnorm == 0.0) return MFS_OK;
  const double one = 1.0;
  bool first = true;
  while (true) {
    double beta;
    if (first) {
      launch_scale_copy<T>(n, b, 1.0, V, c->stream);
      beta = bnorm;
      first = false;
    } else {
      // V0 = b - op x
      sys_apply<T>(c, x, V);
      launch_scale_copy<T>(n, V, -1.0, V, c->stream);
      CUDA_TRY(c, cudaMemcpyAsync(coef, &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
      launch_update<T>(n, 1, b, n, coef, 1.0, V, c->stream);
      CHECK_LAUNCH(c);
      if ((s = dots<T>(c, 1, V, V, hn)) != MFS_OK) return s;
      double r2 = 0;
      CUDA_TRY(c, cudaMemcpyAsync(&r2, hn, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      beta = std::sqrt(r2);
      rel = beta / bnorm;
      if (!std::isfinite(beta)) return c->fail(MFS_ERR_NUMERIC, "non-finite GMRES residual");
      if (rel <= tol || iters >= max_iter || beta == 0.0) break;
    }
    launch_scale_copy<T>(n, V, 1.0 / beta, V, c->stream);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j_used = 0;
    bool done = false;
    for (int j = 0; j < restart; ++j) {
      T* w = V + (size_t)(j + 1) * n;
      sys_apply<T>(c, V + (size_t)j * n, w);
      CHECK_LAUNCH(c);
      if ((s = dots<T>(c, j + 1, V, w, h1)) != MFS_OK) return s;
      launch_update<T>(n, j + 1, V, n, h1, -1.0, w, c->stream);
      if ((s = dots<T>(c, j + 1, V, w, h2)) != MFS_OK) return s;
      launch_update<T>(n, j + 1, V, n, h2, -1.0, w, c->stream);
      if ((s = dots<T>(c, 1, w, w, hn)) != MFS_OK) return s;
      CUDA_TRY(c, cudaMemcpyAsync(hb.data(), c->d_h, sizeof(double) * (2 * ldh + 1), cudaMemcpyDeviceToHost, c->stream));
      CUDA_TRY(c, cudaStreamSynchronize(c->stream));
      double* col = &H[(size_t)j * ldh];
      for (int i = 0; i <= j; ++i) col[i] = hb[i] + hb[ldh + i];
      const double hnext = std::sqrt(std::max(0.0, hb[2 * ldh]));
      if (!std::isfinite(hnext)) return c->fail(MFS_ERR_NUMERIC, "non-finite value in the Arnoldi process");
      col[j + 1] = hnext;
      if (hnext > 0) launch_scale_copy<T>(n, w, 1.0 / hnext, w, c->stream);
      for (int i = 0; i < j; ++i) {
        double t = cs[i] * col[i] + sn[i] * col[i + 1];
        col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
        col[i] = t;
      }
      const double den = std::hypot(col[j], col[j + 1]);
      cs[j] = den > 0 ? col[j] / den : 1.0;
      sn[j] = den > 0 ? col[j + 1] / den : 0.0;
      col[j] = den;
      col[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++iters;
      j_used = j + 1;
      rel = std::fabs(g[j + 1]) / bnorm;
      if (rel <= tol || iters >= max_iter || hnext == 0.0) {
        done = true;
        break;
      }
    }
    // y = R^{-1} g, x += V y
    for (int i = j_used - 1; i >= 0; --i) {
      double t = g[i];
      for (int q = i + 1; q < j_used; ++q) t -= H[(size_t)q * ldh + i] * y[q];
      const double diag = H[(size_t)i * ldh + i];
      y[i] = diag != 0.0 ? t / diag : 0.0;
    }
    if (j_used > 0) {
      CUDA_TRY(c, cudaMemcpyAsync(coef, y.data(), sizeof(double) * j_used, cudaMemcpyHostToDevice, c->stream));
      launch_update<T>(n, j_used, V, n, coef, 1.0, x, c->stream);
      CHECK_LAUNCH(c);
    }
    if (done) break;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MFS_OK;
}

// ||v||_2 of an FP64 device vector
mfs_status norm64(mfs_ctx* c, const double* v, double& out) {
  mfs_status s = dots<double>(c, 1, v, v, c->d_h + 4 * 512);  // over the current system size
  if (s != MFS_OK) return s;
  double r2 = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&r2, c->d_h + 4 * 512, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  out = std::sqrt(r2);
  return MFS_OK;
}

// A bounded wait of the tensor-core kernel ran out (its flag is cleared for the next call).
// The bf16 slices of a store entry's Sigma^+ U^T (and of its far-field Q when it has one), made
// once for every context that holds the entry; the calling context's cap counts them.
mfs_status ensure_tc_slices(mfs_ctx* c, SharedFactor& e) {
  std::lock_guard<std::mutex> g(e.tc_mtx);
  const Factor& F = e.F;
  const int ldk = tc_ldk(F.m);
  if (!e.as[0]) {
    const size_t b = sizeof(uint16_t) * (size_t)F.rank * ldk;
    for (int i = 0; i < 3; ++i)
      if (!(e.as[i] = e.alloc(b))) return c->fail(MFS_ERR_OOM, "device allocation failed: tensor-core slices");
    e.tc_bytes += 3 * b;
    launch_split3_matrix(F.rank, F.m, F.ldA, F.A64, ldk, e.as[0], e.as[1], e.as[2], c->stream);
  }
  if (F.Q32 && !e.qs[0]) {
    const int rows = e.q_rows;
    const size_t b = sizeof(uint16_t) * (size_t)rows * ldk;
    for (int i = 0; i < 3; ++i)
      if (!(e.qs[i] = e.alloc(b))) return c->fail(MFS_ERR_OOM, "device allocation failed: tensor-core slices");
    e.tc_bytes += 3 * b;
    launch_split3_matrix_f32(rows, F.m, F.ldQ, F.Q32, ldk, e.qs[0], e.qs[1], e.qs[2], c->stream);
  }
  e.tc_ldk = ldk;
  CHECK_LAUNCH(c);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // other contexts' streams read them next
  return MFS_OK;
}

mfs_status check_tc_timeout(mfs_ctx* c) {
  if (!c->d_tc_err) return MFS_OK;
  int h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (!h) return MFS_OK;
  CUDA_TRY(c, cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream));
  return c->fail(MFS_ERR_TIMEOUT, "tensor-core step 1: a pipeline wait ran out of time");
}

mfs_status check_state(mfs_ctx* c, int need) {
  if (!c) return MFS_ERR_ARG;
  if (c->state < need) return c->fail(MFS_ERR_STATE, need == 1 ? "spheres not set" : "discretisation not built");
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return c->fail(MFS_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  return MFS_OK;
}

}  // namespace

// ================================================================== lockstep batch of problems
struct BatchPlan {
  std::vector<mfs_ctx*> key;
  std::vector<long long> key_build;
  std::vector<int> mob;            // per problem: 1 = mobility (6P border unknowns after the node rows)
  std::vector<long long> nlen;     // node rows 3 n_colloc per problem
  long long* d_nlen = nullptr;
  int K = 0, nt = 1;
  long long n_total = 0, u_total = 0, t_total = 0;
  std::vector<long long> voff, uoff, toff;
  std::vector<long long> pairs_p, proxy_p, image_p;
  std::vector<void*> allocs;
  std::vector<void*> gs_allocs;
  void* d_args = nullptr;    // per-problem kernel arguments for 4 nodes per thread
  void* d_args1 = nullptr;   // and for 1 node per thread
  int2* d_work = nullptr;    // (problem, tile) lists for both tilings
  int2* d_work1 = nullptr;
  int n_work = 0, n_work1 = 0;
  std::vector<int> tiles4;   // large tiles per problem, to pick the tiling of each launch
  std::vector<int> tiles1;
  std::vector<long long> others_p;  // proxies of the other spheres per problem (source split)
  std::vector<int2> w4_host, w1_host;  // full work lists; the launches use the active problems' part
  int2* d_cwork = nullptr;   // compacted (problem, tile) lists of the active problems
  int2* d_cwork1 = nullptr;
  int2* wpin = nullptr;      // pinned staging for them
  int n_cwork = 0, n_cwork1 = 0;
  double* pparts = nullptr;  // source-split partial sums, kPairMaxParts * n_total
  std::vector<int> cprob_host;  // problem of each vector chunk
  std::vector<int> jprob_host;  // problem of each GEMV job
  int* d_jlist = nullptr;       // compacted GEMV job list of the active problems
  int* jpin = nullptr;          // pinned staging for it
  int* d_cchunk = nullptr;      // compacted chunk list of the active problems (seg.list)
  int* cpin = nullptr;          // pinned staging for it
  GivensState gs;               // device GMRES state (restart_cap columns per problem)
  int gs_restart = 0;
  int* snap = nullptr;          // pinned: kSyncEvery x K active-flag snapshots, then the error flag
  int* d_active = nullptr;
  long long *d_uoff = nullptr, *d_voff = nullptr;
  GemvBatch<double> gA, gV;
  GemvBatch<float> gA32;  // the same jobs over the FP32 copies of Sigma^+ U^T (inner MIXED solves)
  // tensor-core step 1 of the inner MIXED solves: the spheres of every problem whose factor is
  // one store entry form the columns of one product; gA32 then covers the other jobs only
  std::shared_ptr<SharedFactor> tc_ent;  // keeps the entry (and its slices) alive with the plan
  TcGemm tcA;
  int tc_ncap = 0, tc_nact = 0;
  std::vector<int> tc_prob;                // problem of each column
  std::vector<long long> tc_x_host, tc_y_host;
  long long *d_tc_x = nullptr, *d_tc_y = nullptr;  // offsets of the active problems' columns
  long long* tc_pin = nullptr;             // pinned staging for them (2 tc_ncap)
  float* tc_partial = nullptr;
  int* tc_err = nullptr;
  std::vector<char> jtc_host;              // per GEMV job: 1 when it is a tensor column
  // several right-hand sides on one geometry in one pair-kernel pass (double-float): items
  // (lead problem, tile, first index into the right-hand-side list, count) and the 128-node
  // tiles of the problems left single
  int4* d_mwork = nullptr;
  int4* mwork_pin = nullptr;
  int* d_rhs = nullptr;
  int* rhs_pin = nullptr;
  int2* d_swork1 = nullptr;
  int2* swork_pin = nullptr;
  unsigned* d_pcount = nullptr;  // per pair-kernel work item: arrivals of its source parts
  int n_mwork = 0, n_swork1 = 0;
  size_t mwork_cap = 0;
  std::vector<int> rhs_shared;             // per problem: right-hand sides in its pair-kernel item
  std::vector<int> leader;                 // per problem: the first problem on the same context
  std::vector<double> bA32_p, bA2_p, bV_p; // per context (at its leader): factor bytes of one step 1
  int* d_jlist_rest = nullptr;             // compacted list of the active problems' other jobs
  int* jpin_rest = nullptr;
  SegTable seg;
  double *wb = nullptr, *x = nullptr, *r = nullptr, *e = nullptr, *w = nullptr, *lh = nullptr, *tmp = nullptr,
         *lam = nullptr, *partial = nullptr, *hbuf = nullptr, *coef = nullptr, *scl = nullptr;
  float2 *x2 = nullptr, *t2 = nullptr;
  std::vector<long long> boff;           // per problem: offset of its 3 P values in bc / F / T
  double *bc_v = nullptr, *bc_w = nullptr, *out_F = nullptr, *out_T = nullptr;
  double* basis = nullptr;
  size_t basis_cap = 0;
  double* hpin = nullptr;  // pinned host staging for the Arnoldi coefficients
  int* apin = nullptr;     // pinned host staging for the active flags
  cudaEvent_t ev = nullptr;
  ~BatchPlan() {
    for (void* q : allocs) cudaFree(q);
    if (basis) cudaFree(basis);
    if (hpin) cudaFreeHost(hpin);
    if (apin) cudaFreeHost(apin);
    if (wpin) cudaFreeHost(wpin);
    if (cpin) cudaFreeHost(cpin);
    if (jpin) cudaFreeHost(jpin);
    if (tc_pin) cudaFreeHost(tc_pin);
    if (mwork_pin) cudaFreeHost(mwork_pin);
    if (rhs_pin) cudaFreeHost(rhs_pin);
    if (swork_pin) cudaFreeHost(swork_pin);
    if (jpin_rest) cudaFreeHost(jpin_rest);
    if (snap) cudaFreeHost(snap);
    for (void* q : gs_allocs) cudaFree(q);
    if (ev) cudaEventDestroy(ev);
  }
  template <typename T>
  T* alloc(size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    allocs.push_back(q);
    return static_cast<T*>(q);
  }
};

namespace {

constexpr int kMaxBatchVec = 512;  // restart + 1 must fit the segmented update's coefficient cache

template <typename T>
bool put(BatchPlan* B, T*& dst, const std::vector<T>& v) {
  dst = B->alloc<T>(v.size());
  return dst && cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

// Builds the concatenated layout, the pair work list, the GEMV job tables and the vector chunks.
mfs_status make_plan(mfs_ctx* c0, int K, mfs_ctx* const* ctxs, const std::vector<int>& mob, BatchPlan*& out) {
  BatchPlan* B = new (std::nothrow) BatchPlan();
  if (!B) return c0->fail(MFS_ERR_OOM, "host allocation failed: batch plan");
  B->K = K;
  B->key.assign(ctxs, ctxs + K);
  B->mob = mob;
  for (int p = 0; p < K; ++p) B->key_build.push_back(ctxs[p]->build_id);
  B->voff.assign(K + 1, 0);
  B->uoff.assign(K + 1, 0);
  B->toff.assign(K + 1, 0);
  long long tiles_large = 0;
  for (int p = 0; p < K; ++p) {
    mfs_ctx* c = ctxs[p];
    B->nlen.push_back(c->n);
    B->voff[p + 1] = B->voff[p] + c->n + (mob[p] ? 6LL * c->P : 0);
    B->uoff[p + 1] = B->uoff[p] + c->n_unk;
    B->toff[p + 1] = B->toff[p] + c->tmp_len;
    B->pairs_p.push_back(c->pairs_per_apply);
    B->proxy_p.push_back(c->proxy_per_apply);
    B->image_p.push_back(c->image_per_apply);
    tiles_large += c->tg.n_tiles;
  }
  B->n_total = B->voff[K];
  B->u_total = B->uoff[K];
  B->t_total = B->toff[K];
  (void)tiles_large;
  // pair kernel arguments and work lists for both tilings; each launch picks the tiling from
  // the tiles of the problems still active (the lockstep tail may hold a single problem)
  const size_t asz = pair_args64_bytes();
  std::vector<char> args4(asz * K), args1(asz * K);
  std::vector<int2> work4, work1;
  for (int p = 0; p < K; ++p) {
    mfs_ctx* c = ctxs[p];
    fill_pair_args64(args4.data() + asz * p, c->tg, c->src, nullptr, nullptr, nullptr, c->hd.prm.visc, 4);
    fill_pair_args64(args1.data() + asz * p, c->tg, c->src, nullptr, nullptr, nullptr, c->hd.prm.visc, 1);
    for (int t = 0; t < c->tg.n_tiles; ++t) work4.push_back(make_int2(p, t));
    for (int t = 0; t < c->tg.n_tiles1; ++t) work1.push_back(make_int2(p, t));
    B->tiles4.push_back(c->tg.n_tiles);
    B->tiles1.push_back(c->tg.n_tiles1);
    B->others_p.push_back((long long)(c->P - 1) * c->src.N);
  }
  B->w4_host = work4;
  B->w1_host = work1;
  B->n_work = (int)work4.size();
  B->n_work1 = (int)work1.size();
  B->d_args = B->alloc<char>(args4.size());
  B->d_args1 = B->alloc<char>(args1.size());
  bool ok = B->d_args && B->d_args1 &&
            cudaMemcpy(B->d_args, args4.data(), args4.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(B->d_args1, args1.data(), args1.size(), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && put(B, B->d_work, work4) && put(B, B->d_work1, work1) && put(B, B->d_uoff, B->uoff) &&
       put(B, B->d_voff, B->voff) && put(B, B->d_nlen, B->nlen);
  B->d_active = B->alloc<int>(K);
  B->d_cwork = B->alloc<int2>(work4.size());
  B->d_cwork1 = B->alloc<int2>(work1.size());
  ok = ok && B->d_active && B->d_cwork && B->d_cwork1 &&
       cudaMallocHost(&B->wpin, sizeof(int2) * std::max<size_t>(1, work4.size() + work1.size())) == cudaSuccess;
  // GEMV jobs: every sphere of every problem, with the problems that share a context (several
  // right-hand sides on one geometry) adjacent, so a factor matrix is read once for all of them
  std::vector<const double*> mA, mV;
  std::vector<const float*> mA32;
  std::vector<const float2*> mA2, mV2;
  std::vector<int> rA, cA, lA, rV, cV, lV, jp;
  std::vector<long long> xA, yA, xV, yV;
  int maxA = 0, maxV = 0;
  std::vector<std::vector<long long>> ptoff(K);
  for (int p = 0; p < K; ++p) {
    mfs_ctx* c = ctxs[p];
    long long t = 0;
    ptoff[p].push_back(0);
    for (int kk = 0; kk < c->hd.P; ++kk) {
      t += c->factors[c->hd.factor_id[kk]].rank;
      ptoff[p].push_back(t);
    }
  }
  // the store entry shared by most spheres over all problems (contexts built with
  // tensor_step1 = 0 keep their spheres on the GEMV)
  std::shared_ptr<SharedFactor> best;
  {
    std::vector<std::pair<SharedFactor*, int>> cnt;
    bool any2 = false;
    for (int p = 0; p < K; ++p) {
      mfs_ctx* c = ctxs[p];
      if (c->hd.prm.tensor_step1 == 0) continue;
      any2 = any2 || c->hd.prm.tensor_step1 == 2;
      for (int kk = 0; kk < c->hd.P; ++kk) {
        const double* a64 = c->factors[c->hd.factor_id[kk]].A64;
        for (auto& e : c->shared)
          if (e->F.A64 == a64) {
            size_t i = 0;
            while (i < cnt.size() && cnt[i].first != e.get()) ++i;
            if (i == cnt.size()) cnt.push_back({e.get(), 0});
            ++cnt[i].second;
          }
      }
    }
    int bi = -1;
    for (size_t i = 0; i < cnt.size(); ++i)
      if (bi < 0 || cnt[i].second > cnt[bi].second) bi = (int)i;
    if (bi >= 0 && cnt[bi].second >= (any2 ? 1 : 8))
      for (int p = 0; p < K && !best; ++p)
        for (auto& e : ctxs[p]->shared)
          if (e.get() == cnt[bi].first) best = e;
  }
  std::vector<int> seen(K, 0);
  B->leader.assign(K, 0);
  B->bA32_p.assign(K, 0.0);
  B->bA2_p.assign(K, 0.0);
  B->bV_p.assign(K, 0.0);
  for (int p0 = 0; p0 < K && ok; ++p0) {
    if (seen[p0]) continue;
    mfs_ctx* c = ctxs[p0];
    const HostDisc& d = c->hd;
    std::vector<int> group;
    for (int p = p0; p < K; ++p)
      if (ctxs[p] == c) {
        group.push_back(p);
        seen[p] = 1;
        B->leader[p] = p0;
      }
    for (int k = 0; k < d.P; ++k) {
      const Factor& F = c->factors[d.factor_id[k]];
      const bool tc_k = best && c->hd.prm.tensor_step1 != 0 && F.A64 == best->F.A64;
      if (!tc_k) B->bA32_p[p0] += 4.0 * F.rank * F.m;
      B->bA2_p[p0] += 8.0 * F.rank * F.m;
      B->bV_p[p0] += 8.0 * F.ncol * F.rank;
      for (int p : group) {
        mA.push_back(F.A64);
        mV.push_back(F.V64);
        mA2.push_back(F.A2);
        mA32.push_back(F.A32);
        mV2.push_back(F.V2);
        rA.push_back(F.rank); cA.push_back(F.m); lA.push_back(F.ldA);
        xA.push_back(B->voff[p] + 3LL * d.colloc_off[k]);
        yA.push_back(B->toff[p] + ptoff[p][k]);
        rV.push_back(F.ncol); cV.push_back(F.rank); lV.push_back(F.ldV);
        xV.push_back(B->toff[p] + ptoff[p][k]);
        yV.push_back(B->uoff[p] + d.unk_off[k]);
        jp.push_back(p);
        maxA = std::max(maxA, F.rank);
        maxV = std::max(maxV, F.ncol);
        const bool tc = best && ctxs[p]->hd.prm.tensor_step1 != 0 && F.A64 == best->F.A64;
        B->jtc_host.push_back(tc ? 1 : 0);
        if (tc) {
          B->tc_prob.push_back(p);
          B->tc_x_host.push_back(xA.back());
          B->tc_y_host.push_back(yA.back());
        }
      }
    }
  }
  const double** dmA = nullptr;
  const double** dmV = nullptr;
  const float2** dmA2 = nullptr;
  const float2** dmV2 = nullptr;
  const float** dmA32 = nullptr;
  int *drA, *dcA, *dlA, *drV, *dcV, *dlV, *djp;
  long long *dxA, *dyA, *dxV, *dyV;
  B->jprob_host = jp;
  ok = ok && (B->d_jlist = B->alloc<int>(jp.size())) &&
       cudaMallocHost(&B->jpin, sizeof(int) * std::max<size_t>(1, jp.size())) == cudaSuccess;
  ok = ok && put(B, dmA, mA) && put(B, dmV, mV) && put(B, drA, rA) && put(B, dcA, cA) && put(B, dlA, lA) &&
       put(B, drV, rV) && put(B, dcV, cV) && put(B, dlV, lV) && put(B, djp, jp) && put(B, dxA, xA) &&
       put(B, dyA, yA) && put(B, dxV, xV) && put(B, dyV, yV) && put(B, dmA2, mA2) && put(B, dmV2, mV2) &&
       put(B, dmA32, mA32);
  if (ok) {
    B->gA.mat_dw = dmA2;
    B->gV.mat_dw = dmV2;
    B->gA.mat = dmA; B->gA.rows = drA; B->gA.cols = dcA; B->gA.ld = dlA; B->gA.x_off = dxA; B->gA.y_off = dyA;
    B->gA.n_jobs = (int)mA.size(); B->gA.max_rows = maxA; B->gA.job_prob = djp; B->gA.active = B->d_active;
    B->gV.mat = dmV; B->gV.rows = drV; B->gV.cols = dcV; B->gV.ld = dlV; B->gV.x_off = dxV; B->gV.y_off = dyV;
    B->gV.n_jobs = (int)mV.size(); B->gV.max_rows = maxV; B->gV.job_prob = djp; B->gV.active = B->d_active;
    B->gA32.mat = dmA32; B->gA32.rows = drA; B->gA32.cols = dcA; B->gA32.ld = dlA; B->gA32.x_off = dxA;
    B->gA32.y_off = dyA; B->gA32.n_jobs = (int)mA32.size(); B->gA32.max_rows = maxA; B->gA32.job_prob = djp;
    B->gA32.active = B->d_active;
  }
  B->mwork_cap = std::max<size_t>(1, B->w1_host.size());
  ok = ok && (B->d_mwork = B->alloc<int4>(B->mwork_cap)) && (B->d_rhs = B->alloc<int>(K)) &&
       (B->d_swork1 = B->alloc<int2>(B->mwork_cap)) && (B->d_pcount = B->alloc<unsigned>(B->mwork_cap)) &&
       cudaMemset(B->d_pcount, 0, sizeof(unsigned) * B->mwork_cap) == cudaSuccess &&
       cudaMallocHost(&B->mwork_pin, sizeof(int4) * B->mwork_cap) == cudaSuccess &&
       cudaMallocHost(&B->rhs_pin, sizeof(int) * K) == cudaSuccess &&
       cudaMallocHost(&B->swork_pin, sizeof(int2) * B->mwork_cap) == cudaSuccess;
  if (ok && best) {
    const Factor& F = best->F;
    const int ncap = (int)B->tc_prob.size();
    mfs_status st2 = ensure_tc_slices(c0, *best);
    if (st2 != MFS_OK) {
      delete B;
      return st2;
    }
    void* xs[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < 3; ++i)
      if (!(xs[i] = B->alloc<uint16_t>((size_t)ncap * tc_ldk(F.m)))) {
        delete B;
        return c0->fail(MFS_ERR_OOM, "device allocation failed: batch tensor-core slices");
      }
    if (!tc_prepare(B->tcA, best->as, F.rank, xs, ncap, F.m)) {
      delete B;
      return c0->fail(MFS_ERR_CUDA, "tensor-core step 1: tensor maps or shared-memory limit unavailable");
    }
    // the partial-sum buffer for any number of active columns up to ncap
    size_t part = 0;
    for (int n = 1; n <= ncap; ++n) part = std::max(part, tc_partial_floats(B->tcA, n));
    B->tc_ent = best;
    B->tc_ncap = ncap;
    ok = (B->d_tc_x = B->alloc<long long>(ncap)) && (B->d_tc_y = B->alloc<long long>(ncap)) &&
         (B->tc_partial = B->alloc<float>(part)) && (B->tc_err = B->alloc<int>(1)) &&
         (B->d_jlist_rest = B->alloc<int>(jp.size())) &&
         cudaMemset(B->tc_err, 0, sizeof(int)) == cudaSuccess &&
         cudaMallocHost(&B->tc_pin, sizeof(long long) * 2 * ncap) == cudaSuccess &&
         cudaMallocHost(&B->jpin_rest, sizeof(int) * std::max<size_t>(1, jp.size())) == cudaSuccess;
  }
  // vector chunks, each inside one problem
  // 1024-element chunks: enough CTAs for batches of small problems (256 was measured slower: the
  // per-CTA coefficient loads and the per-problem reduction grow with the chunk count)
  const long long chunk = 1024;
  std::vector<int> cprob, pchunk(1, 0);
  std::vector<long long> cs, ce;
  for (int p = 0; p < K; ++p) {
    for (long long a = B->voff[p]; a < B->voff[p + 1]; a += chunk) {
      cprob.push_back(p);
      cs.push_back(a);
      ce.push_back(std::min(B->voff[p + 1], a + chunk));
    }
    pchunk.push_back((int)cprob.size());
  }
  int *dcp = nullptr, *dpc = nullptr;
  long long *dcs = nullptr, *dce = nullptr;
  B->cprob_host = cprob;
  ok = ok && put(B, dcp, cprob) && put(B, dpc, pchunk) && put(B, dcs, cs) && put(B, dce, ce) &&
       (B->d_cchunk = B->alloc<int>(cprob.size()));
  if (ok) {
    B->seg.K = K;
    B->seg.nchunks = (int)cprob.size();
    B->seg.chunk = (int)chunk;
    B->seg.prob = dcp;
    B->seg.start = dcs;
    B->seg.end = dce;
    B->seg.pchunk = dpc;
    B->seg.active = B->d_active;
    B->seg.list = B->d_cchunk;
    B->seg.nlist = 0;
    B->seg.counter = B->alloc<unsigned>(K);
    ok = ok && B->seg.counter && cudaMemset(B->seg.counter, 0, sizeof(unsigned) * K) == cudaSuccess;
  }
  const long long n = B->n_total;
  ok = ok && (B->wb = B->alloc<double>(n)) && (B->x = B->alloc<double>(n)) && (B->r = B->alloc<double>(n)) &&
       (B->e = B->alloc<double>(n)) && (B->w = B->alloc<double>(n)) && (B->lh = B->alloc<double>(B->u_total)) &&
       (B->tmp = B->alloc<double>(B->t_total)) && (B->lam = B->alloc<double>(B->u_total)) &&
       (B->partial = B->alloc<double>((size_t)kMaxBatchVec * B->seg.nchunks)) &&
       (B->hbuf = B->alloc<double>((size_t)(2 * kMaxBatchVec + 1) * K)) &&
       (B->coef = B->alloc<double>((size_t)kMaxBatchVec * K)) && (B->scl = B->alloc<double>(K)) &&
       (B->x2 = B->alloc<float2>(n)) && (B->t2 = B->alloc<float2>(B->t_total)) &&
       (B->pparts = B->alloc<double>((size_t)kPairMaxParts * n));
  B->boff.assign(K + 1, 0);
  for (int p = 0; p < K; ++p) B->boff[p + 1] = B->boff[p] + 3LL * ctxs[p]->P;
  ok = ok && (B->bc_v = B->alloc<double>(B->boff[K])) && (B->bc_w = B->alloc<double>(B->boff[K])) &&
       (B->out_F = B->alloc<double>(B->boff[K])) && (B->out_T = B->alloc<double>(B->boff[K]));
  ok = ok && cudaMallocHost(&B->hpin, sizeof(double) * (2 * kMaxBatchVec + 1) * K) == cudaSuccess &&
       cudaMallocHost(&B->apin, sizeof(int) * K) == cudaSuccess &&
       cudaMallocHost(&B->cpin, sizeof(int) * std::max<size_t>(1, B->cprob_host.size())) == cudaSuccess &&
       cudaEventCreateWithFlags(&B->ev, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    delete B;
    return c0->fail(MFS_ERR_OOM, "device allocation failed: batch plan");
  }
  out = B;
  return MFS_OK;
}

// whether the refinement residual of a solve uses the double-float operator
static bool dw_residual(const mfs_solve_opts& o) {
  if (o.precision != MFS_MIXED) return false;
  if (o.residual == MFS_RESIDUAL_SOLVE) return true;
  if (o.residual == MFS_RESIDUAL_FP64) return false;
  return o.tol >= MFS_DW_RESIDUAL_MIN_TOL;
}

struct BatchRun {
  mfs_ctx* c0;
  BatchPlan* B;
  cudaStream_t st;
  bool dw;
  bool fast_a;           // with dw: Sigma^+ U^T from its FP32 copy
  std::vector<int> act;  // host copy of the active flags
  bool x2_ready = false;  // with dw: the apply's input already split into B->x2 (by the scaling)
};

// Active flags and the compacted pair work lists of the active problems.
mfs_status set_active(BatchRun& R, const std::vector<int>& a) {
  BatchPlan* B = R.B;
  if (!R.act.empty() && R.act == a) return MFS_OK;
  R.act = a;
  for (int p = 0; p < B->K; ++p) B->apin[p] = a[p];
  int n4 = 0, n1 = 0;
  int2* w4 = B->wpin;
  int2* w1 = B->wpin + B->w4_host.size();
  for (const int2& w : B->w4_host)
    if (a[w.x]) w4[n4++] = w;
  for (const int2& w : B->w1_host)
    if (a[w.x]) w1[n1++] = w;
  B->n_cwork = n4;
  B->n_cwork1 = n1;
  // the active problems of a context in chunks of up to kPairRhs: a chunk of two or more shares
  // the pair kernel's work items, a problem alone keeps the single-problem kernel
  {
    int nm = 0, nr = 0, ns = 0;
    std::vector<char> single(B->K, 0);
    B->rhs_shared.assign(B->K, 1);
    for (int L = 0; L < B->K; ++L) {
      if (B->leader[L] != L) continue;
      std::vector<int> mem;
      for (int p = L; p < B->K; ++p)
        if (B->leader[p] == L && a[p]) mem.push_back(p);
      for (size_t c0 = 0; c0 < mem.size(); c0 += kPairRhs) {
        const int cnt = (int)std::min<size_t>(kPairRhs, mem.size() - c0);
        if (cnt == 1) {
          single[mem[c0]] = 1;
          continue;
        }
        const int r0 = nr;
        for (int q = 0; q < cnt; ++q) {
          B->rhs_pin[nr++] = mem[c0 + q];
          B->rhs_shared[mem[c0 + q]] = cnt;
        }
        for (int t = 0; t < B->tiles1[L]; ++t) B->mwork_pin[nm++] = make_int4(L, t, r0, cnt);
      }
    }
    for (const int2& w : B->w1_host)
      if (single[w.x]) B->swork_pin[ns++] = w;
    B->n_mwork = nm;
    B->n_swork1 = ns;
    if (nm) {
      CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_mwork, B->mwork_pin, sizeof(int4) * nm, cudaMemcpyHostToDevice, R.st));
      CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_rhs, B->rhs_pin, sizeof(int) * nr, cudaMemcpyHostToDevice, R.st));
    }
    if (ns) CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_swork1, B->swork_pin, sizeof(int2) * ns, cudaMemcpyHostToDevice, R.st));
  }
  int nc = 0;
  for (int b = 0; b < (int)B->cprob_host.size(); ++b)
    if (a[B->cprob_host[b]]) B->cpin[nc++] = b;
  B->seg.nlist = nc;
  // GEMV jobs of the active problems (the launches' grids cover only those)
  int nj = 0;
  for (int j = 0; j < (int)B->jprob_host.size(); ++j)
    if (a[B->jprob_host[j]]) B->jpin[nj++] = j;
  for (GemvBatch<double>* g : {&B->gA, &B->gV}) {
    g->job_list = B->d_jlist;
    g->n_list = nj;
  }
  B->gA32.job_list = B->d_jlist;
  B->gA32.n_list = nj;
  if (B->tc_ncap > 0) {
    // the FP32 GEMV covers the jobs that are not tensor columns; the columns of the active
    // problems go to the tensor-core product
    int nr = 0, nt = 0;
    for (int j = 0; j < (int)B->jprob_host.size(); ++j)
      if (a[B->jprob_host[j]] && !B->jtc_host[j]) B->jpin_rest[nr++] = j;
    for (int i = 0; i < B->tc_ncap; ++i)
      if (a[B->tc_prob[i]]) {
        B->tc_pin[nt] = B->tc_x_host[i];
        B->tc_pin[B->tc_ncap + nt] = B->tc_y_host[i];
        ++nt;
      }
    B->gA32.job_list = B->d_jlist_rest;
    B->gA32.n_list = nr;
    B->tc_nact = nt;
    if (nr) CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_jlist_rest, B->jpin_rest, sizeof(int) * nr, cudaMemcpyHostToDevice, R.st));
    if (nt) {
      CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_tc_x, B->tc_pin, sizeof(long long) * nt, cudaMemcpyHostToDevice, R.st));
      CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_tc_y, B->tc_pin + B->tc_ncap, sizeof(long long) * nt, cudaMemcpyHostToDevice,
                                     R.st));
    }
  }
  CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_active, B->apin, sizeof(int) * B->K, cudaMemcpyHostToDevice, R.st));
  if (nj) CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_jlist, B->jpin, sizeof(int) * nj, cudaMemcpyHostToDevice, R.st));
  if (nc) CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_cchunk, B->cpin, sizeof(int) * nc, cudaMemcpyHostToDevice, R.st));
  if (n4) CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_cwork, w4, sizeof(int2) * n4, cudaMemcpyHostToDevice, R.st));
  if (n1) CUDA_TRY(R.c0, cudaMemcpyAsync(B->d_cwork1, w1, sizeof(int2) * n1, cudaMemcpyHostToDevice, R.st));
  // the pinned staging buffers are rewritten by the next call: wait for these copies
  CUDA_TRY(R.c0, cudaStreamSynchronize(R.st));
  return MFS_OK;
}

// out = G_hat in for every problem the device flags mark active (the host's R.act picks the tiling)
void batch_apply_kernels(BatchRun& R, const double* in, double* out) {
  mfs_ctx* c = R.c0;
  BatchPlan* B = R.B;
  timed(c, c->ev_gemv, [&] {
    if (R.dw) {
      if (!R.x2_ready) launch_split_dw(B->n_total, in, B->x2, R.st);
      if (R.fast_a) {
        launch_gemv_f32_dw(B->gA32, B->x2, B->t2, R.st);
        if (B->tc_nact > 0) {
          launch_tc_gemm(B->tcA, B->tc_nact, in, B->d_tc_x, B->d_tc_y, nullptr, B->t2, B->tc_partial, B->tc_err, true,
                         R.st);
          c->tm.tc_launches += 1;
          c->tm.tc_columns += B->tc_nact;
        }
      } else {
        launch_gemv_dw(B->gA, B->x2, B->t2, nullptr, R.st);
      }
      launch_gemv_dw(B->gV, B->t2, nullptr, B->lh, R.st);
    } else {
      launch_gemv<double>(B->gA, in, B->tmp, R.st);
      launch_gemv<double>(B->gV, B->tmp, B->lh, R.st);
    }
  });
  long long active_tiles = 0, min_others = -1;
  for (int p = 0; p < B->K; ++p)
    if (R.act[p]) {
      active_tiles += B->tiles4[p];
      if (B->others_p[p] > 0) min_others = min_others < 0 ? B->others_p[p] : std::min(min_others, B->others_p[p]);
    }
  const int nt = pair_nodes_per_thread((int)std::min<long long>(active_tiles, 1 << 30));
  // few tiles left (the lockstep tail): split each tile's sources over several CTAs
  const int parts = R.dw && nt == 1 && min_others > 0 ? pair_split_parts(B->n_cwork1, min_others, kPairMaxParts) : 1;
  timed(c, c->ev_pair, [&] {
    if (R.dw && B->n_mwork > 0) {
      // right-hand sides on one geometry share the pair evaluations; the problems left single
      // run the 1-node-per-thread kernel with the same source split, one reduction for both
      const long long items = (long long)B->n_mwork + B->n_swork1;
      const int mparts = min_others > 0 ? pair_split_parts(items, min_others, kPairMaxParts) : 1;
      // (with split sources the last CTA of each item adds the parts)
      launch_pairs_multi64(B->d_args1, B->d_mwork, B->n_mwork, B->d_rhs, B->d_active, B->lh, in, out, B->d_uoff,
                           B->d_voff, mparts, B->pparts, B->n_total, B->d_nlen, R.st, B->d_pcount);
      launch_pairs_batch64(true, B->d_args1, B->d_swork1, B->n_swork1, B->d_active, 1, B->lh, in, out, B->d_uoff,
                           B->d_voff, mparts, B->pparts, B->n_total, B->seg, R.st, B->d_nlen, true, B->d_pcount);
    } else if (nt == 4)
      launch_pairs_batch64(R.dw, B->d_args, B->d_cwork, B->n_cwork, B->d_active, 4, B->lh, in, out, B->d_uoff,
                           B->d_voff, 1, nullptr, 0, B->seg, R.st);
    else
      launch_pairs_batch64(R.dw, B->d_args1, B->d_cwork1, B->n_cwork1, B->d_active, 1, B->lh, in, out, B->d_uoff,
                           B->d_voff, parts, B->pparts, B->n_total, B->seg, R.st, B->d_nlen, false, B->d_pcount);
  });
  // mobility problems: the rigid motion of the border unknowns, and their force/torque rows
  // (the bordered operator of the single solves, problem by problem)
  for (int p = 0; p < B->K; ++p)
    if (B->mob[p] && R.act[p]) {
      mfs_ctx* cp = B->key[p];
      const double a = cp->a, mu = cp->hd.prm.visc;
      launch_rigid_sub(cp->tg.n, cp->d_owner, cp->tg.pos64, in + B->voff[p] + B->nlen[p], out + B->voff[p], R.st);
      launch_forces_torques_scaled(cp->src, B->lh + B->uoff[p], out + B->voff[p] + B->nlen[p],
                                   out + B->voff[p] + B->nlen[p] + 3, 6, 1.0 / (6.0 * kPi * mu * a),
                                   1.0 / (8.0 * kPi * mu * a * a * a), R.st);
    }
  c->tm.gemv_launches += 2;
  c->tm.pair_launches += 1;
  c->tm.pair_kind = R.dw ? MFS_MIXED : MFS_FP64;
  const int kind = c->tm.pair_kind;
  c->tm.by_kind_launches[kind] += 1;
  if (c->prof) c->ev_pair_kind.push_back(kind);
}

// work counters of one batched apply over the problems of `act`
void batch_apply_count(BatchRun& R, const std::vector<int>& act) {
  mfs_ctx* c = R.c0;
  BatchPlan* B = R.B;
  const int kind = R.dw ? MFS_MIXED : MFS_FP64;
  std::vector<int> per_ctx(B->K, 0);
  for (int p = 0; p < B->K; ++p)
    if (act[p]) {
      if (R.dw) {
        // a geometry shared by r right-hand sides is evaluated once for all of them
        const int r = B->n_mwork > 0 && (int)B->rhs_shared.size() == B->K ? B->rhs_shared[p] : 1;
        c->tm.pair_issued_flops += (double)B->proxy_p[p] * (kDwPairRhsFlops + kDwPairGeomFlops / r) +
                                   (double)B->image_p[p] * (kDwTripleRhsFlops + kDwTripleGeomFlops / r);
        if (r > 1) c->tm.pair_shared_rhs += B->pairs_p[p];
      }
      c->tm.pair_interactions += B->pairs_p[p];
      c->tm.pair_proxy += B->proxy_p[p];
      c->tm.pair_image_nodes += B->image_p[p];
      c->tm.by_kind_proxy[kind] += B->proxy_p[p];
      c->tm.by_kind_image_nodes[kind] += B->image_p[p];
      ++per_ctx[B->leader[p]];
    }
  // factor bytes: the right-hand sides on one geometry run their jobs of a factor in adjacent
  // CTAs, which read it from HBM once (the others hit L2): one read per context and apply
  for (int p = 0; p < B->K; ++p)
    if (per_ctx[p] > 0) c->tm.gemv_bytes += (R.dw && R.fast_a ? B->bA32_p[p] : B->bA2_p[p]) + B->bV_p[p];
}

// Gram-Schmidt traffic of Arnoldi step j over the problems of `act`: two dot-product launches
// against the j + 1 basis vectors (read (j + 1) n and w's n doubles each) and two updates
// (read (j + 1) n, read and write w's n each), n the active problems' summed length
void batch_krylov_count(BatchRun& R, const std::vector<int>& act, int j) {
  BatchPlan* B = R.B;
  long long n_act = 0;
  for (int p = 0; p < B->K; ++p)
    if (act[p]) n_act += B->voff[p + 1] - B->voff[p];
  R.c0->tm.krylov_launches += 4;
  R.c0->tm.krylov_bytes += 8.0 * (4.0 * j + 10.0) * (double)n_act;
}

void batch_apply(BatchRun& R, const double* in, double* out) {
  batch_apply_kernels(R, in, out);
  batch_apply_count(R, R.act);
}

// per-problem 2-norms of v (active problems; others 0)
mfs_status batch_norms(BatchRun& R, const double* v, std::vector<double>& nrm) {
  BatchPlan* B = R.B;
  double* hn = B->hbuf + (size_t)2 * kMaxBatchVec * B->K;
  launch_seg_dots(B->seg, 1, v, B->n_total, v, B->partial, hn, R.st);
  CUDA_TRY(R.c0, cudaMemcpyAsync(B->hpin, hn, sizeof(double) * B->K, cudaMemcpyDeviceToHost, R.st));
  CUDA_TRY(R.c0, cudaStreamSynchronize(R.st));
  nrm.assign(B->K, 0.0);
  // a NaN stays NaN (std::max would turn it into 0 and hide non-finite data)
  for (int p = 0; p < B->K; ++p) {
    const double h = B->hpin[p];
    nrm[p] = R.act[p] ? (std::isnan(h) ? h : std::sqrt(std::max(0.0, h))) : 0.0;
  }
  return MFS_OK;
}

constexpr int kSyncEvery = 4;  // lockstep GMRES steps between host synchronisations

// Device GMRES state for `restart` steps (kept across calls, grown when needed).
mfs_status ensure_givens(BatchRun& R, int restart) {
  BatchPlan* B = R.B;
  if (B->gs_restart >= restart && B->snap) return MFS_OK;
  for (void* q : B->gs_allocs) cudaFree(q);
  B->gs_allocs.clear();
  B->gs_restart = 0;
  const int K = B->K, ldh = restart + 1;
  auto get = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    B->gs_allocs.push_back(q);
    return q;
  };
  GivensState& S = B->gs;
  S.K = K;
  S.ldh = ldh;
  S.restart = restart;
  S.H = (double*)get(sizeof(double) * (size_t)K * restart * ldh);
  S.cs = (double*)get(sizeof(double) * (size_t)K * restart);
  S.sn = (double*)get(sizeof(double) * (size_t)K * restart);
  S.g = (double*)get(sizeof(double) * (size_t)K * ldh);
  S.bn = (double*)get(sizeof(double) * K);
  S.tol = (double*)get(sizeof(double) * K);
  S.est = (double*)get(sizeof(double) * K);
  S.iters = (int*)get(sizeof(int) * K);
  S.jused = (int*)get(sizeof(int) * K);
  S.err = (int*)get(sizeof(int));
  S.active = B->d_active;
  S.scl = B->scl;
  if (!S.H || !S.cs || !S.sn || !S.g || !S.bn || !S.tol || !S.est || !S.iters || !S.jused || !S.err)
    return R.c0->fail(MFS_ERR_OOM, "device allocation failed: batched GMRES state");
  // snapshots, then one slot for the error flag
  if (!B->snap && cudaMallocHost(&B->snap, sizeof(int) * ((size_t)kSyncEvery * K + 1)) != cudaSuccess) {
    cudaGetLastError();
    return R.c0->fail(MFS_ERR_OOM, "pinned allocation failed: batched GMRES flags");
  }
  B->gs_restart = restart;
  return MFS_OK;
}

// One GMRES cycle (at most `restart` iterations) from x = 0 for the problems with solve[p] = 1.
// The Hessenberg updates, the convergence tests and the retirement of converged problems run on
// the device; the host synchronises every kSyncEvery steps to refresh its view of the active
// set (compacted launch lists, work counters) and to stop once every problem has converged.
mfs_status batch_gmres_cycle(BatchRun& R, const double* b, double* x, const std::vector<int>& solve,
                             const std::vector<double>& tol, int restart, int iter_budget, std::vector<int>& iters,
                             std::vector<double>& est) {
  BatchPlan* B = R.B;
  mfs_ctx* c = R.c0;
  const int K = B->K;
  const long long n = B->n_total;
  const int ldh = restart + 1;
  mfs_status s;
  size_t need = (size_t)(restart + 1) * (size_t)n;
  if (B->basis_cap < need) {
    if (B->basis) cudaFree(B->basis);
    B->basis = nullptr;
    B->basis_cap = 0;
    if (cudaMalloc(&B->basis, need * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return c->fail(MFS_ERR_OOM, "device allocation failed: batched Krylov basis");
    }
    B->basis_cap = need;
  }
  if ((s = ensure_givens(R, restart)) != MFS_OK) return s;
  GivensState S = B->gs;
  S.ldh = ldh;
  S.restart = restart;
  double* V = B->basis;
  CUDA_TRY(c, cudaMemsetAsync(x, 0, sizeof(double) * n, R.st));
  if ((s = set_active(R, solve)) != MFS_OK) return s;
  std::vector<double> bn;
  if ((s = batch_norms(R, b, bn)) != MFS_OK) return s;
  std::vector<int> act(solve);
  for (int p = 0; p < K; ++p)
    if (act[p] && !(bn[p] > 0)) {
      if (!std::isfinite(bn[p])) return c->fail(MFS_ERR_NUMERIC, "right-hand side is not finite");
      act[p] = 0;
    }
  if ((s = set_active(R, act)) != MFS_OK) return s;
  const std::vector<int> started(act);
  // initial state: V_0 = b / ||b||, g = (||b||, 0, ...)
  std::vector<double> sc(K, 0.0), g0((size_t)K * ldh, 0.0), bnd(K, 1.0);
  for (int p = 0; p < K; ++p)
    if (act[p]) {
      sc[p] = 1.0 / bn[p];
      g0[(size_t)p * ldh] = bn[p];
      bnd[p] = bn[p];
      est[p] = 1.0;
    }
  CUDA_TRY(c, cudaMemcpyAsync(B->scl, sc.data(), sizeof(double) * K, cudaMemcpyHostToDevice, R.st));
  CUDA_TRY(c, cudaMemcpyAsync(S.g, g0.data(), sizeof(double) * g0.size(), cudaMemcpyHostToDevice, R.st));
  CUDA_TRY(c, cudaMemcpyAsync(const_cast<double*>(S.bn), bnd.data(), sizeof(double) * K, cudaMemcpyHostToDevice, R.st));
  CUDA_TRY(c, cudaMemcpyAsync(const_cast<double*>(S.tol), tol.data(), sizeof(double) * K, cudaMemcpyHostToDevice, R.st));
  CUDA_TRY(c, cudaMemsetAsync(S.iters, 0, sizeof(int) * K, R.st));
  CUDA_TRY(c, cudaMemsetAsync(S.jused, 0, sizeof(int) * K, R.st));
  CUDA_TRY(c, cudaMemsetAsync(S.err, 0, sizeof(int), R.st));
  // v_0 = b / ||b||, split for the first double-float apply at the same time
  if (R.dw) launch_seg_scale_split(B->seg, B->scl, b, V, B->x2, R.st);
  else launch_seg_scale(B->seg, B->scl, b, V, R.st);
  double* h1 = B->hbuf;
  double* h2 = B->hbuf + (size_t)kMaxBatchVec * K;
  double* hn = B->hbuf + (size_t)2 * kMaxBatchVec * K;
  // the steps since the last synchronisation: flags after each step, for the work counters
  std::vector<int> window_start(act);
  int in_window = 0, used = 0, last_j = -1;
  bool any = true;
  for (int j = 0; j < restart && used < iter_budget && any; ++j) {
    last_j = j;
    double* w = V + (size_t)(j + 1) * n;
    R.x2_ready = R.dw;
    batch_apply_kernels(R, V + (size_t)j * n, w);
    R.x2_ready = false;
    timed(c, c->ev_krylov, [&] {
      launch_seg_dots(B->seg, j + 1, V, n, w, B->partial, h1, R.st);
      launch_seg_update(B->seg, j + 1, V, n, h1, -1.0, w, R.st);
      launch_seg_dots(B->seg, j + 1, V, n, w, B->partial, h2, R.st);
      launch_seg_update(B->seg, j + 1, V, n, h2, -1.0, w, R.st);
    });
    launch_seg_dots(B->seg, 1, w, n, w, B->partial, hn, R.st);
    launch_batch_givens(S, j, h1, h2, hn, R.st);
    // v_{j+1} = w / h_{j+1,j}, split for the next apply
    if (R.dw) launch_seg_scale_split(B->seg, B->scl, w, w, B->x2, R.st);
    else launch_seg_scale(B->seg, B->scl, w, w, R.st);
    CHECK_LAUNCH(c);
    CUDA_TRY(c, cudaMemcpyAsync(B->snap + (size_t)in_window * K, B->d_active, sizeof(int) * K, cudaMemcpyDeviceToHost,
                                R.st));
    ++in_window;
    ++used;
    if (in_window == kSyncEvery || j + 1 == restart || used >= iter_budget) {
      int* herr = B->snap + (size_t)kSyncEvery * K;
      CUDA_TRY(c, cudaMemcpyAsync(herr, S.err, sizeof(int), cudaMemcpyDeviceToHost, R.st));
      CUDA_TRY(c, cudaStreamSynchronize(R.st));
      if (*herr) return c->fail(MFS_ERR_NUMERIC, "non-finite value in the batched Arnoldi process");
      // the apply of each step ran over the flags left by the step before it
      std::vector<int> cur(window_start);
      for (int t = 0; t < in_window; ++t) {
        batch_apply_count(R, cur);
        batch_krylov_count(R, cur, j - in_window + 1 + t);
        cur.assign(B->snap + (size_t)t * K, B->snap + (size_t)(t + 1) * K);
      }
      in_window = 0;
      window_start = cur;
      any = false;
      for (int p = 0; p < K; ++p) any = any || cur[p];
      if (any && (s = set_active(R, cur)) != MFS_OK) return s;
    }
  }
  // the device flags were changed by the Givens kernel: the next set_active must upload
  R.act.clear();
  if (in_window > 0) {
    // left the loop between synchronisations (every problem converged): count the last steps
    CUDA_TRY(c, cudaStreamSynchronize(R.st));
    std::vector<int> cur(window_start);
    for (int t = 0; t < in_window; ++t) {
      batch_apply_count(R, cur);
      batch_krylov_count(R, cur, last_j - in_window + 1 + t);
      cur.assign(B->snap + (size_t)t * K, B->snap + (size_t)(t + 1) * K);
    }
  }
  // per-problem counts and estimates, then x = V y with y = R^{-1} g
  std::vector<int> it_dev(K), jused(K);
  std::vector<double> est_dev(K);
  CUDA_TRY(c, cudaMemcpyAsync(it_dev.data(), S.iters, sizeof(int) * K, cudaMemcpyDeviceToHost, R.st));
  CUDA_TRY(c, cudaMemcpyAsync(jused.data(), S.jused, sizeof(int) * K, cudaMemcpyDeviceToHost, R.st));
  CUDA_TRY(c, cudaMemcpyAsync(est_dev.data(), S.est, sizeof(double) * K, cudaMemcpyDeviceToHost, R.st));
  CUDA_TRY(c, cudaStreamSynchronize(R.st));
  int jmax = 0;
  for (int p = 0; p < K; ++p) {
    if (!started[p]) continue;
    iters[p] += it_dev[p];
    if (jused[p] > 0) est[p] = est_dev[p];
    jmax = std::max(jmax, jused[p]);
  }
  if (jmax == 0) return MFS_OK;
  launch_batch_backsolve(S, jmax, B->coef, R.st);
  if ((s = set_active(R, started)) != MFS_OK) return s;
  launch_seg_update(B->seg, jmax, V, n, B->coef, 1.0, x, R.st);
  CHECK_LAUNCH(c);
  return MFS_OK;
}

// Boundary data and outputs of a batch: from and to the contexts themselves (distinct contexts),
// or per problem from caller arrays (contexts may repeat: several right-hand sides per geometry).
struct BatchIO {
  const double* const* v = nullptr;  // null: take each context's own boundary data
  const double* const* w = nullptr;
  bool in_device = false;
  double* const* F = nullptr;        // null: forces/torques go to the contexts
  double* const* T = nullptr;
  bool out_device = false;
  bool repeats = false;
};

mfs_status batch_lockstep_impl(int K, mfs_ctx* const* ctxs, const mfs_solve_opts& o, mfs_solve_info* infos,
                               const BatchIO& io) {
  auto t0 = std::chrono::steady_clock::now();
  mfs_ctx* c0 = ctxs[0];
  for (int p = 0; p < K; ++p) {
    mfs_status s = check_state(ctxs[p], 2);
    if (s != MFS_OK) return s;
    if (!ctxs[p]->factored) return ctxs[p]->fail(MFS_ERR_STATE, "built without one-body factors (build_factors = 0)");
    // a context in the mobility mode (forces and torques prescribed) joins as a mobility problem,
    // unless the batch brings its own rigid velocities
    if (ctxs[p]->device != c0->device) return c0->fail(MFS_ERR_ARG, "batched contexts must share one device");
    if (!io.repeats)
      for (int q = 0; q < p; ++q)
        if (ctxs[q] == ctxs[p]) return c0->fail(MFS_ERR_ARG, "a context appears twice in the batch");
  }
  if (o.restart < 1 || o.restart + 1 > kMaxBatchVec || !(o.tol > 0) || o.max_iter < 1 || o.max_refine < 0 ||
      o.residual < MFS_RESIDUAL_AUTO || o.residual > MFS_RESIDUAL_SOLVE)
    return c0->fail(MFS_ERR_ARG, "invalid solve options (restart must be in [1, 511])");
  check_state(c0, 2);
  // reuse the cached plan when the same contexts with the same builds come back
  std::vector<int> mob(K, 0);
  for (int p = 0; p < K; ++p) mob[p] = !io.v && ctxs[p]->mode == 1 ? 1 : 0;
  BatchPlan* B = c0->batch;
  bool same = B && B->K == K && B->mob == mob;
  for (int p = 0; same && p < K; ++p) same = B->key[p] == ctxs[p] && B->key_build[p] == ctxs[p]->build_id;
  if (!same) {
    if (B) delete B;
    c0->batch = nullptr;
    mfs_status s = make_plan(c0, K, ctxs, mob, B);
    if (s != MFS_OK) return s;
    c0->batch = B;
  }
  BatchRun R{c0, B, c0->stream, o.precision == MFS_MIXED, o.precision == MFS_MIXED, std::vector<int>()};  // act empty: the first set_active uploads
  // order after the work already queued on every context's stream
  for (int p = 0; p < K; ++p)
    if (ctxs[p]->stream != R.st) {
      CUDA_TRY(c0, cudaEventRecord(B->ev, ctxs[p]->stream));
      CUDA_TRY(c0, cudaStreamWaitEvent(R.st, B->ev, 0));
    }
  for (int p = 0; p < K; ++p) {
    mfs_ctx* c = ctxs[p];
    const size_t bytes = sizeof(double) * 3 * c->P;
    if (io.v) {
      const cudaMemcpyKind kind = io.in_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
      if (!io.v[p] || !io.w[p]) return c0->fail(MFS_ERR_ARG, "null boundary data in the batch");
      CUDA_TRY(c0, cudaMemcpyAsync(B->bc_v + B->boff[p], io.v[p], bytes, kind, R.st));
      CUDA_TRY(c0, cudaMemcpyAsync(B->bc_w + B->boff[p], io.w[p], bytes, kind, R.st));
    } else if (mob[p]) {
      // fixed spheres in the background flow, then the prescribed (scaled) forces and torques
      CUDA_TRY(c0, cudaMemcpyAsync(B->bc_v + B->boff[p], c->d_zero, bytes, cudaMemcpyDeviceToDevice, R.st));
      CUDA_TRY(c0, cudaMemcpyAsync(B->bc_w + B->boff[p], c->d_zero, bytes, cudaMemcpyDeviceToDevice, R.st));
      CUDA_TRY(c0, cudaMemcpyAsync(B->wb + B->voff[p] + B->nlen[p], c->d_border, sizeof(double) * 6 * c->P,
                                   cudaMemcpyDeviceToDevice, R.st));
    } else {
      CUDA_TRY(c0, cudaMemcpyAsync(B->bc_v + B->boff[p], c->d_v, bytes, cudaMemcpyDeviceToDevice, R.st));
      CUDA_TRY(c0, cudaMemcpyAsync(B->bc_w + B->boff[p], c->d_om, bytes, cudaMemcpyDeviceToDevice, R.st));
    }
    launch_rhs(c->tg.n, c->d_colloc_abs, c->d_owner, c->d_sqrtw, c->src.cen64, B->bc_v + B->boff[p],
               B->bc_w + B->boff[p], c->bg.data(), B->wb + B->voff[p], R.st);
  }
  CHECK_LAUNCH(c0);
  mfs_status s;
  std::vector<int> all(K, 1);
  if ((s = set_active(R, all)) != MFS_OK) return s;
  std::vector<double> bnorm, rn;
  if ((s = batch_norms(R, B->wb, bnorm)) != MFS_OK) return s;
  const long long n = B->n_total;
  CUDA_TRY(c0, cudaMemsetAsync(B->x, 0, sizeof(double) * n, R.st));
  CUDA_TRY(c0, cudaMemcpyAsync(B->r, B->wb, sizeof(double) * n, cudaMemcpyDeviceToDevice, R.st));
  std::vector<double> rel(K), est(K, 0.0);
  std::vector<int> iters(K, 0), refines(K, 0), stalled(K, 0);
  for (int p = 0; p < K; ++p) {
    if (!std::isfinite(bnorm[p])) return ctxs[p]->fail(MFS_ERR_NUMERIC, "boundary data is not finite");
    rel[p] = bnorm[p] > 0 ? 1.0 : 0.0;
  }
  const int max_outer = std::max(o.max_refine, o.max_iter / o.restart + 2);
  int total_iters = 0;
  for (int outer = 0; outer < max_outer; ++outer) {
    std::vector<int> solve_p(K, 0);
    std::vector<double> tol_p(K, 0.5);
    bool any = false;
    for (int p = 0; p < K; ++p) {
      solve_p[p] = rel[p] > o.tol && !stalled[p];
      tol_p[p] = solve_p[p] ? std::min(0.5, kInnerTol * o.tol / rel[p]) : 0.5;
      any = any || solve_p[p];
    }
    if (!any || total_iters >= o.max_iter) break;
    std::vector<int> it_before(iters);
    if ((s = batch_gmres_cycle(R, B->r, B->e, solve_p, tol_p, o.restart, o.max_iter - total_iters, iters, est)) != MFS_OK)
      return s;
    int cyc = 0;
    for (int p = 0; p < K; ++p) cyc = std::max(cyc, iters[p] - it_before[p]);
    total_iters += cyc;
    launch_axpy64(n, 1.0, B->e, B->x, R.st);
    // true residual of the problems solved in this pass (the others keep theirs; their
    // segments of r are overwritten with unused values below and never read again)
    std::vector<int> live(K);
    for (int p = 0; p < K; ++p) live[p] = bnorm[p] > 0 && solve_p[p];
    if ((s = set_active(R, live)) != MFS_OK) return s;
    {
      // refinement residual with the operator that dw_residual() picks (see mfs_solve)
      const bool dw = R.dw, fa = R.fast_a;
      R.dw = dw_residual(o);
      R.fast_a = false;
      batch_apply(R, B->x, B->w);
      R.dw = dw;
      R.fast_a = fa;
    }
    launch_sub((int)n, B->wb, B->w, B->r, R.st);
    CHECK_LAUNCH(c0);
    if ((s = batch_norms(R, B->r, rn)) != MFS_OK) return s;
    for (int p = 0; p < K; ++p) {
      if (!live[p]) continue;
      double prev = rel[p];
      rel[p] = rn[p] / bnorm[p];
      if (!std::isfinite(rel[p])) return ctxs[p]->fail(MFS_ERR_NUMERIC, "residual is not finite");
      if (solve_p[p]) {
        if (outer > 0) ++refines[p];
        if (rel[p] >= prev && rel[p] > o.tol) stalled[p] = 1;  // a pass that gained nothing
      }
    }
  }
  if (B->tc_err) {
    int h = 0;
    CUDA_TRY(c0, cudaMemcpyAsync(&h, B->tc_err, sizeof(int), cudaMemcpyDeviceToHost, R.st));
    CUDA_TRY(c0, cudaStreamSynchronize(R.st));
    if (h) {
      CUDA_TRY(c0, cudaMemsetAsync(B->tc_err, 0, sizeof(int), R.st));
      return c0->fail(MFS_ERR_TIMEOUT, "tensor-core step 1: a pipeline wait ran out of time");
    }
  }
  // lambda = B^+ mu, then per-context outputs
  std::vector<int> live(K);
  for (int p = 0; p < K; ++p) live[p] = 1;
  if ((s = set_active(R, live)) != MFS_OK) return s;
  timed(c0, c0->ev_gemv, [&] {
    if (o.precision == MFS_MIXED) {
      // double-float factors (~2^-46 relative) instead of the FP64 pipes
      launch_split_dw(B->n_total, B->x, B->x2, R.st);
      launch_gemv_dw(B->gA, B->x2, B->t2, nullptr, R.st);
      launch_gemv_dw(B->gV, B->t2, nullptr, B->lam, R.st);
    } else {
      launch_gemv<double>(B->gA, B->x, B->tmp, R.st);
      launch_gemv<double>(B->gV, B->tmp, B->lam, R.st);
    }
  });
  for (int p = 0; p < K; ++p) {
    mfs_ctx* c = ctxs[p];
    // each context keeps the solution of its last problem in the batch
    CUDA_TRY(c0, cudaMemcpyAsync(c->d_mu, B->x + B->voff[p], sizeof(double) * (B->voff[p + 1] - B->voff[p]),
                                 cudaMemcpyDeviceToDevice, R.st));
    if (B->mob[p]) {
      // rigid velocities from the border unknowns (V_k, Omega_k) per sphere
      const double* xb = B->x + B->voff[p] + B->nlen[p];
      CUDA_TRY(c0, cudaMemcpy2DAsync(c->d_v, 3 * sizeof(double), xb, 6 * sizeof(double), 3 * sizeof(double), c->P,
                                     cudaMemcpyDeviceToDevice, R.st));
      CUDA_TRY(c0, cudaMemcpy2DAsync(c->d_om, 3 * sizeof(double), xb + 3, 6 * sizeof(double), 3 * sizeof(double), c->P,
                                     cudaMemcpyDeviceToDevice, R.st));
    }
    CUDA_TRY(c0, cudaMemcpyAsync(c->d_lam, B->lam + B->uoff[p], sizeof(double) * c->n_unk, cudaMemcpyDeviceToDevice, R.st));
    launch_forces_torques(c->src, B->lam + B->uoff[p], B->out_F + B->boff[p], B->out_T + B->boff[p], R.st);
    const size_t bytes = sizeof(double) * 3 * c->P;
    CUDA_TRY(c0, cudaMemcpyAsync(c->d_F, B->out_F + B->boff[p], bytes, cudaMemcpyDeviceToDevice, R.st));
    CUDA_TRY(c0, cudaMemcpyAsync(c->d_T, B->out_T + B->boff[p], bytes, cudaMemcpyDeviceToDevice, R.st));
    if (io.F && io.F[p])
      CUDA_TRY(c0, cudaMemcpyAsync(io.F[p], B->out_F + B->boff[p], bytes,
                                   io.out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, R.st));
    if (io.T && io.T[p])
      CUDA_TRY(c0, cudaMemcpyAsync(io.T[p], B->out_T + B->boff[p], bytes,
                                   io.out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, R.st));
  }
  CHECK_LAUNCH(c0);
  CUDA_TRY(c0, cudaEventRecord(B->ev, R.st));
  for (int p = 0; p < K; ++p)
    if (ctxs[p]->stream != R.st) CUDA_TRY(c0, cudaStreamWaitEvent(ctxs[p]->stream, B->ev, 0));
  CUDA_TRY(c0, cudaStreamSynchronize(R.st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  mfs_status first = MFS_OK;
  for (int p = 0; p < K; ++p) {
    mfs_ctx* c = ctxs[p];
    c->solved = true;
    bool conv = rel[p] <= o.tol;
    if (infos) {
      infos[p].iters = iters[p];
      infos[p].refinements = refines[p];
      infos[p].rel_residual = rel[p];
      infos[p].seconds = secs;
      infos[p].converged = conv ? 1 : 0;
    }
    if (!conv) {
      char buf[160];
      std::snprintf(buf, sizeof buf, "not converged: relative residual %.3e after %d iterations", rel[p], iters[p]);
      c->fail(MFS_ERR_NOT_CONVERGED, buf);
      if (first == MFS_OK) first = MFS_ERR_NOT_CONVERGED;
    }
  }
  return first;
}

mfs_status batch_lockstep(int K, mfs_ctx* const* ctxs, const mfs_solve_opts& o, mfs_solve_info* infos,
                          const BatchIO& io = BatchIO()) {
  mfs_ctx* c0 = ctxs[0];
  const long long l0 = launches_on_this_thread();
  mfs_status s = batch_lockstep_impl(K, ctxs, o, infos, io);
  c0->tm.kernel_launches += launches_on_this_thread() - l0;
  if (c0->prof) {
    cudaStreamSynchronize(c0->stream);
    collect_events(c0);
  }
  return s;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

void mfs_default_params(mfs_params* p) {
  if (!p) return;
  p->n_proxy = 686;
  p->r_proxy = 0.63;
  p->m_basic = 823;
  p->delta_offset = 0.05;
  p->alpha1 = 6;
  p->alpha2 = 6;
  p->beta1 = kPi / 5.0;
  p->beta2 = kPi / 60.0;
  p->eps_trunc = 5e-12;
  p->nim_a = 8.72;
  p->nim_b = 6.15;
  p->nim_cut = 0.15;
  p->nim_max = 20;
  p->nim_fixed = -1;
  p->left_precond = 1;
  p->visc = 1.0;
  p->build_factors = 1;
  p->nim_min = 0;
  p->far_dist = 0.0;
  p->far_n_eq = 300;
  p->far_r_eq = 1.0;
  p->far_r_chk = 2.0;
  p->far_eps = 1e-6;
  p->tensor_step1 = 1;
}

void mfs_default_solve_opts(mfs_solve_opts* o) {
  if (!o) return;
  o->precision = MFS_MIXED;
  o->tol = 1e-6;
  o->max_iter = 2000;
  o->restart = 300;
  o->max_refine = 20;
  o->inner_tol = 1e-4;
  o->residual = MFS_RESIDUAL_AUTO;
}


mfs_status mfs_create(mfs_ctx** out, int device, void* cuda_stream) {
  if (!out) return MFS_ERR_ARG;
  *out = nullptr;
  mfs_ctx* c = new (std::nothrow) mfs_ctx();
  if (!c) return MFS_ERR_OOM;
  c->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MFS_ERR_CUDA;
  }
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return MFS_ERR_CUDA;
    }
    c->own_stream = true;
  }
  *out = c;
  return MFS_OK;
}

void mfs_destroy(mfs_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  delete c->batch;
  c->batch = nullptr;
  c->free_build();
  for (auto* lst : {&c->ev_pair, &c->ev_gemv, &c->ev_krylov, &c->ev_far, &c->ev_pool})
    for (auto& e : *lst) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  if (c->solver) cusolverDnDestroy(c->solver);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* mfs_last_error(const mfs_ctx* c) { return c ? c->err.c_str() : "null context"; }

mfs_status mfs_set_spheres(mfs_ctx* c, int P, const double* centres, const double* radii) {
  if (!c) return MFS_ERR_ARG;
  if (P <= 0 || !centres || !radii) return c->fail(MFS_ERR_ARG, "P must be positive and arrays non-null");
  double a = radii[0];
  if (!(a > 0) || !std::isfinite(a)) return c->fail(MFS_ERR_ARG, "radius must be positive");
  for (int k = 0; k < P; ++k) {
    if (std::fabs(radii[k] - a) > 1e-12 * a) return c->fail(MFS_ERR_UNSUPPORTED, "all spheres must have the same radius");
    for (int q = 0; q < 3; ++q)
      if (!std::isfinite(centres[3 * k + q])) return c->fail(MFS_ERR_ARG, "non-finite centre");
  }
  c->free_build();
  c->P = P;
  c->a = a;
  c->centres.assign(centres, centres + 3 * (size_t)P);
  c->state = 1;
  c->have_bc = false;
  c->err.clear();
  return MFS_OK;
}

mfs_status mfs_set_background_flow(mfs_ctx* c, const double* U, const double* E, const double* Om) {
  if (!c) return MFS_ERR_ARG;
  for (int i = 0; i < 9; ++i)
    if ((U && i < 3 && !std::isfinite(U[i])) || (E && !std::isfinite(E[i])) || (Om && i < 3 && !std::isfinite(Om[i])))
      return c->fail(MFS_ERR_ARG, "non-finite background flow");
  std::fill(c->bg.begin(), c->bg.end(), 0.0);
  if (U) std::copy(U, U + 3, c->bg.begin());
  if (E) std::copy(E, E + 9, c->bg.begin() + 3);
  if (Om) std::copy(Om, Om + 3, c->bg.begin() + 12);
  c->solved = false;
  return MFS_OK;
}

static mfs_status build_impl(mfs_ctx* c, const mfs_params* params);

mfs_status mfs_build(mfs_ctx* c, const mfs_params* params) {
  mfs_status s = check_state(c, 1);
  if (s != MFS_OK) return s;
  s = build_impl(c, params);
  if (s != MFS_OK) {
    // a failed build releases whatever it had allocated; the spheres stay set
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    c->free_build();
    c->state = 1;
  }
  return s;
}

static mfs_status build_impl(mfs_ctx* c, const mfs_params* params) {
  mfs_status s = MFS_OK;
  mfs_params p;
  if (params) p = *params; else mfs_default_params(&p);
  c->free_build();
  c->state = 1;
  HostDisc hd;
  s = build_discretisation(c->centres.data(), c->P, c->a, p, hd, c->err);
  if (s != MFS_OK) return s;
  c->hd = std::move(hd);
  HostDisc& d = c->hd;
  const int P = d.P, N = p.n_proxy, nc = d.n_colloc(), ni = d.n_img();
  c->n = 3 * nc;
  c->n_unk = d.n_unknowns();

  // ---- targets: positions relative to the owner centre, tiles inside one sphere
  std::vector<float4> t32(nc);
  std::vector<double> t64(4 * (size_t)nc), cabs(d.colloc), sw(nc);
  std::vector<int> ts, tst, tcn, ts1, tst1, tcn1;
  for (int k = 0; k < P; ++k) {
    for (int i = d.colloc_off[k]; i < d.colloc_off[k + 1]; ++i) {
      double r[3];
      for (int q = 0; q < 3; ++q) r[q] = d.colloc[3 * i + q] - d.centres[3 * k + q];
      double w = p.left_precond ? std::sqrt(d.weight[i]) : 1.0;
      sw[i] = w;
      t32[i] = make_float4((float)r[0], (float)r[1], (float)r[2], (float)w);
      t64[4 * i] = r[0]; t64[4 * i + 1] = r[1]; t64[4 * i + 2] = r[2]; t64[4 * i + 3] = w;
    }
    for (int s0 = d.colloc_off[k]; s0 < d.colloc_off[k + 1]; s0 += kTileTargets) {
      ts.push_back(k);
      tst.push_back(s0);
      tcn.push_back(std::min(kTileTargets, d.colloc_off[k + 1] - s0));
    }
    for (int s0 = d.colloc_off[k]; s0 < d.colloc_off[k + 1]; s0 += kTileTargets / 4) {
      ts1.push_back(k);
      tst1.push_back(s0);
      tcn1.push_back(std::min(kTileTargets / 4, d.colloc_off[k + 1] - s0));
    }
  }
  c->tg.n_tiles1 = (int)ts1.size();
  if ((s = upload(c, c->tg.tile1_sphere, ts1)) != MFS_OK) return s;
  if ((s = upload(c, c->tg.tile1_start, tst1)) != MFS_OK) return s;
  if ((s = upload(c, c->tg.tile1_count, tcn1)) != MFS_OK) return s;
  c->tg.n = nc;
  c->tg.n_tiles = (int)ts.size();
  if ((s = upload(c, c->tg.pos32, t32)) != MFS_OK) return s;
  if ((s = upload(c, c->tg.pos64, t64)) != MFS_OK) return s;
  if ((s = upload(c, c->tg.tile_sphere, ts)) != MFS_OK) return s;
  if ((s = upload(c, c->tg.tile_start, tst)) != MFS_OK) return s;
  if ((s = upload(c, c->tg.tile_count, tcn)) != MFS_OK) return s;
  if ((s = upload(c, c->d_colloc_abs, cabs)) != MFS_OK) return s;
  if ((s = upload(c, c->d_owner, d.owner)) != MFS_OK) return s;
  if ((s = upload(c, c->d_sqrtw, sw)) != MFS_OK) return s;

  // ---- sources
  std::vector<float4> p32(N), i32(std::max(ni, 1));
  std::vector<double> p64(4 * (size_t)N), i64(4 * (size_t)std::max(ni, 1), 0.0);
  for (int j = 0; j < N; ++j) {
    p32[j] = make_float4((float)d.proxy_rel[3 * j], (float)d.proxy_rel[3 * j + 1], (float)d.proxy_rel[3 * j + 2], 0.f);
    for (int q = 0; q < 3; ++q) p64[4 * j + q] = d.proxy_rel[3 * j + q];
    p64[4 * j + 3] = 0;
  }
  for (int j = 0; j < ni; ++j) {
    int o = d.img_owner[j];
    double r[3];
    for (int q = 0; q < 3; ++q) r[q] = d.image[3 * j + q] - d.centres[3 * o + q];
    i32[j] = make_float4((float)r[0], (float)r[1], (float)r[2], 0.f);
    for (int q = 0; q < 3; ++q) i64[4 * j + q] = r[q];
  }
  std::vector<float> chi(3 * (size_t)P), clo(3 * (size_t)P);
  for (int i = 0; i < 3 * P; ++i) {
    chi[i] = (float)d.centres[i];
    clo[i] = (float)(d.centres[i] - (double)chi[i]);
  }
  std::vector<int> io = d.img_owner;
  if (io.empty()) io.push_back(0);
  c->src.P = P;
  c->src.N = N;
  c->src.n_img = ni;
  if ((s = upload(c, c->src.proxy32, p32)) != MFS_OK) return s;
  if ((s = upload(c, c->src.proxy64, p64)) != MFS_OK) return s;
  if ((s = upload(c, c->src.img32, i32)) != MFS_OK) return s;
  if ((s = upload(c, c->src.img64, i64)) != MFS_OK) return s;
  if ((s = upload(c, c->src.img_owner, io)) != MFS_OK) return s;
  if ((s = upload(c, c->src.unk_off, d.unk_off)) != MFS_OK) return s;
  if ((s = upload(c, c->src.img_off, d.img_off)) != MFS_OK) return s;
  if ((s = upload(c, c->src.cen_hi, chi)) != MFS_OK) return s;
  if ((s = upload(c, c->src.cen_lo, clo)) != MFS_OK) return s;
  if ((s = upload(c, c->src.cen64, d.centres)) != MFS_OK) return s;

  // ---- one-body factors: B_k = W_k G^(kk), thin SVD in FP64 (Golub-Kahan bidiagonalisation
  // with implicit QR, backward stable), truncation at eps_trunc sigma_max, packing.  The
  // distinct blocks are spread over host worker threads, each with its own stream, cuSOLVER
  // handle and scratch, so the latency-bound parts of the SVDs overlap on the GPU.
  const int nf = p.build_factors ? (int)d.factor_rep.size() : 0;
  int max_m = 0, max_nc = 0;
  for (int f = 0; f < nf; ++f) {
    int k = d.factor_rep[f];
    int m = 3 * (d.colloc_off[k + 1] - d.colloc_off[k]);
    int ncol = (int)(d.unk_off[k + 1] - d.unk_off[k]);
    if (m < ncol) return c->fail(MFS_ERR_ARG, "more unknowns than collocation equations on a sphere; raise m_basic");
    max_m = std::max(max_m, m);
    max_nc = std::max(max_nc, ncol);
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // geometry uploads done before workers start

  // ---- far field, the part every sphere shares: the pseudo-inverse of the Stokeslet block from
  // the equivalent points to the check points, truncated at far_eps of its largest singular value
  const bool far_on = p.far_dist > 0 && nf > 0;
  const int n_eq = far_on ? p.far_n_eq : 0, n_chk = 2 * n_eq;
  std::vector<void*> far_tmp;  // build-time buffers of the far field, freed at the end of the build
  struct FarTmpFree {
    std::vector<void*>& v;
    ~FarTmpFree() {
      for (void* q : v) cudaFree(q);
    }
  } far_tmp_free{far_tmp};
  auto far_alloc = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    far_tmp.push_back(q);
    return q;
  };
  double *d_pinv = nullptr, *d_chk = nullptr, *d_ones = nullptr;
  std::vector<double> eq_host;
  if (far_on) {
    std::vector<double> chk, ones(n_chk, 1.0);
    std::vector<int> ty0(n_eq, 0);
    fibonacci_sphere(n_eq, p.far_r_eq * c->a, eq_host);
    fibonacci_sphere(n_chk, p.far_r_chk * c->a, chk);
    const int me = 3 * n_chk, ne = 3 * n_eq;
    d_chk = (double*)far_alloc(sizeof(double) * chk.size());
    d_ones = (double*)far_alloc(sizeof(double) * n_chk);
    double* d_eq = (double*)far_alloc(sizeof(double) * eq_host.size());
    int* d_ty0 = (int*)far_alloc(sizeof(int) * n_eq);
    double* d_S = (double*)far_alloc(sizeof(double) * (size_t)me * ne);
    double* d_U = (double*)far_alloc(sizeof(double) * (size_t)me * ne);
    double* d_VT = (double*)far_alloc(sizeof(double) * (size_t)ne * ne);
    double* d_s = (double*)far_alloc(sizeof(double) * ne);
    double* d_sinv = (double*)far_alloc(sizeof(double) * ne);
    double* d_rw = (double*)far_alloc(sizeof(double) * ne);
    int* d_info = (int*)far_alloc(sizeof(int));
    d_pinv = (double*)far_alloc(sizeof(double) * (size_t)ne * me);
    if (!d_chk || !d_ones || !d_eq || !d_ty0 || !d_S || !d_U || !d_VT || !d_s || !d_sinv || !d_rw || !d_info || !d_pinv)
      return c->fail(MFS_ERR_OOM, "device allocation failed: far-field fit");
    CUDA_TRY(c, cudaMemcpyAsync(d_chk, chk.data(), sizeof(double) * chk.size(), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(d_ones, ones.data(), sizeof(double) * n_chk, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(d_eq, eq_host.data(), sizeof(double) * eq_host.size(), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(d_ty0, ty0.data(), sizeof(int) * n_eq, cudaMemcpyHostToDevice, c->stream));
    launch_assemble_block(n_chk, n_eq, d_chk, d_ones, d_eq, d_ty0, p.visc, d_S, me, c->stream);
    CHECK_LAUNCH(c);
    cusolverDnHandle_t hs = nullptr;
    cublasHandle_t hb = nullptr;
    struct Handles {
      cusolverDnHandle_t& s;
      cublasHandle_t& b;
      ~Handles() {
        if (s) cusolverDnDestroy(s);
        if (b) cublasDestroy(b);
      }
    } handles{hs, hb};
    if (cusolverDnCreate(&hs) != CUSOLVER_STATUS_SUCCESS || cusolverDnSetStream(hs, c->stream) != CUSOLVER_STATUS_SUCCESS ||
        cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS || cublasSetStream(hb, c->stream) != CUBLAS_STATUS_SUCCESS)
      return c->fail(MFS_ERR_CUDA, "far field: cuSOLVER / cuBLAS handle creation failed");
    int lw = 0;
    CUSOLVER_TRY(c, cusolverDnDgesvd_bufferSize(hs, me, ne, &lw));
    double* d_work = (double*)far_alloc(sizeof(double) * (size_t)std::max(lw, 1));
    if (!d_work) return c->fail(MFS_ERR_OOM, "device allocation failed: far-field SVD workspace");
    CUSOLVER_TRY(c, cusolverDnDgesvd(hs, 'S', 'S', me, ne, d_S, me, d_s, d_U, me, d_VT, ne, d_work, lw, d_rw, d_info));
    std::vector<double> hsv(ne);
    int hinfo = 0;
    CUDA_TRY(c, cudaMemcpyAsync(hsv.data(), d_s, sizeof(double) * ne, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(&hinfo, d_info, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (hinfo != 0) return c->fail(MFS_ERR_CUDA, "far field: SVD of the equivalent-source block failed");
    double smax = 0;
    for (double v : hsv) smax = std::max(smax, v);
    std::vector<double> sinv(ne, 0.0);
    for (int i = 0; i < ne; ++i)
      if (hsv[i] >= p.far_eps * smax && hsv[i] > 0) sinv[i] = 1.0 / hsv[i];
    CUDA_TRY(c, cudaMemcpyAsync(d_sinv, sinv.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, c->stream));
    // Pinv = V diag(sinv) U^T: scale the columns of U, then (VT)^T (U diag(sinv))^T
    // (d_S, overwritten by the SVD, receives U diag(sinv))
    if (cublasDdgmm(hb, CUBLAS_SIDE_RIGHT, me, ne, d_U, me, d_sinv, 1, d_S, me) != CUBLAS_STATUS_SUCCESS)
      return c->fail(MFS_ERR_CUDA, "far field: cublasDdgmm failed");
    const double one = 1.0, zero = 0.0;
    if (cublasDgemm(hb, CUBLAS_OP_T, CUBLAS_OP_T, ne, me, ne, &one, d_VT, ne, d_S, me, &zero, d_pinv, ne) !=
        CUBLAS_STATUS_SUCCESS)
      return c->fail(MFS_ERR_CUDA, "far field: cublasDgemm (pseudo-inverse) failed");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  c->factors.assign(nf, Factor());
  const int n_workers = std::max(0, std::min(nf, 8));
  std::mutex mtx;
  std::string werr;
  mfs_status wstat = MFS_OK;
  auto worker = [&](int wid) {
    auto fail_w = [&](mfs_status st, const std::string& msg) {
      std::lock_guard<std::mutex> g(mtx);
      if (wstat == MFS_OK) {
        wstat = st;
        werr = msg;
      }
    };
    if (cudaSetDevice(c->device) != cudaSuccess) return fail_w(MFS_ERR_CUDA, "cudaSetDevice in factor worker");
    cudaStream_t st = nullptr;
    cusolverDnHandle_t h = nullptr;
    cublasHandle_t hb = nullptr;
    std::vector<void*> scratch;
    auto salloc = [&](size_t bytes) -> void* {
      void* q = nullptr;
      if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      scratch.push_back(q);
      return q;
    };
    auto cleanup = [&]() {
      if (st) cudaStreamSynchronize(st);
      for (void* q : scratch) cudaFree(q);
      if (h) cusolverDnDestroy(h);
      if (hb) cublasDestroy(hb);
      if (st) cudaStreamDestroy(st);
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cusolverDnCreate(&h) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnSetStream(h, st) != CUSOLVER_STATUS_SUCCESS ||
        (far_on && (cublasCreate(&hb) != CUBLAS_STATUS_SUCCESS || cublasSetStream(hb, st) != CUBLAS_STATUS_SUCCESS))) {
      cudaGetLastError();
      cleanup();
      return fail_w(MFS_ERR_CUDA, "factor worker: stream or cuSOLVER handle creation failed");
    }
    // B = QR (blocked Householder), R = U_R Sigma V^T (square SVD), U = Q [U_R; 0]: the route of
    // LAPACK's SVD for tall matrices, backward stable like the SVD of B itself
    double* dB = (double*)salloc(sizeof(double) * (size_t)max_m * max_nc);
    double* dR = (double*)salloc(sizeof(double) * (size_t)max_nc * max_nc);
    double* dUR = (double*)salloc(sizeof(double) * (size_t)max_nc * max_nc);
    double* dtau = (double*)salloc(sizeof(double) * max_nc);
    int lwork = 0, lw_qr = 0, lw_orm = 0;
    if (!dB || !dR || !dUR || !dtau || cusolverDnDgesvd_bufferSize(h, max_nc, max_nc, &lwork) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDgeqrf_bufferSize(h, max_m, max_nc, dB, max_m, &lw_qr) != CUSOLVER_STATUS_SUCCESS ||
        cusolverDnDormqr_bufferSize(h, CUBLAS_SIDE_LEFT, CUBLAS_OP_N, max_m, max_nc, max_nc, dB, max_m, dtau, dB, max_m,
                                    &lw_orm) != CUSOLVER_STATUS_SUCCESS) {
      cleanup();
      return fail_w(MFS_ERR_CUDA, "factor worker: cuSOLVER workspace query failed");
    }
    lwork = std::max(lwork, std::max(lw_qr, lw_orm));
    double* dU = (double*)salloc(sizeof(double) * (size_t)max_m * max_nc);
    double* dVT = (double*)salloc(sizeof(double) * (size_t)max_nc * max_nc);
    double* dS = (double*)salloc(sizeof(double) * max_nc);
    double* drw = (double*)salloc(sizeof(double) * max_nc);
    double* dwork = (double*)salloc(sizeof(double) * (size_t)lwork);
    int* dinfo = (int*)salloc(3 * sizeof(int));
    double* dxr = (double*)salloc(sizeof(double) * (size_t)max_m);
    double* dsw = (double*)salloc(sizeof(double) * ((size_t)max_m / 3 + 1));
    double* dyr = (double*)salloc(sizeof(double) * (size_t)max_nc);
    int* dty = (int*)salloc(sizeof(int) * ((size_t)max_nc / 3 + 1));
    int* dkeep = (int*)salloc(sizeof(int) * (size_t)max_nc);
    if (!dB || !dU || !dVT || !dS || !drw || !dwork || !dinfo || !dxr || !dsw || !dyr || !dty || !dkeep) {
      cleanup();
      return fail_w(MFS_ERR_OOM, "device allocation failed: factorisation scratch");
    }
    // far field: the check-point field of the sphere's sources, its products with V and
    // Sigma^+ U^T, and Q in FP64 before rounding
    double *dG = nullptr, *dT1 = nullptr, *dT2 = nullptr, *dQ64 = nullptr;
    if (far_on) {
      dG = (double*)salloc(sizeof(double) * 3 * (size_t)n_chk * max_nc);
      dT1 = (double*)salloc(sizeof(double) * 3 * (size_t)n_chk * max_nc);
      dT2 = (double*)salloc(sizeof(double) * 3 * (size_t)n_chk * max_m);
      dQ64 = (double*)salloc(sizeof(double) * (size_t)pad4(max_m) * 3 * n_eq);
      if (!dG || !dT1 || !dT2 || !dQ64) {
        cleanup();
        return fail_w(MFS_ERR_OOM, "device allocation failed: far-field scratch");
      }
    }
    std::vector<double> hS(max_nc);
    for (int f = wid; f < nf; f += n_workers) {
      {
        std::lock_guard<std::mutex> g(mtx);
        if (wstat != MFS_OK) break;
      }
      const int k = d.factor_rep[f];
      const int m_nodes = d.colloc_off[k + 1] - d.colloc_off[k];
      const int m = 3 * m_nodes;
      const int ncol = (int)(d.unk_off[k + 1] - d.unk_off[k]);
      const int n_src = ncol / 3;
      // rows: collocation nodes of k relative to c_k; columns: strength order (proxies, then S, R, D per image node)
      std::vector<double> xr(3 * (size_t)m_nodes), swk(m_nodes), yr(3 * (size_t)n_src);
      std::vector<int> ty(n_src);
      for (int i = 0; i < m_nodes; ++i) {
        int gi = d.colloc_off[k] + i;
        for (int q = 0; q < 3; ++q) xr[3 * i + q] = d.colloc[3 * gi + q] - d.centres[3 * k + q];
        swk[i] = sw[gi];
      }
      for (int j = 0; j < N; ++j) {
        for (int q = 0; q < 3; ++q) yr[3 * j + q] = d.proxy_rel[3 * j + q];
        ty[j] = 0;
      }
      for (int j = d.img_off[k]; j < d.img_off[k + 1]; ++j) {
        int base = N + 3 * (j - d.img_off[k]);
        for (int t = 0; t < 3; ++t) {
          for (int q = 0; q < 3; ++q) yr[3 * (base + t) + q] = d.image[3 * j + q] - d.centres[3 * k + q];
          ty[base + t] = t;
        }
      }
      // a sphere without images has the basic block, fixed by the radius, the viscosity, the
      // proxy sphere (N, R_p), the basic grid (M0, its weights), the truncation and the far-field
      // settings (the grids are global-frame, so the block does not depend on the centre): its
      // factor may already be in the store; otherwise it is computed into a new store entry
      std::shared_ptr<SharedFactor> ent;
      if (d.img_off[k + 1] == d.img_off[k]) {
        std::vector<double> key = {c->a,        p.visc,       p.eps_trunc,        (double)N,
                                   p.r_proxy,   (double)p.m_basic, (double)p.left_precond, (double)m_nodes,
                                   far_on ? 1.0 : 0.0, (double)n_eq, p.far_r_eq, p.far_r_chk,
                                   p.far_eps};
        if (std::shared_ptr<SharedFactor> hit = store_find(c->device, key)) {
          std::lock_guard<std::mutex> g(mtx);
          if (c->mem_limit && c->mem_used + hit->bytes > c->mem_limit) {
            if (wstat == MFS_OK) {
              wstat = MFS_ERR_OOM;
              werr = "device allocation failed: one-body factors (memory cap)";
            }
            break;
          }
          c->mem_used += hit->bytes;
          c->shared.push_back(hit);
          c->factors[f] = hit->F;
          ++c->factors_reused;
          continue;
        }
        ent = std::make_shared<SharedFactor>();
        ent->device = c->device;
        ent->key = std::move(key);
        ent->q_rows = far_on ? 3 * n_eq : 0;
      }
      // device memory of the factor: the context's own, or the new store entry's (held by the
      // context and counted against its cap)
      auto falloc = [&](size_t bytes) -> void* {
        if (!ent) return c->dalloc<char>(bytes);
        if (c->mem_limit && c->mem_used + bytes > c->mem_limit) return nullptr;
        void* q = ent->alloc(bytes);
        if (q) {
          c->mem_used += bytes;
          ent->bytes += bytes;
        }
        return q;
      };
      cudaError_t e1 = cudaMemcpyAsync(dxr, xr.data(), xr.size() * 8, cudaMemcpyHostToDevice, st);
      cudaError_t e2 = cudaMemcpyAsync(dsw, swk.data(), swk.size() * 8, cudaMemcpyHostToDevice, st);
      cudaError_t e3 = cudaMemcpyAsync(dyr, yr.data(), yr.size() * 8, cudaMemcpyHostToDevice, st);
      cudaError_t e4 = cudaMemcpyAsync(dty, ty.data(), ty.size() * 4, cudaMemcpyHostToDevice, st);
      if (e1 || e2 || e3 || e4) {
        fail_w(MFS_ERR_CUDA, "upload of self-block geometry failed");
        break;
      }
      launch_assemble_self(d, k, dxr, dsw, dyr, dty, n_src, dB, m, st);
      cusolverStatus_t sst = cusolverDnDgeqrf(h, m, ncol, dB, m, dtau, dwork, lwork, dinfo);
      upper_copy_kernel<<<256, 256, 0, st>>>(ncol, dB, m, dR);
      if (sst == CUSOLVER_STATUS_SUCCESS)
        sst = cusolverDnDgesvd(h, 'S', 'S', ncol, ncol, dR, ncol, dS, dUR, ncol, dVT, ncol, dwork, lwork, drw, dinfo + 1);
      // U = Q [U_R; 0]
      cudaMemsetAsync(dU, 0, sizeof(double) * (size_t)m * ncol, st);
      cudaMemcpy2DAsync(dU, sizeof(double) * m, dUR, sizeof(double) * ncol, sizeof(double) * ncol, ncol,
                        cudaMemcpyDeviceToDevice, st);
      if (sst == CUSOLVER_STATUS_SUCCESS)
        sst = cusolverDnDormqr(h, CUBLAS_SIDE_LEFT, CUBLAS_OP_N, m, ncol, ncol, dB, m, dtau, dU, m, dwork, lwork,
                               dinfo + 2);
      int hinfo3[3] = {0, 0, 0};
      cudaMemcpyAsync(hinfo3, dinfo, 3 * sizeof(int), cudaMemcpyDeviceToHost, st);
      cudaMemcpyAsync(hS.data(), dS, sizeof(double) * ncol, cudaMemcpyDeviceToHost, st);
      cudaError_t es = cudaStreamSynchronize(st);
      const int hinfo = hinfo3[0] ? hinfo3[0] : (hinfo3[1] ? hinfo3[1] : hinfo3[2]);
      if (sst != CUSOLVER_STATUS_SUCCESS || es != cudaSuccess || hinfo != 0) {
        fail_w(MFS_ERR_CUDA, "one-body SVD failed (cusolver status " + std::to_string((int)sst) + ", info " +
                                 std::to_string(hinfo) + ")");
        break;
      }
      // keep sigma >= eps * sigma_max (no assumption on the order the SVD returns them in)
      double smax = 0;
      for (int i = 0; i < ncol; ++i) smax = std::max(smax, hS[i]);
      std::vector<int> keep;
      for (int i = 0; i < ncol; ++i)
        if (hS[i] >= p.eps_trunc * smax && hS[i] > 0) keep.push_back(i);
      const int r = (int)keep.size();
      if (r == 0) {
        fail_w(MFS_ERR_NUMERIC, "one-body block has no singular value above the truncation level");
        break;
      }
      if (cudaMemcpyAsync(dkeep, keep.data(), sizeof(int) * r, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        fail_w(MFS_ERR_CUDA, "upload of the retained singular indices failed");
        break;
      }
      Factor F;
      F.m = m;
      F.ncol = ncol;
      F.rank = r;
      F.ldA = pad4(m);
      F.ldV = pad4(r);
      {
        std::lock_guard<std::mutex> g(mtx);
        F.A64 = (double*)falloc(sizeof(double) * (size_t)r * F.ldA);
        F.A32 = (float*)falloc(sizeof(float) * (size_t)r * F.ldA);
        F.V64 = (double*)falloc(sizeof(double) * (size_t)ncol * F.ldV);
        F.V32 = (float*)falloc(sizeof(float) * (size_t)ncol * F.ldV);
        F.A2 = (float2*)falloc(sizeof(float2) * (size_t)r * F.ldA);
        F.V2 = (float2*)falloc(sizeof(float2) * (size_t)ncol * F.ldV);
      }
      if (!F.A64 || !F.A32 || !F.V64 || !F.V32 || !F.A2 || !F.V2) {
        fail_w(MFS_ERR_OOM, "device allocation failed: one-body factors");
        break;
      }
      pack_A_kernel<<<1024, 256, 0, st>>>(r, m, F.ldA, dU, dS, dkeep, F.A64, F.A32, F.A2);
      pack_V_kernel<<<1024, 256, 0, st>>>(ncol, r, F.ldV, dVT, dkeep, F.V64, F.V32, F.V2);
      if (far_on) {
        // Q = Pinv (G_chk (V (Sigma^+ U^T))): the check-point field of B^+ first, in FP64, so the
        // amplified directions of B^+ only ever meet fields that are correspondingly weak
        F.ldQ = pad4(m);
        {
          std::lock_guard<std::mutex> g(mtx);
          F.Q32 = (float*)falloc(sizeof(float) * (size_t)3 * n_eq * F.ldQ);
        }
        if (!F.Q32) {
          fail_w(MFS_ERR_OOM, "device allocation failed: far-field matrices");
          break;
        }
        const int mc = 3 * n_chk, ne = 3 * n_eq;
        const double one = 1.0, zero = 0.0;
        launch_assemble_block(n_chk, n_src, d_chk, d_ones, dyr, dty, p.visc, dG, mc, st);
        cudaMemsetAsync(dQ64, 0, sizeof(double) * (size_t)F.ldQ * ne, st);
        bool okb = cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_T, mc, r, ncol, &one, dG, mc, F.V64, F.ldV, &zero, dT1, mc) ==
                       CUBLAS_STATUS_SUCCESS &&
                   cublasDgemm(hb, CUBLAS_OP_N, CUBLAS_OP_T, mc, m, r, &one, dT1, mc, F.A64, F.ldA, &zero, dT2, mc) ==
                       CUBLAS_STATUS_SUCCESS &&
                   cublasDgemm(hb, CUBLAS_OP_T, CUBLAS_OP_T, m, ne, mc, &one, dT2, mc, d_pinv, ne, &zero, dQ64,
                               F.ldQ) == CUBLAS_STATUS_SUCCESS;
        if (!okb) {
          fail_w(MFS_ERR_CUDA, "far field: cublasDgemm (Q) failed");
          break;
        }
        launch_convert<double, float>((long long)F.ldQ * ne, dQ64, 1.0, F.Q32, st);
      }
      cudaError_t el = cudaGetLastError();
      if (el == cudaSuccess) el = cudaStreamSynchronize(st);  // keep and hS are reused next round
      if (el != cudaSuccess) {
        fail_w(MFS_ERR_CUDA, std::string("factor packing: ") + cudaGetErrorString(el));
        break;
      }
      c->factors[f] = F;
      if (ent) {
        ent->F = F;
        store_add(ent);
        std::lock_guard<std::mutex> g(mtx);
        c->shared.push_back(ent);
      }
    }
    cleanup();
  };
  {
    std::vector<std::thread> pool;
    for (int w = 0; w < n_workers; ++w) pool.emplace_back(worker, w);
    for (auto& t : pool) t.join();
  }
  if (wstat != MFS_OK) return c->fail(wstat, werr);

  // ---- far field: neighbour lists, equivalent points, the per-sphere Q GEMV
  if (far_on) {
    FarField& ff = c->ff;
    ff.n_eq = n_eq;
    std::vector<float4> e32(n_eq);
    for (int e = 0; e < n_eq; ++e)
      e32[e] = make_float4((float)eq_host[3 * e], (float)eq_host[3 * e + 1], (float)eq_host[3 * e + 2], 0.f);
    std::vector<int> noff(1, 0), nidx, xoff(1, 0), xidx;
    const double fd2 = (p.far_dist * c->a) * (p.far_dist * c->a);
    long long np = 0, ni = 0, nfar = 0;
    for (int k = 0; k < P; ++k) {
      const long long mk = d.colloc_off[k + 1] - d.colloc_off[k];
      int n_near = 0;
      for (int k2 = 0; k2 < P; ++k2) {
        if (k2 == k) {
          xidx.push_back(k);
          continue;
        }
        double r2 = 0;
        for (int q = 0; q < 3; ++q) {
          const double dq = d.centres[3 * k + q] - d.centres[3 * k2 + q];
          r2 += dq * dq;
        }
        if (r2 < fd2) {
          nidx.push_back(k2);
          xidx.push_back(k2);
          ++n_near;
          np += mk * N;
          ni += mk * (d.img_off[k2 + 1] - d.img_off[k2]);
        }
      }
      noff.push_back((int)nidx.size());
      xoff.push_back((int)xidx.size());
      nfar += mk * (long long)n_eq * (P - 1 - n_near);
    }
    if (nidx.empty()) nidx.push_back(0);
    if ((s = upload(c, ff.eq32, e32)) != MFS_OK || (s = upload(c, ff.near_off, noff)) != MFS_OK ||
        (s = upload(c, ff.near_idx, nidx)) != MFS_OK || (s = upload(c, ff.excl_off, xoff)) != MFS_OK ||
        (s = upload(c, ff.excl_idx, xidx)) != MFS_OK)
      return s;
    ALLOC_TRY(c, c->d_q, float, 3 * (size_t)n_eq * P);
    ff.q = c->d_q;
    c->near_proxy_per_apply = np;
    c->near_image_per_apply = ni;
    c->near_pairs_per_apply = np + 3 * ni;
    c->far_pairs_per_apply = nfar;
    std::vector<const float*> mQ(P);
    std::vector<int> rQ(P, 3 * n_eq), cQ(P), lQ(P);
    std::vector<long long> xQ(P), yQ(P);
    for (int k = 0; k < P; ++k) {
      const Factor& F = c->factors[d.factor_id[k]];
      mQ[k] = F.Q32;
      cQ[k] = F.m;
      lQ[k] = F.ldQ;
      xQ[k] = 3LL * d.colloc_off[k];
      yQ[k] = 3LL * n_eq * k;
    }
    const float** dmQ = nullptr;
    int *drQ, *dcQ, *dlQ;
    long long *dxQ, *dyQ;
    if ((s = upload(c, dmQ, mQ)) || (s = upload(c, drQ, rQ)) || (s = upload(c, dcQ, cQ)) || (s = upload(c, dlQ, lQ)) ||
        (s = upload(c, dxQ, xQ)) || (s = upload(c, dyQ, yQ)))
      return s;
    c->gQ.mat = dmQ;
    c->gQ.rows = drQ;
    c->gQ.cols = dcQ;
    c->gQ.ld = dlQ;
    c->gQ.x_off = dxQ;
    c->gQ.y_off = dyQ;
    c->gQ.n_jobs = P;
    c->gQ.max_rows = 3 * n_eq;
  }

  // ---- GEMV batches for step 1
  std::vector<long long> tmp_off(P + 1, 0);
  if (nf > 0)
    for (int k = 0; k < P; ++k) tmp_off[k + 1] = tmp_off[k] + c->factors[d.factor_id[k]].rank;
  c->tmp_len = tmp_off[P];
  if (nf > 0) {
    std::vector<const double*> mA64(P), mV64(P);
    std::vector<const float*> mA32(P), mV32(P);
    std::vector<const float2*> mA2(P), mV2(P);
    std::vector<int> rA(P), cA(P), lA(P), rV(P), cV(P), lV(P);
    std::vector<long long> xA(P), yA(P), xV(P), yV(P);
    int maxA = 0, maxV = 0;
    for (int k = 0; k < P; ++k) {
      const Factor& F = c->factors[d.factor_id[k]];
      mA64[k] = F.A64; mA32[k] = F.A32; mV64[k] = F.V64; mV32[k] = F.V32;
      mA2[k] = F.A2; mV2[k] = F.V2;
      rA[k] = F.rank; cA[k] = F.m; lA[k] = F.ldA;
      xA[k] = 3LL * d.colloc_off[k]; yA[k] = tmp_off[k];
      rV[k] = F.ncol; cV[k] = F.rank; lV[k] = F.ldV;
      xV[k] = tmp_off[k]; yV[k] = d.unk_off[k];
      maxA = std::max(maxA, F.rank);
      maxV = std::max(maxV, F.ncol);
    }
    const double** dm64 = nullptr;
    const float** dm32 = nullptr;
    if ((s = upload(c, dm64, mA64)) != MFS_OK) return s;
    c->gA64.mat = dm64;
    if ((s = upload(c, dm32, mA32)) != MFS_OK) return s;
    c->gA32.mat = dm32;
    if ((s = upload(c, dm64, mV64)) != MFS_OK) return s;
    c->gV64.mat = dm64;
    if ((s = upload(c, dm32, mV32)) != MFS_OK) return s;
    c->gV32.mat = dm32;
    const float2** dm2 = nullptr;
    if ((s = upload(c, dm2, mA2)) != MFS_OK) return s;
    c->gA64.mat_dw = dm2;
    if ((s = upload(c, dm2, mV2)) != MFS_OK) return s;
    c->gV64.mat_dw = dm2;
    int *d_rA, *d_cA, *d_lA, *d_rV, *d_cV, *d_lV;
    long long *d_xA, *d_yA, *d_xV, *d_yV;
    if ((s = upload(c, d_rA, rA)) || (s = upload(c, d_cA, cA)) || (s = upload(c, d_lA, lA)) || (s = upload(c, d_rV, rV)) ||
        (s = upload(c, d_cV, cV)) || (s = upload(c, d_lV, lV)) || (s = upload(c, d_xA, xA)) || (s = upload(c, d_yA, yA)) ||
        (s = upload(c, d_xV, xV)) || (s = upload(c, d_yV, yV)))
      return s;
    c->gA64.rows = c->gA32.rows = d_rA;
    c->gA64.cols = c->gA32.cols = d_cA;
    c->gA64.ld = c->gA32.ld = d_lA;
    c->gA64.x_off = c->gA32.x_off = d_xA;
    c->gA64.y_off = c->gA32.y_off = d_yA;
    c->gA64.n_jobs = c->gA32.n_jobs = P;
    c->gA64.max_rows = c->gA32.max_rows = maxA;
    c->gV64.rows = c->gV32.rows = d_rV;
    c->gV64.cols = c->gV32.cols = d_cV;
    c->gV64.ld = c->gV32.ld = d_lV;
    c->gV64.x_off = c->gV32.x_off = d_xV;
    c->gV64.y_off = c->gV32.y_off = d_yV;
    c->gV64.n_jobs = c->gV32.n_jobs = P;
    c->gV64.max_rows = c->gV32.max_rows = maxV;
  }

  // ---- tensor-core step 1: the spheres without contacts share the basic factor; their
  // Sigma^+ U^T (and far-field Q) products in the passes become one matrix product each
  {
    int shared_f = -1;
    for (int k = 0; k < P && nf > 0; ++k)
      if (d.img_off[k + 1] == d.img_off[k] && d.colloc_off[k + 1] - d.colloc_off[k] == p.m_basic) {
        shared_f = d.factor_id[k];
        break;
      }
    std::vector<int> tck, rest;
    for (int k = 0; k < P; ++k) {
      if (shared_f >= 0 && d.factor_id[k] == shared_f) tck.push_back(k);
      else rest.push_back(k);
    }
    const int tc_min = p.tensor_step1 == 2 ? 1 : 8;
    if (nf > 0 && p.tensor_step1 != 0 && (int)tck.size() >= tc_min) {
      const Factor& F = c->factors[shared_f];
      const int ldk = tc_ldk(F.m), ncap = (int)tck.size();
      // the factor of spheres without images lives in the store, with its bf16 slices
      SharedFactor* se = nullptr;
      for (auto& e : c->shared)
        if (e->F.A64 == F.A64) se = e.get();
      if (!se) return c->fail(MFS_ERR_STATE, "tensor-core step 1: the shared factor is not in the store");
      if ((s = ensure_tc_slices(c, *se)) != MFS_OK) return s;
      if (c->mem_limit && c->mem_used + se->tc_bytes > c->mem_limit)
        return c->fail(MFS_ERR_OOM, "device allocation failed: tensor-core slices (memory cap)");
      c->mem_used += se->tc_bytes;
      void* xs[3];
      for (int i = 0; i < 3; ++i) {
        xs[i] = c->dalloc<uint16_t>((size_t)ncap * ldk);
        if (!xs[i]) return c->fail(MFS_ERR_OOM, "device allocation failed: tensor-core slices");
      }
      if (!tc_prepare(c->tcA, se->as, F.rank, xs, ncap, F.m))
        return c->fail(MFS_ERR_CUDA, "tensor-core step 1: tensor maps or shared-memory limit unavailable");
      size_t part = tc_partial_floats(c->tcA, ncap);
      std::vector<long long> xo(ncap), ya(ncap), yq(ncap);
      for (int i = 0; i < ncap; ++i) {
        const int k = tck[i];
        xo[i] = 3LL * d.colloc_off[k];
        ya[i] = tmp_off[k];
        yq[i] = 3LL * n_eq * k;
      }
      if (far_on) {
        if (!tc_prepare(c->tcQ, se->qs, 3 * n_eq, xs, ncap, F.m))
          return c->fail(MFS_ERR_CUDA, "tensor-core step 1: tensor maps unavailable");
        part = std::max(part, tc_partial_floats(c->tcQ, ncap));
        if ((s = upload(c, c->d_tc_yQ, yq)) != MFS_OK) return s;
      }
      if ((s = upload(c, c->d_tc_xoff, xo)) != MFS_OK || (s = upload(c, c->d_tc_yA, ya)) != MFS_OK) return s;
      ALLOC_TRY(c, c->d_tc_partial, float, part);
      ALLOC_TRY(c, c->d_tc_err, int, 1);
      CUDA_TRY(c, cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream));
      CHECK_LAUNCH(c);
      // GEMV jobs of the other spheres
      auto sub_batch = [&](GemvBatch<float>& out, bool q) -> mfs_status {
        std::vector<const float*> mm;
        std::vector<int> rr, cc, ll;
        std::vector<long long> xx, yy;
        int mx = 0;
        for (int k : rest) {
          const Factor& G = c->factors[d.factor_id[k]];
          mm.push_back(q ? G.Q32 : G.A32);
          rr.push_back(q ? 3 * n_eq : G.rank);
          cc.push_back(G.m);
          ll.push_back(q ? G.ldQ : G.ldA);
          xx.push_back(3LL * d.colloc_off[k]);
          yy.push_back(q ? 3LL * n_eq * k : tmp_off[k]);
          mx = std::max(mx, rr.back());
        }
        out = GemvBatch<float>();
        out.n_jobs = (int)mm.size();
        out.max_rows = mx;
        if (mm.empty()) return MFS_OK;
        const float** dm = nullptr;
        int *dr, *dc, *dl;
        long long *dx, *dy;
        mfs_status st2;
        if ((st2 = upload(c, dm, mm)) || (st2 = upload(c, dr, rr)) || (st2 = upload(c, dc, cc)) ||
            (st2 = upload(c, dl, ll)) || (st2 = upload(c, dx, xx)) || (st2 = upload(c, dy, yy)))
          return st2;
        out.mat = dm;
        out.rows = dr;
        out.cols = dc;
        out.ld = dl;
        out.x_off = dx;
        out.y_off = dy;
        return MFS_OK;
      };
      if ((s = sub_batch(c->gA32_rest, false)) != MFS_OK) return s;
      if (far_on && (s = sub_batch(c->gQ_rest, true)) != MFS_OK) return s;
      c->tc_ncols = ncap;
    }
  }

  // ---- work vectors
  const int n = c->n;
  ALLOC_TRY(c, c->d_v, double, 3 * (size_t)P);
  ALLOC_TRY(c, c->d_om, double, 3 * (size_t)P);
  // system vectors hold the 6P border unknowns of the mobility problem as well
  ALLOC_TRY(c, c->d_wb, double, n + 6 * (size_t)P);
  ALLOC_TRY(c, c->d_mu, double, n + 6 * (size_t)P);
  ALLOC_TRY(c, c->d_r, double, n + 6 * (size_t)P);
  ALLOC_TRY(c, c->d_w64, double, n + 6 * (size_t)P);
  ALLOC_TRY(c, c->d_border, double, 6 * (size_t)P);
  ALLOC_TRY(c, c->d_zero, double, 3 * (size_t)P);
  ALLOC_TRY(c, c->d_pparts, double, (size_t)kPairMaxParts * n);
  ALLOC_TRY(c, c->d_tmp64, double, c->tmp_len);
  ALLOC_TRY(c, c->d_lh64, double, c->n_unk);
  ALLOC_TRY(c, c->d_lam, double, c->n_unk);
  ALLOC_TRY(c, c->d_F, double, 3 * (size_t)P);
  ALLOC_TRY(c, c->d_T, double, 3 * (size_t)P);
  ALLOC_TRY(c, c->d_tmp32, float, c->tmp_len);
  ALLOC_TRY(c, c->d_lh32, float, c->n_unk);
  ALLOC_TRY(c, c->d_in32, float, std::max<long long>(n, c->n_unk));
  ALLOC_TRY(c, c->d_out32, float, std::max<long long>(n, c->n_unk));
  ALLOC_TRY(c, c->d_mu32, float, n);
  ALLOC_TRY(c, c->d_x2, float2, n);
  ALLOC_TRY(c, c->d_t2, float2, c->tmp_len);
  c->nblk = std::max(1, std::min(1024, (n + 4095) / 4096));
  ALLOC_TRY(c, c->d_partial, double, (size_t)c->nblk * 512);
  ALLOC_TRY(c, c->d_h, double, 5 * 512);
  CUDA_TRY(c, cudaMemsetAsync(c->d_v, 0, sizeof(double) * 3 * P, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_zero, 0, sizeof(double) * 3 * P, c->stream));
  c->n_sys = n;
  c->mode = 0;
  CUDA_TRY(c, cudaMemsetAsync(c->d_om, 0, sizeof(double) * 3 * P, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  {
    mfs_sizes_t sz;
    c->state = 2;
    mfs_sizes(c, &sz);
    c->pairs_per_apply = sz.pairs_fp;
    long long pp = 0, ip = 0;
    for (int k = 0; k < P; ++k) {
      long long mk = d.colloc_off[k + 1] - d.colloc_off[k];
      pp += mk * (long long)(P - 1) * N;
      ip += mk * (long long)(ni - (d.img_off[k + 1] - d.img_off[k]));
    }
    c->proxy_per_apply = pp;
    c->image_per_apply = ip;
    static std::atomic<long long> g_build_counter{0};
    c->build_id = ++g_build_counter;
    double b32 = 0, b64 = 0, bf = 0;
    for (int k = 0; k < P && nf > 0; ++k) {
      const Factor& F = c->factors[d.factor_id[k]];
      double elems = (double)F.rank * F.m + (double)F.ncol * F.rank;
      b32 += 4.0 * elems;
      b64 += 8.0 * elems;
      bf += 4.0 * F.rank * F.m + 8.0 * F.ncol * F.rank;
    }
    c->gemv_bytes32 = b32;
    c->gemv_bytes64 = b64;
    c->gemv_bytes_fast = bf;
  }
  c->factored = nf > 0;
  c->solved = false;
  c->have_bc = false;
  return MFS_OK;
}

mfs_status mfs_discretise_host(int P, const double* centres, double radius, const mfs_params* params, int* n_colloc,
                               int* n_sources, double* x, double* w, int* owner, double* pos, int* type) {
  if (P < 1 || !centres || !(radius > 0) || !std::isfinite(radius)) return MFS_ERR_ARG;
  for (int i = 0; i < 3 * P; ++i)
    if (!std::isfinite(centres[i])) return MFS_ERR_ARG;
  mfs_params p;
  if (params) p = *params; else mfs_default_params(&p);
  HostDisc d;
  std::string err;
  mfs_status s = build_discretisation(centres, P, radius, p, d, err);
  if (s != MFS_OK) return s;
  const int N = d.prm.n_proxy;
  if (n_colloc) *n_colloc = d.n_colloc();
  if (n_sources) *n_sources = P * N + 3 * d.n_img();
  if (x) std::copy(d.colloc.begin(), d.colloc.end(), x);
  if (w) std::copy(d.weight.begin(), d.weight.end(), w);
  if (owner) std::copy(d.owner.begin(), d.owner.end(), owner);
  if (pos || type) {
    // the strength order of mfs_get_strengths: per sphere its proxies, then S, R, D per image node
    long long v = 0;
    for (int k = 0; k < P; ++k) {
      for (int j = 0; j < N; ++j, ++v) {
        if (pos)
          for (int q = 0; q < 3; ++q) pos[3 * v + q] = d.centres[3 * k + q] + d.proxy_rel[3 * j + q];
        if (type) type[v] = 0;
      }
      for (int j = d.img_off[k]; j < d.img_off[k + 1]; ++j)
        for (int t = 0; t < 3; ++t, ++v) {
          if (pos)
            for (int q = 0; q < 3; ++q) pos[3 * v + q] = d.image[3 * j + q];
          if (type) type[v] = t;
        }
    }
  }
  return MFS_OK;
}

mfs_status mfs_sizes(const mfs_ctx* cc, mfs_sizes_t* out) {
  mfs_ctx* c = const_cast<mfs_ctx*>(cc);
  if (!c || !out) return MFS_ERR_ARG;
  if (c->state < 2) return c->fail(MFS_ERR_STATE, "discretisation not built");
  const HostDisc& d = c->hd;
  out->P = d.P;
  out->n_contacts = (int)d.contacts.size();
  out->n_colloc = d.n_colloc();
  out->n_proxy_total = d.P * d.prm.n_proxy;
  out->n_image_nodes = d.n_img();
  out->n_unknowns = (int)d.n_unknowns();
  out->n_factors = (int)c->factors.size();
  long long pairs = 0;
  for (int k = 0; k < d.P; ++k) {
    long long mk = d.colloc_off[k + 1] - d.colloc_off[k];
    long long other = (long long)(d.P - 1) * d.prm.n_proxy + 3LL * (d.n_img() - (d.img_off[k + 1] - d.img_off[k]));
    pairs += mk * other;
  }
  out->pairs_fp = pairs;
  out->pairs_near_fp = c->ff.n_eq > 0 ? c->near_pairs_per_apply : pairs;
  out->pairs_far_eq = c->ff.n_eq > 0 ? c->far_pairs_per_apply : 0;
  out->n_factors_shared = (int)c->shared.size();
  out->n_factors_reused = c->factors_reused;
  return MFS_OK;
}

mfs_status mfs_set_rigid_velocities(mfs_ctx* c, const double* v, const double* om) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (!v || !om) return c->fail(MFS_ERR_ARG, "null velocity array");
  for (long long i = 0; i < 3LL * c->P; ++i)
    if (!std::isfinite(v[i]) || !std::isfinite(om[i])) return c->fail(MFS_ERR_ARG, "non-finite rigid velocity");
  CUDA_TRY(c, cudaMemcpyAsync(c->d_v, v, sizeof(double) * 3 * c->P, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_om, om, sizeof(double) * 3 * c->P, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->mode = 0;
  c->have_bc = true;
  c->solved = false;
  return MFS_OK;
}

mfs_status mfs_set_rigid_velocities_device(mfs_ctx* c, const double* v, const double* om) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (!v || !om) return c->fail(MFS_ERR_ARG, "null velocity array");
  CUDA_TRY(c, cudaMemcpyAsync(c->d_v, v, sizeof(double) * 3 * c->P, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_om, om, sizeof(double) * 3 * c->P, cudaMemcpyDeviceToDevice, c->stream));
  c->mode = 0;
  c->have_bc = true;
  c->solved = false;
  return MFS_OK;
}

static mfs_status solve_impl(mfs_ctx* c, const mfs_solve_opts* opts, mfs_solve_info* info);

mfs_status mfs_set_forces_torques(mfs_ctx* c, const double* F, const double* T) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (!F || !T) return c->fail(MFS_ERR_ARG, "null force/torque array");
  const double a = c->a, mu = c->hd.prm.visc;
  const double sF = 1.0 / (6.0 * kPi * mu * a), sT = 1.0 / (8.0 * kPi * mu * a * a * a);
  std::vector<double> b(6 * (size_t)c->P);
  for (int k = 0; k < c->P; ++k)
    for (int q = 0; q < 3; ++q) {
      if (!std::isfinite(F[3 * k + q]) || !std::isfinite(T[3 * k + q])) return c->fail(MFS_ERR_ARG, "non-finite force/torque");
      b[6 * k + q] = sF * F[3 * k + q];
      b[6 * k + 3 + q] = sT * T[3 * k + q];
    }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_border, b.data(), sizeof(double) * b.size(), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->mode = 1;
  c->have_bc = true;
  c->solved = false;
  return MFS_OK;
}

mfs_status mfs_get_rigid_velocities(mfs_ctx* c, double* v, double* omega) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (!c->solved || c->mode != 1) return c->fail(MFS_ERR_STATE, "no mobility solution yet");
  if (!v || !omega) return c->fail(MFS_ERR_ARG, "null output");
  CUDA_TRY(c, cudaMemcpyAsync(v, c->d_v, sizeof(double) * 3 * c->P, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(omega, c->d_om, sizeof(double) * 3 * c->P, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MFS_OK;
}

mfs_status mfs_solve(mfs_ctx* c, const mfs_solve_opts* opts, mfs_solve_info* info) {
  const long long l0 = launches_on_this_thread();
  mfs_status s = solve_impl(c, opts, info);
  if (c) {
    c->tm.kernel_launches += launches_on_this_thread() - l0;
    if (c->prof) {
      cudaStreamSynchronize(c->stream);
      collect_events(c);
    }
  }
  return s;
}

static mfs_status solve_impl(mfs_ctx* c, const mfs_solve_opts* opts, mfs_solve_info* info) {
  auto t0 = std::chrono::steady_clock::now();
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (!c->factored) return c->fail(MFS_ERR_STATE, "built without one-body factors (build_factors = 0)");
  mfs_solve_opts o;
  if (opts) o = *opts; else mfs_default_solve_opts(&o);
  if (o.restart < 1 || o.restart > 500 || !(o.tol > 0) || o.max_iter < 1 || o.max_refine < 0 ||
      (o.precision != MFS_FP64 && o.precision != MFS_MIXED && o.precision != MFS_FP32) ||
      o.residual < MFS_RESIDUAL_AUTO || o.residual > MFS_RESIDUAL_SOLVE)
    return c->fail(MFS_ERR_ARG, "invalid solve options (restart must be in [1, 500])");
  if (c->mode == 1 && o.precision == MFS_FP32)
    return c->fail(MFS_ERR_UNSUPPORTED, "the mobility problem is solved in MFS_FP64 or MFS_MIXED");
  c->n_sys = c->n + (c->mode == 1 ? 6 * c->P : 0);
  const int n = c->n_sys;
  if (c->mode == 1) {
    // fixed spheres in the background flow, plus the prescribed forces and torques
    launch_rhs(c->tg.n, c->d_colloc_abs, c->d_owner, c->d_sqrtw, c->src.cen64, c->d_zero, c->d_zero, c->bg.data(),
               c->d_wb, c->stream);
    CUDA_TRY(c, cudaMemcpyAsync(c->d_wb + c->n, c->d_border, sizeof(double) * 6 * c->P, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    launch_rhs(c->tg.n, c->d_colloc_abs, c->d_owner, c->d_sqrtw, c->src.cen64, c->d_v, c->d_om, c->bg.data(), c->d_wb,
               c->stream);
  }
  CHECK_LAUNCH(c);
  double bnorm = 0;
  if ((s = norm64(c, c->d_wb, bnorm)) != MFS_OK) return s;
  int iters = 0, refinements = 0;
  double rel = 0;
  bool converged = false;
  if (!(bnorm > 0)) {
    CUDA_TRY(c, cudaMemsetAsync(c->d_mu, 0, sizeof(double) * n, c->stream));
    converged = std::isfinite(bnorm);
    if (!converged) return c->fail(MFS_ERR_NUMERIC, "boundary data is not finite");
  } else if (o.precision == MFS_FP64 || o.precision == MFS_MIXED) {
    // FP64 GMRES; MIXED evaluates the pair sums in double-float on the FP32 pipes.  The
    // residual is re-evaluated with the same operator after each pass and the correction
    // equation solved again if a restart-limited pass fell short (iterative refinement).
    c->dw_pairs = (o.precision == MFS_MIXED);
    c->dw_fast_a = c->dw_pairs;
    c->ff_pass = c->dw_pairs;  // far field (if built) in the passes only
    CUDA_TRY(c, cudaMemsetAsync(c->d_mu, 0, sizeof(double) * n, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_r, c->d_wb, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    double rn = bnorm;
    rel = 1.0;
    for (int it = 0; it <= o.max_refine; ++it) {
      if (rel <= o.tol) break;
      if (it == o.max_refine || iters >= o.max_iter) break;
      int it_in = 0;
      double est = 0;
      // solve G_hat e = r with the relative accuracy still missing, then mu += e
      if ((s = gmres<double>(c, c->d_r, c->d_w64, std::min(0.5, kInnerTol * o.tol / rel), o.restart, o.max_iter - iters,
                             it_in, est)) != MFS_OK) {
        c->dw_pairs = c->dw_fast_a = c->ff_pass = false;
        return s;
      }
      iters += it_in;
      {
        double one = 1.0;
        CUDA_TRY(c, cudaMemcpyAsync(c->d_h + 4 * 512 + 8, &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
        launch_update<double>(n, 1, c->d_w64, n, c->d_h + 4 * 512 + 8, 1.0, c->d_mu, c->stream);
      }
      // refinement residual with the native FP64 operator (the double-float passes then only
      // have to contract the error, and the final accuracy is that of FP64), or, at tolerances
      // far above its accuracy floor, with the double-float operator
      c->dw_pairs = dw_residual(o);
      c->dw_fast_a = c->ff_pass = false;
      sys_apply<double>(c, c->d_mu, c->d_w64);
      c->dw_pairs = (o.precision == MFS_MIXED);
      c->dw_fast_a = c->ff_pass = c->dw_pairs;
      launch_sub(n, c->d_wb, c->d_w64, c->d_r, c->stream);
      CHECK_LAUNCH(c);
      double rprev = rn;
      if ((s = norm64(c, c->d_r, rn)) != MFS_OK) {
        c->dw_pairs = c->dw_fast_a = c->ff_pass = false;
        return s;
      }
      rel = rn / bnorm;
      if (it > 0) ++refinements;
      if (!std::isfinite(rn)) {
        c->dw_pairs = c->dw_fast_a = c->ff_pass = false;
        return c->fail(MFS_ERR_NUMERIC, "residual is not finite");
      }
      if (rn > 0.9 * rprev && rel > o.tol) break;
    }
    c->dw_pairs = c->dw_fast_a = c->ff_pass = false;
    converged = rel <= o.tol;
  } else {
    // MFS_FP32: FP64 residual, FP32 inner GMRES on the normalised residual
    CUDA_TRY(c, cudaMemsetAsync(c->d_mu, 0, sizeof(double) * n, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_r, c->d_wb, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    double rn = bnorm;
    rel = 1.0;
    for (int it = 0; it <= o.max_refine; ++it) {
      if (rel <= o.tol) {
        converged = true;
        break;
      }
      if (it == o.max_refine || iters >= o.max_iter) break;
      launch_convert<double, float>(n, c->d_r, 1.0 / rn, c->d_in32, c->stream);
      int it_in = 0;
      double est = 0;
      if ((s = gmres<float>(c, c->d_in32, c->d_out32, std::max(o.inner_tol, o.tol / rel * 0.5), o.restart,
                            o.max_iter - iters, it_in, est)) != MFS_OK)
        return s;
      iters += it_in;
      launch_axpy_mixed(n, rn, c->d_out32, c->d_mu, c->stream);
      apply_op<double>(c, c->d_mu, c->d_w64);
      launch_sub(n, c->d_wb, c->d_w64, c->d_r, c->stream);
      CHECK_LAUNCH(c);
      double rprev = rn;
      if ((s = norm64(c, c->d_r, rn)) != MFS_OK) return s;
      rel = rn / bnorm;
      ++refinements;
      if (!std::isfinite(rn)) return c->fail(MFS_ERR_NUMERIC, "refinement residual is not finite");
      if (rn > 0.9 * rprev && rel > o.tol) break;  // refinement stagnates at the FP32 operator's accuracy
    }
    if (rel <= o.tol) converged = true;
  }
  // lambda = B^+ mu (double-float factors for MFS_MIXED, FP64 otherwise), then forces and torques
  c->dw_pairs = (o.precision == MFS_MIXED);
  precond<double>(c, c->d_mu, c->d_lam);
  c->dw_pairs = c->dw_fast_a = false;
  launch_forces_torques(c->src, c->d_lam, c->d_F, c->d_T, c->stream);
  if (c->mode == 1) {
    // rigid velocities from the border unknowns (V_k, Omega_k) per sphere
    CUDA_TRY(c, cudaMemcpy2DAsync(c->d_v, 3 * sizeof(double), c->d_mu + c->n, 6 * sizeof(double), 3 * sizeof(double),
                                  c->P, cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpy2DAsync(c->d_om, 3 * sizeof(double), c->d_mu + c->n + 3, 6 * sizeof(double),
                                  3 * sizeof(double), c->P, cudaMemcpyDeviceToDevice, c->stream));
  }
  CHECK_LAUNCH(c);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if ((s = check_tc_timeout(c)) != MFS_OK) return s;
  c->solved = true;
  if (info) {
    info->iters = iters;
    info->refinements = refinements;
    info->rel_residual = rel;
    info->converged = converged ? 1 : 0;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  if (!converged) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "not converged: relative residual %.3e after %d iterations", rel, iters);
    return c->fail(MFS_ERR_NOT_CONVERGED, buf);
  }
  return MFS_OK;
}

mfs_status mfs_get_forces_torques(mfs_ctx* c, double* F, double* T) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (!c->solved) return c->fail(MFS_ERR_STATE, "no solution yet");
  if (!F || !T) return c->fail(MFS_ERR_ARG, "null output");
  CUDA_TRY(c, cudaMemcpyAsync(F, c->d_F, sizeof(double) * 3 * c->P, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(T, c->d_T, sizeof(double) * 3 * c->P, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MFS_OK;
}

mfs_status mfs_get_forces_torques_device(mfs_ctx* c, double* F, double* T) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (!c->solved) return c->fail(MFS_ERR_STATE, "no solution yet");
  if (!F || !T) return c->fail(MFS_ERR_ARG, "null output");
  CUDA_TRY(c, cudaMemcpyAsync(F, c->d_F, sizeof(double) * 3 * c->P, cudaMemcpyDeviceToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(T, c->d_T, sizeof(double) * 3 * c->P, cudaMemcpyDeviceToDevice, c->stream));
  return MFS_OK;
}

mfs_status mfs_eval_velocity(mfs_ctx* c, int npts, const double* x, double* u) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (!c->solved) return c->fail(MFS_ERR_STATE, "no solution yet");
  if (npts < 0 || (npts > 0 && (!x || !u))) return c->fail(MFS_ERR_ARG, "bad evaluation arrays");
  if (npts == 0) return MFS_OK;
  // temporary target set: absolute positions, no self exclusion (sphere index -1)
  std::vector<double> t64(4 * (size_t)npts);
  for (int i = 0; i < npts; ++i) {
    for (int q = 0; q < 3; ++q) t64[4 * i + q] = x[3 * i + q];
    t64[4 * i + 3] = 1.0;
  }
  int nt = (npts + kTileTargets - 1) / kTileTargets;
  std::vector<int> ts(nt, -1), tst(nt), tcn(nt);
  for (int t = 0; t < nt; ++t) {
    tst[t] = t * kTileTargets;
    tcn[t] = std::min(kTileTargets, npts - t * kTileTargets);
  }
  std::vector<void*> tmp;
  auto ta = [&](size_t bytes) -> void* {
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    tmp.push_back(q);
    return q;
  };
  auto done = [&](mfs_status st) {
    cudaStreamSynchronize(c->stream);
    for (void* q : tmp) cudaFree(q);
    return st;
  };
  TargetSet tg;
  tg.n = npts;
  tg.n_tiles = nt;
  tg.pos64 = (double*)ta(t64.size() * 8);
  tg.tile_sphere = (int*)ta(nt * 4);
  tg.tile_start = (int*)ta(nt * 4);
  tg.tile_count = (int*)ta(nt * 4);
  double* du = (double*)ta(3 * (size_t)npts * 8);
  if (!tg.pos64 || !tg.tile_sphere || !tg.tile_start || !tg.tile_count || !du)
    return done(c->fail(MFS_ERR_OOM, "device allocation failed: evaluation points"));
  cudaMemcpyAsync(tg.pos64, t64.data(), t64.size() * 8, cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(tg.tile_sphere, ts.data(), nt * 4, cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(tg.tile_start, tst.data(), nt * 4, cudaMemcpyHostToDevice, c->stream);
  cudaMemcpyAsync(tg.tile_count, tcn.data(), nt * 4, cudaMemcpyHostToDevice, c->stream);
  launch_pairs<double>(tg, c->src, c->d_lam, nullptr, du, c->hd.prm.visc, c->stream);
  cudaMemcpyAsync(u, du, 3 * (size_t)npts * 8, cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return done(c->fail(MFS_ERR_CUDA, std::string("eval: ") + cudaGetErrorString(e)));
  return done(MFS_OK);
}

mfs_status mfs_get_strengths(mfs_ctx* c, double* lambda, double* pos, int* type) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  const HostDisc& d = c->hd;
  if (lambda) {
    if (!c->solved) return c->fail(MFS_ERR_STATE, "no solution yet");
    CUDA_TRY(c, cudaMemcpyAsync(lambda, c->d_lam, sizeof(double) * c->n_unk, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  if (pos || type) {
    long long v = 0;
    const int N = d.prm.n_proxy;
    for (int k = 0; k < d.P; ++k) {
      for (int j = 0; j < N; ++j, ++v) {
        if (pos)
          for (int q = 0; q < 3; ++q) pos[3 * v + q] = d.centres[3 * k + q] + d.proxy_rel[3 * j + q];
        if (type) type[v] = 0;
      }
      for (int j = d.img_off[k]; j < d.img_off[k + 1]; ++j)
        for (int t = 0; t < 3; ++t, ++v) {
          if (pos)
            for (int q = 0; q < 3; ++q) pos[3 * v + q] = d.image[3 * j + q];
          if (type) type[v] = t;
        }
    }
  }
  return MFS_OK;
}

mfs_status mfs_get_collocation(mfs_ctx* c, double* x, double* w, int* owner) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  const HostDisc& d = c->hd;
  if (x) std::copy(d.colloc.begin(), d.colloc.end(), x);
  if (w) std::copy(d.weight.begin(), d.weight.end(), w);
  if (owner) std::copy(d.owner.begin(), d.owner.end(), owner);
  return MFS_OK;
}

mfs_status mfs_get_rhs(mfs_ctx* c, double* wb) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (!wb) return c->fail(MFS_ERR_ARG, "null output");
  launch_rhs(c->tg.n, c->d_colloc_abs, c->d_owner, c->d_sqrtw, c->src.cen64, c->d_v, c->d_om, c->bg.data(), c->d_wb, c->stream);
  CHECK_LAUNCH(c);
  CUDA_TRY(c, cudaMemcpyAsync(wb, c->d_wb, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MFS_OK;
}

// Runs one step of the operator on host data: stage inputs, compute, read back.
static mfs_status run_step(mfs_ctx* c, int precision, int which, const double* in1, const double* in2, double* out) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (precision != MFS_FP64 && precision != MFS_MIXED && precision != MFS_FP32 && precision != MFS_MIXED_PASS)
    return c->fail(MFS_ERR_ARG, "precision must be MFS_FP64, MFS_MIXED, MFS_FP32 or MFS_MIXED_PASS");
  if (!in1 || !out || (which == 2 && !in2)) return c->fail(MFS_ERR_ARG, "null array");
  if (which != 2 && !c->factored) return c->fail(MFS_ERR_STATE, "built without one-body factors (build_factors = 0)");
  const long long n = c->n, nu = c->n_unk;
  const long long len1 = which == 2 ? nu : n;      // pairs: first input is lambda_hat
  const long long lenout = which == 1 ? nu : n;    // precond: output in source space
  double* d1 = which == 2 ? c->d_lam : c->d_mu;
  // the operator-step entry points reuse the solution buffers; a later get_* must re-solve
  c->solved = false;
  CUDA_TRY(c, cudaMemcpyAsync(d1, in1, sizeof(double) * len1, cudaMemcpyHostToDevice, c->stream));
  if (which == 2) CUDA_TRY(c, cudaMemcpyAsync(c->d_mu, in2, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
  double* dout = which == 1 ? c->d_lh64 : c->d_w64;
  if (precision != MFS_FP32) {
    c->dw_pairs = (precision == MFS_MIXED || precision == MFS_MIXED_PASS);
    c->dw_fast_a = c->ff_pass = (precision == MFS_MIXED_PASS);
    if (which == 0) apply_op<double>(c, c->d_mu, c->d_w64);
    else if (which == 1) precond<double>(c, c->d_mu, c->d_lh64);
    else pairs_step<double>(c, c->d_lam, c->d_mu, c->d_w64);
    c->dw_pairs = c->dw_fast_a = c->ff_pass = false;
  } else {
    launch_convert<double, float>(len1, d1, 1.0, c->d_in32, c->stream);
    if (which == 0) {
      apply_op<float>(c, c->d_in32, c->d_out32);
    } else if (which == 1) {
      precond<float>(c, c->d_in32, c->d_out32);
    } else {
      launch_convert<double, float>(n, c->d_mu, 1.0, c->d_mu32, c->stream);
      pairs_step<float>(c, c->d_in32, c->d_mu32, c->d_out32);
    }
    launch_convert<float, double>(lenout, c->d_out32, 1.0, dout, c->stream);
  }
  CHECK_LAUNCH(c);
  CUDA_TRY(c, cudaMemcpyAsync(out, dout, sizeof(double) * lenout, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->prof) collect_events(c);
  return check_tc_timeout(c);
}

mfs_status mfs_batch_solve(int n_problems, mfs_ctx* const* ctxs, const mfs_solve_opts* opts, mfs_solve_info* infos) {
  if (n_problems < 0 || (n_problems > 0 && !ctxs)) return MFS_ERR_ARG;
  for (int i = 0; i < n_problems; ++i)
    if (!ctxs[i]) return MFS_ERR_ARG;
  if (n_problems == 0) return MFS_OK;
  mfs_solve_opts o;
  if (opts) o = *opts; else mfs_default_solve_opts(&o);
  if (o.precision == MFS_FP64 || o.precision == MFS_MIXED) return batch_lockstep(n_problems, ctxs, o, infos);
  // MFS_FP32: independent solves, concurrently on the contexts' own streams
  std::vector<mfs_status> st(n_problems, MFS_OK);
  std::atomic<int> next{0};
  unsigned hw = std::thread::hardware_concurrency();
  int n_threads = std::max(1, std::min(n_problems, (int)std::max(4u, std::min(hw ? 2 * hw : 16u, 64u))));
  auto work = [&]() {
    for (int i = next++; i < n_problems; i = next++) st[i] = mfs_solve(ctxs[i], &o, infos ? &infos[i] : nullptr);
  };
  std::vector<std::thread> pool;
  for (int t = 0; t < n_threads; ++t) pool.emplace_back(work);
  for (auto& t : pool) t.join();
  for (int i = 0; i < n_problems; ++i)
    if (st[i] != MFS_OK) return st[i];
  return MFS_OK;
}

static mfs_status batch_rhs_common(int n, mfs_ctx* const* ctxs, const double* const* v, const double* const* omega,
                                   bool dev, const mfs_solve_opts* opts, mfs_solve_info* infos, double* const* F,
                                   double* const* T) {
  if (n < 0 || (n > 0 && (!ctxs || !v || !omega))) return MFS_ERR_ARG;
  for (int i = 0; i < n; ++i)
    if (!ctxs[i]) return MFS_ERR_ARG;
  if (n == 0) return MFS_OK;
  mfs_solve_opts o;
  if (opts) o = *opts; else mfs_default_solve_opts(&o);
  if (o.precision != MFS_FP64 && o.precision != MFS_MIXED)
    return ctxs[0]->fail(MFS_ERR_UNSUPPORTED, "batched right-hand sides support MFS_FP64 and MFS_MIXED");
  BatchIO io;
  io.v = v;
  io.w = omega;
  io.in_device = dev;
  io.F = F;
  io.T = T;
  io.out_device = dev;
  io.repeats = true;
  return batch_lockstep(n, ctxs, o, infos, io);
}

mfs_status mfs_batch_solve_rhs(int n_problems, mfs_ctx* const* ctxs, const double* const* v, const double* const* omega,
                               const mfs_solve_opts* opts, mfs_solve_info* infos, double* const* F, double* const* T) {
  return batch_rhs_common(n_problems, ctxs, v, omega, false, opts, infos, F, T);
}

mfs_status mfs_batch_solve_rhs_device(int n_problems, mfs_ctx* const* ctxs, const double* const* d_v,
                                      const double* const* d_omega, const mfs_solve_opts* opts, mfs_solve_info* infos,
                                      double* const* d_F, double* const* d_T) {
  return batch_rhs_common(n_problems, ctxs, d_v, d_omega, true, opts, infos, d_F, d_T);
}

mfs_status mfs_probe_alu_peak(int device, int which, double* tflops, double* ms) {
  if ((which != 0 && which != 1) || !tflops) return MFS_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return MFS_ERR_CUDA;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return MFS_ERR_CUDA;
  }
  void* sink = nullptr;
  if (cudaMalloc(&sink, 16) != cudaSuccess) {
    cudaGetLastError();
    return MFS_ERR_OOM;
  }
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mfs_status out = MFS_OK;
  const int blocks = sms * 8;                   // 8 CTAs of 256 threads per SM
  const int iters = which == 0 ? 40000 : 1200;  // ~0.2 s at the respective peak
  float t = 0.f;
  double flops = 0;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    out = MFS_ERR_CUDA;
  } else {
    launch_fma_probe(which, blocks, iters / 8, sink, st);  // warm-up
    cudaEventRecord(e0, st);
    flops = launch_fma_probe(which, blocks, iters, sink, st);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || !(t > 0.f))
      out = MFS_ERR_CUDA;
  }
  cudaGetLastError();
  if (out == MFS_OK) {
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(sink);
  return out;
}

mfs_status mfs_tune_pairs(mfs_ctx* c, mfs_pair_shapes* out) {
  mfs_status s = check_state(c, 2);
  if (s != MFS_OK) return s;
  if (c->tg.n_tiles == 0) return c->fail(MFS_ERR_STATE, "no collocation nodes to tune on");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(c, cudaEventCreate(&e0));
  CUDA_TRY(c, cudaEventCreate(&e1));
  struct EvFree {
    cudaEvent_t a, b;
    ~EvFree() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evf{e0, e1};
  // inputs: the context's work buffers, zeroed (the launches' cost does not depend on the values)
  CUDA_TRY(c, cudaMemsetAsync(c->d_lh64, 0, sizeof(double) * c->n_unk, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_mu, 0, sizeof(double) * c->n, c->stream));
  if (c->d_q) CUDA_TRY(c, cudaMemsetAsync(c->d_q, 0, sizeof(float) * 3 * (size_t)c->ff.n_eq * c->P, c->stream));
  const double visc = c->hd.prm.visc;
  // each candidate: one warm-up and two timed launches
  auto time_it = [&](auto&& launch, double& ms) -> mfs_status {
    launch();
    CUDA_TRY(c, cudaEventRecord(e0, c->stream));
    launch();
    launch();
    CUDA_TRY(c, cudaEventRecord(e1, c->stream));
    CHECK_LAUNCH(c);
    CUDA_TRY(c, cudaEventSynchronize(e1));
    float t = 0;
    CUDA_TRY(c, cudaEventElapsedTime(&t, e0, e1));
    ms = t / 2.0;
    return MFS_OK;
  };
  // parts 0: the wave-filling rule; packed -1: the scalar far kernel
  const std::vector<PairShape> cands = {{1, 1, 0}, {1, 0, 0}, {4, 1, 0}, {4, 0, 0}};
  const std::vector<PairShape> far_cands = {{1, 1, 0}, {1, 0, 0}, {4, 1, 0}, {4, 0, 0}, {4, 1, -1}, {4, 0, -1}};
  auto tune = [&](auto&& launch_with, PairShape& best, double& best_ms, const std::vector<PairShape>& cs) -> mfs_status {
    best_ms = -1;
    for (const PairShape& sh : cs) {
      if (sh.nt == 1 && c->tg.n_tiles1 == 0) continue;
      double ms = 0;
      mfs_status st = time_it([&] { launch_with(sh); }, ms);
      if (st != MFS_OK) return st;
      if (best_ms < 0 || ms < best_ms) {
        best_ms = ms;
        best = sh;
      }
    }
    return MFS_OK;
  };
  mfs_pair_shapes r{};
  double ms = 0;
  PairShape best;
  if ((s = tune([&](PairShape sh) { launch_pairs_dw(c->tg, c->src, c->d_lh64, c->d_mu, c->d_w64, visc, c->d_pparts,
                                                    kPairMaxParts, c->stream, sh); },
                best, ms, cands)) != MFS_OK)
    return s;
  c->shape_all = best;
  PairShape ra = resolve_dw_shape(c->tg, c->src, best, kPairMaxParts);
  r.all_nodes_per_thread = ra.nt;
  r.all_parts = ra.parts;
  r.all_ms = ms;
  if (c->ff.n_eq > 0) {
    if ((s = tune([&](PairShape sh) { launch_pairs_dw_near(c->tg, c->src, c->ff, c->d_lh64, c->d_mu, c->d_w64, visc,
                                                           c->d_pparts, kPairMaxParts, c->stream, sh); },
                  best, ms, cands)) != MFS_OK)
      return s;
    c->shape_near = best;
    PairShape rn = resolve_near_shape(c->tg, best, kPairMaxParts);
    r.near_nodes_per_thread = rn.nt;
    r.near_parts = rn.parts;
    r.near_ms = ms;
    if ((s = tune([&](PairShape sh) { launch_pairs_far(c->tg, c->src, c->ff, c->d_w64, visc, c->d_pparts,
                                                       kPairMaxParts, c->stream, sh); },
                  best, ms, far_cands)) != MFS_OK)
      return s;
    c->shape_far = best;
    PairShape rf = resolve_far_shape(c->tg, best, kPairMaxParts);
    r.far_nodes_per_thread = rf.nt;
    r.far_parts = rf.parts;
    r.far_packed = rf.packed;
    r.far_ms = ms;
  }
  c->solved = false;  // the work buffers were overwritten
  if (out) *out = r;
  return MFS_OK;
}

mfs_status mfs_set_memory_limit(mfs_ctx* c, unsigned long long bytes) {
  if (!c) return MFS_ERR_ARG;
  c->mem_limit = bytes;
  return MFS_OK;
}

mfs_status mfs_memory_in_use(const mfs_ctx* c, unsigned long long* bytes) {
  if (!c || !bytes) return MFS_ERR_ARG;
  *bytes = c->mem_used;
  return MFS_OK;
}

mfs_status mfs_set_profiling(mfs_ctx* c, int on) {
  if (!c) return MFS_ERR_ARG;
  c->prof = on != 0;
  return MFS_OK;
}

mfs_status mfs_get_timing(mfs_ctx* c, mfs_timing_t* out, int reset) {
  if (!c || !out) return MFS_ERR_ARG;
  if (c->prof && c->stream) {
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    collect_events(c);
  }
  *out = c->tm;
  if (reset) c->tm = mfs_timing_t{};
  return MFS_OK;
}

// ---- pseudo-inverse apply that allocates nothing
// Scratch for the intermediate Sigma^+ U^T mu of every sphere, resident on each GPU that
// loads the library until the process exits.  Host code reaches it only through the device
// address looked up below; the array's host-side name is a stand-in, not a device pointer.
constexpr long long kNoAllocScratch = 1LL << 21;  // doubles (16 MiB)
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

static std::mutex g_noalloc_mtx;
static double* g_noalloc_ptr[64] = {nullptr};
static void* g_noalloc_cuctx[64] = {nullptr};  // driver context of each cached lookup

// The calling thread's current driver context (CUcontext), through the runtime's entry-point
// query so that the library does not link the driver library itself; null if unavailable.
static void* current_driver_context() {
  using GetCurrent = int (*)(void**);
  static GetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<GetCurrent>(f);
  }();
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

mfs_status mfs_apply_precond_noalloc(mfs_ctx* c, const double* d_mu, double* d_lambda_hat) {
  mfs_status s = check_state(c, 2);  // also makes the context's device current
  if (s != MFS_OK) return s;
  if (!c->factored) return c->fail(MFS_ERR_STATE, "built without one-body factors (build_factors = 0)");
  if (!d_mu || !d_lambda_hat) return c->fail(MFS_ERR_ARG, "null device pointer");
  if (c->tmp_len > kNoAllocScratch)
    return c->fail(MFS_ERR_ARG, "mfs_apply_precond_noalloc: the summed retained ranks (" + std::to_string(c->tmp_len) +
                                    ") exceed its fixed scratch of " + std::to_string(kNoAllocScratch) + " doubles");
  if (c->device < 0 || c->device >= 64) return c->fail(MFS_ERR_ARG, "device index out of range for the static scratch table");
  double* scratch = nullptr;
  {
    // first call on this device (or in a new driver context of it, e.g. after a device reset):
    // resolve the array's device address with the device current
    std::lock_guard<std::mutex> g(g_noalloc_mtx);
    void* cu = current_driver_context();
    if (!g_noalloc_ptr[c->device] || !cu || cu != g_noalloc_cuctx[c->device]) {
      double* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return c->fail(MFS_ERR_CUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
      }
      g_noalloc_ptr[c->device] = ptr;
      g_noalloc_cuctx[c->device] = cu;
    }
    scratch = g_noalloc_ptr[c->device];
  }
  // every scratch entry that the second GEMV reads is written by the first one of the same
  // call, so nothing has to be cleared between calls
  launch_gemv<double>(c->gA64, d_mu, scratch, c->stream);
  launch_gemv<double>(c->gV64, scratch, d_lambda_hat, c->stream);
  CHECK_LAUNCH(c);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MFS_OK;
}

mfs_status mfs_apply_operator(mfs_ctx* c, int precision, const double* mu, double* out) {
  return run_step(c, precision, 0, mu, nullptr, out);
}
mfs_status mfs_apply_precond(mfs_ctx* c, int precision, const double* mu, double* lambda_hat) {
  return run_step(c, precision, 1, mu, nullptr, lambda_hat);
}
mfs_status mfs_apply_pairs(mfs_ctx* c, int precision, const double* lambda_hat, const double* mu, double* out) {
  return run_step(c, precision, 2, lambda_hat, mu, out);
}

}  // extern "C"
