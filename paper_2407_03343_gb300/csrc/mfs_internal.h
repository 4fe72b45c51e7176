// Internal declarations shared by the translation units of libmfs.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mfs.h"

namespace mfs {

// One near contact (Sec. 2.3): spheres k < kp with gap delta (radius units) and n_im
// image nodes on each sphere's half of the centre-centre line.
struct Contact {
  int k, kp;
  double delta;
  int nim;
};

// Host copy of the discretisation (Sec. 2.1, 2.3, 5.1).  Everything the device needs
// is derived from this once per build.
struct HostDisc {
  int P = 0;
  double a = 1.0;
  mfs_params prm{};
  std::vector<double> centres;        // 3P
  std::vector<Contact> contacts;
  std::vector<int> colloc_off;        // P+1, node offsets
  std::vector<double> colloc;         // 3 * n_colloc, absolute positions
  std::vector<double> weight;         // n_colloc, area weights w_i
  std::vector<int> owner;             // n_colloc
  std::vector<double> proxy_rel;      // 3N, proxy positions relative to the owner centre
  std::vector<int> img_off;           // P+1, image-node offsets
  std::vector<double> image;          // 3 * n_img, absolute positions
  std::vector<int> img_owner;         // n_img
  std::vector<long long> unk_off;     // P+1, offsets in the strength vector (3N + 9 n_img_k per sphere)
  std::vector<int> factor_id;         // P, which one-body factor serves sphere k
  std::vector<int> factor_rep;        // per factor, a sphere whose self block defines it
  int n_colloc() const { return colloc_off.empty() ? 0 : colloc_off.back(); }
  int n_img() const { return img_off.empty() ? 0 : img_off.back(); }
  long long n_unknowns() const { return unk_off.empty() ? 0 : unk_off.back(); }
};

// Builds the discretisation; returns MFS_OK or MFS_ERR_GEOMETRY / MFS_ERR_ARG with err set.
mfs_status build_discretisation(const double* centres, int P, double a, const mfs_params& p,
                                HostDisc& out, std::string& err);

// n points of the quasi-uniform Fibonacci grid (the basic-grid construction of Sec. 2.1) on the
// sphere of radius r about the origin, 3 n values.
void fibonacci_sphere(int n, double r, std::vector<double>& out);

// ---------------------------------------------------------------- device-side views

// Target (collocation) nodes grouped by sphere, processed in tiles that never straddle
// a sphere, so the self block of step 2 can be skipped per tile (Sec. 2.2, direct summation).
struct TargetSet {
  int n = 0;             // nodes
  int n_tiles = 0;       // tiles of up to 512 nodes (4 per thread)
  int n_tiles1 = 0;      // tiles of up to 128 nodes (1 per thread), used when there are few large tiles
  float4* pos32 = nullptr;   // (x - c_k, y - c_k, z - c_k, sqrt w) per node, FP32
  double* pos64 = nullptr;   // same, 4 doubles per node
  int* tile_sphere = nullptr;
  int* tile_start = nullptr;
  int* tile_count = nullptr;
  int* tile1_sphere = nullptr;
  int* tile1_start = nullptr;
  int* tile1_count = nullptr;
};

// Tile size choice: 4 nodes per thread once the large tiles fill the GPU twice over.
inline int pair_nodes_per_thread(int n_tiles_large) { return n_tiles_large >= 2 * 152 ? 4 : 1; }

struct SourceSet {
  int P = 0, N = 0, n_img = 0;
  float4* proxy32 = nullptr;   // N positions relative to the owner centre (same for every sphere)
  double* proxy64 = nullptr;   // 4 doubles per proxy (x, y, z, 0)
  float4* img32 = nullptr;     // image node positions relative to the owner centre
  double* img64 = nullptr;     // 4 doubles per node (x, y, z, 0)
  int* img_owner = nullptr;
  long long* unk_off = nullptr;  // P+1
  int* img_off = nullptr;        // P+1
  float* cen_hi = nullptr;       // 3P, centres split into FP32 hi + lo parts
  float* cen_lo = nullptr;
  double* cen64 = nullptr;       // 3P
};

// Far-field representation of the other spheres' sources in the GMRES passes (built when
// mfs_params.far_dist > 0): for target sphere k the spheres within far_dist of it ("near") are
// summed directly in double-float; every other sphere k' acts through n_eq equivalent
// Stokeslets on a sphere about c_k' whose strengths q_k' = Q_f mu_k' come from one FP32
// matrix per distinct one-body factor (Q_f maps the sphere's collocation data to the
// equivalent sources reproducing the field of B_f^+ mu outside the check sphere).
struct FarField {
  int n_eq = 0;
  float4* eq32 = nullptr;   // equivalent-source positions relative to the owner centre
  int* near_off = nullptr;  // P+1: CSR of the near spheres of each sphere, ascending
  int* near_idx = nullptr;
  int* excl_off = nullptr;  // P+1: the near spheres and the sphere itself, ascending (far: the rest)
  int* excl_idx = nullptr;
  const float* q = nullptr; // equivalent strengths, 3 n_eq per sphere, sphere-major
};

// Kernels launched so far by the calling host thread (every launcher below counts itself).
long long launches_on_this_thread();
void note_launch();

// Tensor-core product C = A X^T for the spheres sharing the basic factor (mfs_tc.cu): A (M x K)
// and X (n_cap x K) as three bf16 slices each (row-major, leading dimension ldk = K rounded up to
// the 64-element pipeline chunk, zero-padded), tensor maps prepared once.
struct TcGemm {
  int M = 0, K = 0, ldk = 0, n_cap = 0, nk = 0;
  alignas(64) unsigned char maps[6][128];  // CUtensorMap of A0 A1 A2 X0 X1 X2
  void* x_slices[3] = {nullptr, nullptr, nullptr};
};
int tc_ldk(int cols);
// slices of a row-major FP64 matrix (rows x cols, leading dimension ld) into rows x ldk bf16 matrices
void launch_split3_matrix(int rows, int cols, long long ld, const double* in, int ldk, void* s0, void* s1, void* s2,
                          cudaStream_t st);
void launch_split3_matrix_f32(int rows, int cols, long long ld, const float* in, int ldk, void* s0, void* s1, void* s2,
                              cudaStream_t st);
// tensor maps of the A slices (M rows) and X slices (n_cap rows), K columns; false if the driver
// cannot encode them or the kernel's shared memory cannot be raised
bool tc_prepare(TcGemm& g, const void* const a_slices[3], int M, const void* const x_slices[3], int n_cap, int K);
// FP32 partial-sum scratch (floats) that launch_tc_gemm needs for ncols columns
size_t tc_partial_floats(const TcGemm& g, int ncols);
// column n = x[x_off[n] ...]: slices it, multiplies on the tensor cores, and writes
// (A x_n)[m] to y32[y_off[n] + m] (FP32) or y2[y_off[n] + m] = (value, 0); err set on a wait timeout.
// slice_x = false reuses the X slices the previous product over the same x wrote.
void launch_tc_gemm(const TcGemm& g, int ncols, const double* x, const long long* x_off, const long long* y_off,
                    float* y32, float2* y2, float* partial, int* err, bool slice_x, cudaStream_t st);

// A launch shape: nodes per thread (4: 512-node tiles, 1: 128-node tiles, 0: by rule) and source
// parts per tile (0: the wave-filling rule, 1: no split, > 1: that many).
struct PairShape {
  int nt = 0;
  int parts = 0;
  int packed = 0;  // far kernel with 4 nodes per thread: 0 packed-FP32 (default), -1 scalar; resolved: 1 / 0
};

// Kernel launchers (mfs_kernels.cu).  All run on `st`.
template <typename T>
void launch_pairs(const TargetSet& tg, const SourceSet& src, const T* lam_hat, const T* mu,
                  T* out, double visc, cudaStream_t st);

// Same sums as launch_pairs<double> (FP64 in and out) computed in double-float arithmetic on
// the FP32 pipes.  With few target tiles the sources of each tile are split over up to
// max_parts CTAs whose partial sums go to `partial` (max_parts * 3 n doubles; null: no split)
// and are added in a second, deterministic pass.
void launch_pairs_dw(const TargetSet& tg, const SourceSet& src, const double* lam_hat, const double* mu,
                     double* out, double visc, double* partial, int max_parts, cudaStream_t st,
                     PairShape shape = PairShape());
// Source split of the 1-node-per-thread tiling: as many parts as keep the CTAs within one wave
// (152 SMs x 7 resident CTAs of the double-float kernel: 72 registers x 128 threads, 28 KB of
// shared memory), at least kPairSplitMinSources sources per part, at most max_parts.
constexpr int kPairSplitTarget = 152 * 7;
constexpr int kPairSplitMinSources = 64;
constexpr int kPairMaxParts = 16;
int pair_split_parts(long long n_tiles1, long long min_sources, int max_parts);

// Near part of the far-field split, double-float: out = mu + W sum over the near spheres of the
// target's sphere (their proxies and image triples) of G lambda_hat.
// Both split each tile's sources over up to max_parts CTAs (partial: max_parts * 3 n doubles, or
// null for no split) so that the grid fills whole waves of resident CTAs; the parts are added in
// a fixed order by a second kernel.
void launch_pairs_dw_near(const TargetSet& tg, const SourceSet& src, const FarField& ff, const double* lam_hat,
                          const double* mu, double* out, double visc, double* partial, int max_parts, cudaStream_t st,
                          PairShape shape = PairShape());
// Far part, FP32 with compensated cross-tile sums: out += W sum over the far spheres of the
// equivalent Stokeslets' field.
void launch_pairs_far(const TargetSet& tg, const SourceSet& src, const FarField& ff, double* out, double visc,
                      double* partial, int max_parts, cudaStream_t st, PairShape shape = PairShape());
// the shape a launch with `shape` resolves to (nodes per thread, parts), for reporting
PairShape resolve_near_shape(const TargetSet& tg, PairShape shape, int max_parts);
PairShape resolve_far_shape(const TargetSet& tg, PairShape shape, int max_parts);
PairShape resolve_dw_shape(const TargetSet& tg, const SourceSet& src, PairShape shape, int max_parts);

// Many problems per launch (FP64 data): a device table of per-problem kernel arguments, a work
// list of (problem, tile) pairs and a per-problem active flag.
size_t pair_args64_bytes();
void fill_pair_args64(void* host_dst, const TargetSet& tg, const SourceSet& src, const double* lam_hat,
                      const double* mu, double* out, double visc, int nodes_per_thread);
struct SegTable;
// parts > 1 (double-float, 1 node per thread only): sources split as in launch_pairs_dw, the
// partial sums in `partial` (parts slices of pstride doubles) reduced over the chunks of `seg`.
void launch_pairs_batch64(bool double_float, const void* d_args, const int2* d_work, int n_work, const int* d_active,
                          int nodes_per_thread, const double* lam, const double* mu, double* out,
                          const long long* d_uoff, const long long* d_voff, int parts, double* partial,
                          long long pstride, const SegTable& seg, cudaStream_t st, const long long* d_nlen = nullptr,
                          bool skip_reduce = false, unsigned* d_counter = nullptr);
// Several right-hand sides on one geometry (double-float, 1 node per thread): work[b] = (lead
// problem, tile, first index into rhs_prob, count <= kPairRhs); each pair's Green's function is
// formed once for all of the item's right-hand sides.  parts > 1 writes partial sums as
// launch_pairs_batch64 does; with d_counter (zeros, one per item) the last CTA of each item adds
// them, else the caller runs launch_pair_parts_reduce_batch once.
constexpr int kPairRhs = 3;
void launch_pairs_multi64(const void* d_args1, const int4* d_work, int n_work, const int* d_rhs, const int* d_active,
                          const double* lam, const double* mu, double* out, const long long* d_uoff,
                          const long long* d_voff, int parts, double* partial, long long pstride,
                          const long long* d_nlen, cudaStream_t st, unsigned* d_counter = nullptr);
void launch_pair_parts_reduce_batch(const void* d_args1, const SegTable& seg, const double* lam, const double* mu,
                                    double* out, const long long* d_uoff, const long long* d_voff, int parts,
                                    double* partial, long long pstride, const long long* d_nlen, cudaStream_t st);

// Batched GEMV: for every job j, y_j = M_j x_j with M_j row-major (rows_j x cols_j, leading dim ld_j).
template <typename T>
struct GemvBatch {
  const T** mat = nullptr;  // device array of device pointers
  int* rows = nullptr;
  int* cols = nullptr;
  int* ld = nullptr;
  long long* x_off = nullptr;
  long long* y_off = nullptr;
  int n_jobs = 0;
  int max_rows = 0;
  const int* job_prob = nullptr;  // optional: problem of each job, with
  const int* active = nullptr;    //   per-problem flags (jobs of inactive problems are skipped)
  const float2** mat_dw = nullptr;  // optional: the same matrices as (hi, lo) float pairs
  const int* job_list = nullptr;    // optional: the jobs to run (n_list of them); the grid then
  int n_list = 0;                   //   covers only those
};
template <typename T>
void launch_gemv(const GemvBatch<T>& b, const T* x, T* y, cudaStream_t st);
// Double-float GEMV on the FP32 pipes over b.mat_dw: x as (hi, lo) pairs; the result goes to
// y_dw as pairs, or to y64 joined into doubles when y_dw is null.
void launch_gemv_dw(const GemvBatch<double>& b, const float2* x, float2* y_dw, double* y64, cudaStream_t st);
// Double-float GEMV over an FP32 matrix (b.mat): x as (hi, lo) pairs, y_dw as pairs.  The matrix
// rows must start 16-byte aligned (ld a multiple of 4).
void launch_gemv_f32_dw(const GemvBatch<float>& b, const float2* x, float2* y_dw, cudaStream_t st);
// (hi, lo) float pairs of a double vector.
void launch_split_dw(long long n, const double* in, float2* out, cudaStream_t st);

// Self block B_k = W_k G^(kk) assembled column-major FP64 (rows 3 M_k, cols 3 N_k, lda rows)
// with columns in the strength order of the library.
void launch_assemble_self(const HostDisc& hd, int k, const double* d_colloc_rel, const double* d_sqrtw,
                          const double* d_src_rel, const int* d_src_type, int n_src, double* B, int lda,
                          cudaStream_t st);

// The same kernel matrix for m arbitrary targets (xrel, 3 m, row scale sqrtw, m) and n_src sources
// (yrel, 3 n_src, types 0 S / 1 R / 2 D), column-major with leading dimension lda.
void launch_assemble_block(int m, int n_src, const double* xrel, const double* sqrtw, const double* yrel,
                           const int* type, double visc, double* B, long long lda, cudaStream_t st);

// Krylov helpers.
template <typename T>
void launch_multidot(int n, int nvec, const T* V, long long ldv, const T* w, double* partial, int nblk,
                     cudaStream_t st);
void launch_reduce_partials(int nvec, int nblk, const double* partial, double* h, cudaStream_t st);
template <typename T>
void launch_update(int n, int nvec, const T* V, long long ldv, const double* h, double sign, T* w,
                   cudaStream_t st);
template <typename T>
void launch_scale_copy(int n, const T* w, double s, T* out, cudaStream_t st);
template <typename Tin, typename Tout>
void launch_convert(long long n, const Tin* in, double s, Tout* out, cudaStream_t st);
void launch_axpy_mixed(int n, double a, const float* x, double* y, cudaStream_t st);
void launch_sub(int n, const double* a, const double* b, double* out, cudaStream_t st);

// Segmented vector kernels over a concatenation of independent problems: chunk b covers
// [start[b], end[b]) and belongs to problem prob[b]; per-problem coefficients are stored
// vector-major, c[i * K + p].  Chunks of inactive problems do nothing.
struct SegTable {
  int K = 0, nchunks = 0;
  int chunk = 1024;             // longest chunk (at most 1024 elements)
  const int* prob = nullptr;
  const long long* start = nullptr;
  const long long* end = nullptr;
  const int* pchunk = nullptr;  // K+1 chunk offsets per problem
  const int* active = nullptr;
  const int* list = nullptr;    // optional: the chunks of the active problems (nlist of them); the
  int nlist = 0;                //   launches then cover only those
  unsigned* counter = nullptr;  // optional, K zeros: the dot products are then reduced per problem by
                                //   the last CTA of each problem instead of a second kernel
};
void launch_seg_dots(const SegTable& t, int nvec, const double* V, long long ldv, const double* w, double* partial,
                     double* h, cudaStream_t st);
void launch_seg_update(const SegTable& t, int nvec, const double* V, long long ldv, const double* coef, double sign,
                       double* w, cudaStream_t st);
void launch_seg_scale(const SegTable& t, const double* s, const double* in, double* out, cudaStream_t st);
// the same scaling, also writing the (hi, lo) float split of the result to x2 (the input of the
// next double-float apply, which then skips its own split)
void launch_seg_scale_split(const SegTable& t, const double* s, const double* in, double* out, float2* x2,
                            cudaStream_t st);
void launch_axpy64(long long n, double a, const double* x, double* y, cudaStream_t st);

// Device-resident GMRES state of a lockstep batch of K problems: per problem `restart`
// Hessenberg columns of ldh = restart + 1 entries, the Givens rotations, the rotated right-hand
// side g (g_0 = ||b||), its norm bn, the tolerance, the residual estimate, the step counts, the
// active flags (shared with the batch kernels), the scale of the next basis vector and an error
// flag (a non-finite Arnoldi value).
constexpr int kMaxGmresCol = 512;  // restart + 1 must not exceed this (the batch limit)
struct GivensState {
  double* H = nullptr;
  double* cs = nullptr;
  double* sn = nullptr;
  double* g = nullptr;
  const double* bn = nullptr;
  const double* tol = nullptr;
  double* est = nullptr;
  int* iters = nullptr;
  int* jused = nullptr;
  int* active = nullptr;
  double* scl = nullptr;
  int* err = nullptr;
  int K = 0, ldh = 0, restart = 0;
};
// Arnoldi step j from the CGS2 dot products h1, h2 (vector-major, h[i K + p]) and the squared
// norm hn of the orthogonalised vector; deactivates converged problems.
void launch_batch_givens(const GivensState& S, int j, const double* h1, const double* h2, const double* hn,
                         cudaStream_t st);
// coef[i K + p] = (R^{-1} g)_i over each problem's jused steps, zero up to jmax.
void launch_batch_backsolve(const GivensState& S, int jmax, double* coef, cudaStream_t st);

// Arithmetic-peak probe (which 0: FP32 FFMA, 1: FP64 DFMA) of `blocks` CTAs x 256 threads,
// `iters` loop trips; returns the flops the launch performs.  sink: 8 writable bytes.
double launch_fma_probe(int which, int blocks, int iters, void* sink, cudaStream_t st);

// Forces and torques (Sec. 2.3 remark), FP64, one CTA per sphere.
void launch_forces_torques(const SourceSet& src, const double* lam, double* F, double* T, cudaStream_t st);
// the same with F, T written every `stride` doubles per sphere and scaled by sF, sT
void launch_forces_torques_scaled(const SourceSet& src, const double* lam, double* F, double* T, int stride, double sF,
                                  double sT, cudaStream_t st);
// out[node] -= sqrt(w) (V_k + Omega_k x (x - c_k)), U = (V_k, Omega_k) per sphere, pos64 = targets' (x - c, sqrt w)
void launch_rigid_sub(int n, const int* owner, const double* pos64, const double* U, double* out, cudaStream_t st);
// Right-hand side W (v + omega x (x - c) - u_inf(x)), FP64.
void launch_rhs(int n, const double* colloc_abs, const int* owner, const double* sqrtw, const double* cen,
                const double* v, const double* om, const double* bg /* 15 doubles: U, E, Omega */,
                double* wb, cudaStream_t st);

}  // namespace mfs
