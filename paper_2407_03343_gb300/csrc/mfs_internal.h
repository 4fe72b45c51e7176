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

// ---------------------------------------------------------------- device-side views

// Target (collocation) nodes grouped by sphere, processed in tiles that never straddle
// a sphere, so the self block of step 2 can be skipped per tile (Sec. 2.2, direct summation).
struct TargetSet {
  int n = 0;             // nodes
  int n_tiles = 0;
  float4* pos32 = nullptr;   // (x - c_k, y - c_k, z - c_k, sqrt w) per node, FP32
  double* pos64 = nullptr;   // same, 4 doubles per node
  int* tile_sphere = nullptr;
  int* tile_start = nullptr;
  int* tile_count = nullptr;
};

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

// Kernels launched so far by the calling host thread (every launcher below counts itself).
long long launches_on_this_thread();

// Kernel launchers (mfs_kernels.cu).  All run on `st`.
template <typename T>
void launch_pairs(const TargetSet& tg, const SourceSet& src, const T* lam_hat, const T* mu,
                  T* out, double visc, cudaStream_t st);

// Same sums as launch_pairs<double> (FP64 in and out) computed in double-float arithmetic on
// the FP32 pipes.
void launch_pairs_dw(const TargetSet& tg, const SourceSet& src, const double* lam_hat, const double* mu,
                     double* out, double visc, cudaStream_t st);

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
};
template <typename T>
void launch_gemv(const GemvBatch<T>& b, const T* x, T* y, cudaStream_t st);

// Self block B_k = W_k G^(kk) assembled column-major FP64 (rows 3 M_k, cols 3 N_k, lda rows)
// with columns in the strength order of the library.
void launch_assemble_self(const HostDisc& hd, int k, const double* d_colloc_rel, const double* d_sqrtw,
                          const double* d_src_rel, const int* d_src_type, int n_src, double* B, int lda,
                          cudaStream_t st);

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

// Forces and torques (Sec. 2.3 remark), FP64, one CTA per sphere.
void launch_forces_torques(const SourceSet& src, const double* lam, double* F, double* T, cudaStream_t st);
// Right-hand side W (v + omega x (x - c) - u_inf(x)), FP64.
void launch_rhs(int n, const double* colloc_abs, const int* owner, const double* sqrtw, const double* cen,
                const double* v, const double* om, const double* bg /* 15 doubles: U, E, Omega */,
                double* wb, cudaStream_t st);

}  // namespace mfs
