// Tensor-core part of step 1 (sm_103a tcgen05): the spheres that share the basic one-body factor.
//
// Equal spheres without contacts have identical self blocks, so one truncated pseudo-inverse
// B^+ = V Sigma^+ U^T serves all of them (Sec. 2.2; Sec. 4 needs a single SVD for equal spheres),
// and the products of one of its factors with every such sphere's collocation data mu_k form one
// matrix product instead of a batch of matrix-vector products:
//     C = A X^T,   A: M x K (Sigma^+ U^T, or the far-field matrix Q), row n of X: mu of sphere n.
// The GMRES passes apply Sigma^+ U^T at FP32 accuracy (FP32 entries, FP32-accurate sums), so the
// product is formed at that accuracy on the bf16 tensor cores: every operand is split into three
// bf16 slices (a = a0 + a1 + a2 holds an FP32 value exactly; x likewise to 24 bits) and the six
// slice products a_i x_j with i + j <= 2 accumulate in FP32 in tensor memory (the dropped ones are
// below 2^-24 of the product).
//
// Kernel: one CTA of 128 threads per (128-row, 128-column, K-range) tile.  Thread 0 drives a
// two-stage pipeline: TMA loads of the six 128 x 64 bf16 slice tiles of a K-chunk (128-byte
// swizzle) complete on a "full" mbarrier, 24 tcgen05.mma (6 slice pairs x 4 steps of K = 16)
// read them from shared memory and accumulate into a 128 x 128 FP32 tile in tensor memory, and a
// tcgen05.commit on the stage's "empty" mbarrier releases its buffers for the next load.  After
// the last chunk the four warps read the accumulator back with tcgen05.ld (warp w owns rows
// 32 w .. 32 w + 31) and write their partial tile; a second kernel adds the K-range partials in a
// fixed order (deterministic) and scatters the columns to the spheres' vectors.  Every wait is
// bounded by a clock limit; a CTA that runs out sets an error flag, drains what it issued (again
// bounded), frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "mfs_internal.h"

namespace mfs {
namespace {

constexpr int kTcM = 128;   // rows per tile (tensor-memory lanes)
constexpr int kTcN = 128;   // columns per tile (tensor-memory columns of the FP32 accumulator)
constexpr int kTcK = 64;    // K per pipeline stage: one 128-byte swizzle span of bf16
constexpr int kTcStages = 2;
constexpr int kTcSlices = 3;
constexpr int kTileBytes = kTcM * kTcK * 2;                      // 16 KB, A and X tiles alike
constexpr int kStageBytes = 2 * kTcSlices * kTileBytes;          // 96 KB: A0 A1 A2 X0 X1 X2
constexpr int kTcSmem = kTcStages * kStageBytes + 1024 + 256;    // + alignment slack + barriers
constexpr long long kWaitCycles = 4000000000LL;                  // ~2 s at 2 GHz

// slice pairs (i, j) with i + j <= 2, largest first
__constant__ int kPairI[6] = {0, 0, 1, 0, 1, 2};
__constant__ int kPairJ[6] = {0, 1, 0, 2, 1, 0};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// true once the phase of the given parity has completed; false after kWaitCycles
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor of a K-major operand tile written by TMA with 128-byte swizzle:
// rows of 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;            // leading byte offset (not used by swizzled K-major layouts)
  d |= (uint64_t)(1024u >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1u << 46;            // version
  d |= (uint64_t)2u << 61;            // 128-byte swizzle
  return d;
}
// instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), bf16 A and B (bits 7-9,
// 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// partial[ks][m][n] (M_pad x N_pad per K-range) of the tile (blockIdx.x, blockIdx.y) over the
// K-chunks [blockIdx.z * nk_per, ...)
__global__ void __launch_bounds__(128, 1)
    tc_gemm3_kernel(const __grid_constant__ CUtensorMap ta0, const __grid_constant__ CUtensorMap ta1,
                    const __grid_constant__ CUtensorMap ta2, const __grid_constant__ CUtensorMap tx0,
                    const __grid_constant__ CUtensorMap tx1, const __grid_constant__ CUtensorMap tx2, int nk,
                    int nk_per, float* __restrict__ partial, int m_pad, int n_pad, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kTcStages * kStageBytes);
  uint64_t* empty = full + kTcStages;
  uint64_t* done = empty + kTcStages;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  int* ok_flag = reinterpret_cast<int*>(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * kTcN;
  const int kc0 = blockIdx.z * nk_per, kc1 = min(nk, kc0 + nk_per);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *ok_flag = 1;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(kTcN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (threadIdx.x == 0) {
    const CUtensorMap* ma[3] = {&ta0, &ta1, &ta2};
    const CUtensorMap* mx[3] = {&tx0, &tx1, &tx2};
    bool ok = true;
    int loaded = kc0;  // next chunk to load
    auto load = [&](int kc) {
      const int s = (kc - kc0) % kTcStages;
      uint8_t* base = smem + s * kStageBytes;
      mbar_expect_tx(&full[s], kStageBytes);
      for (int i = 0; i < kTcSlices; ++i) tma_load_2d(base + i * kTileBytes, ma[i], kc * kTcK, m0, &full[s]);
      for (int j = 0; j < kTcSlices; ++j)
        tma_load_2d(base + (kTcSlices + j) * kTileBytes, mx[j], kc * kTcK, n0, &full[s]);
    };
    for (; loaded < kc1 && loaded < kc0 + kTcStages - 1; ++loaded) load(loaded);
    int consumed = kc0;
    for (int kc = kc0; kc < kc1; ++kc) {
      const int u = kc - kc0;
      if (loaded < kc1) {
        const int ul = loaded - kc0;
        // the stage was last read by the MMAs of chunk loaded - kTcStages
        if (ul >= kTcStages && !mbar_wait(&empty[ul % kTcStages], ((ul / kTcStages) - 1) & 1)) {
          ok = false;
          break;
        }
        load(loaded);
        ++loaded;
      }
      const int s = u % kTcStages;
      if (!mbar_wait(&full[s], (u / kTcStages) & 1)) {
        ok = false;
        break;
      }
      consumed = kc + 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(smem + s * kStageBytes);
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk)
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const uint64_t a = sw128_desc(base + kPairI[p] * kTileBytes + kk * 32);
          const uint64_t b = sw128_desc(base + (kTcSlices + kPairJ[p]) * kTileBytes + kk * 32);
          umma_bf16(tmem, a, b, (u > 0 || kk > 0 || p > 0) ? 1u : 0u);
        }
      umma_commit(&empty[s]);
    }
    // every MMA issued so far arrives on `done` when it has completed
    umma_commit(done);
    if (!ok) {
      *ok_flag = 0;
      atomicExch(err, 1);
      // drain the loads issued but not consumed, so no copy lands after the CTA has exited
      for (int kc = consumed; kc < loaded; ++kc) {
        const int u = kc - kc0;
        mbar_wait(&full[u % kTcStages], (u / kTcStages) & 1);
      }
    }
  }
  __syncthreads();
  const bool fin = mbar_wait(done, 0);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!fin && lane == 0) atomicExch(err, 1);
  const bool write = fin && *ok_flag;
  // epilogue: warp w holds rows 32 w .. 32 w + 31 of the tile, 16 columns per tensor-memory load
  const int m = m0 + 32 * warp + lane;
  float* dst = partial + (long long)blockIdx.z * m_pad * n_pad;
#pragma unroll 1
  for (int c = 0; c < kTcN / 16; ++c) {
    float v[16];
    tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * c), v);
    if (write && m < m_pad)
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int n = n0 + 16 * c + q;
        if (n < n_pad) dst[(long long)n * m_pad + m] = v[q];
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN) : "memory");
}

// out column n (sphere n): element m < rows of sum over the K-ranges of partial[ks][n][m], added
// in K-range order, written as FP32 (y32) or as a (hi, 0) float pair (y2) at y_off[n] + m
__global__ void tc_reduce_kernel(const float* __restrict__ partial, int ksplit, int m_pad, int n_pad, int rows, int ncols,
                                 const long long* __restrict__ y_off, float* __restrict__ y32, float2* __restrict__ y2) {
  const int n = blockIdx.y;
  if (n >= ncols) return;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < rows; m += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int k = 0; k < ksplit; ++k) s += partial[((long long)k * n_pad + n) * m_pad + m];
    if (y32) y32[y_off[n] + m] = s;
    else y2[y_off[n] + m] = make_float2(s, 0.f);
  }
}

// three bf16 slices of each row of a matrix (rows x cols, leading dimension ld) into rows x ldk
// slice matrices (zero beyond cols): s0 = bf16(v), s1 = bf16(v - s0), s2 = bf16(v - s0 - s1)
template <typename Tin>
__global__ void split3_matrix_kernel(int rows, int cols, long long ld, const Tin* __restrict__ in, int ldk,
                                     __nv_bfloat16* __restrict__ s0, __nv_bfloat16* __restrict__ s1,
                                     __nv_bfloat16* __restrict__ s2) {
  const long long tot = (long long)rows * ldk;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / ldk), k = (int)(e - (long long)r * ldk);
    const double v = k < cols ? (double)in[(long long)r * ld + k] : 0.0;
    const __nv_bfloat16 a = __double2bfloat16(v);
    const double r1 = v - (double)__bfloat162float(a);
    const __nv_bfloat16 b = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(b);
    s0[e] = a;
    s1[e] = b;
    s2[e] = __double2bfloat16(r2);
  }
}

// the same for the spheres' collocation data: row n = x[x_off[n] .. x_off[n] + cols)
__global__ void split3_gather_kernel(int nrows, int cols, const double* __restrict__ x, const long long* __restrict__ x_off,
                                     int ldk, __nv_bfloat16* __restrict__ s0, __nv_bfloat16* __restrict__ s1,
                                     __nv_bfloat16* __restrict__ s2) {
  const int n = blockIdx.y;
  if (n >= nrows) return;
  const double* xr = x + x_off[n];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ldk; k += gridDim.x * blockDim.x) {
    const double v = k < cols ? xr[k] : 0.0;
    const __nv_bfloat16 a = __double2bfloat16(v);
    const double r1 = v - (double)__bfloat162float(a);
    const __nv_bfloat16 b = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(b);
    const long long e = (long long)n * ldk + k;
    s0[e] = a;
    s1[e] = b;
    s2[e] = __double2bfloat16(r2);
  }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<EncodeTiled>(f);
  }();
  return fn;
}

// 2-D bf16 tensor map over a rows x ldk row-major matrix, 128 x 64 boxes, 128-byte swizzle;
// rows beyond the matrix read as zeros
bool make_map(CUtensorMap* map, const void* base, int rows, int ldk) {
  EncodeTiled enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ldk, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ldk * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int tc_ldk(int cols) { return (cols + kTcK - 1) / kTcK * kTcK; }

size_t tc_smem_bytes() { return kTcSmem; }

void launch_split3_matrix(int rows, int cols, long long ld, const double* in, int ldk, void* s0, void* s1, void* s2,
                          cudaStream_t st) {
  note_launch();
  split3_matrix_kernel<double><<<152 * 8, 256, 0, st>>>(rows, cols, ld, in, ldk, static_cast<__nv_bfloat16*>(s0),
                                                         static_cast<__nv_bfloat16*>(s1), static_cast<__nv_bfloat16*>(s2));
}
void launch_split3_matrix_f32(int rows, int cols, long long ld, const float* in, int ldk, void* s0, void* s1, void* s2,
                              cudaStream_t st) {
  note_launch();
  split3_matrix_kernel<float><<<152 * 8, 256, 0, st>>>(rows, cols, ld, in, ldk, static_cast<__nv_bfloat16*>(s0),
                                                        static_cast<__nv_bfloat16*>(s1), static_cast<__nv_bfloat16*>(s2));
}

bool tc_prepare(TcGemm& g, const void* const a_slices[3], int M, const void* const x_slices[3], int n_cap, int K) {
  g.M = M;
  g.K = K;
  g.ldk = tc_ldk(K);
  g.n_cap = n_cap;
  g.nk = g.ldk / kTcK;
  static_assert(sizeof(CUtensorMap) <= sizeof(g.maps[0]), "tensor-map storage");
  for (int i = 0; i < 3; ++i) {
    CUtensorMap m;
    if (!make_map(&m, a_slices[i], M, g.ldk)) return false;
    std::memcpy(g.maps[i], &m, sizeof(m));
    if (!make_map(&m, x_slices[i], n_cap, g.ldk)) return false;
    std::memcpy(g.maps[3 + i], &m, sizeof(m));
  }
  g.x_slices[0] = const_cast<void*>(x_slices[0]);
  g.x_slices[1] = const_cast<void*>(x_slices[1]);
  g.x_slices[2] = const_cast<void*>(x_slices[2]);
  // the shared-memory limit is a per-device attribute of the kernel: set it on the current device
  if (cudaFuncSetAttribute(tc_gemm3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// K-ranges per tile so that the grid covers about one wave of the 152 SMs
int tc_ksplit(const TcGemm& g, int ncols) {
  const int tiles = ((g.M + kTcM - 1) / kTcM) * ((ncols + kTcN - 1) / kTcN);
  int ks = std::max(1, 152 / std::max(1, tiles));
  ks = std::min(ks, g.nk);
  return ks;
}

void launch_tc_gemm(const TcGemm& g, int ncols, const double* x, const long long* x_off, const long long* y_off,
                    float* y32, float2* y2, float* partial, int* err, bool slice_x, cudaStream_t st) {
  if (ncols <= 0) return;
  // slices of the spheres' data (skipped when another product just wrote them from the same x)
  if (slice_x) {
    note_launch();
    split3_gather_kernel<<<dim3((g.ldk + 255) / 256, ncols), 256, 0, st>>>(
        ncols, g.K, x, x_off, g.ldk, static_cast<__nv_bfloat16*>(g.x_slices[0]),
        static_cast<__nv_bfloat16*>(g.x_slices[1]), static_cast<__nv_bfloat16*>(g.x_slices[2]));
  }
  const int ks = tc_ksplit(g, ncols);
  const int nk_per = (g.nk + ks - 1) / ks;
  const int ks_used = (g.nk + nk_per - 1) / nk_per;
  const int m_tiles = (g.M + kTcM - 1) / kTcM, n_tiles = (ncols + kTcN - 1) / kTcN;
  const int m_pad = m_tiles * kTcM, n_pad = n_tiles * kTcN;
  CUtensorMap m[6];
  for (int i = 0; i < 6; ++i) std::memcpy(&m[i], g.maps[i], sizeof(CUtensorMap));
  note_launch();
  tc_gemm3_kernel<<<dim3(m_tiles, n_tiles, ks_used), 128, kTcSmem, st>>>(m[0], m[1], m[2], m[3], m[4], m[5], g.nk, nk_per,
                                                                       partial, m_pad, n_pad, err);
  note_launch();
  tc_reduce_kernel<<<dim3((g.M + 255) / 256, ncols), 256, 0, st>>>(partial, ks_used, m_pad, n_pad, g.M, ncols, y_off,
                                                                  y32, y2);
}

size_t tc_partial_floats(const TcGemm& g, int ncols) {
  const int ks = tc_ksplit(g, ncols);
  const int nk_per = (g.nk + ks - 1) / ks;
  const int ks_used = (g.nk + nk_per - 1) / nk_per;
  const size_t m_pad = (size_t)((g.M + kTcM - 1) / kTcM) * kTcM, n_pad = (size_t)((ncols + kTcN - 1) / kTcN) * kTcN;
  return (size_t)ks_used * m_pad * n_pad;
}

}  // namespace mfs
