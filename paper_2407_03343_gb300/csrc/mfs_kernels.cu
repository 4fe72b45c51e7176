// CUDA kernels of the hot path (sm_103a).
//
//  pairs_kernel<T>     steps 2+3 of the G_hat apply (Sec. 2.2, eq. uAll): for every
//                      collocation node x_i of sphere k,
//                        out_i = mu_i + sqrt(w_i) sum_{k' != k} [S f + R t + D d](x_i - y)
//                      over the proxy Stokeslets and the image S/R/D triples of all other
//                      spheres (eq. lin_comb).  Direct summation, so the self block is
//                      skipped instead of being added and subtracted (allowed by Sec. 2.2).
//                      Sources are staged through shared memory in tiles; each thread owns
//                      NT target nodes in registers; 1/|r| comes from rsqrt (FP32) or an
//                      FP32 seed refined by Newton-Raphson (FP64).  FP32 sums run per tile
//                      and are folded into Kahan-compensated accumulators across tiles.
//                      Positions are stored relative to their sphere centre and shifted into
//                      the target sphere's frame while staging, with the centre difference
//                      taken in float-float, so near-contact distances keep FP32 accuracy.
//  gemv_kernel<T>      batched row-major GEMV for the one-body pseudo-inverse factors
//                      (eq. transform), HBM-bound.
//  Krylov kernels      multi-dot, update, scale (GMRES with CGS2), FP64 partial sums.
//  ft_kernel           forces and torques from the strengths (Sec. 2.3 remark), FP64.
//  rhs_kernel          W u_bc (eq. bc, eq. lq2), FP64.
//  assemble_self       B_k = W_k G^(kk) column-major FP64 for the one-time factorisation.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "mfs_internal.h"

namespace mfs {
namespace {

constexpr int kPairThreads = 128;
constexpr int kTileProxy = 256; // proxy sources staged per round
constexpr int kTileImg = 128;   // image nodes staged per round
constexpr double kPi = 3.14159265358979323846;

// four doubles moved as one 32-byte-aligned unit
struct __align__(32) D4 {
  double x, y, z, w;
};

template <typename T> struct Prec;
template <> struct Prec<float> {
  using V4 = float4;
  static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
  static __device__ __forceinline__ V4 mk(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
};
template <> struct Prec<double> {
  using V4 = D4;
  // 1/sqrt(x): FP32 hardware estimate refined by two Newton-Raphson steps
  // y <- y (3 - x y^2) / 2, each of which roughly doubles the number of correct bits.
  static __device__ __forceinline__ double rsq(double x) {
    double y = (double)rsqrtf((float)x);
    y = y * (1.5 - 0.5 * x * y * y);
    y = y * (1.5 - 0.5 * x * y * y);
    return y;
  }
  static __device__ __forceinline__ V4 mk(double a, double b, double c, double d) { return D4{a, b, c, d}; }
};

// Kahan-compensated s += x.  FP64 accumulates directly.
__device__ __forceinline__ void comp_add(float& s, float& c, float x) {
  float y = x - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
}
__device__ __forceinline__ void comp_add(double& s, double& c, double x) { (void)c; s += x; }

// Centre of sphere o minus centre of the target frame, in the working precision.
struct CentreShift32 {
  const float* hi;
  const float* lo;
  float kh[3], kl[3];
  __device__ void init(int k) {
    for (int c = 0; c < 3; ++c) {
      kh[c] = k >= 0 ? hi[3 * k + c] : 0.f;
      kl[c] = k >= 0 ? lo[3 * k + c] : 0.f;
    }
  }
  __device__ __forceinline__ float d(int o, int c) const { return (hi[3 * o + c] - kh[c]) + (lo[3 * o + c] - kl[c]); }
};
struct CentreShift64 {
  const double* cen;
  double kc[3];
  __device__ void init(int k) {
    for (int c = 0; c < 3; ++c) kc[c] = k >= 0 ? cen[3 * k + c] : 0.0;
  }
  __device__ __forceinline__ double d(int o, int c) const { return cen[3 * o + c] - kc[c]; }
};
template <typename T> struct ShiftOf;
template <> struct ShiftOf<float> { using type = CentreShift32; };
template <> struct ShiftOf<double> { using type = CentreShift64; };

template <typename T>
struct PairArgs {
  const typename Prec<T>::V4* tgt;  // (x, y, z, sqrt w) relative to the tile's sphere (absolute if sphere < 0)
  const int* tile_sphere;
  const int* tile_start;
  const int* tile_count;
  const typename Prec<T>::V4* proxy;  // N, relative to the owner centre
  int N, P;
  const typename Prec<T>::V4* img;    // image nodes relative to the owner centre
  const int* img_owner;
  const int* img_off;
  int n_img;
  const long long* unk_off;
  const float* cen_hi;
  const float* cen_lo;
  const double* cen64;
  const T* lam;
  const T* mu;   // may be null: then out = scale * sum (no W, no identity)
  T* out;
  T scale;       // 1 / (8 pi mu)
  T dip;         // 2 mu: dipole strengths rescaled so that scale * dip = 1 / (4 pi)
};

// One target tile (NT nodes per thread) against every source of every other sphere.
template <typename T, int NT>
__device__ __forceinline__ void pair_tile(const PairArgs<T>& A, const int t) {
  using V4 = typename Prec<T>::V4;
  __shared__ V4 sp[kTileProxy];
  __shared__ V4 sf[kTileProxy];
  __shared__ V4 si[3 * kTileImg];

  const int k = A.tile_sphere[t];
  const int start = A.tile_start[t];
  const int cnt = A.tile_count[t];
  typename ShiftOf<T>::type sh;
  if constexpr (sizeof(T) == 4) { sh.hi = A.cen_hi; sh.lo = A.cen_lo; } else { sh.cen = A.cen64; }
  sh.init(k);

  T x[NT], y[NT], z[NT], ux[NT], uy[NT], uz[NT];
  T sx[NT], sy[NT], sz[NT], cx[NT], cy[NT], cz[NT];
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    int idx = threadIdx.x + q * kPairThreads;
    int node = start + (idx < cnt ? idx : cnt - 1);
    V4 p = A.tgt[node];
    x[q] = p.x; y[q] = p.y; z[q] = p.z;
    ux[q] = uy[q] = uz[q] = T(0);
    sx[q] = sy[q] = sz[q] = T(0);
    cx[q] = cy[q] = cz[q] = T(0);
  }
  const T far = T(1e18);

  // ---- proxy Stokeslets of every sphere but k
  const int total = A.P * A.N;
  // the proxies before and after sphere k's own, in tiles with exact trip counts
  for (int rr = 0; rr < 2; ++rr) {
  const int r_lo = rr == 0 ? 0 : (k < 0 ? total : (k + 1) * A.N);
  const int r_hi = rr == 0 ? (k < 0 ? total : k * A.N) : total;
  for (int s0 = r_lo; s0 < r_hi; s0 += kTileProxy) {
    const int ns = min(kTileProxy, r_hi - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < ns; i += kPairThreads) {
      int j = s0 + i;
      V4 pos = Prec<T>::mk(far, far, far, T(0)), str = Prec<T>::mk(T(0), T(0), T(0), T(0));
      if (j < total) {
        int o = j / A.N;
        int jj = j - o * A.N;
        V4 pr = A.proxy[jj];
        pos = Prec<T>::mk(pr.x + sh.d(o, 0), pr.y + sh.d(o, 1), pr.z + sh.d(o, 2), T(0));
        if (o != k) {
          const T* l = A.lam + A.unk_off[o] + 3LL * jj;
          str = Prec<T>::mk(l[0], l[1], l[2], T(0));
        }
      }
      sp[i] = pos;
      sf[i] = str;
    }
    __syncthreads();
#pragma unroll 2
    for (int j = 0; j < ns; ++j) {
      const V4 p = sp[j];
      const V4 f = sf[j];
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        T dx = x[q] - p.x, dy = y[q] - p.y, dz = z[q] - p.z;
        T r2 = dx * dx + dy * dy + dz * dz;
        T ir = Prec<T>::rsq(r2);
        T ir2 = ir * ir;
        T rf = dx * f.x + dy * f.y + dz * f.z;
        T c = rf * ir2;
        ux[q] += ir * (f.x + c * dx);
        uy[q] += ir * (f.y + c * dy);
        uz[q] += ir * (f.z + c * dz);
      }
    }
#pragma unroll
    for (int q = 0; q < NT; ++q) {
      comp_add(sx[q], cx[q], ux[q]);
      comp_add(sy[q], cy[q], uy[q]);
      comp_add(sz[q], cz[q], uz[q]);
      ux[q] = uy[q] = uz[q] = T(0);
    }
  }
  }

  // ---- image nodes (Stokeslet + rotlet + potential dipole at one position)
  const int self_lo = k >= 0 ? A.img_off[k] : 0, self_hi = k >= 0 ? A.img_off[k + 1] : 0;
  for (int rr = 0; rr < 2; ++rr) {
  const int r_lo = rr == 0 ? 0 : self_hi;
  const int r_hi = rr == 0 ? self_lo : A.n_img;
  for (int s0 = r_lo; s0 < r_hi; s0 += kTileImg) {
    const int ns = min(kTileImg, r_hi - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < ns; i += kPairThreads) {
      int j = s0 + i;
      V4 a = Prec<T>::mk(far, far, far, T(0)), b = Prec<T>::mk(T(0), T(0), T(0), T(0)), c = b;
      if (j < A.n_img) {
        int o = A.img_owner[j];
        V4 pr = A.img[j];
        T px = pr.x + sh.d(o, 0), py = pr.y + sh.d(o, 1), pz = pr.z + sh.d(o, 2);
        if (o != k) {
          const T* l = A.lam + A.unk_off[o] + 3LL * A.N + 9LL * (j - A.img_off[o]);
          a = Prec<T>::mk(px, py, pz, l[0]);
          b = Prec<T>::mk(l[1], l[2], l[3], l[4]);
          c = Prec<T>::mk(l[5], A.dip * l[6], A.dip * l[7], A.dip * l[8]);
        } else {
          a = Prec<T>::mk(px, py, pz, T(0));
        }
      }
      si[3 * i] = a;
      si[3 * i + 1] = b;
      si[3 * i + 2] = c;
    }
    __syncthreads();
    for (int j = 0; j < ns; ++j) {
      const V4 a = si[3 * j], b = si[3 * j + 1], c = si[3 * j + 2];
      // f = (a.w, b.x, b.y), t = (b.z, b.w, c.x), d = (c.y, c.z, c.w)
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        T dx = x[q] - a.x, dy = y[q] - a.y, dz = z[q] - a.z;
        T r2 = dx * dx + dy * dy + dz * dz;
        T ir = Prec<T>::rsq(r2);
        T ir2 = ir * ir;
        T ir3 = ir * ir2;
        // Stokeslet
        T rf = dx * a.w + dy * b.x + dz * b.y;
        T cs = rf * ir2;
        T vx = ir * (a.w + cs * dx), vy = ir * (b.x + cs * dy), vz = ir * (b.y + cs * dz);
        // rotlet: (t x r) / r^3
        vx += ir3 * (b.w * dz - c.x * dy);
        vy += ir3 * (c.x * dx - b.z * dz);
        vz += ir3 * (b.z * dy - b.w * dx);
        // potential dipole: -d / r^3 + 3 (d.r) r / r^5
        T rd = dx * c.y + dy * c.z + dz * c.w;
        T c3 = T(3) * rd * ir3 * ir2;
        vx += c3 * dx - ir3 * c.y;
        vy += c3 * dy - ir3 * c.z;
        vz += c3 * dz - ir3 * c.w;
        ux[q] += vx;
        uy[q] += vy;
        uz[q] += vz;
      }
    }
#pragma unroll
    for (int q = 0; q < NT; ++q) {
      comp_add(sx[q], cx[q], ux[q]);
      comp_add(sy[q], cy[q], uy[q]);
      comp_add(sz[q], cz[q], uz[q]);
      ux[q] = uy[q] = uz[q] = T(0);
    }
  }
  }

#pragma unroll
  for (int q = 0; q < NT; ++q) {
    int idx = threadIdx.x + q * kPairThreads;
    if (idx < cnt) {
      long long node = start + idx;
      T sw = A.tgt[node].w;
      T gx = (sx[q] + cx[q]) * A.scale, gy = (sy[q] + cy[q]) * A.scale, gz = (sz[q] + cz[q]) * A.scale;
      if (A.mu) {
        A.out[3 * node] = A.mu[3 * node] + sw * gx;
        A.out[3 * node + 1] = A.mu[3 * node + 1] + sw * gy;
        A.out[3 * node + 2] = A.mu[3 * node + 2] + sw * gz;
      } else {
        A.out[3 * node] = gx;
        A.out[3 * node + 1] = gy;
        A.out[3 * node + 2] = gz;
      }
    }
  }
}

template <typename T>
PairArgs<T> make_args(const TargetSet& tg, const SourceSet& src, const T* lam, const T* mu, T* out, double visc,
                      int nt = 4) {
  PairArgs<T> A;
  if constexpr (sizeof(T) == 4) {
    A.tgt = tg.pos32;
    A.proxy = src.proxy32;
    A.img = src.img32;
  } else {
    A.tgt = reinterpret_cast<const D4*>(tg.pos64);
    A.proxy = reinterpret_cast<const D4*>(src.proxy64);
    A.img = reinterpret_cast<const D4*>(src.img64);
  }
  A.tile_sphere = nt == 4 ? tg.tile_sphere : tg.tile1_sphere;
  A.tile_start = nt == 4 ? tg.tile_start : tg.tile1_start;
  A.tile_count = nt == 4 ? tg.tile_count : tg.tile1_count;
  A.N = src.N;
  A.P = src.P;
  A.img_owner = src.img_owner;
  A.img_off = src.img_off;
  A.n_img = src.n_img;
  A.unk_off = src.unk_off;
  A.cen_hi = src.cen_hi;
  A.cen_lo = src.cen_lo;
  A.cen64 = src.cen64;
  A.lam = lam;
  A.mu = mu;
  A.out = out;
  A.scale = T(1.0 / (8.0 * kPi * visc));
  A.dip = T(2.0 * visc);
  return A;
}

// ------------------------------------------------------------------ double-float pair kernel
// FP64-accurate pair sums on the FP32 pipes.  A value is an unevaluated sum hi + lo of two
// floats (double-word arithmetic).  Error-free transforms: TwoSum (Knuth, TAOCP vol. 2),
// FastTwoSum and TwoProd via FMA (Dekker 1971); DW+DW and DW*DW follow the "sloppy" sum
// and the FMA-based product of Joldes, Muller and Popescu (ACM TOMS 44, 2017), whose
// absolute errors stay at ~2^-46 of the operands even under cancellation, which is what
// the pair sums need: the strengths lambda_hat = B^+ mu can exceed the field they produce
// by 1e9 or more (Sec. 2.2, truncation 5e-12), so every term must be accurate to ~1e-14.
struct dw {
  float h, l;
};
// The _rn intrinsics are never contracted into FMAs, which the error-free transforms
// rely on (a fused a*b + w would break the rounded product they assume).
__device__ __forceinline__ dw two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ dw two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ dw dw_add(dw x, dw y) {
  dw s = two_sum(x.h, y.h);
  float v = __fadd_rn(x.l, y.l);
  return fast_two_sum(s.h, __fadd_rn(s.l, v));
}
__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw{-y.h, -y.l}); }
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
  dw c = two_prod(x.h, y.h);
  float t = __fmul_rn(x.h, y.l);
  t = __fmaf_rn(x.l, y.h, t);
  return fast_two_sum(c.h, __fadd_rn(c.l, t));
}
__device__ __forceinline__ dw dw_mul_f(dw x, float y) {
  dw c = two_prod(x.h, y);
  return fast_two_sum(c.h, __fmaf_rn(x.l, y, c.l));
}
__device__ __forceinline__ dw dw_split(double v) {
  float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double dw_join(dw x) { return (double)x.h + (double)x.l; }
// 1/sqrt(x): FP32 estimate, one FP32 Newton step, one double-word Newton step
// y <- y + y (1 - x y^2) / 2.
__device__ __forceinline__ dw dw_rsqrt(dw x) {
  float s = rsqrtf(x.h);
  s = __fmul_rn(s, __fmaf_rn(__fmul_rn(-0.5f, x.h), __fmul_rn(s, s), 1.5f));
  dw s2 = two_prod(s, s);
  dw e = dw_mul(x, s2);
  float h = __fsub_rn(__fsub_rn(1.0f, e.h), e.l);
  return fast_two_sum(s, __fmul_rn(__fmul_rn(0.5f, s), h));
}

// Compensated evaluation for the pair kernel (in the style of Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 2005): a product keeps its exact
// rounding error plus the first-order cross terms, a sum keeps the TwoSum error plus the low
// parts, and neither renormalises; the low part then stays within a few ulps of the high part
// scaled by the operands' magnitude, which bounds every absolute error by ~2^-46 of the
// operands.  Renormalisation is kept where cancellation could let the low part outgrow the
// high part (differences of positions and dot products) and at every accumulation.
__device__ __forceinline__ dw mul_u(dw x, dw y) {
  float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return {p, e};
}
__device__ __forceinline__ dw add_u(dw x, dw y) {
  dw s = two_sum(x.h, y.h);
  return {s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l))};
}
__device__ __forceinline__ dw neg(dw x) { return {-x.h, -x.l}; }
// u += t with the running sum renormalised every time: its partial sums can exceed the final
// value by ~1e9 under cancellation, so its low word must stay within an ulp of the high word
__device__ __forceinline__ void acc_u(dw& u, dw t) { u = dw_add(u, t); }
// x - y for positions: the difference is never below ~1e-3 of the radius, far above the low parts
__device__ __forceinline__ dw sub_pos(dw x, dw y) {
  dw s = two_sum(x.h, -y.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fsub_rn(x.l, y.l)));
}
// a.b for three double-word pairs, renormalised (the sum may cancel)
__device__ __forceinline__ dw dot3_u(dw a0, dw a1, dw a2, dw b0, dw b1, dw b2) {
  dw p0 = mul_u(a0, b0), p1 = mul_u(a1, b1), p2 = mul_u(a2, b2);
  dw s1 = two_sum(p0.h, p1.h);
  dw s2 = two_sum(s1.h, p2.h);
  float lo = __fadd_rn(__fadd_rn(__fadd_rn(p0.l, p1.l), __fadd_rn(p2.l, s1.l)), s2.l);
  return two_sum(s2.h, lo);
}
// |d|^2 (all terms positive, no cancellation)
__device__ __forceinline__ dw norm2_u(dw d0, dw d1, dw d2) {
  dw p0 = two_prod(d0.h, d0.h), p1 = two_prod(d1.h, d1.h), p2 = two_prod(d2.h, d2.h);
  p0.l = __fmaf_rn(__fadd_rn(d0.h, d0.h), d0.l, p0.l);
  p1.l = __fmaf_rn(__fadd_rn(d1.h, d1.h), d1.l, p1.l);
  p2.l = __fmaf_rn(__fadd_rn(d2.h, d2.h), d2.l, p2.l);
  dw s1 = two_sum(p0.h, p1.h);
  dw s2 = two_sum(s1.h, p2.h);
  float lo = __fadd_rn(__fadd_rn(__fadd_rn(p0.l, p1.l), __fadd_rn(p2.l, s1.l)), s2.l);
  return fast_two_sum(s2.h, lo);
}
__device__ __forceinline__ dw rsqrt_u(dw x) {
  float s = rsqrtf(x.h);
  s = __fmul_rn(s, __fmaf_rn(__fmul_rn(-0.5f, x.h), __fmul_rn(s, s), 1.5f));
  dw e = mul_u(x, two_prod(s, s));
  float h = __fsub_rn(__fsub_rn(1.0f, e.h), e.l);
  return fast_two_sum(s, __fmul_rn(__fmul_rn(0.5f, s), h));
}
__device__ __forceinline__ dw times3_u(dw x) {
  dw c = two_prod(x.h, 3.0f);
  return {c.h, __fmaf_rn(x.l, 3.0f, c.l)};
}

struct __align__(16) DWPos {
  float xh, yh, zh, pad0;
  float xl, yl, zl, pad1;
};

// Target nodes of one tile in double-float, with their running sums.
template <int NT>
struct DWTile {
  dw x[NT], y[NT], z[NT], ux[NT], uy[NT], uz[NT];
};

template <int NT>
__device__ __forceinline__ void dw_load_targets(const PairArgs<double>& A, int start, int cnt, DWTile<NT>& T) {
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    int idx = threadIdx.x + q * kPairThreads;
    int node = start + (idx < cnt ? idx : cnt - 1);
    D4 p = A.tgt[node];
    T.x[q] = dw_split(p.x);
    T.y[q] = dw_split(p.y);
    T.z[q] = dw_split(p.z);
    T.ux[q] = T.uy[q] = T.uz[q] = dw{0.f, 0.f};
  }
}

// Proxy Stokeslets [r_lo, r_hi) of the flattened proxy index (sphere o = j / N, proxy j - o N),
// staged through shared memory in tiles of kTileProxy; sphere k's own proxies carry no strength.
template <int NT>
__device__ __forceinline__ void dw_proxy_range(const PairArgs<double>& A, const CentreShift64& sh, int k, int r_lo,
                                               int r_hi, float4* sp, float4* sf, DWTile<NT>& T) {
  const double far = 1e18;
  const int total = A.P * A.N;
  for (int s0 = r_lo; s0 < r_hi; s0 += kTileProxy) {
    const int ns = min(kTileProxy, r_hi - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < ns; i += kPairThreads) {
      int j = s0 + i;
      double px = far, py = far, pz = far, fx = 0, fy = 0, fz = 0;
      if (j < total) {
        int o = j / A.N;
        int jj = j - o * A.N;
        D4 pr = A.proxy[jj];
        px = pr.x + sh.d(o, 0);
        py = pr.y + sh.d(o, 1);
        pz = pr.z + sh.d(o, 2);
        if (o != k) {
          const double* l = A.lam + A.unk_off[o] + 3LL * jj;
          fx = l[0]; fy = l[1]; fz = l[2];
        }
      }
      dw a = dw_split(px), b = dw_split(py), c = dw_split(pz);
      sp[2 * i] = make_float4(a.h, b.h, c.h, 0.f);
      sp[2 * i + 1] = make_float4(a.l, b.l, c.l, 0.f);
      a = dw_split(fx); b = dw_split(fy); c = dw_split(fz);
      sf[2 * i] = make_float4(a.h, b.h, c.h, 0.f);
      sf[2 * i + 1] = make_float4(a.l, b.l, c.l, 0.f);
    }
    __syncthreads();
    for (int j = 0; j < ns; ++j) {
      const float4 ph = sp[2 * j], pl = sp[2 * j + 1];
      const float4 fh = sf[2 * j], fl = sf[2 * j + 1];
      const dw fx{fh.x, fl.x}, fy{fh.y, fl.y}, fz{fh.z, fl.z};
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        dw dx = sub_pos(T.x[q], dw{ph.x, pl.x});
        dw dy = sub_pos(T.y[q], dw{ph.y, pl.y});
        dw dz = sub_pos(T.z[q], dw{ph.z, pl.z});
        dw ir = rsqrt_u(norm2_u(dx, dy, dz));
        dw ir2 = mul_u(ir, ir);
        dw c = mul_u(dot3_u(dx, dy, dz, fx, fy, fz), ir2);
        acc_u(T.ux[q], mul_u(ir, add_u(fx, mul_u(c, dx))));
        acc_u(T.uy[q], mul_u(ir, add_u(fy, mul_u(c, dy))));
        acc_u(T.uz[q], mul_u(ir, add_u(fz, mul_u(c, dz))));
      }
    }
#pragma unroll
    for (int q = 0; q < NT; ++q) {
      T.ux[q] = two_sum(T.ux[q].h, T.ux[q].l);
      T.uy[q] = two_sum(T.uy[q].h, T.uy[q].l);
      T.uz[q] = two_sum(T.uz[q].h, T.uz[q].l);
    }
  }
}

// Image nodes [r_lo, r_hi) (Stokeslet + rotlet + potential dipole at one position), staged in
// tiles of kTileImg; sphere k's own nodes carry no strength.
template <int NT>
__device__ __forceinline__ void dw_image_range(const PairArgs<double>& A, const CentreShift64& sh, int k, int r_lo,
                                               int r_hi, float4* si, DWTile<NT>& T) {
  const double far = 1e18;
  for (int s0 = r_lo; s0 < r_hi; s0 += kTileImg) {
    const int ns = min(kTileImg, r_hi - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < ns; i += kPairThreads) {
      int j = s0 + i;
      double v[12] = {far, far, far, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      if (j < A.n_img) {
        int o = A.img_owner[j];
        D4 pr = A.img[j];
        v[0] = pr.x + sh.d(o, 0);
        v[1] = pr.y + sh.d(o, 1);
        v[2] = pr.z + sh.d(o, 2);
        if (o != k) {
          const double* l = A.lam + A.unk_off[o] + 3LL * A.N + 9LL * (j - A.img_off[o]);
          for (int q = 0; q < 6; ++q) v[3 + q] = l[q];
          for (int q = 6; q < 9; ++q) v[3 + q] = A.dip * l[q];
        }
      }
      // node i occupies si[6i .. 6i+5]: hi of (x, y, z, f, t, d) then lo of the same 12 values
      float hv[12], lv[12];
      for (int q = 0; q < 12; ++q) {
        dw s = dw_split(v[q]);
        hv[q] = s.h;
        lv[q] = s.l;
      }
      si[6 * i] = make_float4(hv[0], hv[1], hv[2], hv[3]);
      si[6 * i + 1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
      si[6 * i + 2] = make_float4(hv[8], hv[9], hv[10], hv[11]);
      si[6 * i + 3] = make_float4(lv[0], lv[1], lv[2], lv[3]);
      si[6 * i + 4] = make_float4(lv[4], lv[5], lv[6], lv[7]);
      si[6 * i + 5] = make_float4(lv[8], lv[9], lv[10], lv[11]);
    }
    __syncthreads();
    for (int j = 0; j < ns; ++j) {
      const float4 h0 = si[6 * j], h1 = si[6 * j + 1], h2 = si[6 * j + 2];
      const float4 l0 = si[6 * j + 3], l1 = si[6 * j + 4], l2 = si[6 * j + 5];
      const dw px{h0.x, l0.x}, py{h0.y, l0.y}, pz{h0.z, l0.z};
      const dw fx{h0.w, l0.w}, fy{h1.x, l1.x}, fz{h1.y, l1.y};
      const dw tx{h1.z, l1.z}, ty{h1.w, l1.w}, tz{h2.x, l2.x};
      const dw qx{h2.y, l2.y}, qy{h2.z, l2.z}, qz{h2.w, l2.w};
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        dw dx = sub_pos(T.x[q], px), dy = sub_pos(T.y[q], py), dz = sub_pos(T.z[q], pz);
        dw ir = rsqrt_u(norm2_u(dx, dy, dz));
        dw ir2 = mul_u(ir, ir);
        dw ir3 = mul_u(ir, ir2);
        // Stokeslet
        dw cs = mul_u(dot3_u(dx, dy, dz, fx, fy, fz), ir2);
        acc_u(T.ux[q], mul_u(ir, add_u(fx, mul_u(cs, dx))));
        acc_u(T.uy[q], mul_u(ir, add_u(fy, mul_u(cs, dy))));
        acc_u(T.uz[q], mul_u(ir, add_u(fz, mul_u(cs, dz))));
        // rotlet (t x r) / r^3
        acc_u(T.ux[q], mul_u(ir3, add_u(mul_u(ty, dz), neg(mul_u(tz, dy)))));
        acc_u(T.uy[q], mul_u(ir3, add_u(mul_u(tz, dx), neg(mul_u(tx, dz)))));
        acc_u(T.uz[q], mul_u(ir3, add_u(mul_u(tx, dy), neg(mul_u(ty, dx)))));
        // potential dipole -d / r^3 + 3 (d.r) r / r^5
        dw c3 = times3_u(mul_u(mul_u(dot3_u(dx, dy, dz, qx, qy, qz), ir3), ir2));
        acc_u(T.ux[q], mul_u(c3, dx));
        acc_u(T.uy[q], mul_u(c3, dy));
        acc_u(T.uz[q], mul_u(c3, dz));
        acc_u(T.ux[q], neg(mul_u(ir3, qx)));
        acc_u(T.uy[q], neg(mul_u(ir3, qy)));
        acc_u(T.uz[q], neg(mul_u(ir3, qz)));
      }
    }
#pragma unroll
    for (int q = 0; q < NT; ++q) {
      T.ux[q] = two_sum(T.ux[q].h, T.ux[q].l);
      T.uy[q] = two_sum(T.uy[q].h, T.uy[q].l);
      T.uz[q] = two_sum(T.uz[q].h, T.uz[q].l);
    }
  }
}

// out = mu + sqrt(w) scale u per node (or the scaled partial sum of this source part, or the
// plain scaled sum when mu is null)
template <int NT>
__device__ __forceinline__ void dw_write_out(const PairArgs<double>& A, int start, int cnt, const DWTile<NT>& T,
                                             int part, int nparts, double* __restrict__ partial, long long pstride) {
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    int idx = threadIdx.x + q * kPairThreads;
    if (idx < cnt) {
      long long node = start + idx;
      double sw = A.tgt[node].w;
      double gx = dw_join(T.ux[q]) * A.scale, gy = dw_join(T.uy[q]) * A.scale, gz = dw_join(T.uz[q]) * A.scale;
      if (nparts > 1) {
        double* o = partial + part * pstride + 3 * node;
        o[0] = gx;
        o[1] = gy;
        o[2] = gz;
      } else if (A.mu) {
        A.out[3 * node] = A.mu[3 * node] + sw * gx;
        A.out[3 * node + 1] = A.mu[3 * node + 1] + sw * gy;
        A.out[3 * node + 2] = A.mu[3 * node + 2] + sw * gz;
      } else {
        A.out[3 * node] = gx;
        A.out[3 * node + 1] = gy;
        A.out[3 * node + 2] = gz;
      }
    }
  }
}

// Sources may be split over `nparts` CTAs per target tile (when there are too few tiles to
// fill the GPU): part `part` takes a contiguous share of the tile's source list (the sources of
// every other sphere) and, for nparts > 1, writes its scaled partial sum to
// partial[part * pstride + 3 node + c] for pair_parts_reduce to finish.
template <int NT>
__device__ __forceinline__ void pair_tile_dw(const PairArgs<double>& A, const int t, const int part, const int nparts,
                                             double* __restrict__ partial, const long long pstride) {
  __shared__ float4 sp[2 * kTileProxy];   // position hi, lo
  __shared__ float4 sf[2 * kTileProxy];   // strength hi, lo
  __shared__ float4 si[6 * kTileImg];     // image node: 12 hi values (3 float4), then 12 lo values (3 float4)

  const int k = A.tile_sphere[t];
  const int start = A.tile_start[t];
  const int cnt = A.tile_count[t];
  CentreShift64 sh;
  sh.cen = A.cen64;
  sh.init(k);
  DWTile<NT> T;
  dw_load_targets<NT>(A, start, cnt, T);

  const int total = A.P * A.N;
  // the proxies before and after sphere k's own (this part's share of them), in tiles with
  // exact trip counts
  const int p_lo = k < 0 ? total : k * A.N, p_w = k < 0 ? 0 : A.N;
  const long long p_eff = total - p_w;
  const int pe0 = (int)(p_eff * part / nparts), pe1 = (int)(p_eff * (part + 1) / nparts);
  dw_proxy_range<NT>(A, sh, k, min(pe0, p_lo), min(pe1, p_lo), sp, sf, T);
  dw_proxy_range<NT>(A, sh, k, max(pe0, p_lo) + p_w, max(pe1, p_lo) + p_w, sp, sf, T);

  // image nodes before and after sphere k's own, this part's share
  const int i_lo = k >= 0 ? A.img_off[k] : 0, i_w = k >= 0 ? A.img_off[k + 1] - i_lo : 0;
  const long long i_eff = A.n_img - i_w;
  const int ie0 = (int)(i_eff * part / nparts), ie1 = (int)(i_eff * (part + 1) / nparts);
  dw_image_range<NT>(A, sh, k, min(ie0, i_lo), min(ie1, i_lo), si, T);
  dw_image_range<NT>(A, sh, k, max(ie0, i_lo) + i_w, max(ie1, i_lo) + i_w, si, T);

  dw_write_out<NT>(A, start, cnt, T, part, nparts, partial, pstride);
}

// The near part of the far-field split: only the spheres of the target sphere's near list
// (ascending; runs of consecutive spheres are staged as one range).
template <int NT>
__device__ __forceinline__ void pair_tile_dw_near(const PairArgs<double>& A, const int* __restrict__ near_off,
                                                  const int* __restrict__ near_idx, const int t, const int part,
                                                  const int nparts, double* __restrict__ partial,
                                                  const long long pstride) {
  __shared__ float4 sp[2 * kTileProxy];
  __shared__ float4 sf[2 * kTileProxy];
  __shared__ float4 si[6 * kTileImg];
  const int k = A.tile_sphere[t];
  const int start = A.tile_start[t];
  const int cnt = A.tile_count[t];
  CentreShift64 sh;
  sh.cen = A.cen64;
  sh.init(k);
  DWTile<NT> T;
  dw_load_targets<NT>(A, start, cnt, T);
  // this part's share of the near list
  const int b0 = near_off[k], nn = near_off[k + 1] - b0;
  const int a1 = b0 + (int)((long long)nn * (part + 1) / nparts);
  for (int a = b0 + (int)((long long)nn * part / nparts); a < a1;) {
    const int o0 = near_idx[a];
    int o1 = o0;
    while (a + 1 < a1 && near_idx[a + 1] == o1 + 1) {
      ++a;
      ++o1;
    }
    ++a;
    dw_proxy_range<NT>(A, sh, k, o0 * A.N, (o1 + 1) * A.N, sp, sf, T);
    dw_image_range<NT>(A, sh, k, A.img_off[o0], A.img_off[o1 + 1], si, T);
  }
  dw_write_out<NT>(A, start, cnt, T, part, nparts, partial, pstride);
}

// ------------------------------------------------------------------ far-field kernel (FP32)
constexpr int kTileFar = 256;  // equivalent sources staged per round

struct FarArgs {
  const float4* tgt;     // (x - c_k, sqrt w) per node, FP32
  const double* tgt64;   // the same in FP64 (sqrt w taken from here)
  const int* tile_sphere;
  const int* tile_start;
  const int* tile_count;
  const float4* eq;      // n_eq equivalent-source positions relative to the owner centre
  int n_eq, P;
  const int* excl_off;
  const int* excl_idx;
  const float* cen_hi;
  const float* cen_lo;
  const float* q;        // 3 n_eq strengths per sphere
  double* out;
  float scale;           // 1 / (8 pi mu)
};

// out += sqrt(w) scale sum over every sphere outside the target sphere's exclusion list (its
// near spheres and itself) of the Stokeslet field of its equivalent sources.  The excluded
// spheres split the flattened equivalent-source index into runs, each staged in tiles.
template <int NT>
__global__ void __launch_bounds__(kPairThreads) pairs_far_kernel(FarArgs A, int nparts, double* __restrict__ partial,
                                                                 long long pstride) {
  __shared__ float4 sp[kTileFar];
  __shared__ float4 sf[kTileFar];
  const int t = blockIdx.x / nparts, part = blockIdx.x % nparts;
  const int k = A.tile_sphere[t];
  const int start = A.tile_start[t];
  const int cnt = A.tile_count[t];
  CentreShift32 sh;
  sh.hi = A.cen_hi;
  sh.lo = A.cen_lo;
  sh.init(k);
  float x[NT], y[NT], z[NT], ux[NT], uy[NT], uz[NT], sx[NT], sy[NT], sz[NT], cx[NT], cy[NT], cz[NT];
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    int idx = threadIdx.x + q * kPairThreads;
    float4 p = A.tgt[start + (idx < cnt ? idx : cnt - 1)];
    x[q] = p.x; y[q] = p.y; z[q] = p.z;
    ux[q] = uy[q] = uz[q] = sx[q] = sy[q] = sz[q] = cx[q] = cy[q] = cz[q] = 0.f;
  }
  const int e0 = A.excl_off[k], e1 = A.excl_off[k + 1];
  // this part's share [f0, f1) of the far sources, counted in the order of the runs between
  // excluded spheres
  const long long n_far = (long long)(A.P - (e1 - e0)) * A.n_eq;
  const long long f0 = n_far * part / nparts, f1 = n_far * (part + 1) / nparts;
  long long before = 0;  // far sources in the runs before the current one
  int prev = -1;
  for (int a = e0; a <= e1; ++a) {
    const int nxt = a < e1 ? A.excl_idx[a] : A.P;
    const int run_lo = (prev + 1) * A.n_eq, run_hi = nxt * A.n_eq;
    prev = nxt;
    const long long len = run_hi - run_lo;
    const int lo = run_lo + (int)max(0LL, min(len, f0 - before));
    const int hi = run_lo + (int)max(0LL, min(len, f1 - before));
    before += len;
    for (int s0 = lo; s0 < hi; s0 += kTileFar) {
      const int ns = min(kTileFar, hi - s0);
      __syncthreads();
      for (int i = threadIdx.x; i < ns; i += kPairThreads) {
        const int j = s0 + i;
        const int o = j / A.n_eq;
        const int e = j - o * A.n_eq;
        const float4 z0 = A.eq[e];
        sp[i] = make_float4(z0.x + sh.d(o, 0), z0.y + sh.d(o, 1), z0.z + sh.d(o, 2), 0.f);
        const float* g = A.q + 3LL * j;
        sf[i] = make_float4(g[0], g[1], g[2], 0.f);
      }
      __syncthreads();
#pragma unroll 2
      for (int j = 0; j < ns; ++j) {
        const float4 p = sp[j];
        const float4 f = sf[j];
#pragma unroll
        for (int q = 0; q < NT; ++q) {
          float dx = x[q] - p.x, dy = y[q] - p.y, dz = z[q] - p.z;
          float r2 = dx * dx + dy * dy + dz * dz;
          float ir = rsqrtf(r2);
          float ir2 = ir * ir;
          float rf = dx * f.x + dy * f.y + dz * f.z;
          float c = rf * ir2;
          ux[q] += ir * (f.x + c * dx);
          uy[q] += ir * (f.y + c * dy);
          uz[q] += ir * (f.z + c * dz);
        }
      }
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        comp_add(sx[q], cx[q], ux[q]);
        comp_add(sy[q], cy[q], uy[q]);
        comp_add(sz[q], cz[q], uz[q]);
        ux[q] = uy[q] = uz[q] = 0.f;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    int idx = threadIdx.x + q * kPairThreads;
    if (idx < cnt) {
      long long node = start + idx;
      double sw = A.tgt64[4 * node + 3] * (double)A.scale;
      const double gx = sw * ((double)sx[q] + (double)cx[q]), gy = sw * ((double)sy[q] + (double)cy[q]),
                   gz = sw * ((double)sz[q] + (double)cz[q]);
      if (nparts > 1) {
        double* o = partial + part * pstride + 3 * node;
        o[0] = gx;
        o[1] = gy;
        o[2] = gz;
      } else {
        A.out[3 * node] += gx;
        A.out[3 * node + 1] += gy;
        A.out[3 * node + 2] += gz;
      }
    }
  }
}

// Packed-FP32 variant (sm_100+ f32x2 instructions): the four targets of a thread form two pairs,
// each operation of the pair math runs on both lanes of a pair with one instruction (the FMA pipe
// still does one lane-operation per target, but the issue slots are halved, which is what bounds
// the scalar kernel).  Sources are staged with every component duplicated into both lanes.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2sub(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2mul(f2x a, f2x b) {
  f2x d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x f2fma(f2x a, f2x b, f2x c) {
  f2x d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2x f2make(float lo, float hi) {
  f2x d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
  return d;
}
__device__ __forceinline__ void f2split(f2x v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__global__ void __launch_bounds__(kPairThreads) pairs_far2_kernel(FarArgs A, int nparts, double* __restrict__ partial,
                                                                  long long pstride) {
  __shared__ ulonglong2 sa[kTileFar];  // (px, px | py, py)
  __shared__ ulonglong2 sb[kTileFar];  // (pz, pz | fx, fx)
  __shared__ ulonglong2 sc[kTileFar];  // (fy, fy | fz, fz)
  constexpr int NT = 4;
  const int t = blockIdx.x / nparts, part = blockIdx.x % nparts;
  const int k = A.tile_sphere[t];
  const int start = A.tile_start[t];
  const int cnt = A.tile_count[t];
  CentreShift32 sh;
  sh.hi = A.cen_hi;
  sh.lo = A.cen_lo;
  sh.init(k);
  float x[NT], y[NT], z[NT], sx[NT], sy[NT], sz[NT], cx[NT], cy[NT], cz[NT];
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    int idx = threadIdx.x + q * kPairThreads;
    float4 p = A.tgt[start + (idx < cnt ? idx : cnt - 1)];
    x[q] = p.x; y[q] = p.y; z[q] = p.z;
    sx[q] = sy[q] = sz[q] = cx[q] = cy[q] = cz[q] = 0.f;
  }
  const f2x X0 = f2make(x[0], x[1]), X1 = f2make(x[2], x[3]);
  const f2x Y0 = f2make(y[0], y[1]), Y1 = f2make(y[2], y[3]);
  const f2x Z0 = f2make(z[0], z[1]), Z1 = f2make(z[2], z[3]);
  const f2x zero2 = f2make(0.f, 0.f);
  const int e0 = A.excl_off[k], e1 = A.excl_off[k + 1];
  const long long n_far = (long long)(A.P - (e1 - e0)) * A.n_eq;
  const long long f0 = n_far * part / nparts, f1 = n_far * (part + 1) / nparts;
  long long before = 0;
  int prev = -1;
  for (int a = e0; a <= e1; ++a) {
    const int nxt = a < e1 ? A.excl_idx[a] : A.P;
    const int run_lo = (prev + 1) * A.n_eq, run_hi = nxt * A.n_eq;
    prev = nxt;
    const long long len = run_hi - run_lo;
    const int lo = run_lo + (int)max(0LL, min(len, f0 - before));
    const int hi = run_lo + (int)max(0LL, min(len, f1 - before));
    before += len;
    for (int s0 = lo; s0 < hi; s0 += kTileFar) {
      const int ns = min(kTileFar, hi - s0);
      __syncthreads();
      for (int i = threadIdx.x; i < ns; i += kPairThreads) {
        const int j = s0 + i;
        const int o = j / A.n_eq;
        const int e = j - o * A.n_eq;
        const float4 z0 = A.eq[e];
        const float px = z0.x + sh.d(o, 0), py = z0.y + sh.d(o, 1), pz = z0.z + sh.d(o, 2);
        const float* g = A.q + 3LL * j;
        const float fx = g[0], fy = g[1], fz = g[2];
        sa[i] = make_ulonglong2(f2make(px, px), f2make(py, py));
        sb[i] = make_ulonglong2(f2make(pz, pz), f2make(fx, fx));
        sc[i] = make_ulonglong2(f2make(fy, fy), f2make(fz, fz));
      }
      __syncthreads();
      f2x ux0 = zero2, uy0 = zero2, uz0 = zero2, ux1 = zero2, uy1 = zero2, uz1 = zero2;
#pragma unroll 2
      for (int j = 0; j < ns; ++j) {
        const ulonglong2 a2 = sa[j], b2 = sb[j], c2 = sc[j];
#define MFS_FAR2_PAIR(X, Y, Z, UX, UY, UZ)                                        \
  {                                                                               \
    const f2x dx = f2sub(X, a2.x), dy = f2sub(Y, a2.y), dz = f2sub(Z, b2.x);      \
    const f2x r2 = f2fma(dz, dz, f2fma(dy, dy, f2mul(dx, dx)));                   \
    float rl, rh;                                                                 \
    f2split(r2, rl, rh);                                                          \
    const f2x ir = f2make(rsqrtf(rl), rsqrtf(rh));                                \
    const f2x ir2 = f2mul(ir, ir);                                                \
    const f2x rf = f2fma(dz, c2.y, f2fma(dy, c2.x, f2mul(dx, b2.y)));             \
    const f2x cc = f2mul(rf, ir2);                                                \
    UX = f2fma(ir, f2fma(cc, dx, b2.y), UX);                                      \
    UY = f2fma(ir, f2fma(cc, dy, c2.x), UY);                                      \
    UZ = f2fma(ir, f2fma(cc, dz, c2.y), UZ);                                      \
  }
        MFS_FAR2_PAIR(X0, Y0, Z0, ux0, uy0, uz0)
        MFS_FAR2_PAIR(X1, Y1, Z1, ux1, uy1, uz1)
#undef MFS_FAR2_PAIR
      }
      float u[3][NT];
      f2split(ux0, u[0][0], u[0][1]);
      f2split(ux1, u[0][2], u[0][3]);
      f2split(uy0, u[1][0], u[1][1]);
      f2split(uy1, u[1][2], u[1][3]);
      f2split(uz0, u[2][0], u[2][1]);
      f2split(uz1, u[2][2], u[2][3]);
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        comp_add(sx[q], cx[q], u[0][q]);
        comp_add(sy[q], cy[q], u[1][q]);
        comp_add(sz[q], cz[q], u[2][q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NT; ++q) {
    int idx = threadIdx.x + q * kPairThreads;
    if (idx < cnt) {
      long long node = start + idx;
      double sw = A.tgt64[4 * node + 3] * (double)A.scale;
      const double gx = sw * ((double)sx[q] + (double)cx[q]), gy = sw * ((double)sy[q] + (double)cy[q]),
                   gz = sw * ((double)sz[q] + (double)cz[q]);
      if (nparts > 1) {
        double* o = partial + part * pstride + 3 * node;
        o[0] = gx;
        o[1] = gy;
        o[2] = gz;
      } else {
        A.out[3 * node] += gx;
        A.out[3 * node + 1] += gy;
        A.out[3 * node + 2] += gz;
      }
    }
  }
}

// out[e] (+)= the parts in order: with mu, out = mu + sqrt(w) * sum (the near kernel's unscaled
// parts); without, out += sum (the far kernel's parts, already scaled)
__global__ void parts_add_kernel(long long n3, const D4* __restrict__ tgt, int nparts, const double* __restrict__ partial,
                                 long long pstride, const double* __restrict__ mu, double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += partial[q * pstride + e];
    out[e] = mu ? mu[e] + tgt[e / 3].w * s : out[e] + s;
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(kPairThreads) pairs_kernel(PairArgs<T> A) {
  pair_tile<T, NT>(A, blockIdx.x);
}
template <int NT>
__global__ void __launch_bounds__(kPairThreads) pairs_dw_kernel(PairArgs<double> A, int nparts, double* partial,
                                                                long long pstride) {
  pair_tile_dw<NT>(A, blockIdx.x / nparts, blockIdx.x % nparts, nparts, partial, pstride);
}
template <int NT>
__global__ void __launch_bounds__(kPairThreads) pairs_dw_near_kernel(PairArgs<double> A, const int* near_off,
                                                                     const int* near_idx, int nparts, double* partial,
                                                                     long long pstride) {
  pair_tile_dw_near<NT>(A, near_off, near_idx, blockIdx.x / nparts, blockIdx.x % nparts, nparts, partial, pstride);
}
// out = mu + sqrt(w) * (sum of the parts), or the plain sum when mu is null; parts added in order
__global__ void pair_parts_reduce_kernel(long long n3, const D4* __restrict__ tgt, int nparts,
                                         const double* __restrict__ partial, long long pstride,
                                         const double* __restrict__ mu, double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3; e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nparts; ++q) s += partial[q * pstride + e];
    out[e] = mu ? mu[e] + tgt[e / 3].w * s : s;
  }
}
// Many problems in one launch: work[b] = (problem, tile); problems whose flag is 0 are skipped.
// The per-problem vectors are segments of concatenated ones: lam at lam + uoff[p], mu and out
// at mu + voff[p], out + voff[p].
struct BatchVecs {
  const double* lam;
  const double* mu;
  double* out;
  const long long* uoff;
  const long long* voff;
  double* partial;     // split sources: nparts slices of the concatenated vector length
  long long pstride;
  const long long* nlen;  // node rows (3 n_colloc) of each problem; a mobility problem's border follows
  unsigned* counter;      // optional, zeros, one per work item: with split sources the last CTA of an
                          // item adds the parts (in part order) itself and re-arms its counter
};

// Split sources, fused reduction: every CTA of work item `item` has written its partial sums of the
// tile's nodes; the last one to arrive adds the parts in part order and writes out = mu + sqrt(w) s.
// Returns whether this CTA was the last (all threads see the same answer).
__device__ __forceinline__ bool parts_last_arrival(unsigned* counter, int item, int nparts) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(&counter[item], 1u) == (unsigned)nparts - 1;
    if (last) counter[item] = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}
__device__ __forceinline__ void parts_finish_node(const D4* tgt, long long node, int nparts, const double* partial,
                                                  long long pstride, const double* mu, double* out) {
  const double sw = tgt[node].w;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double sum = 0.0;
    for (int q = 0; q < nparts; ++q) sum += __ldcg(&partial[q * pstride + 3 * node + c]);
    out[3 * node + c] = mu[3 * node + c] + sw * sum;
  }
}
template <typename T, int NT>
__global__ void __launch_bounds__(kPairThreads) pairs_batch_kernel(const PairArgs<T>* __restrict__ args,
                                                                   const int2* __restrict__ work,
                                                                   const int* __restrict__ active, BatchVecs bv) {
  const int2 w = work[blockIdx.x];
  if (!active[w.x]) return;
  PairArgs<T> A = args[w.x];
  A.lam = bv.lam + bv.uoff[w.x];
  A.mu = bv.mu + bv.voff[w.x];
  A.out = bv.out + bv.voff[w.x];
  pair_tile<T, NT>(A, w.y);
}
// (register bounds as the compiler chose them before the fused reduction: 7 CTAs per SM for 1 node
// per thread, 4 for 4)
template <int NT>
__global__ void __launch_bounds__(kPairThreads, NT == 1 ? 7 : 4) pairs_dw_batch_kernel(const PairArgs<double>* __restrict__ args,
                                                                      const int2* __restrict__ work,
                                                                      const int* __restrict__ active, BatchVecs bv,
                                                                      int nparts) {
  const int2 w = work[blockIdx.x / nparts];
  if (!active[w.x]) return;
  PairArgs<double> A = args[w.x];
  A.lam = bv.lam + bv.uoff[w.x];
  A.mu = bv.mu + bv.voff[w.x];
  A.out = bv.out + bv.voff[w.x];
  pair_tile_dw<NT>(A, w.y, blockIdx.x % nparts, nparts, bv.partial + bv.voff[w.x], bv.pstride);
  if constexpr (NT == 1) {  // only the 1-node tiling splits sources
    if (nparts > 1 && bv.counter && parts_last_arrival(bv.counter, blockIdx.x / nparts, nparts)) {
      const int start = A.tile_start[w.y], cnt = A.tile_count[w.y];
      for (int i = threadIdx.x; i < cnt; i += blockDim.x)
        parts_finish_node(A.tgt, start + i, nparts, bv.partial + bv.voff[w.x], bv.pstride, A.mu, A.out);
    }
  }
}
// ------------------------------------------------------------------ several right-hand sides on one geometry
// The problems of a batch that share a context (the motions of one geometry) have the same
// targets and sources and differ only in their strengths.  Work item (lead problem, 128-node
// tile, first index into the right-hand-side list, count <= kPairRhs): the position
// differences, the distance and its powers of each (node, source) pair are formed once in
// double-float and applied to the strengths of every listed right-hand side (~85 of the ~204
// FP32 operations of a Stokeslet pair, ~89 of ~436 of an image triple, are shared).  Each
// right-hand side's sums follow the operation order of pair_tile_dw.
constexpr int kTileProxyM = 128;  // proxy sources staged per round
constexpr int kTileImgM = 64;     // image nodes staged per round

template <int R>
struct DWMulti {
  dw x, y, z;
  dw ux[R], uy[R], uz[R];
};

template <int R>
__device__ __forceinline__ void dwm_proxy_range(const PairArgs<double>& A, const CentreShift64& sh, int k,
                                                const double* const (&lam)[R], unsigned mask, int r_lo, int r_hi,
                                                float4* sp, float4 (*sf)[2 * kTileProxyM], DWMulti<R>& T) {
  const double far = 1e18;
  const int total = A.P * A.N;
  for (int s0 = r_lo; s0 < r_hi; s0 += kTileProxyM) {
    const int ns = min(kTileProxyM, r_hi - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < ns; i += kPairThreads) {
      const int j = s0 + i;
      double px = far, py = far, pz = far;
      int o = -1, jj = 0;
      if (j < total) {
        o = j / A.N;
        jj = j - o * A.N;
        const D4 pr = A.proxy[jj];
        px = pr.x + sh.d(o, 0);
        py = pr.y + sh.d(o, 1);
        pz = pr.z + sh.d(o, 2);
      }
      dw a = dw_split(px), b = dw_split(py), c = dw_split(pz);
      sp[2 * i] = make_float4(a.h, b.h, c.h, 0.f);
      sp[2 * i + 1] = make_float4(a.l, b.l, c.l, 0.f);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        double fx = 0, fy = 0, fz = 0;
        if ((mask >> r & 1u) && o >= 0 && o != k) {
          const double* l = lam[r] + A.unk_off[o] + 3LL * jj;
          fx = l[0];
          fy = l[1];
          fz = l[2];
        }
        a = dw_split(fx);
        b = dw_split(fy);
        c = dw_split(fz);
        sf[r][2 * i] = make_float4(a.h, b.h, c.h, 0.f);
        sf[r][2 * i + 1] = make_float4(a.l, b.l, c.l, 0.f);
      }
    }
    __syncthreads();
    for (int j = 0; j < ns; ++j) {
      const float4 ph = sp[2 * j], pl = sp[2 * j + 1];
      const dw dx = sub_pos(T.x, dw{ph.x, pl.x});
      const dw dy = sub_pos(T.y, dw{ph.y, pl.y});
      const dw dz = sub_pos(T.z, dw{ph.z, pl.z});
      const dw ir = rsqrt_u(norm2_u(dx, dy, dz));
      const dw ir2 = mul_u(ir, ir);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(mask >> r & 1u)) continue;
        const float4 fh = sf[r][2 * j], fl = sf[r][2 * j + 1];
        const dw fx{fh.x, fl.x}, fy{fh.y, fl.y}, fz{fh.z, fl.z};
        const dw c = mul_u(dot3_u(dx, dy, dz, fx, fy, fz), ir2);
        acc_u(T.ux[r], mul_u(ir, add_u(fx, mul_u(c, dx))));
        acc_u(T.uy[r], mul_u(ir, add_u(fy, mul_u(c, dy))));
        acc_u(T.uz[r], mul_u(ir, add_u(fz, mul_u(c, dz))));
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T.ux[r] = two_sum(T.ux[r].h, T.ux[r].l);
      T.uy[r] = two_sum(T.uy[r].h, T.uy[r].l);
      T.uz[r] = two_sum(T.uz[r].h, T.uz[r].l);
    }
  }
}

// image node strengths of one right-hand side in 5 float4: hi of (f, t, d) then lo of the same
template <int R>
__device__ __forceinline__ void dwm_image_range(const PairArgs<double>& A, const CentreShift64& sh, int k,
                                                const double* const (&lam)[R], unsigned mask, int r_lo, int r_hi,
                                                float4* sip, float4 (*sis)[5 * kTileImgM], DWMulti<R>& T) {
  const double far = 1e18;
  for (int s0 = r_lo; s0 < r_hi; s0 += kTileImgM) {
    const int ns = min(kTileImgM, r_hi - s0);
    __syncthreads();
    for (int i = threadIdx.x; i < ns; i += kPairThreads) {
      const int j = s0 + i;
      double px = far, py = far, pz = far;
      int o = -1;
      if (j < A.n_img) {
        o = A.img_owner[j];
        const D4 pr = A.img[j];
        px = pr.x + sh.d(o, 0);
        py = pr.y + sh.d(o, 1);
        pz = pr.z + sh.d(o, 2);
      }
      dw a = dw_split(px), b = dw_split(py), c = dw_split(pz);
      sip[2 * i] = make_float4(a.h, b.h, c.h, 0.f);
      sip[2 * i + 1] = make_float4(a.l, b.l, c.l, 0.f);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float hv[9], lv[9];
        const double* l = nullptr;
        if ((mask >> r & 1u) && o >= 0 && o != k) l = lam[r] + A.unk_off[o] + 3LL * A.N + 9LL * (j - A.img_off[o]);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          const double v = l ? (q < 6 ? l[q] : A.dip * l[q]) : 0.0;
          const dw sv = dw_split(v);
          hv[q] = sv.h;
          lv[q] = sv.l;
        }
        sis[r][5 * i] = make_float4(hv[0], hv[1], hv[2], hv[3]);
        sis[r][5 * i + 1] = make_float4(hv[4], hv[5], hv[6], hv[7]);
        sis[r][5 * i + 2] = make_float4(hv[8], lv[0], lv[1], lv[2]);
        sis[r][5 * i + 3] = make_float4(lv[3], lv[4], lv[5], lv[6]);
        sis[r][5 * i + 4] = make_float4(lv[7], lv[8], 0.f, 0.f);
      }
    }
    __syncthreads();
    for (int j = 0; j < ns; ++j) {
      const float4 ph = sip[2 * j], pl = sip[2 * j + 1];
      const dw dx = sub_pos(T.x, dw{ph.x, pl.x}), dy = sub_pos(T.y, dw{ph.y, pl.y}), dz = sub_pos(T.z, dw{ph.z, pl.z});
      const dw ir = rsqrt_u(norm2_u(dx, dy, dz));
      const dw ir2 = mul_u(ir, ir);
      const dw ir3 = mul_u(ir, ir2);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (!(mask >> r & 1u)) continue;
        const float4 v0 = sis[r][5 * j], v1 = sis[r][5 * j + 1], v2 = sis[r][5 * j + 2], v3 = sis[r][5 * j + 3],
                     v4 = sis[r][5 * j + 4];
        const dw fx{v0.x, v2.y}, fy{v0.y, v2.z}, fz{v0.z, v2.w};
        const dw tx{v0.w, v3.x}, ty{v1.x, v3.y}, tz{v1.y, v3.z};
        const dw qx{v1.z, v3.w}, qy{v1.w, v4.x}, qz{v2.x, v4.y};
        // Stokeslet
        const dw cs = mul_u(dot3_u(dx, dy, dz, fx, fy, fz), ir2);
        acc_u(T.ux[r], mul_u(ir, add_u(fx, mul_u(cs, dx))));
        acc_u(T.uy[r], mul_u(ir, add_u(fy, mul_u(cs, dy))));
        acc_u(T.uz[r], mul_u(ir, add_u(fz, mul_u(cs, dz))));
        // rotlet (t x r) / r^3
        acc_u(T.ux[r], mul_u(ir3, add_u(mul_u(ty, dz), neg(mul_u(tz, dy)))));
        acc_u(T.uy[r], mul_u(ir3, add_u(mul_u(tz, dx), neg(mul_u(tx, dz)))));
        acc_u(T.uz[r], mul_u(ir3, add_u(mul_u(tx, dy), neg(mul_u(ty, dx)))));
        // potential dipole -d / r^3 + 3 (d.r) r / r^5
        const dw c3 = times3_u(mul_u(mul_u(dot3_u(dx, dy, dz, qx, qy, qz), ir3), ir2));
        acc_u(T.ux[r], mul_u(c3, dx));
        acc_u(T.uy[r], mul_u(c3, dy));
        acc_u(T.uz[r], mul_u(c3, dz));
        acc_u(T.ux[r], neg(mul_u(ir3, qx)));
        acc_u(T.uy[r], neg(mul_u(ir3, qy)));
        acc_u(T.uz[r], neg(mul_u(ir3, qz)));
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      T.ux[r] = two_sum(T.ux[r].h, T.ux[r].l);
      T.uy[r] = two_sum(T.uy[r].h, T.uy[r].l);
      T.uz[r] = two_sum(T.uz[r].h, T.uz[r].l);
    }
  }
}

// work[b] = (lead problem, tile of the 1-node-per-thread tiling, first index into rhs_prob, count);
// the sources are split over nparts CTAs per item as in pairs_dw_batch_kernel
template <int R>
__global__ void __launch_bounds__(kPairThreads) pairs_dw_multi_kernel(const PairArgs<double>* __restrict__ args,
                                                                      const int4* __restrict__ work,
                                                                      const int* __restrict__ rhs_prob,
                                                                      const int* __restrict__ active, BatchVecs bv,
                                                                      int nparts) {
  __shared__ float4 sp[2 * kTileProxyM];
  __shared__ float4 sf[R][2 * kTileProxyM];
  __shared__ float4 sip[2 * kTileImgM];
  __shared__ float4 sis[R][5 * kTileImgM];
  const int4 w = work[blockIdx.x / nparts];
  const int part = blockIdx.x % nparts;
  int prob[R];
  unsigned mask = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    prob[r] = rhs_prob[w.z + min(r, w.w - 1)];
    if (r < w.w && active[prob[r]]) mask |= 1u << r;
  }
  if (!mask) return;
  const PairArgs<double> A = args[w.x];
  const double* lam[R];
#pragma unroll
  for (int r = 0; r < R; ++r) lam[r] = bv.lam + bv.uoff[prob[r]];
  const int t = w.y;
  const int k = A.tile_sphere[t];
  const int start = A.tile_start[t];
  const int cnt = A.tile_count[t];
  CentreShift64 sh;
  sh.cen = A.cen64;
  sh.init(k);
  DWMulti<R> T;
  {
    const int idx = threadIdx.x;
    const int node = start + (idx < cnt ? idx : cnt - 1);
    const D4 p = A.tgt[node];
    T.x = dw_split(p.x);
    T.y = dw_split(p.y);
    T.z = dw_split(p.z);
#pragma unroll
    for (int r = 0; r < R; ++r) T.ux[r] = T.uy[r] = T.uz[r] = dw{0.f, 0.f};
  }
  const int total = A.P * A.N;
  const int p_lo = k < 0 ? total : k * A.N, p_w = k < 0 ? 0 : A.N;
  const long long p_eff = total - p_w;
  const int pe0 = (int)(p_eff * part / nparts), pe1 = (int)(p_eff * (part + 1) / nparts);
  dwm_proxy_range<R>(A, sh, k, lam, mask, min(pe0, p_lo), min(pe1, p_lo), sp, sf, T);
  dwm_proxy_range<R>(A, sh, k, lam, mask, max(pe0, p_lo) + p_w, max(pe1, p_lo) + p_w, sp, sf, T);
  const int i_lo = k >= 0 ? A.img_off[k] : 0, i_w = k >= 0 ? A.img_off[k + 1] - i_lo : 0;
  const long long i_eff = A.n_img - i_w;
  const int ie0 = (int)(i_eff * part / nparts), ie1 = (int)(i_eff * (part + 1) / nparts);
  dwm_image_range<R>(A, sh, k, lam, mask, min(ie0, i_lo), min(ie1, i_lo), sip, sis, T);
  dwm_image_range<R>(A, sh, k, lam, mask, max(ie0, i_lo) + i_w, max(ie1, i_lo) + i_w, sip, sis, T);
  const int idx = threadIdx.x;
  if (idx < cnt) {
    const long long node = start + idx;
    const double sw = A.tgt[node].w;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!(mask >> r & 1u)) continue;
      const double gx = dw_join(T.ux[r]) * A.scale, gy = dw_join(T.uy[r]) * A.scale, gz = dw_join(T.uz[r]) * A.scale;
      const long long off = bv.voff[prob[r]];
      if (nparts > 1) {
        double* o = bv.partial + off + part * bv.pstride + 3 * node;
        o[0] = gx;
        o[1] = gy;
        o[2] = gz;
      } else {
        const double* mu = bv.mu + off;
        double* out = bv.out + off;
        out[3 * node] = mu[3 * node] + sw * gx;
        out[3 * node + 1] = mu[3 * node + 1] + sw * gy;
        out[3 * node + 2] = mu[3 * node + 2] + sw * gz;
      }
    }
  }
  if (nparts > 1 && bv.counter && parts_last_arrival(bv.counter, blockIdx.x / nparts, nparts)) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!(mask >> r & 1u)) continue;
      const long long off = bv.voff[prob[r]];
      for (int i = threadIdx.x; i < cnt; i += blockDim.x)
        parts_finish_node(A.tgt, start + i, nparts, bv.partial + off, bv.pstride, bv.mu + off, bv.out + off);
    }
  }
}

// the batched counterpart of pair_parts_reduce_kernel: CTA (chunk of an active problem, piece of
// blockDim elements), so that a single short problem still gets enough CTAs
__global__ void pair_parts_reduce_batch_kernel(SegTable t, const PairArgs<double>* __restrict__ args, BatchVecs bv,
                                               int nparts) {
  const int b = t.list ? t.list[blockIdx.x] : blockIdx.x;
  const int p = t.prob[b];
  if (!t.active[p]) return;
  const long long e = t.start[b] + (long long)blockIdx.y * blockDim.x + threadIdx.x;
  if (e >= t.end[b]) return;
  if (bv.nlen && e - bv.voff[p] >= bv.nlen[p]) return;  // a mobility problem's border rows
  const D4* tgt = args[p].tgt;
  double s = 0.0;
  for (int q = 0; q < nparts; ++q) s += bv.partial[q * bv.pstride + e];
  bv.out[e] = bv.mu[e] + tgt[(e - bv.voff[p]) / 3].w * s;
}

// ------------------------------------------------------------------ batched GEMV
constexpr int kGemvThreads = 256;
constexpr int kGemvRowsPerWarp = 2;
constexpr int kGemvDepth = 4;  // 16-byte loads per row and lane in flight in the double-float GEMVs

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int w = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int w = 2; };

template <typename T>
__device__ __forceinline__ T dot_vec(const typename Vec<T>::type& m, const T* x);
template <> __device__ __forceinline__ float dot_vec<float>(const float4& m, const float* x) {
  return m.x * __ldg(x) + m.y * __ldg(x + 1) + m.z * __ldg(x + 2) + m.w * __ldg(x + 3);
}
template <> __device__ __forceinline__ double dot_vec<double>(const double2& m, const double* x) {
  return m.x * __ldg(x) + m.y * __ldg(x + 1);
}

template <typename T>
__global__ void __launch_bounds__(kGemvThreads) gemv_kernel(GemvBatch<T> B, const T* __restrict__ x, T* __restrict__ y) {
  using VT = typename Vec<T>::type;
  constexpr int W = Vec<T>::w;
  // jobs sharing a matrix are adjacent, so its rows are read once; with a compacted list the grid
  // covers the active problems' jobs only
  const int job = B.job_list ? B.job_list[blockIdx.x] : blockIdx.x;
  if (B.active && !B.active[B.job_prob[job]]) return;
  const int nr = B.rows[job], nc = B.cols[job], ld = B.ld[job];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = (blockIdx.y * (kGemvThreads / 32) + warp) * kGemvRowsPerWarp;
  if (r0 >= nr) return;
  const T* M = B.mat[job];
  const T* xv = x + B.x_off[job];
  T acc[kGemvRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) acc[r] = T(0);
  const int nvec = nc / W;
  for (int v = lane; v < nvec; v += 32) {
#pragma unroll
    for (int r = 0; r < kGemvRowsPerWarp; ++r) {
      int row = r0 + r;
      if (row < nr) {
        VT m = reinterpret_cast<const VT*>(M + (long long)row * ld)[v];
        acc[r] += dot_vec<T>(m, xv + v * W);
      }
    }
  }
  for (int c = nvec * W + lane; c < nc; c += 32) {
#pragma unroll
    for (int r = 0; r < kGemvRowsPerWarp; ++r) {
      int row = r0 + r;
      if (row < nr) acc[r] += M[(long long)row * ld + c] * xv[c];
    }
  }
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) {
    T s = acc[r];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && r0 + r < nr) y[B.y_off[job] + r0 + r] = s;
  }
}

// Double-float GEMV: each matrix element and each x element is a (hi, lo) float pair; products
// and sums use the error-free double-word operations above, so the result carries ~2^-46
// relative accuracy while reading the same 8 bytes per element as FP64.
template <bool OUT64>
__global__ void __launch_bounds__(kGemvThreads) gemv_dw_kernel(GemvBatch<double> B, const float2* __restrict__ x,
                                                                float2* __restrict__ y2, double* __restrict__ y64) {
  // jobs sharing a matrix are adjacent, so its rows are read once; with a compacted list the grid
  // covers the active problems' jobs only
  const int job = B.job_list ? B.job_list[blockIdx.x] : blockIdx.x;
  if (B.active && !B.active[B.job_prob[job]]) return;
  const int nr = B.rows[job], nc = B.cols[job], ld = B.ld[job];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = (blockIdx.y * (kGemvThreads / 32) + warp) * kGemvRowsPerWarp;
  if (r0 >= nr) return;
  const float2* M = B.mat_dw[job];
  const float2* xv = x + B.x_off[job];
  dw acc[kGemvRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) acc[r] = dw{0.f, 0.f};
  const int npair = nc / 2;  // two elements per 16-byte load
  // kGemvDepth loads per row and lane issued before they are used, so that enough bytes are
  // in flight even when few jobs are active (the lockstep tail)
  for (int v0 = lane; v0 < npair; v0 += 32 * kGemvDepth) {
    float4 m[kGemvDepth][kGemvRowsPerWarp];
#pragma unroll
    for (int u = 0; u < kGemvDepth; ++u)
#pragma unroll
      for (int r = 0; r < kGemvRowsPerWarp; ++r)
        if (v0 + 32 * u < npair && r0 + r < nr)
          m[u][r] = reinterpret_cast<const float4*>(M + (long long)(r0 + r) * ld)[v0 + 32 * u];
#pragma unroll
    for (int u = 0; u < kGemvDepth; ++u) {
      const int v = v0 + 32 * u;
      if (v >= npair) break;
      const float2 xa = xv[2 * v], xb = xv[2 * v + 1];
#pragma unroll
      for (int r = 0; r < kGemvRowsPerWarp; ++r)
        if (r0 + r < nr) {
          acc[r] = dw_add(acc[r], dw_mul(dw{m[u][r].x, m[u][r].y}, dw{xa.x, xa.y}));
          acc[r] = dw_add(acc[r], dw_mul(dw{m[u][r].z, m[u][r].w}, dw{xb.x, xb.y}));
        }
    }
  }
  for (int cidx = 2 * npair + lane; cidx < nc; cidx += 32) {
    const float2 xa = xv[cidx];
#pragma unroll
    for (int r = 0; r < kGemvRowsPerWarp; ++r) {
      int row = r0 + r;
      if (row < nr) {
        float2 m = M[(long long)row * ld + cidx];
        acc[r] = dw_add(acc[r], dw_mul(dw{m.x, m.y}, dw{xa.x, xa.y}));
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) {
    dw s = acc[r];
    for (int o = 16; o > 0; o >>= 1) {
      dw t{__shfl_xor_sync(0xffffffffu, s.h, o), __shfl_xor_sync(0xffffffffu, s.l, o)};
      s = dw_add(s, t);
    }
    if (lane == 0 && r0 + r < nr) {
      long long idx = B.y_off[job] + r0 + r;
      if (OUT64) y64[idx] = dw_join(s);
      else y2[idx] = make_float2(s.h, s.l);
    }
  }
}

// The same product with the matrix in FP32 (4 bytes per element).  Per element the product
// m (x_hi + x_lo) is formed exactly up to the rounding of its small part (TwoProd), the running
// FP32 sum's rounding error is captured by TwoSum, and the error terms are summed in a second
// float that is folded in once per lane: ~11 instructions per element instead of a full
// double-word product and sum, with an accumulation error (~n^2 eps^2 for n terms per lane)
// far below the FP32 rounding of the matrix itself, which is the only real error.  Used for Sigma^+ U^T in the inner solves of MFS_MIXED,
// whose rounding (relative 6e-8 per element, amplified by Sigma^+ only along right singular
// vectors whose fields on the other spheres are correspondingly weak) leaves the operator
// accurate to ~1e-7; the refinement residual is evaluated with the double-float factors.
__global__ void __launch_bounds__(kGemvThreads) gemv_f32dw_kernel(GemvBatch<float> B, const float2* __restrict__ x,
                                                                  float2* __restrict__ y2) {
  const int job = B.job_list ? B.job_list[blockIdx.x] : blockIdx.x;
  if (B.active && !B.active[B.job_prob[job]]) return;
  const int nr = B.rows[job], nc = B.cols[job], ld = B.ld[job];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = (blockIdx.y * (kGemvThreads / 32) + warp) * kGemvRowsPerWarp;
  if (r0 >= nr) return;
  const float* M = B.mat[job];
  const float2* xv = x + B.x_off[job];
  float sh[kGemvRowsPerWarp], sl[kGemvRowsPerWarp];
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) sh[r] = sl[r] = 0.f;
  auto add = [](float& h, float& l, float m, float2 xe) {
    dw p = two_prod(m, xe.x);
    p.l = __fmaf_rn(m, xe.y, p.l);
    dw t = two_sum(h, p.h);
    h = t.h;
    l = __fadd_rn(l, __fadd_rn(t.l, p.l));
  };
  const int nq = nc / 4;  // four elements per 16-byte load
  for (int v0 = lane; v0 < nq; v0 += 32 * kGemvDepth) {
    float4 m[kGemvDepth][kGemvRowsPerWarp];
#pragma unroll
    for (int u = 0; u < kGemvDepth; ++u)
#pragma unroll
      for (int r = 0; r < kGemvRowsPerWarp; ++r)
        if (v0 + 32 * u < nq && r0 + r < nr)
          m[u][r] = reinterpret_cast<const float4*>(M + (long long)(r0 + r) * ld)[v0 + 32 * u];
#pragma unroll
    for (int u = 0; u < kGemvDepth; ++u) {
      const int v = v0 + 32 * u;
      if (v >= nq) break;
      const float2 x0 = xv[4 * v], x1 = xv[4 * v + 1], x2 = xv[4 * v + 2], x3 = xv[4 * v + 3];
#pragma unroll
      for (int r = 0; r < kGemvRowsPerWarp; ++r)
        if (r0 + r < nr) {
          add(sh[r], sl[r], m[u][r].x, x0);
          add(sh[r], sl[r], m[u][r].y, x1);
          add(sh[r], sl[r], m[u][r].z, x2);
          add(sh[r], sl[r], m[u][r].w, x3);
        }
    }
  }
  for (int cidx = 4 * nq + lane; cidx < nc; cidx += 32) {
    const float2 xa = xv[cidx];
#pragma unroll
    for (int r = 0; r < kGemvRowsPerWarp; ++r) {
      int row = r0 + r;
      if (row < nr) add(sh[r], sl[r], M[(long long)row * ld + cidx], xa);
    }
  }
#pragma unroll
  for (int r = 0; r < kGemvRowsPerWarp; ++r) {
    dw s = two_sum(sh[r], sl[r]);
    for (int o = 16; o > 0; o >>= 1) {
      dw t{__shfl_xor_sync(0xffffffffu, s.h, o), __shfl_xor_sync(0xffffffffu, s.l, o)};
      s = dw_add(s, t);
    }
    if (lane == 0 && r0 + r < nr) y2[B.y_off[job] + r0 + r] = make_float2(s.h, s.l);
  }
}

__global__ void split_dw_kernel(long long n, const double* __restrict__ in, float2* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    dw s = dw_split(in[e]);
    out[e] = make_float2(s.h, s.l);
  }
}

// ------------------------------------------------------------------ Krylov helpers
constexpr int kRedThreads = 256;

template <typename T>
__global__ void multidot_kernel(int n, const T* __restrict__ V, long long ldv, const T* __restrict__ w,
                                double* __restrict__ partial, int nblk) {
  const int b = blockIdx.x, i = blockIdx.y;
  const int chunk = (n + nblk - 1) / nblk;
  const int lo = b * chunk, hi = min(n, lo + chunk);
  const T* v = V + (long long)i * ldv;
  T s = T(0);
  for (int e = lo + threadIdx.x; e < hi; e += blockDim.x) s += v[e] * w[e];
  double d = (double)s;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  __shared__ double red[kRedThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    partial[(long long)i * nblk + b] = t;
  }
}

__global__ void reduce_partials_kernel(int nvec, int nblk, const double* __restrict__ partial, double* __restrict__ h) {
  const int i = blockIdx.x;
  double s = 0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(long long)i * nblk + b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    h[i] = t;
  }
}

template <typename T>
__global__ void update_kernel(int n, int nvec, const T* __restrict__ V, long long ldv, const double* __restrict__ h,
                              double sign, T* __restrict__ w) {
  __shared__ T hs[512];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) hs[i] = T(sign * h[i]);
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    T acc = w[e];
    for (int i = 0; i < nvec; ++i) acc += hs[i] * V[(long long)i * ldv + e];
    w[e] = acc;
  }
}

template <typename T>
__global__ void scale_copy_kernel(int n, const T* __restrict__ w, double s, T* __restrict__ out) {
  T ss = T(s);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = ss * w[e];
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(long long n, const Tin* __restrict__ in, double s, Tout* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = (Tout)(s * (double)in[e]);
}

__global__ void axpy_mixed_kernel(int n, double a, const float* __restrict__ x, double* __restrict__ y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] += a * (double)x[e];
}

__global__ void sub_kernel(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    out[e] = a[e] - b[e];
}

// ------------------------------------------------------------------ segmented (batched) vector kernels
constexpr int kSegThreads = 256;

// The chunk a CTA works on: blockIdx.x indexes the compacted list of the active problems'
// chunks when the table carries one, else all chunks (inactive ones return at once).
__device__ __forceinline__ int seg_chunk(const SegTable& t) { return t.list ? t.list[blockIdx.x] : blockIdx.x; }

// Partial dot products of w with basis vectors over one chunk: CTA (chunk, vector block) stages
// the chunk of w (at most kSegChunkMax elements) in shared memory and each warp takes vectors of
// its block, so the launch has enough CTAs to keep HBM busy even for a single short problem.
constexpr int kSegChunkMax = 1024;
constexpr int kSegDotVecs = 16;   // basis vectors per CTA
constexpr int kSegUpdSub = 128;   // elements per CTA of the update (one per thread)
__global__ void seg_dots_kernel(SegTable t, int nvec, const double* __restrict__ V, long long ldv,
                                const double* __restrict__ w, double* __restrict__ partial, double* __restrict__ h) {
  const int b = seg_chunk(t);
  const int p = t.prob[b];
  if (!t.active[p]) return;
  const long long lo = t.start[b];
  const int len = (int)(t.end[b] - lo);
  __shared__ double ws[kSegChunkMax];
  for (int e = threadIdx.x; e < len; e += blockDim.x) ws[e] = w[lo + e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int i1 = min(nvec, (int)(blockIdx.y + 1) * kSegDotVecs);
  // two vectors per warp at a time, so that twice the loads are in flight
  for (int i = blockIdx.y * kSegDotVecs + warp; i < i1; i += 2 * nwarps) {
    const int i2 = i + nwarps;
    const double* v = V + (long long)i * ldv + lo;
    const double* v2 = V + (long long)min(i2, i1 - 1) * ldv + lo;
    double d = 0.0, d2 = 0.0;
#pragma unroll 8
    for (int e = lane; e < len; e += 32) {
      const double x = ws[e];
      d += v[e] * x;
      d2 += v2[e] * x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      d += __shfl_xor_sync(0xffffffffu, d, o);
      d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    }
    if (lane == 0) {
      partial[(long long)i * t.nchunks + b] = d;
      if (i2 < i1) partial[(long long)i2 * t.nchunks + b] = d2;
    }
  }
  if (!t.counter) return;
  // the last CTA of problem p to finish adds its partial dots in chunk order (so the result does
  // not depend on which CTA that is) and re-arms the counter for the next launch
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned total = (unsigned)(t.pchunk[p + 1] - t.pchunk[p]) * gridDim.y;
    last = atomicAdd(&t.counter[p], 1u) == total - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    double sum = 0.0;
    for (int c = t.pchunk[p]; c < t.pchunk[p + 1]; ++c) sum += __ldcg(&partial[(long long)i * t.nchunks + c]);
    h[(long long)i * t.K + p] = sum;
  }
  if (threadIdx.x == 0) t.counter[p] = 0u;
}

// h[i K + p] = sum over problem p's chunks (in order) of the partial dots of vector i
__global__ void seg_reduce_kernel(SegTable t, int nvec, const double* __restrict__ partial, double* __restrict__ h) {
  const int p = blockIdx.x;
  if (!t.active[p]) return;
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    double s = 0.0;
    for (int b = t.pchunk[p]; b < t.pchunk[p + 1]; ++b) s += partial[(long long)i * t.nchunks + b];
    h[(long long)i * t.K + p] = s;
  }
}

// w += sign * sum_i coef[i K + p] V_i over one kSegUpdSub-element piece of a chunk per CTA.  The
// CTA's kSegUpdGroups thread groups take interleaved vectors (more loads in flight when a short
// problem has few pieces) and their sums are added in group order.
constexpr int kSegUpdGroups = 4;
__global__ void __launch_bounds__(kSegUpdSub* kSegUpdGroups)
    seg_update_kernel(SegTable t, int nvec, const double* __restrict__ V, long long ldv,
                      const double* __restrict__ coef, double sign, double* __restrict__ w) {
  const int b = seg_chunk(t);
  const int p = t.prob[b];
  if (!t.active[p]) return;
  const int tl = threadIdx.x % kSegUpdSub, g = threadIdx.x / kSegUpdSub;
  const long long e = t.start[b] + (long long)blockIdx.y * kSegUpdSub + tl;
  if (t.start[b] + (long long)blockIdx.y * kSegUpdSub >= t.end[b]) return;  // whole CTA past the chunk
  __shared__ double c[512];
  __shared__ double red[kSegUpdGroups][kSegUpdSub];
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) c[i] = sign * coef[(long long)i * t.K + p];
  __syncthreads();
  double a = 0.0;
  if (e < t.end[b]) {
#pragma unroll 8
    for (int i = g; i < nvec; i += kSegUpdGroups) a += c[i] * V[(long long)i * ldv + e];
  }
  red[g][tl] = a;
  __syncthreads();
  if (g == 0 && e < t.end[b]) {
    double s = w[e];
#pragma unroll
    for (int q = 0; q < kSegUpdGroups; ++q) s += red[q][tl];
    w[e] = s;
  }
}

inline int seg_ctas(const SegTable& t) { return t.list ? t.nlist : t.nchunks; }

__global__ void seg_scale_kernel(SegTable t, const double* __restrict__ s, const double* __restrict__ in,
                                 double* __restrict__ out) {
  const int b = seg_chunk(t);
  const int p = t.prob[b];
  if (!t.active[p]) return;
  const double f = s[p];
  for (long long e = t.start[b] + threadIdx.x; e < t.end[b]; e += blockDim.x) out[e] = f * in[e];
}

__global__ void seg_scale_split_kernel(SegTable t, const double* __restrict__ s, const double* __restrict__ in,
                                       double* __restrict__ out, float2* __restrict__ x2) {
  const int b = seg_chunk(t);
  const int p = t.prob[b];
  if (!t.active[p]) return;
  const double f = s[p];
  for (long long e = t.start[b] + threadIdx.x; e < t.end[b]; e += blockDim.x) {
    const double v = f * in[e];
    out[e] = v;
    const dw d = dw_split(v);
    x2[e] = make_float2(d.h, d.l);
  }
}

__global__ void axpy64_kernel(long long n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    y[e] += a * x[e];
}

// ------------------------------------------------------------------ batched Givens (device)
// One Arnoldi step for every active problem of a lockstep batch, one thread per problem: the
// Hessenberg column h = h1 + h2 (the two classical Gram-Schmidt passes) with the subdiagonal
// sqrt(hn), the earlier Givens rotations applied, a new rotation formed, the least-squares
// right-hand side g rotated and the residual estimate |g_{j+1}| / ||b|| updated.  A problem that
// meets its tolerance (or breaks down) is deactivated here, on the device, so the host need
// not wait for every step; scl = 1 / h_{j+1,j} normalises the new basis vector.
// One CTA per problem.  Applying the earlier rotations to the new column is the first-order
// linear recurrence r_{i+1} = -sn_i r_i + cs_i h_{i+1} (r_0 = h_0) with outputs
// h'_i = cs_i r_i + sn_i h_{i+1}; the CTA evaluates it as a parallel prefix of the affine maps
// r -> a r + b (each thread composes a contiguous run, a warp scan and the warp totals give every
// run its starting r), so its FP64 work is a few dependent operations per thread instead of a
// chain of j on one thread.
__global__ void batch_givens_kernel(GivensState S, int j, const double* __restrict__ h1, const double* __restrict__ h2,
                                    const double* __restrict__ hn) {
  const int p = blockIdx.x;
  if (!S.active[p]) return;
  __shared__ double col[kMaxGmresCol + 1], cs[kMaxGmresCol], sn[kMaxGmresCol];
  __shared__ double wa[32], wb[32], rj, hnext;
  __shared__ int bad;
  double* colg = S.H + ((long long)p * S.restart + j) * S.ldh;
  double* csg = S.cs + (long long)p * S.restart;
  double* sng = S.sn + (long long)p * S.restart;
  double* g = S.g + (long long)p * S.ldh;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) col[i] = h1[(long long)i * S.K + p] + h2[(long long)i * S.K + p];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    cs[i] = csg[i];
    sn[i] = sng[i];
  }
  if (threadIdx.x == 0) {
    hnext = sqrt(fmax(0.0, hn[p]));
    bad = !isfinite(hnext);
    if (j == 0) rj = 0.0;
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) {
      S.err[0] = 1;
      S.active[p] = 0;
    }
    return;
  }
  // this thread's run [i0, i1) of the rotations, composed into r -> A r + B
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (j + blockDim.x - 1) / blockDim.x;
  const int i0 = min(j, tid * per), i1 = min(j, i0 + per);
  double A = 1.0, B = 0.0;
  for (int i = i0; i < i1; ++i) {
    const double a = -sn[i];
    B = fma(a, B, cs[i] * col[i + 1]);
    A *= a;
  }
  // inclusive scan over the warp's runs (a later run applies after an earlier one)
  for (int o = 1; o < 32; o <<= 1) {
    const double Ap = __shfl_up_sync(0xffffffffu, A, o), Bp = __shfl_up_sync(0xffffffffu, B, o);
    if (lane >= o) {
      B = fma(A, Bp, B);
      A *= Ap;
    }
  }
  if (lane == 31) {
    wa[warp] = A;
    wb[warp] = B;
  }
  __syncthreads();
  // the composition of every run before this thread's: the earlier warps', then the earlier lanes'
  double PA = 1.0, PB = 0.0;
  for (int q = 0; q < warp; ++q) {
    PB = fma(wa[q], PB, wb[q]);
    PA *= wa[q];
  }
  double EA = __shfl_up_sync(0xffffffffu, A, 1), EB = __shfl_up_sync(0xffffffffu, B, 1);
  if (lane == 0) {
    EA = 1.0;
    EB = 0.0;
  }
  double r = fma(EA, fma(PA, col[0], PB), EB);  // r at i0
  for (int i = i0; i < i1; ++i) {
    const double x = col[i + 1];
    colg[i] = fma(cs[i], r, sn[i] * x);
    r = fma(-sn[i], r, cs[i] * x);
  }
  if (i1 == j && i0 < i1) rj = r;
  if (j == 0 && tid == 0) rj = col[0];
  __syncthreads();
  if (tid == 0) {
    const double cj = rj, hx = hnext;
    const double den = hypot(cj, hx);
    const double c = den > 0 ? cj / den : 1.0, sj = den > 0 ? hx / den : 0.0;
    csg[j] = c;
    sng[j] = sj;
    colg[j] = den;
    colg[j + 1] = 0.0;
    g[j + 1] = -sj * g[j];
    g[j] = c * g[j];
    S.jused[p] = j + 1;
    S.iters[p] += 1;
    S.est[p] = fabs(g[j + 1]) / S.bn[p];
    S.scl[p] = hx > 0 ? 1.0 / hx : 0.0;
    if (S.est[p] <= S.tol[p] || hx == 0.0) S.active[p] = 0;
  }
}

// y = R^{-1} g per problem (back substitution over its own jused steps): coef[i K + p] = y_i,
// zero for jused <= i < jmax
__global__ void batch_backsolve_kernel(GivensState S, int jmax, double* __restrict__ coef) {
  const int p = blockIdx.x;
  const int J = S.jused[p];
  const double* H = S.H + (long long)p * S.restart * S.ldh;
  const double* g = S.g + (long long)p * S.ldh;
  __shared__ double t[kMaxGmresCol];
  // column-oriented back substitution: after y_i is known, every thread updates t[q] -= R[q][i] y_i
  for (int q = threadIdx.x; q < J; q += blockDim.x) t[q] = g[q];
  __syncthreads();
  for (int i = J - 1; i >= 0; --i) {
    const double d = H[(long long)i * S.ldh + i];
    const double yi = d != 0.0 ? t[i] / d : 0.0;
    __syncthreads();
    for (int q = threadIdx.x; q < i; q += blockDim.x) t[q] -= H[(long long)i * S.ldh + q] * yi;
    if (threadIdx.x == 0) coef[(long long)i * S.K + p] = yi;
    __syncthreads();
  }
  for (int i = J + threadIdx.x; i < jmax; i += blockDim.x) coef[(long long)i * S.K + p] = 0.0;
}

// ------------------------------------------------------------------ forces / torques
__global__ void ft_kernel(int N, const double* __restrict__ proxy64, const double* __restrict__ img64,
                          const int* __restrict__ img_off, const long long* __restrict__ unk_off,
                          const double* __restrict__ lam, double* __restrict__ F, double* __restrict__ Tq, int stride,
                          double sF, double sT) {
  const int k = blockIdx.x;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const double* l = lam + unk_off[k];
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const double* y = proxy64 + 4LL * j;
    double fx = l[3 * j], fy = l[3 * j + 1], fz = l[3 * j + 2];
    acc[0] += fx; acc[1] += fy; acc[2] += fz;
    acc[3] += y[1] * fz - y[2] * fy;
    acc[4] += y[2] * fx - y[0] * fz;
    acc[5] += y[0] * fy - y[1] * fx;
  }
  const int i0 = img_off[k], i1 = img_off[k + 1];
  for (int j = i0 + threadIdx.x; j < i1; j += blockDim.x) {
    const double* y = img64 + 4LL * j;
    const double* s = l + 3LL * N + 9LL * (j - i0);
    double fx = s[0], fy = s[1], fz = s[2];
    acc[0] += fx; acc[1] += fy; acc[2] += fz;
    acc[3] += s[3] + y[1] * fz - y[2] * fy;
    acc[4] += s[4] + y[2] * fx - y[0] * fz;
    acc[5] += s[5] + y[0] * fy - y[1] * fx;
  }
  __shared__ double red[6][32];
  for (int c = 0; c < 6; ++c) {
    double s = acc[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[c][threadIdx.x >> 5] = s;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[threadIdx.x][q];
    if (threadIdx.x < 3) F[(long long)stride * k + threadIdx.x] = sF * s;
    else Tq[(long long)stride * k + threadIdx.x - 3] = sT * s;
  }
}

// out[node] -= sqrt(w) (V_k + Omega_k x (x - c_k)) with U = (V_k, Omega_k) per sphere
__global__ void rigid_sub_kernel(int n, const int* __restrict__ owner, const double* __restrict__ pos64,
                                 const double* __restrict__ U, double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double* u = U + 6LL * owner[i];
    const double* r = pos64 + 4LL * i;
    const double sw = r[3];
    out[3LL * i] -= sw * (u[0] + u[4] * r[2] - u[5] * r[1]);
    out[3LL * i + 1] -= sw * (u[1] + u[5] * r[0] - u[3] * r[2]);
    out[3LL * i + 2] -= sw * (u[2] + u[3] * r[1] - u[4] * r[0]);
  }
}

struct Bg { double v[15]; };

__global__ void rhs_kernel(int n, const double* __restrict__ xabs, const int* __restrict__ owner,
                           const double* __restrict__ sqrtw, const double* __restrict__ cen,
                           const double* __restrict__ v, const double* __restrict__ om, Bg bg, double* __restrict__ wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int o = owner[i];
    double x0 = xabs[3 * i], x1 = xabs[3 * i + 1], x2 = xabs[3 * i + 2];
    double r0 = x0 - cen[3 * o], r1 = x1 - cen[3 * o + 1], r2 = x2 - cen[3 * o + 2];
    const double* w = om + 3 * o;
    double u0 = v[3 * o] + w[1] * r2 - w[2] * r1;
    double u1 = v[3 * o + 1] + w[2] * r0 - w[0] * r2;
    double u2 = v[3 * o + 2] + w[0] * r1 - w[1] * r0;
    // background u_inf = U + E x + Omega x x, subtracted (eq. bc)
    const double* E = bg.v + 3;
    const double* Om = bg.v + 12;
    u0 -= bg.v[0] + E[0] * x0 + E[1] * x1 + E[2] * x2 + Om[1] * x2 - Om[2] * x1;
    u1 -= bg.v[1] + E[3] * x0 + E[4] * x1 + E[5] * x2 + Om[2] * x0 - Om[0] * x2;
    u2 -= bg.v[2] + E[6] * x0 + E[7] * x1 + E[8] * x2 + Om[0] * x1 - Om[1] * x0;
    double s = sqrtw[i];
    wb[3 * i] = s * u0;
    wb[3 * i + 1] = s * u1;
    wb[3 * i + 2] = s * u2;
  }
}

// B[(3 s + c) lda + 3 i + r] = sqrt(w_i) K_type(x_i - y_s)[r][c]
__global__ void assemble_self_kernel(int m, int n_src, const double* __restrict__ xrel, const double* __restrict__ sqrtw,
                                     const double* __restrict__ yrel, const int* __restrict__ type, double scale,
                                     double* __restrict__ B, long long lda) {
  long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (id >= (long long)m * n_src) return;
  int i = (int)(id % m);
  int s = (int)(id / m);
  double r[3] = {xrel[3 * i] - yrel[3 * s], xrel[3 * i + 1] - yrel[3 * s + 1], xrel[3 * i + 2] - yrel[3 * s + 2]};
  double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  double ir = 1.0 / sqrt(r2);
  double ir3 = ir * ir * ir;
  double K[3][3];
  int ty = type[s];
  if (ty == 0) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) K[a][b] = scale * ((a == b ? ir : 0.0) + r[a] * r[b] * ir3);
  } else if (ty == 1) {
    double c = scale * ir3;
    K[0][0] = 0; K[0][1] = c * r[2]; K[0][2] = -c * r[1];
    K[1][0] = -c * r[2]; K[1][1] = 0; K[1][2] = c * r[0];
    K[2][0] = c * r[1]; K[2][1] = -c * r[0]; K[2][2] = 0;
  } else {
    double c = 1.0 / (4.0 * kPi);
    double ir5 = ir3 * ir * ir;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) K[a][b] = c * ((a == b ? -ir3 : 0.0) + 3.0 * r[a] * r[b] * ir5);
  }
  double w = sqrtw[i];
  for (int c = 0; c < 3; ++c)
    for (int rr = 0; rr < 3; ++rr) B[(3LL * s + c) * lda + 3LL * i + rr] = w * K[rr][c];
}

// Arithmetic-peak probe: 8 independent fused multiply-add chains per thread, 16 steps of each
// per loop trip, enough warps per SM to hide the FMA latency.  The result is stored only when it
// equals a value it never takes, so the chains cannot be removed.
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, T a, T b, T* __restrict__ sink) {
  T x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = T(threadIdx.x + q) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if constexpr (sizeof(T) == 4) x[q] = __fmaf_rn(x[q], a, b);
        else x[q] = __fma_rn(x[q], a, b);
      }
  }
  T s = T(0);
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  if (s == T(-1.25e30)) sink[0] = s;
}

thread_local long long t_launches = 0;

inline int grid_for(long long n, int threads, int cap = 152 * 16) {
  long long g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

long long launches_on_this_thread() { return t_launches; }
void note_launch() { ++t_launches; }

template <typename T>
void launch_pairs(const TargetSet& tg, const SourceSet& src, const T* lam_hat, const T* mu, T* out, double visc,
                  cudaStream_t st) {
  if (tg.n_tiles == 0) return;
  const int nt = tg.n_tiles1 > 0 ? pair_nodes_per_thread(tg.n_tiles) : 4;
  PairArgs<T> A = make_args<T>(tg, src, lam_hat, mu, out, visc, nt);
  ++t_launches;
  if (nt == 4) pairs_kernel<T, 4><<<tg.n_tiles, kPairThreads, 0, st>>>(A);
  else pairs_kernel<T, 1><<<tg.n_tiles1, kPairThreads, 0, st>>>(A);
}
template void launch_pairs<float>(const TargetSet&, const SourceSet&, const float*, const float*, float*, double, cudaStream_t);
template void launch_pairs<double>(const TargetSet&, const SourceSet&, const double*, const double*, double*, double, cudaStream_t);

int pair_split_parts(long long n_tiles1, long long min_sources, int max_parts) {
  if (n_tiles1 <= 0) return 1;
  long long s = kPairSplitTarget / n_tiles1;  // at most one wave of resident CTAs
  s = std::min<long long>(s, min_sources / kPairSplitMinSources);
  s = std::min<long long>(s, max_parts);
  return (int)std::max<long long>(s, 1);
}

// nodes per thread of a launch: the requested shape, else the rule (512-node tiles once they fill
// the GPU twice; 128-node tiles only when they exist)
static int shape_nt(const TargetSet& tg, const PairShape& shape) {
  if (tg.n_tiles1 == 0) return 4;
  if (shape.nt == 1 || shape.nt == 4) return shape.nt;
  return pair_nodes_per_thread(tg.n_tiles);
}

PairShape resolve_dw_shape(const TargetSet& tg, const SourceSet& src, PairShape shape, int max_parts) {
  PairShape r;
  r.nt = shape_nt(tg, shape);
  if (shape.parts > 0) r.parts = std::min(shape.parts, max_parts);
  else if (r.nt == 4) r.parts = 1;
  else r.parts = pair_split_parts(tg.n_tiles1, (long long)(src.P - 1) * src.N, max_parts);
  return r;
}

void launch_pairs_dw(const TargetSet& tg, const SourceSet& src, const double* lam_hat, const double* mu, double* out,
                     double visc, double* partial, int max_parts, cudaStream_t st, PairShape shape) {
  if (tg.n_tiles == 0) return;
  const PairShape r = resolve_dw_shape(tg, src, shape, max_parts);
  const int nt = r.nt;
  const int parts = partial ? r.parts : 1;
  PairArgs<double> A = make_args<double>(tg, src, lam_hat, mu, out, visc, nt);
  const long long n3 = 3LL * tg.n;
  ++t_launches;
  if (nt == 4) pairs_dw_kernel<4><<<tg.n_tiles * parts, kPairThreads, 0, st>>>(A, parts, partial, n3);
  else pairs_dw_kernel<1><<<tg.n_tiles1 * parts, kPairThreads, 0, st>>>(A, parts, partial, n3);
  if (parts > 1) {
    ++t_launches;
    pair_parts_reduce_kernel<<<grid_for(n3, 256), 256, 0, st>>>(n3, A.tgt, parts, partial, n3, mu, out);
  }
}

// resident CTAs of a pair kernel on the current device (SMs x CTAs per SM), looked up once per
// (device, kernel)
static double resident_ctas(const void* kernel) {
  static std::mutex mtx;
  static std::vector<std::pair<std::pair<int, const void*>, double>> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> g(mtx);
  for (const auto& e : cache)
    if (e.first.first == dev && e.first.second == kernel) return e.second;
  int per_sm = 0, sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kPairThreads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  cache.push_back({{dev, kernel}, (double)sms * per_sm});
  return cache.back().second;
}

// source parts per tile so that tiles x parts fill whole waves of the resident CTAs (ties: fewer)
int wave_parts(long long tiles, const void* kernel, int max_parts) {
  const double wave = resident_ctas(kernel);
  if (wave <= 0) return 1;
  int best = 1;
  double best_eff = 0;
  for (int p = 1; p <= max_parts; ++p) {
    const double w = (double)tiles * p / wave;
    const double eff = w / std::ceil(w);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = p;
    }
  }
  return best;
}

PairShape resolve_near_shape(const TargetSet& tg, PairShape shape, int max_parts) {
  PairShape r;
  r.nt = shape_nt(tg, shape);
  const long long tiles = r.nt == 4 ? tg.n_tiles : tg.n_tiles1;
  r.parts = shape.parts > 0 ? std::min(shape.parts, max_parts)
                            : wave_parts(tiles, r.nt == 4 ? (const void*)pairs_dw_near_kernel<4>
                                                          : (const void*)pairs_dw_near_kernel<1>, max_parts);
  return r;
}

void launch_pairs_dw_near(const TargetSet& tg, const SourceSet& src, const FarField& ff, const double* lam_hat,
                          const double* mu, double* out, double visc, double* partial, int max_parts, cudaStream_t st,
                          PairShape shape) {
  if (tg.n_tiles == 0) return;
  const PairShape r = resolve_near_shape(tg, shape, max_parts);
  const int nt = r.nt;
  PairArgs<double> A = make_args<double>(tg, src, lam_hat, mu, out, visc, nt);
  const long long tiles = nt == 4 ? tg.n_tiles : tg.n_tiles1;
  const int parts = partial ? r.parts : 1;
  const long long n3 = 3LL * tg.n;
  ++t_launches;
  if (nt == 4)
    pairs_dw_near_kernel<4><<<tiles * parts, kPairThreads, 0, st>>>(A, ff.near_off, ff.near_idx, parts, partial, n3);
  else
    pairs_dw_near_kernel<1><<<tiles * parts, kPairThreads, 0, st>>>(A, ff.near_off, ff.near_idx, parts, partial, n3);
  if (parts > 1) {
    ++t_launches;
    parts_add_kernel<<<grid_for(n3, 256), 256, 0, st>>>(n3, A.tgt, parts, partial, n3, mu, out);
  }
}

PairShape resolve_far_shape(const TargetSet& tg, PairShape shape, int max_parts) {
  PairShape r;
  r.nt = shape_nt(tg, shape);
  // 4 nodes per thread run the packed-FP32 kernel unless the scalar one is asked for
  r.packed = r.nt == 4 && shape.packed >= 0 ? 1 : 0;
  const long long tiles = r.nt == 4 ? tg.n_tiles : tg.n_tiles1;
  const void* kern = r.nt == 4 ? (r.packed ? (const void*)pairs_far2_kernel : (const void*)pairs_far_kernel<4>)
                               : (const void*)pairs_far_kernel<1>;
  r.parts = shape.parts > 0 ? std::min(shape.parts, max_parts) : wave_parts(tiles, kern, max_parts);
  return r;
}

void launch_pairs_far(const TargetSet& tg, const SourceSet& src, const FarField& ff, double* out, double visc,
                      double* partial, int max_parts, cudaStream_t st, PairShape shape) {
  if (tg.n_tiles == 0 || ff.n_eq == 0) return;
  const PairShape r = resolve_far_shape(tg, shape, max_parts);
  const int nt = r.nt;
  FarArgs A;
  A.tgt = tg.pos32;
  A.tgt64 = tg.pos64;
  A.tile_sphere = nt == 4 ? tg.tile_sphere : tg.tile1_sphere;
  A.tile_start = nt == 4 ? tg.tile_start : tg.tile1_start;
  A.tile_count = nt == 4 ? tg.tile_count : tg.tile1_count;
  A.eq = ff.eq32;
  A.n_eq = ff.n_eq;
  A.P = src.P;
  A.excl_off = ff.excl_off;
  A.excl_idx = ff.excl_idx;
  A.cen_hi = src.cen_hi;
  A.cen_lo = src.cen_lo;
  A.q = ff.q;
  A.out = out;
  A.scale = (float)(1.0 / (8.0 * kPi * visc));
  const long long tiles = nt == 4 ? tg.n_tiles : tg.n_tiles1;
  const int parts = partial ? r.parts : 1;
  const long long n3 = 3LL * tg.n;
  ++t_launches;
  if (nt == 4 && r.packed) pairs_far2_kernel<<<tiles * parts, kPairThreads, 0, st>>>(A, parts, partial, n3);
  else if (nt == 4) pairs_far_kernel<4><<<tiles * parts, kPairThreads, 0, st>>>(A, parts, partial, n3);
  else pairs_far_kernel<1><<<tiles * parts, kPairThreads, 0, st>>>(A, parts, partial, n3);
  if (parts > 1) {
    ++t_launches;
    parts_add_kernel<<<grid_for(n3, 256), 256, 0, st>>>(n3, reinterpret_cast<const D4*>(tg.pos64), parts, partial, n3,
                                                        nullptr, out);
  }
}

size_t pair_args64_bytes() { return sizeof(PairArgs<double>); }

void fill_pair_args64(void* host_dst, const TargetSet& tg, const SourceSet& src, const double* lam_hat,
                      const double* mu, double* out, double visc, int nodes_per_thread) {
  PairArgs<double> A = make_args<double>(tg, src, lam_hat, mu, out, visc, nodes_per_thread);
  std::memcpy(host_dst, &A, sizeof(A));
}

void launch_pairs_batch64(bool double_float, const void* d_args, const int2* d_work, int n_work, const int* d_active,
                          int nodes_per_thread, const double* lam, const double* mu, double* out,
                          const long long* d_uoff, const long long* d_voff, int parts, double* partial,
                          long long pstride, const SegTable& seg, cudaStream_t st, const long long* d_nlen,
                          bool skip_reduce, unsigned* d_counter) {
  if (n_work == 0) return;
  const PairArgs<double>* args = static_cast<const PairArgs<double>*>(d_args);
  BatchVecs bv{lam, mu, out, d_uoff, d_voff, partial, pstride, d_nlen, d_counter};
  if (d_counter) skip_reduce = true;  // the last CTA of each item adds the parts
  ++t_launches;
  if (double_float) {
    if (nodes_per_thread == 4) {
      pairs_dw_batch_kernel<4><<<n_work, kPairThreads, 0, st>>>(args, d_work, d_active, bv, 1);
    } else {
      if (!partial) parts = 1;
      pairs_dw_batch_kernel<1><<<n_work * parts, kPairThreads, 0, st>>>(args, d_work, d_active, bv, parts);
      if (parts > 1 && !skip_reduce) {
        ++t_launches;
        if (seg_ctas(seg) > 0)
          pair_parts_reduce_batch_kernel<<<dim3(seg_ctas(seg), (seg.chunk + 127) / 128), 128, 0, st>>>(seg, args, bv, parts);
      }
    }
  } else {
    if (nodes_per_thread == 4) pairs_batch_kernel<double, 4><<<n_work, kPairThreads, 0, st>>>(args, d_work, d_active, bv);
    else pairs_batch_kernel<double, 1><<<n_work, kPairThreads, 0, st>>>(args, d_work, d_active, bv);
  }
}

void launch_pairs_multi64(const void* d_args1, const int4* d_work, int n_work, const int* d_rhs, const int* d_active,
                          const double* lam, const double* mu, double* out, const long long* d_uoff,
                          const long long* d_voff, int parts, double* partial, long long pstride,
                          const long long* d_nlen, cudaStream_t st, unsigned* d_counter) {
  if (n_work == 0) return;
  if (!partial) parts = 1;
  const PairArgs<double>* args = static_cast<const PairArgs<double>*>(d_args1);
  BatchVecs bv{lam, mu, out, d_uoff, d_voff, partial, pstride, d_nlen, d_counter};
  ++t_launches;
  pairs_dw_multi_kernel<kPairRhs><<<n_work * parts, kPairThreads, 0, st>>>(args, d_work, d_rhs, d_active, bv, parts);
}

void launch_pair_parts_reduce_batch(const void* d_args1, const SegTable& seg, const double* lam, const double* mu,
                                    double* out, const long long* d_uoff, const long long* d_voff, int parts,
                                    double* partial, long long pstride, const long long* d_nlen, cudaStream_t st) {
  if (parts <= 1 || seg_ctas(seg) == 0) return;
  const PairArgs<double>* args = static_cast<const PairArgs<double>*>(d_args1);
  BatchVecs bv{lam, mu, out, d_uoff, d_voff, partial, pstride, d_nlen, nullptr};
  ++t_launches;
  pair_parts_reduce_batch_kernel<<<dim3(seg_ctas(seg), (seg.chunk + 127) / 128), 128, 0, st>>>(seg, args, bv, parts);
}

void launch_seg_dots(const SegTable& t, int nvec, const double* V, long long ldv, const double* w, double* partial,
                     double* h, cudaStream_t st) {
  if (seg_ctas(t) == 0 || nvec == 0) return;
  ++t_launches;
  seg_dots_kernel<<<dim3(seg_ctas(t), (nvec + kSegDotVecs - 1) / kSegDotVecs), kSegThreads, 0, st>>>(t, nvec, V, ldv,
                                                                                                     w, partial, h);
  if (!t.counter) {
    ++t_launches;
    seg_reduce_kernel<<<t.K, 128, 0, st>>>(t, nvec, partial, h);
  }
}
void launch_seg_update(const SegTable& t, int nvec, const double* V, long long ldv, const double* coef, double sign,
                       double* w, cudaStream_t st) {
  if (seg_ctas(t) == 0 || nvec == 0) return;
  ++t_launches;
  seg_update_kernel<<<dim3(seg_ctas(t), (t.chunk + kSegUpdSub - 1) / kSegUpdSub), kSegUpdSub * kSegUpdGroups, 0, st>>>(
      t, nvec, V, ldv, coef, sign, w);
}
void launch_seg_scale_split(const SegTable& t, const double* s, const double* in, double* out, float2* x2,
                            cudaStream_t st) {
  if (seg_ctas(t) == 0) return;
  ++t_launches;
  seg_scale_split_kernel<<<seg_ctas(t), kSegThreads, 0, st>>>(t, s, in, out, x2);
}
void launch_seg_scale(const SegTable& t, const double* s, const double* in, double* out, cudaStream_t st) {
  if (seg_ctas(t) == 0) return;
  ++t_launches;
  seg_scale_kernel<<<seg_ctas(t), kSegThreads, 0, st>>>(t, s, in, out);
}
void launch_batch_givens(const GivensState& S, int j, const double* h1, const double* h2, const double* hn,
                         cudaStream_t st) {
  ++t_launches;
  batch_givens_kernel<<<S.K, 128, 0, st>>>(S, j, h1, h2, hn);
}
void launch_batch_backsolve(const GivensState& S, int jmax, double* coef, cudaStream_t st) {
  ++t_launches;
  batch_backsolve_kernel<<<S.K, 128, 0, st>>>(S, jmax, coef);
}
void launch_axpy64(long long n, double a, const double* x, double* y, cudaStream_t st) {
  ++t_launches;
  axpy64_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, a, x, y);
}

template <typename T>
void launch_gemv(const GemvBatch<T>& b, const T* x, T* y, cudaStream_t st) {
  if (b.n_jobs == 0 || b.max_rows == 0) return;
  const int rows_per_cta = (kGemvThreads / 32) * kGemvRowsPerWarp;
  const int jobs = b.job_list ? b.n_list : b.n_jobs;
  if (jobs == 0) return;
  dim3 grid(jobs, (b.max_rows + rows_per_cta - 1) / rows_per_cta);
  ++t_launches;
  gemv_kernel<T><<<grid, kGemvThreads, 0, st>>>(b, x, y);
}
template void launch_gemv<float>(const GemvBatch<float>&, const float*, float*, cudaStream_t);

void launch_gemv_dw(const GemvBatch<double>& b, const float2* x, float2* y_dw, double* y64, cudaStream_t st) {
  if (b.n_jobs == 0 || b.max_rows == 0) return;
  const int rows_per_cta = (kGemvThreads / 32) * kGemvRowsPerWarp;
  const int jobs = b.job_list ? b.n_list : b.n_jobs;
  if (jobs == 0) return;
  dim3 grid(jobs, (b.max_rows + rows_per_cta - 1) / rows_per_cta);
  ++t_launches;
  if (y_dw) gemv_dw_kernel<false><<<grid, kGemvThreads, 0, st>>>(b, x, y_dw, nullptr);
  else gemv_dw_kernel<true><<<grid, kGemvThreads, 0, st>>>(b, x, nullptr, y64);
}

void launch_gemv_f32_dw(const GemvBatch<float>& b, const float2* x, float2* y_dw, cudaStream_t st) {
  if (b.n_jobs == 0 || b.max_rows == 0) return;
  const int rows_per_cta = (kGemvThreads / 32) * kGemvRowsPerWarp;
  const int jobs = b.job_list ? b.n_list : b.n_jobs;
  if (jobs == 0) return;
  dim3 grid(jobs, (b.max_rows + rows_per_cta - 1) / rows_per_cta);
  ++t_launches;
  gemv_f32dw_kernel<<<grid, kGemvThreads, 0, st>>>(b, x, y_dw);
}

void launch_split_dw(long long n, const double* in, float2* out, cudaStream_t st) {
  ++t_launches;
  split_dw_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, in, out);
}
template void launch_gemv<double>(const GemvBatch<double>&, const double*, double*, cudaStream_t);

template <typename T>
void launch_multidot(int n, int nvec, const T* V, long long ldv, const T* w, double* partial, int nblk, cudaStream_t st) {
  dim3 grid(nblk, nvec);
  ++t_launches;
  multidot_kernel<T><<<grid, kRedThreads, 0, st>>>(n, V, ldv, w, partial, nblk);
}
template void launch_multidot<float>(int, int, const float*, long long, const float*, double*, int, cudaStream_t);
template void launch_multidot<double>(int, int, const double*, long long, const double*, double*, int, cudaStream_t);

void launch_reduce_partials(int nvec, int nblk, const double* partial, double* h, cudaStream_t st) {
  ++t_launches;
  reduce_partials_kernel<<<nvec, 256, 0, st>>>(nvec, nblk, partial, h);
}

template <typename T>
void launch_update(int n, int nvec, const T* V, long long ldv, const double* h, double sign, T* w, cudaStream_t st) {
  ++t_launches;
  update_kernel<T><<<grid_for(n, 256), 256, 0, st>>>(n, nvec, V, ldv, h, sign, w);
}
template void launch_update<float>(int, int, const float*, long long, const double*, double, float*, cudaStream_t);
template void launch_update<double>(int, int, const double*, long long, const double*, double, double*, cudaStream_t);

template <typename T>
void launch_scale_copy(int n, const T* w, double s, T* out, cudaStream_t st) {
  ++t_launches;
  scale_copy_kernel<T><<<grid_for(n, 256), 256, 0, st>>>(n, w, s, out);
}
template void launch_scale_copy<float>(int, const float*, double, float*, cudaStream_t);
template void launch_scale_copy<double>(int, const double*, double, double*, cudaStream_t);

template <typename Tin, typename Tout>
void launch_convert(long long n, const Tin* in, double s, Tout* out, cudaStream_t st) {
  ++t_launches;
  convert_kernel<Tin, Tout><<<grid_for(n, 256), 256, 0, st>>>(n, in, s, out);
}
template void launch_convert<double, float>(long long, const double*, double, float*, cudaStream_t);
template void launch_convert<float, double>(long long, const float*, double, double*, cudaStream_t);
template void launch_convert<double, double>(long long, const double*, double, double*, cudaStream_t);

void launch_axpy_mixed(int n, double a, const float* x, double* y, cudaStream_t st) {
  ++t_launches;
  axpy_mixed_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, a, x, y);
}
void launch_sub(int n, const double* a, const double* b, double* out, cudaStream_t st) {
  ++t_launches;
  sub_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, a, b, out);
}

void launch_forces_torques(const SourceSet& src, const double* lam, double* F, double* T, cudaStream_t st) {
  ++t_launches;
  ft_kernel<<<src.P, 256, 0, st>>>(src.N, src.proxy64, src.img64, src.img_off, src.unk_off, lam, F, T, 3, 1.0, 1.0);
}
void launch_forces_torques_scaled(const SourceSet& src, const double* lam, double* F, double* T, int stride, double sF,
                                  double sT, cudaStream_t st) {
  ++t_launches;
  ft_kernel<<<src.P, 256, 0, st>>>(src.N, src.proxy64, src.img64, src.img_off, src.unk_off, lam, F, T, stride, sF, sT);
}
void launch_rigid_sub(int n, const int* owner, const double* pos64, const double* U, double* out, cudaStream_t st) {
  ++t_launches;
  rigid_sub_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, owner, pos64, U, out);
}

void launch_rhs(int n, const double* colloc_abs, const int* owner, const double* sqrtw, const double* cen,
                const double* v, const double* om, const double* bg, double* wb, cudaStream_t st) {
  Bg b;
  for (int i = 0; i < 15; ++i) b.v[i] = bg[i];
  ++t_launches;
  rhs_kernel<<<grid_for(n, 256), 256, 0, st>>>(n, colloc_abs, owner, sqrtw, cen, v, om, b, wb);
}

double launch_fma_probe(int which, int blocks, int iters, void* sink, cudaStream_t st) {
  ++t_launches;
  if (which == 0) fma_probe_kernel<float><<<blocks, 256, 0, st>>>(iters, 0.9999f, 1e-4f, static_cast<float*>(sink));
  else fma_probe_kernel<double><<<blocks, 256, 0, st>>>(iters, 0.9999, 1e-4, static_cast<double*>(sink));
  return 2.0 * 8.0 * 16.0 * (double)iters * (double)blocks * 256.0;  // flops
}

void launch_assemble_block(int m, int n_src, const double* xrel, const double* sqrtw, const double* yrel,
                           const int* type, double visc, double* B, long long lda, cudaStream_t st) {
  long long tot = (long long)m * n_src;
  int threads = 256;
  long long blocks = (tot + threads - 1) / threads;
  if (blocks == 0) return;
  ++t_launches;
  assemble_self_kernel<<<(unsigned)blocks, threads, 0, st>>>(m, n_src, xrel, sqrtw, yrel, type, 1.0 / (8.0 * kPi * visc),
                                                             B, lda);
}

void launch_assemble_self(const HostDisc& hd, int k, const double* d_colloc_rel, const double* d_sqrtw,
                          const double* d_src_rel, const int* d_src_type, int n_src, double* B, int lda,
                          cudaStream_t st) {
  int m = hd.colloc_off[k + 1] - hd.colloc_off[k];
  long long tot = (long long)m * n_src;
  int threads = 256;
  long long blocks = (tot + threads - 1) / threads;
  ++t_launches;
  assemble_self_kernel<<<(unsigned)blocks, threads, 0, st>>>(m, n_src, d_colloc_rel, d_sqrtw, d_src_rel, d_src_type,
                                                             1.0 / (8.0 * kPi * hd.prm.visc), B, lda);
}

}  // namespace mfs
