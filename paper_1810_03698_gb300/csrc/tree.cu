// Treecode matrix-vector product (Sec. "The treecode algorithm").
//
// Sources are the Gauss nodes, targets the collocation points; both live in the
// octree over the Morton-ordered panels.  For a target batch (a leaf) and a cell
// C with radius R_C, the cell is accepted (far field) when
//     R_C < theta * (|c_T - c_C| - R_T),
// i.e. the paper's acceptance criterion theta > R_b / R_tb holds for every target
// of the batch; otherwise C is opened, and leaves that are never accepted are
// summed directly (near field).
//
// Far field (Cartesian Taylor expansion about the cell centre c, order P):
// with Delta = x - c and h = y - c,
//     G(x - y) = sum_{|k| <= P} a_k(Delta) h^k,   a_k = (1/k!) d^k/dh^k G(Delta - h) at h = 0,
// so  V = sum_k a_k M_k   with M_k = sum_s m_s h_s^k             (single layer),
//     K = sum_k a_k D_k   with D_k = sum_s sum_j k_j d_sj h_s^(k - e_j)  (double layer:
//         the moments of the dipole layer, since d . grad_y G = d . grad_h of the series).
// Coefficients by recurrence in |k| = n, written for f(h) = e^{-kappa r}/r, r = |Delta - h|
// (kappa = 0 gives Laplace).  From r^2 grad f = (Delta - h)(f + kappa e^{-kappa r}) and
// grad e^{-kappa r} = kappa (Delta - h) f one gets, with b_k the coefficients of e^{-kappa r},
//     n |Delta|^2 a_k = (2n - 1) sum_j Delta_j a_{k-e_j} - (n - 1) sum_j a_{k-2e_j}
//                       + kappa sum_j (Delta_j b_{k-e_j} - b_{k-2e_j}),
//     n b_k           = kappa sum_j (Delta_j a_{k-e_j} - a_{k-2e_j}),
// a_0 = e^{-kappa|Delta|}/|Delta|, b_0 = e^{-kappa|Delta|} (terms with a negative index vanish).
// Moments of a parent follow from its children's by the exact shift
//     M_k(c_p) = sum_{l <= k} prod_i C(k_i, l_i) (c_c - c_p)_i^(k_i - l_i) M_l(c_c)
// (and the same for D_k).
//
// Precision: the FP32 form takes every coordinate difference relative to a
// nearby centre subtracted in FP64 (target-leaf centre for the near field,
// Delta = (x - c_T) + (c_T - c_C) for the far field), keeps per-cell and per-tile
// sums in FP32 and per-target sums in FP64.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace bp {

namespace {

constexpr int TB = 128;      // threads per block of the moment kernels
constexpr int TBT = 128;     // targets per block of the near/far kernels (up to four warps of one
                             // leaf); warps with no target skip the arithmetic and only help
                             // stage shared data, so only the last warp of a leaf has idle lanes
constexpr int MAXP = 6;      // highest Taylor order compiled

// ---------------------------------------------------------------- multi-index tables
template <int P>
struct MI {
  static constexpr int NC = (P + 1) * (P + 2) * (P + 3) / 6;
  int k[NC][3];
  int ord[NC];
  int m1[NC][3];  // index of k - e_j, or -1
  int m2[NC][3];  // index of k - 2 e_j, or -1
  int idx[P + 1][P + 1][P + 1];
  constexpr MI() : k{}, ord{}, m1{}, m2{}, idx{} {
    int t = 0;
    for (int a = 0; a <= P; ++a)
      for (int b = 0; b <= P; ++b)
        for (int c = 0; c <= P; ++c) idx[a][b][c] = -1;
    for (int n = 0; n <= P; ++n)
      for (int a = n; a >= 0; --a)
        for (int b = n - a; b >= 0; --b) {
          k[t][0] = a;
          k[t][1] = b;
          k[t][2] = n - a - b;
          ord[t] = n;
          idx[a][b][n - a - b] = t;
          ++t;
        }
    for (int u = 0; u < NC; ++u)
      for (int j = 0; j < 3; ++j) {
        int q[3] = {k[u][0], k[u][1], k[u][2]};
        m1[u][j] = -1;
        m2[u][j] = -1;
        if (q[j] >= 1) {
          q[j] -= 1;
          m1[u][j] = idx[q[0]][q[1]][q[2]];
          q[j] += 1;
        }
        if (q[j] >= 2) {
          q[j] -= 2;
          m2[u][j] = idx[q[0]][q[1]][q[2]];
          q[j] += 2;
        }
      }
  }
};

__host__ __device__ constexpr int ncoef(int P) { return (P + 1) * (P + 2) * (P + 3) / 6; }

// constant-memory copies for kernels that index the tables at run time
template <int P>
__constant__ MI<P> c_mi{};

struct Binom {
  int b[MAXP + 1][MAXP + 1];
  constexpr Binom() : b{} {
    for (int a = 0; a <= MAXP; ++a) {
      b[a][0] = 1;
      for (int q = 1; q <= a; ++q) b[a][q] = b[a - 1][q - 1] + (q <= a - 1 ? b[a - 1][q] : 0);
    }
  }
};
__constant__ Binom c_binom{};

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float exp2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float inv_sqrt(float x) { return rsqrt_approx(x); }
__device__ __forceinline__ double inv_sqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float exp_neg(float kr) { return exp2_approx(-1.4426950408889634f * kr); }
__device__ __forceinline__ double exp_neg(double kr) { return exp(-kr); }

template <typename R4>
struct Vec4;
template <>
struct Vec4<float> {
  typedef float4 T;
};
template <>
struct Vec4<double> {
  typedef double4 T;
};

// ---------------------------------------------------------------- cell geometry
// centre = midpoint of the bounding box of the cell's Gauss nodes; radius = max distance to them
__global__ void cell_geometry_kernel(const int* __restrict__ begin, const int* __restrict__ end, int K,
                                     const double4* __restrict__ src64, double4* __restrict__ center) {
  __shared__ double sh[6][256];
  const int cidx = blockIdx.x;
  const int s0 = begin[cidx] * K, s1 = end[cidx] * K;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int j = s0 + threadIdx.x; j < s1; j += 256) {
    double4 y = src64[j];
    lo[0] = fmin(lo[0], y.x); hi[0] = fmax(hi[0], y.x);
    lo[1] = fmin(lo[1], y.y); hi[1] = fmax(hi[1], y.y);
    lo[2] = fmin(lo[2], y.z); hi[2] = fmax(hi[2], y.z);
  }
  for (int d = 0; d < 3; ++d) {
    sh[d][threadIdx.x] = lo[d];
    sh[3 + d][threadIdx.x] = hi[d];
  }
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int d = 0; d < 3; ++d) {
        sh[d][threadIdx.x] = fmin(sh[d][threadIdx.x], sh[d][threadIdx.x + s]);
        sh[3 + d][threadIdx.x] = fmax(sh[3 + d][threadIdx.x], sh[3 + d][threadIdx.x + s]);
      }
    __syncthreads();
  }
  const double cx = 0.5 * (sh[0][0] + sh[3][0]), cy = 0.5 * (sh[1][0] + sh[4][0]), cz = 0.5 * (sh[2][0] + sh[5][0]);
  __syncthreads();
  double r2 = 0.0;
  for (int j = s0 + threadIdx.x; j < s1; j += 256) {
    double4 y = src64[j];
    double dx = y.x - cx, dy = y.y - cy, dz = y.z - cz;
    r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
  }
  sh[0][threadIdx.x] = r2;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[0][threadIdx.x] = fmax(sh[0][threadIdx.x], sh[0][threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) center[cidx] = make_double4(cx, cy, cz, sqrt(sh[0][0]));
}

// FP32 position of every Gauss node relative to the centre of its leaf (FP64 subtraction)
__global__ void src_rel_kernel(const int* __restrict__ leaf_cell, int nleaf, const int* __restrict__ begin,
                               const int* __restrict__ end, const double4* __restrict__ center, int K,
                               const double4* __restrict__ src64, float4* __restrict__ rel) {
  const int l = blockIdx.x;
  if (l >= nleaf) return;
  const int cl = leaf_cell[l];
  const double4 c = center[cl];
  for (int j = begin[cl] * K + threadIdx.x; j < end[cl] * K; j += blockDim.x) {
    const double4 y = src64[j];
    rel[j] = make_float4((float)(y.x - c.x), (float)(y.y - c.y), (float)(y.z - c.z), 0.f);
  }
}

// ---------------------------------------------------------------- moments
// Leaf moments from the sources: one block per leaf, thread o owns moments o, o + TB, ...
template <int P, typename Real>
__global__ void __launch_bounds__(TB) leaf_moments_kernel(const int* __restrict__ leaf_cell,
                                                          const int* __restrict__ begin, const int* __restrict__ end,
                                                          const double4* __restrict__ center, int K,
                                                          const double4* __restrict__ src64,
                                                          const typename Vec4<Real>::T* __restrict__ str,
                                                          const int* __restrict__ active,
                                                          const int* __restrict__ leaf_sys, Real* __restrict__ mom) {
  const MI<P>& mi = c_mi<P>;
  constexpr int NC = MI<P>::NC;
  __shared__ Real pw[TB][3][P + 1];
  __shared__ Real sd[TB][4];
  if (active && !active[leaf_sys[blockIdx.x]]) return;  // system not being solved
  const int cidx = leaf_cell[blockIdx.x];
  const double4 c = center[cidx];
  const int s0 = begin[cidx] * K, s1 = end[cidx] * K;
  Real acc[(2 * NC + TB - 1) / TB];
  for (int u = 0; u < (2 * NC + TB - 1) / TB; ++u) acc[u] = 0;
  for (int t0 = s0; t0 < s1; t0 += TB) {
    int j = t0 + threadIdx.x;
    if (j < s1) {
      double4 y = src64[j];
      Real h[3] = {(Real)(y.x - c.x), (Real)(y.y - c.y), (Real)(y.z - c.z)};
      for (int d = 0; d < 3; ++d) {
        Real p = 1;
        for (int e = 0; e <= P; ++e) {
          pw[threadIdx.x][d][e] = p;
          p *= h[d];
        }
      }
      auto s = str[j];
      sd[threadIdx.x][0] = s.x;
      sd[threadIdx.x][1] = s.y;
      sd[threadIdx.x][2] = s.z;
      sd[threadIdx.x][3] = s.w;
    }
    __syncthreads();
    const int lim = min(TB, s1 - t0);
    for (int u = 0; u < (2 * NC + TB - 1) / TB; ++u) {
      const int o = threadIdx.x + u * TB;
      if (o >= 2 * NC) break;
      const bool dbl = o >= NC;
      const int t = dbl ? o - NC : o;
      const int kx = mi.k[t][0], ky = mi.k[t][1], kz = mi.k[t][2];
      Real a = 0;
      for (int q = 0; q < lim; ++q) {
        if (!dbl) {
          a += sd[q][0] * pw[q][0][kx] * pw[q][1][ky] * pw[q][2][kz];
        } else {
          Real v = 0;
          if (kx) v += (Real)kx * sd[q][1] * pw[q][0][kx - 1] * pw[q][1][ky] * pw[q][2][kz];
          if (ky) v += (Real)ky * sd[q][2] * pw[q][0][kx] * pw[q][1][ky - 1] * pw[q][2][kz];
          if (kz) v += (Real)kz * sd[q][3] * pw[q][0][kx] * pw[q][1][ky] * pw[q][2][kz - 1];
          a += v;
        }
      }
      acc[u] += a;
    }
    __syncthreads();
  }
  for (int u = 0; u < (2 * NC + TB - 1) / TB; ++u) {
    const int o = threadIdx.x + u * TB;
    if (o < 2 * NC) mom[(size_t)cidx * 2 * NC + o] = acc[u];
  }
}

// Parent moments by shifting the children's: one block per parent cell of one depth.
template <int P, typename Real>
__global__ void __launch_bounds__(TB) m2m_kernel(int first_cell, const int* __restrict__ child0,
                                                 const int* __restrict__ nchild, const double4* __restrict__ center,
                                                 Real* __restrict__ mom) {
  const MI<P>& mi = c_mi<P>;
  constexpr int NC = MI<P>::NC;
  __shared__ Real dp[8][3][P + 1];
  __shared__ Real cm[8][2 * NC];
  const int pc = first_cell + blockIdx.x;
  const int nch = nchild[pc];
  if (nch == 0) return;  // leaf (uniform across the block)
  const int c0 = child0[pc];
  const double4 cp = center[pc];
  if (threadIdx.x < nch) {
    double4 cc = center[c0 + threadIdx.x];
    Real dl[3] = {(Real)(cc.x - cp.x), (Real)(cc.y - cp.y), (Real)(cc.z - cp.z)};
    for (int d = 0; d < 3; ++d) {
      Real p = 1;
      for (int e = 0; e <= P; ++e) {
        dp[threadIdx.x][d][e] = p;
        p *= dl[d];
      }
    }
  }
  for (int q = threadIdx.x; q < nch * 2 * NC; q += TB) cm[q / (2 * NC)][q % (2 * NC)] = mom[(size_t)(c0 + q / (2 * NC)) * 2 * NC + q % (2 * NC)];
  __syncthreads();
  const auto& binom = c_binom.b;
  for (int o = threadIdx.x; o < 2 * NC; o += TB) {
    const int t = o < NC ? o : o - NC;
    const int off = o < NC ? 0 : NC;
    const int kx = mi.k[t][0], ky = mi.k[t][1], kz = mi.k[t][2];
    Real a = 0;
    for (int ch = 0; ch < nch; ++ch)
      for (int lx = 0; lx <= kx; ++lx)
        for (int ly = 0; ly <= ky; ++ly)
          for (int lz = 0; lz <= kz; ++lz) {
            const int l = mi.idx[lx][ly][lz];
            a += (Real)(binom[kx][lx] * binom[ky][ly] * binom[kz][lz]) * dp[ch][0][kx - lx] * dp[ch][1][ky - ly] *
                 dp[ch][2][kz - lz] * cm[ch][off + l];
          }
    mom[(size_t)pc * 2 * NC + o] = a;
  }
}

// ---------------------------------------------------------------- far field
// One (target, cell) interaction of one kernel: the Laplace coefficients a_k, or the
// Yukawa a_k with their companions b_k, each dotted with the cell's single-layer (M)
// and double-layer (Dm) moments.  Fully unrolled for a compile-time order, so every
// table index is a constant; the per-order factors (2n-1)/(n|Delta|^2),
// (n-1)/(n|Delta|^2), kappa/(n|Delta|^2) and kappa/n are formed once per order.
// The two kernels run as separate launches so each body stays small.
template <int P, typename Real>
__device__ __forceinline__ void far_eval_laplace(const Real D[3], const Real* __restrict__ M,
                                                 const Real* __restrict__ Dm, Real& v, Real& k) {
  constexpr MI<P> mi{};
  constexpr int NC = MI<P>::NC;
  const Real r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
  const Real rinv = inv_sqrt(r2);
  const Real ir2 = rinv * rinv;
  Real q1[P + 1], q2[P + 1];
#pragma unroll
  for (int n = 1; n <= P; ++n) {
    q1[n] = ir2 * (Real)((2.0 * n - 1.0) / n);
    q2[n] = ir2 * (Real)((n - 1.0) / n);
  }
  Real a[NC];
  a[0] = rinv;
  Real sV = a[0] * M[0], sK = a[0] * Dm[0];
#pragma unroll
  for (int t = 1; t < NC; ++t) {
    const int n = mi.ord[t];
    Real s1 = 0, s2 = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (mi.m1[t][j] >= 0) s1 += D[j] * a[mi.m1[t][j]];
      if (mi.m2[t][j] >= 0) s2 += a[mi.m2[t][j]];
    }
    a[t] = q1[n] * s1 - q2[n] * s2;
    sV += a[t] * M[t];
    sK += a[t] * Dm[t];
  }
  v += sV;
  k += sK;
}

template <int P, typename Real>
__device__ __forceinline__ void far_eval_yukawa(const Real D[3], const Real* __restrict__ M,
                                                const Real* __restrict__ Dm, Real kappa, Real& v, Real& k) {
  constexpr MI<P> mi{};
  constexpr int NC = MI<P>::NC;
  const Real r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
  const Real rinv = inv_sqrt(r2);
  const Real ir2 = rinv * rinv;
  Real q1[P + 1], q2[P + 1], q3[P + 1], kn[P + 1];
#pragma unroll
  for (int n = 1; n <= P; ++n) {
    q1[n] = ir2 * (Real)((2.0 * n - 1.0) / n);
    q2[n] = ir2 * (Real)((n - 1.0) / n);
    kn[n] = kappa * (Real)(1.0 / n);
    q3[n] = kn[n] * ir2;
  }
  const Real e = exp_neg(kappa * (r2 * rinv));
  Real A[NC], Bc[NC];
  A[0] = e * rinv;
  Bc[0] = e;
  Real sV = A[0] * M[0], sK = A[0] * Dm[0];
#pragma unroll
  for (int t = 1; t < NC; ++t) {
    const int n = mi.ord[t];
    Real s1a = 0, s2a = 0, s1b = 0, s2b = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (mi.m1[t][j] >= 0) {
        s1a += D[j] * A[mi.m1[t][j]];
        s1b += D[j] * Bc[mi.m1[t][j]];
      }
      if (mi.m2[t][j] >= 0) {
        s2a += A[mi.m2[t][j]];
        s2b += Bc[mi.m2[t][j]];
      }
    }
    Bc[t] = kn[n] * (s1a - s2a);
    A[t] = q1[n] * s1a - q2[n] * s2a + q3[n] * (s1b - s2b);
    sV += A[t] * M[t];
    sK += A[t] * Dm[t];
  }
  v += sV;
  k += sK;
}

constexpr int FCH = 8;  // far cells staged in shared memory per pass

// One block per target block (<= 128 targets of one leaf); loops over the leaf's far
// cells.  YUK = 0 evaluates the Laplace kernel into rows (V_L, K_L), YUK = 1 the
// Yukawa kernel into rows (V_Y, K_Y) of `out` ([4][n]).
template <int P, typename Real, int YUK>
__global__ void __launch_bounds__(TBT) far_kernel(const int4* __restrict__ blk, const double4* __restrict__ tgt64,
                                                 const int* __restrict__ leaf_cell, const double4* __restrict__ center,
                                                 const int* __restrict__ far_ptr, const int* __restrict__ far_list,
                                                 const Real* __restrict__ mom, Real kappa, int n,
                                                 const int* __restrict__ active, const int* __restrict__ leaf_sys,
                                                 double* __restrict__ out) {
  constexpr int NC = MI<P>::NC;
  __shared__ Real sm[FCH][2 * NC];
  __shared__ Real so[FCH][3];
  const int4 B = blk[blockIdx.x];
  const int leaf = B.x;
  if (active && !active[leaf_sys[leaf]]) return;
  const double4 ct = center[leaf_cell[leaf]];
  const int i = B.y + threadIdx.x;
  const bool act = (int)threadIdx.x < B.z;
  Real xr[3] = {0, 0, 0};
  if (act) {
    double4 x = tgt64[i];
    xr[0] = (Real)(x.x - ct.x);
    xr[1] = (Real)(x.y - ct.y);
    xr[2] = (Real)(x.z - ct.z);
  }
  double aV = 0, aK = 0;
  const int f0 = far_ptr[leaf], f1 = far_ptr[leaf + 1];
  for (int fb = f0; fb < f1; fb += FCH) {
    const int cnt = min(FCH, f1 - fb);
    for (int q = threadIdx.x; q < cnt * 2 * NC; q += TBT)
      sm[q / (2 * NC)][q % (2 * NC)] = mom[(size_t)far_list[fb + q / (2 * NC)] * 2 * NC + q % (2 * NC)];
    if ((int)threadIdx.x < cnt) {
      double4 cc = center[far_list[fb + threadIdx.x]];
      so[threadIdx.x][0] = (Real)(ct.x - cc.x);
      so[threadIdx.x][1] = (Real)(ct.y - cc.y);
      so[threadIdx.x][2] = (Real)(ct.z - cc.z);
    }
    __syncthreads();
    Real v = 0, k = 0;
    if ((int)(threadIdx.x & ~31u) < B.z) {  // warp holds at least one target
      for (int q = 0; q < cnt; ++q) {
        const Real D[3] = {xr[0] + so[q][0], xr[1] + so[q][1], xr[2] + so[q][2]};
        if (YUK)
          far_eval_yukawa<P, Real>(D, sm[q], sm[q] + NC, kappa, v, k);
        else
          far_eval_laplace<P, Real>(D, sm[q], sm[q] + NC, v, k);
      }
    }
    aV += (double)v;
    aK += (double)k;
    __syncthreads();
  }
  if (act) {
    out[(2 * YUK) * (size_t)n + i] = aV;
    out[(2 * YUK + 1) * (size_t)n + i] = aK;
  }
}

// ---------------------------------------------------------------- near field
__device__ __forceinline__ void pair_accum(const float x[3], float4 p, float4 s, float kappa, float nk_log2e,
                                           float& vl, float& kl, float& vy, float& ky) {
  float dx = x[0] - p.x, dy = x[1] - p.y, dz = x[2] - p.z;
  float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float rinv = r2 > 0.f ? rsqrt_approx(r2) : 0.f;
  float r = r2 * rinv;
  float e = exp2_approx(r * nk_log2e);
  float mr = s.x * rinv;
  vl = fmaf(mr, p.w, vl);  // p.w: 1 for a source of the target's body, 0 for another body
  vy = fmaf(mr, e, vy);
  float dR = fmaf(s.y, dx, fmaf(s.z, dy, s.w * dz));
  float t = dR * (rinv * rinv) * rinv;
  kl = fmaf(t, p.w, kl);
  ky = fmaf(t * fmaf(kappa, r, 1.f), e, ky);
}

__device__ __forceinline__ void pair_accum(const double x[3], double4 p, double4 s, double kappa, double,
                                           double& vl, double& kl, double& vy, double& ky) {
  double dx = x[0] - p.x, dy = x[1] - p.y, dz = x[2] - p.z;
  double r2 = dx * dx + dy * dy + dz * dz;
  if (r2 == 0.0) return;
  double R = sqrt(r2);
  double rinv = 1.0 / R;
  double e = exp(-kappa * R);
  double mr = s.x * rinv;
  vl = fma(mr, p.w, vl);
  vy += mr * e;
  double t = (s.y * dx + s.z * dy + s.w * dz) * rinv * rinv * rinv;
  kl = fma(t, p.w, kl);
  ky += t * (1.0 + kappa * R) * e;
}

// One warp per target block of <= 32 targets of one leaf.  The leaf's near list is
// cut into gridDim.y consecutive pieces; piece s writes its partial sums to
// out + s * 4n (no atomics: the combine kernel adds the pieces in order).
constexpr int NTB = 32;
template <typename Real>
__global__ void __launch_bounds__(NTB) near_kernel(const int4* __restrict__ blk, const double4* __restrict__ tgt64,
                                                  const int* __restrict__ leaf_cell,
                                                  const double4* __restrict__ center, const int* __restrict__ begin,
                                                  const int* __restrict__ end, const int* __restrict__ near_ptr,
                                                  const int* __restrict__ near_list, int K,
                                                  const double4* __restrict__ src64,
                                                  const typename Vec4<Real>::T* __restrict__ str, Real kappa,
                                                  Real nk_log2e, int n, const float4* __restrict__ src_rel,
                                                  const int* __restrict__ active, const int* __restrict__ leaf_sys,
                                                  double* __restrict__ out) {
  typedef typename Vec4<Real>::T R4;
  __shared__ R4 sp[NTB];
  __shared__ R4 ss[NTB];
  const int4 B = blk[blockIdx.x];
  const int leaf = B.x;
  if (active && !active[leaf_sys[leaf]]) return;
  const double4 ct = center[leaf_cell[leaf]];
  const int i = B.y + threadIdx.x;
  const bool act = (int)threadIdx.x < B.z;
  Real xr[3] = {0, 0, 0};
  if (act) {
    double4 x = tgt64[i];
    xr[0] = (Real)(x.x - ct.x);
    xr[1] = (Real)(x.y - ct.y);
    xr[2] = (Real)(x.z - ct.z);
  }
  // The sources of up to NLC near leaves are streamed as one concatenated sequence,
  // so every tile but the last of a pass is full and runs the unrolled loop.
  constexpr int NLC = 64;
  __shared__ int lb[NLC];       // first source index of each leaf of the pass
  __shared__ int lc[NLC + 1];   // cumulative source counts
  __shared__ float lo3[NLC][3]; // FP32 offset (source-leaf centre - target-leaf centre)
  __shared__ float lw[NLC];     // Laplace weight of the leaf: 1 same body, 0 another body
  double acc[4] = {0, 0, 0, 0};
  const int nl = near_ptr[leaf + 1] - near_ptr[leaf];
  const int e0 = near_ptr[leaf] + (int)(((long long)nl * blockIdx.y) / gridDim.y);
  const int e1 = near_ptr[leaf] + (int)(((long long)nl * (blockIdx.y + 1)) / gridDim.y);
  for (int eb = e0; eb < e1; eb += NLC) {
    const int cnt = min(NLC, e1 - eb);
    __syncthreads();  // the previous pass is done with lb / lc
    for (int q = threadIdx.x; q < cnt; q += NTB) {
      const int ent = near_list[eb + q];
      const int cl = leaf_cell[ent & ~NEAR_CROSS];
      lw[q] = (ent & NEAR_CROSS) ? 0.f : 1.f;
      lb[q] = begin[cl] * K;
      lc[q + 1] = (end[cl] - begin[cl]) * K;
      const double4 cs = center[cl];
      lo3[q][0] = (float)(cs.x - ct.x);
      lo3[q][1] = (float)(cs.y - ct.y);
      lo3[q][2] = (float)(cs.z - ct.z);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      lc[0] = 0;
      for (int q = 1; q <= cnt; ++q) lc[q] += lc[q - 1];
    }
    __syncthreads();
    const int total = lc[cnt];
    for (int t0 = 0; t0 < total; t0 += NTB) {
      const int j = t0 + threadIdx.x;
      R4 pz, sz;
      pz.x = pz.y = pz.z = pz.w = 0;
      sz = pz;
      if (j < total) {
        int lo = 0, hi = cnt - 1;  // largest q with lc[q] <= j
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (lc[mid] <= j)
            lo = mid;
          else
            hi = mid - 1;
        }
        const int src = lb[lo] + (j - lc[lo]);
        if constexpr (sizeof(Real) == 4) {
          // leaf-relative FP32 position plus the leaf-pair offset: no FP64 work per source
          const float4 r = src_rel[src];
          pz.x = r.x + lo3[lo][0];
          pz.y = r.y + lo3[lo][1];
          pz.z = r.z + lo3[lo][2];
        } else {
          const double4 y = src64[src];
          pz.x = (Real)(y.x - ct.x);
          pz.y = (Real)(y.y - ct.y);
          pz.z = (Real)(y.z - ct.z);
        }
        pz.w = (Real)lw[lo];
        sz = str[src];
      }
      sp[threadIdx.x] = pz;
      ss[threadIdx.x] = sz;
      __syncthreads();
      Real vl = 0, kl = 0, vy = 0, ky = 0;
      if (t0 + NTB <= total) {
#pragma unroll 8
        for (int k = 0; k < NTB; ++k) pair_accum(xr, sp[k], ss[k], kappa, nk_log2e, vl, kl, vy, ky);
      } else {
        const int lim = total - t0;
        for (int k = 0; k < lim; ++k) pair_accum(xr, sp[k], ss[k], kappa, nk_log2e, vl, kl, vy, ky);
      }
      acc[0] += (double)vl;
      acc[1] += (double)kl;
      acc[2] += (double)vy;
      acc[3] += (double)ky;
      __syncthreads();
    }
  }
  if (act) {
    double* o = out + (size_t)blockIdx.y * 4 * n;
    o[i] = acc[0];
    o[n + i] = acc[1];
    o[2 * n + i] = acc[2];
    o[3 * n + i] = acc[3];
  }
}

// ---------------------------------------------------------------- transposed product
// A^T puts charges at the collocation points and evaluates at the Gauss nodes: per
// panel j, sum_g W_g V(y_g) and sum_g W_g n_j . grad V(y_g) with V the potential of the
// charges u (u1 for the Laplace kernel, u2 for Yukawa).  Far field: V(y) = sum_k a_k(D) M_k
// with D = y - c_C and M_k the charge moments of cell C; since da_k/dD_j = -(k_j + 1) a_{k+e_j},
// grad V = -sum_k (k_j + 1) a_{k+e_j} M_k e_j, so the coefficients run to order P + 1.
template <int P, typename Real, int YUK>
__device__ __forceinline__ void farT_eval(const Real D[3], const Real* __restrict__ M, Real kappa, Real& V,
                                          Real G[3]) {
  constexpr int Q = P + 1;
  constexpr MI<Q> mi{};
  constexpr int NCQ = MI<Q>::NC;
  constexpr int NC = MI<P>::NC;
  const Real r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
  const Real rinv = inv_sqrt(r2);
  const Real ir2 = rinv * rinv;
  Real A[NCQ], Bc[YUK ? NCQ : 1];
  Real q1[Q + 1], q2[Q + 1], q3[Q + 1], kn[Q + 1];
#pragma unroll
  for (int nn = 1; nn <= Q; ++nn) {
    q1[nn] = ir2 * (Real)((2.0 * nn - 1.0) / nn);
    q2[nn] = ir2 * (Real)((nn - 1.0) / nn);
    kn[nn] = kappa * (Real)(1.0 / nn);
    q3[nn] = kn[nn] * ir2;
  }
  if (YUK) {
    const Real e = exp_neg(kappa * (r2 * rinv));
    A[0] = e * rinv;
    Bc[0] = e;
  } else {
    A[0] = rinv;
  }
#pragma unroll
  for (int t = 1; t < NCQ; ++t) {
    const int nn = mi.ord[t];
    Real s1a = 0, s2a = 0, s1b = 0, s2b = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (mi.m1[t][j] >= 0) {
        s1a += D[j] * A[mi.m1[t][j]];
        if (YUK) s1b += D[j] * Bc[mi.m1[t][j]];
      }
      if (mi.m2[t][j] >= 0) {
        s2a += A[mi.m2[t][j]];
        if (YUK) s2b += Bc[mi.m2[t][j]];
      }
    }
    if (YUK) {
      Bc[t] = kn[nn] * (s1a - s2a);
      A[t] = q1[nn] * s1a - q2[nn] * s2a + q3[nn] * (s1b - s2b);
    } else {
      A[t] = q1[nn] * s1a - q2[nn] * s2a;
    }
  }
  Real v = 0, g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
  for (int t = 0; t < NC; ++t) {
    const int kx = mi.k[t][0], ky = mi.k[t][1], kz = mi.k[t][2];
    const Real m = M[t];
    v += A[t] * m;
    g0 -= (Real)(kx + 1) * A[mi.idx[kx + 1][ky][kz]] * m;
    g1 -= (Real)(ky + 1) * A[mi.idx[kx][ky + 1][kz]] * m;
    g2 -= (Real)(kz + 1) * A[mi.idx[kx][ky][kz + 1]] * m;
  }
  V = v;
  G[0] = g0;
  G[1] = g1;
  G[2] = g2;
}

// One thread per panel of a target block (<= 128 panels of one leaf), K Gauss nodes
// each; loops over the leaf's far cells (Laplace list for YUK = 0, Yukawa list for 1)
// with the charge moments `mom` ([cell][2][NC], first NC used).  Writes rows
// (2 YUK, 2 YUK + 1) = (sum_g W V, sum_g W n . grad V) of `out` ([4][n]).
template <int P, typename Real, int YUK>
__global__ void __launch_bounds__(TBT) farT_kernel(const int4* __restrict__ blk, const float4* __restrict__ node_rel,
                                                  const double4* __restrict__ node64, const double4* __restrict__ nrm,
                                                  int K, const int* __restrict__ leaf_cell,
                                                  const double4* __restrict__ center, const int* __restrict__ far_ptr,
                                                  const int* __restrict__ far_list, const Real* __restrict__ mom,
                                                  Real kappa, int n, const int* __restrict__ active,
                                                  const int* __restrict__ leaf_sys, double* __restrict__ out) {
  constexpr int NC = MI<P>::NC;
  __shared__ Real sm[FCH][NC];
  __shared__ Real so[FCH][3];
  const int4 B = blk[blockIdx.x];
  const int leaf = B.x;
  if (active && !active[leaf_sys[leaf]]) return;
  const double4 ct = center[leaf_cell[leaf]];
  const int i = B.y + threadIdx.x;
  const bool act = (int)threadIdx.x < B.z;
  Real yr[4][3], w[4], nv[3] = {0, 0, 0};
  for (int g = 0; g < 4; ++g) {
    yr[g][0] = yr[g][1] = yr[g][2] = 0;
    w[g] = 0;
  }
  if (act) {
    for (int g = 0; g < K; ++g) {
      if (sizeof(Real) == 4) {
        const float4 r = node_rel[(size_t)K * i + g];
        yr[g][0] = r.x;
        yr[g][1] = r.y;
        yr[g][2] = r.z;
      } else {
        const double4 y = node64[(size_t)K * i + g];
        yr[g][0] = (Real)(y.x - ct.x);
        yr[g][1] = (Real)(y.y - ct.y);
        yr[g][2] = (Real)(y.z - ct.z);
      }
      w[g] = (Real)node64[(size_t)K * i + g].w;
    }
    const double4 nn = nrm[i];
    nv[0] = (Real)nn.x;
    nv[1] = (Real)nn.y;
    nv[2] = (Real)nn.z;
  }
  double aV = 0, aK = 0;
  const int f0 = far_ptr[leaf], f1 = far_ptr[leaf + 1];
  for (int fb = f0; fb < f1; fb += FCH) {
    const int cnt = min(FCH, f1 - fb);
    for (int q = threadIdx.x; q < cnt * NC; q += TBT)
      sm[q / NC][q % NC] = mom[(size_t)far_list[fb + q / NC] * 2 * NC + q % NC];
    if ((int)threadIdx.x < cnt) {
      const double4 cc = center[far_list[fb + threadIdx.x]];
      so[threadIdx.x][0] = (Real)(ct.x - cc.x);
      so[threadIdx.x][1] = (Real)(ct.y - cc.y);
      so[threadIdx.x][2] = (Real)(ct.z - cc.z);
    }
    __syncthreads();
    Real v = 0, k = 0;
    if ((int)(threadIdx.x & ~31u) < B.z) {
      for (int q = 0; q < cnt; ++q) {
        for (int g = 0; g < K; ++g) {
          const Real D[3] = {yr[g][0] + so[q][0], yr[g][1] + so[q][1], yr[g][2] + so[q][2]};
          Real V, G[3];
          farT_eval<P, Real, YUK>(D, sm[q], kappa, V, G);
          v += w[g] * V;
          k += w[g] * (nv[0] * G[0] + nv[1] * G[1] + nv[2] * G[2]);
        }
      }
    }
    aV += (double)v;
    aK += (double)k;
    __syncthreads();
  }
  if (act) {
    out[(2 * YUK) * (size_t)n + i] = aV;
    out[(2 * YUK + 1) * (size_t)n + i] = aK;
  }
}

// Near field of the transposed product: one warp per target block of <= 32 panels of
// one leaf, the leaf's near list cut into gridDim.y pieces as in near_kernel; the
// sources are the collocation points (charges u1 masked to the target's body, u2),
// the targets each panel's K Gauss nodes.  Writes the four rows of `out + y * 4n`.
template <typename Real>
__global__ void __launch_bounds__(NTB) nearT_kernel(const int4* __restrict__ blk, const float4* __restrict__ node_rel,
                                                   const double4* __restrict__ node64,
                                                   const double4* __restrict__ nrm, int K,
                                                   const int* __restrict__ leaf_cell,
                                                   const double4* __restrict__ center, const int* __restrict__ begin,
                                                   const int* __restrict__ end, const int* __restrict__ near_ptr,
                                                   const int* __restrict__ near_list,
                                                   const float4* __restrict__ cen_rel, const double4* __restrict__ cen64,
                                                   const double* __restrict__ u, Real kappa, int n,
                                                   const int* __restrict__ active, const int* __restrict__ leaf_sys,
                                                   double* __restrict__ out) {
  typedef typename Vec4<Real>::T R4;
  __shared__ R4 sp[NTB];  // source position (rel. target-leaf centre), u2 in w
  __shared__ Real s1[NTB];
  const int4 B = blk[blockIdx.x];
  const int leaf = B.x;
  if (active && !active[leaf_sys[leaf]]) return;
  const double4 ct = center[leaf_cell[leaf]];
  const int i = B.y + threadIdx.x;
  const bool act = (int)threadIdx.x < B.z;
  Real yr[4][3], w[4], nv[3] = {0, 0, 0};
  for (int g = 0; g < 4; ++g) {
    yr[g][0] = yr[g][1] = yr[g][2] = 0;
    w[g] = 0;
  }
  if (act) {
    for (int g = 0; g < K; ++g) {
      if (sizeof(Real) == 4) {
        const float4 r = node_rel[(size_t)K * i + g];
        yr[g][0] = r.x;
        yr[g][1] = r.y;
        yr[g][2] = r.z;
      } else {
        const double4 y = node64[(size_t)K * i + g];
        yr[g][0] = (Real)(y.x - ct.x);
        yr[g][1] = (Real)(y.y - ct.y);
        yr[g][2] = (Real)(y.z - ct.z);
      }
      w[g] = (Real)node64[(size_t)K * i + g].w;
    }
    const double4 nn = nrm[i];
    nv[0] = (Real)nn.x;
    nv[1] = (Real)nn.y;
    nv[2] = (Real)nn.z;
  }
  constexpr int NLC = 64;
  __shared__ int lb[NLC];
  __shared__ int lc[NLC + 1];
  __shared__ float lo3[NLC][3];
  __shared__ float lw[NLC];
  double acc[4] = {0, 0, 0, 0};
  const int nl = near_ptr[leaf + 1] - near_ptr[leaf];
  const int e0 = near_ptr[leaf] + (int)(((long long)nl * blockIdx.y) / gridDim.y);
  const int e1 = near_ptr[leaf] + (int)(((long long)nl * (blockIdx.y + 1)) / gridDim.y);
  for (int eb = e0; eb < e1; eb += NLC) {
    const int cnt = min(NLC, e1 - eb);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += NTB) {
      const int ent = near_list[eb + q];
      const int cl = leaf_cell[ent & ~NEAR_CROSS];
      lw[q] = (ent & NEAR_CROSS) ? 0.f : 1.f;
      lb[q] = begin[cl];
      lc[q + 1] = end[cl] - begin[cl];
      const double4 cs = center[cl];
      lo3[q][0] = (float)(cs.x - ct.x);
      lo3[q][1] = (float)(cs.y - ct.y);
      lo3[q][2] = (float)(cs.z - ct.z);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      lc[0] = 0;
      for (int q = 1; q <= cnt; ++q) lc[q] += lc[q - 1];
    }
    __syncthreads();
    const int total = lc[cnt];
    for (int t0 = 0; t0 < total; t0 += NTB) {
      const int j = t0 + threadIdx.x;
      R4 pz;
      pz.x = pz.y = pz.z = pz.w = 0;
      Real a1 = 0;
      if (j < total) {
        int lo = 0, hi = cnt - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (lc[mid] <= j)
            lo = mid;
          else
            hi = mid - 1;
        }
        const int src = lb[lo] + (j - lc[lo]);
        if constexpr (sizeof(Real) == 4) {
          const float4 r = cen_rel[src];
          pz.x = r.x + lo3[lo][0];
          pz.y = r.y + lo3[lo][1];
          pz.z = r.z + lo3[lo][2];
        } else {
          const double4 x = cen64[src];
          pz.x = (Real)(x.x - ct.x);
          pz.y = (Real)(x.y - ct.y);
          pz.z = (Real)(x.z - ct.z);
        }
        pz.w = (Real)u[n + src];
        a1 = (Real)(lw[lo] * u[src]);
      }
      sp[threadIdx.x] = pz;
      s1[threadIdx.x] = a1;
      __syncthreads();
      Real vl = 0, kl = 0, vy = 0, ky = 0;
      const int lim = min(NTB, total - t0);
      for (int k = 0; k < lim; ++k) {
        const R4 p = sp[k];
        const Real u1 = s1[k], u2 = p.w;
        for (int g = 0; g < K; ++g) {
          const Real dx = p.x - yr[g][0], dy = p.y - yr[g][1], dz = p.z - yr[g][2];
          const Real r2 = dx * dx + dy * dy + dz * dz;
          if (sizeof(Real) == 4) {
            const float ri = r2 > 0.f ? rsqrt_approx((float)r2) : 0.f;
            const float r = (float)r2 * ri;
            const float e = exp2_approx(-1.4426950408889634f * (float)kappa * r);
            const float ww = (float)w[g] * ri;
            const float nR = (float)(nv[0] * dx + nv[1] * dy + nv[2] * dz) * ri * ri;
            vl += (Real)(ww * (float)u1);
            vy += (Real)(ww * (float)u2 * e);
            kl += (Real)(ww * nR * (float)u1);
            ky += (Real)(ww * nR * (float)u2 * fmaf((float)kappa, r, 1.f) * e);
          } else {
            if (r2 == 0) continue;
            const double r = sqrt((double)r2);
            const double ri = 1.0 / r;
            const double e = exp(-(double)kappa * r);
            const double ww = (double)w[g] * ri;
            const double nR = (double)(nv[0] * dx + nv[1] * dy + nv[2] * dz) * ri * ri;
            vl += (Real)(ww * (double)u1);
            vy += (Real)(ww * (double)u2 * e);
            kl += (Real)(ww * nR * (double)u1);
            ky += (Real)(ww * nR * (double)u2 * (1.0 + (double)kappa * r) * e);
          }
        }
      }
      acc[0] += (double)vl;
      acc[1] += (double)kl;
      acc[2] += (double)vy;
      acc[3] += (double)ky;
      __syncthreads();
    }
  }
  if (act) {
    double* o = out + (size_t)blockIdx.y * 4 * n;
    o[i] = acc[0];
    o[n + i] = acc[1];
    o[2 * n + i] = acc[2];
    o[3 * n + i] = acc[3];
  }
}

// charges u1 (Laplace) and u2 (Yukawa) at the collocation points as (u, 0, 0, 0) strengths
template <typename R4>
__global__ void centroid_charges_kernel(const double* __restrict__ u, int n, R4* __restrict__ sL,
                                        R4* __restrict__ sY) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  R4 a, b;
  a.x = u[i];
  a.y = a.z = a.w = 0;
  b.x = u[n + i];
  b.y = b.z = b.w = 0;
  sL[i] = a;
  sY[i] = b;
}

}  // namespace

namespace {

// Octree topology from the sorted 30-bit Morton codes (10 levels of 3 bits).
// With several groups the root's children are the groups (each with its own
// Morton codes); below that a cell with more than `leaf` panels is split by the
// next Morton digit.  Digits shared by every panel of the cell are skipped, so no
// cell has a single child.
void build_topology(Ctx& c) {
  Tree& T = c.tree;
  const int n = c.n;
  const std::vector<unsigned>& m = c.h_morton;
  T.h_begin.assign(1, 0);
  T.h_end.assign(1, n);
  T.h_child0.assign(1, -1);
  T.h_nchild.assign(1, 0);
  T.h_cell_grp.assign(1, c.ngroup > 1 ? -1 : 0);
  std::vector<int> lev(1, 0), depth(1, 0);
  auto add_child = [&](int q, int b, int e, int l, int g) {
    T.h_begin.push_back(b);
    T.h_end.push_back(e);
    T.h_child0.push_back(-1);
    T.h_nchild.push_back(0);
    T.h_cell_grp.push_back(g);
    lev.push_back(l);
    depth.push_back(depth[q] + 1);
    ++T.h_nchild[q];
  };
  for (size_t q = 0; q < T.h_begin.size(); ++q) {
    const int b = T.h_begin[q], e = T.h_end[q];
    if (q == 0 && c.ngroup > 1) {
      T.h_child0[q] = 1;
      for (int g = 0; g < c.ngroup; ++g) add_child((int)q, c.h_gpan[g], c.h_gpan[g + 1], 0, g);
      continue;
    }
    if (e - b <= c.par.leaf) continue;
    int l = lev[q];
    auto digit = [&](int i, int L) { return (int)((m[i] >> (27 - 3 * L)) & 7u); };
    while (l < 10 && digit(b, l) == digit(e - 1, l)) ++l;
    if (l >= 10) continue;  // identical codes: keep as an oversized leaf
    T.h_child0[q] = (int)T.h_begin.size();
    int start = b;
    for (int i = b + 1; i <= e; ++i) {
      if (i == e || digit(i, l) != digit(start, l)) {
        add_child((int)q, start, i, l + 1, T.h_cell_grp[q]);
        start = i;
      }
    }
  }
  T.ncell = (int)T.h_begin.size();
  T.h_depth_begin.clear();
  for (int q = 0; q < T.ncell; ++q)
    while ((int)T.h_depth_begin.size() <= depth[q]) T.h_depth_begin.push_back(q);
  T.ndepth = (int)T.h_depth_begin.size();
  T.h_depth_begin.push_back(T.ncell);
  T.h_leaf_cell.clear();
  for (int q = 0; q < T.ncell; ++q)
    if (T.h_nchild[q] == 0) T.h_leaf_cell.push_back(q);
  T.nleaf = (int)T.h_leaf_cell.size();
}

template <typename V>
void upload(DBuf<V>& d, const std::vector<V>& h, cudaStream_t s) {
  d.alloc(std::max<size_t>(1, h.size()));
  if (!h.empty()) BP_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, s));
}

// Interaction lists of every leaf under the batch acceptance criterion.  Cells of
// another system are skipped, cells of another body of the same system enter the
// Yukawa lists only (Laplace layers act within a body), and the multi-group root
// is always opened.
void build_lists(Ctx& c, cudaStream_t s) {
  Tree& T = c.tree;
  const double theta = c.par.theta;
  std::vector<int> leaf_of(T.ncell, -1);
  for (int l = 0; l < T.nleaf; ++l) leaf_of[T.h_leaf_cell[l]] = l;
  std::vector<int> fptr(T.nleaf + 1, 0), lptr(T.nleaf + 1, 0), nptr(T.nleaf + 1, 0), flist, llist, nlist;
  std::vector<int4> blk, blk32;
  std::vector<int> stack;
  long long pairs = 0, fars = 0, farsL = 0;
  for (int l = 0; l < T.nleaf; ++l) {
    const int ct = T.h_leaf_cell[l];
    const int g = T.h_cell_grp[ct];
    const int sy = c.h_grp_sys[g];
    const double4 a = T.h_center[ct];
    const int ntgt = T.h_end[ct] - T.h_begin[ct];
    stack.assign(1, 0);
    while (!stack.empty()) {
      const int q = stack.back();
      stack.pop_back();
      const int cg = T.h_cell_grp[q];
      if (cg < 0) {
        for (int k = T.h_nchild[q] - 1; k >= 0; --k) stack.push_back(T.h_child0[q] + k);
        continue;
      }
      if (c.h_grp_sys[cg] != sy) continue;
      const double4 b = T.h_center[q];
      const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
      const double gap = std::sqrt(dx * dx + dy * dy + dz * dz) - a.w;
      if (q != ct && gap > 0.0 && b.w < theta * gap) {
        flist.push_back(q);
        fars += ntgt;
        if (cg == g) {
          llist.push_back(q);
          farsL += ntgt;
        }
      } else if (T.h_nchild[q] == 0) {
        nlist.push_back(leaf_of[q] | (cg == g ? 0 : NEAR_CROSS));
        pairs += (long long)ntgt * (T.h_end[q] - T.h_begin[q]) * c.K;
      } else {
        for (int k = T.h_nchild[q] - 1; k >= 0; --k) stack.push_back(T.h_child0[q] + k);
      }
    }
    fptr[l + 1] = (int)flist.size();
    lptr[l + 1] = (int)llist.size();
    nptr[l + 1] = (int)nlist.size();
    for (int off = 0; off < ntgt; off += TBT)
      blk.push_back(make_int4(l, T.h_begin[ct] + off, std::min(TBT, ntgt - off), 0));
    for (int off = 0; off < ntgt; off += 32)
      blk32.push_back(make_int4(l, T.h_begin[ct] + off, std::min(32, ntgt - off), 0));
  }
  // largest blocks first: the grids are only one or two waves deep, so launching the
  // long blocks early shortens the tail (each block's result does not depend on order)
  std::vector<long long> far_work(T.nleaf), near_work(T.nleaf, 0);
  for (int l = 0; l < T.nleaf; ++l) {
    far_work[l] = fptr[l + 1] - fptr[l];
    for (int e = nptr[l]; e < nptr[l + 1]; ++e) {
      const int q = T.h_leaf_cell[nlist[e] & ~NEAR_CROSS];
      near_work[l] += T.h_end[q] - T.h_begin[q];
    }
  }
  std::stable_sort(blk.begin(), blk.end(), [&](const int4& u, const int4& v) {
    return far_work[u.x] * u.z > far_work[v.x] * v.z;
  });
  std::stable_sort(blk32.begin(), blk32.end(), [&](const int4& u, const int4& v) {
    return near_work[u.x] * u.z > near_work[v.x] * v.z;
  });
  // shallowest tree depth that holds an accepted cell: moments above it are never read
  T.m2m_min_depth = T.ndepth;
  for (int q : flist) {
    int d = 0;
    while (d + 1 < T.ndepth && T.h_depth_begin[d + 1] <= q) ++d;
    T.m2m_min_depth = std::min(T.m2m_min_depth, d);
  }
  T.nblk = (int)blk.size();
  T.nblk32 = (int)blk32.size();
  // split each near-field block's source stream so the grid holds ~56 warps per SM
  T.near_splits = std::max(1, std::min(4, cdiv((long long)num_sms(c.device) * 56, std::max(1, T.nblk32))));
  upload(T.blk32, blk32, s);
  T.pairs_per_matvec = pairs;
  T.far_per_matvec = fars;
  T.farL_per_matvec = farsL;
  upload(T.far_ptr, fptr, s);
  upload(T.far_list, flist, s);
  T.farL_same = llist.size() == flist.size();
  if (!T.farL_same) {
    upload(T.farL_ptr, lptr, s);
    upload(T.farL_list, llist, s);
  }
  upload(T.near_ptr, nptr, s);
  upload(T.near_list, nlist, s);
  upload(T.blk, blk, s);
  std::vector<int> lsys(T.nleaf);
  for (int l = 0; l < T.nleaf; ++l) lsys[l] = c.h_grp_sys[T.h_cell_grp[T.h_leaf_cell[l]]];
  upload(T.leaf_sys, lsys, s);
  T.theta_built = theta;
}

template <int P, typename Real>
void run_tree(Ctx& c, DBuf<Real>& mom, cudaStream_t s) {
  Tree& T = c.tree;
  constexpr int NC = MI<P>::NC;
  if (T.mom_order != P || mom.n < (size_t)T.ncell * 2 * NC) {
    mom.alloc((size_t)T.ncell * 2 * NC);
    T.mom_order = P;
  }
  typedef typename Vec4<Real>::T R4;
  const R4* str = nullptr;
  if (sizeof(Real) == 4)
    str = reinterpret_cast<const R4*>(c.str32.p);
  else
    str = reinterpret_cast<const R4*>(c.str64.p);
  launch(leaf_moments_kernel<P, Real>, T.nleaf, TB, 0, s, T.leaf_cell.p, T.begin.p, T.end.p, T.center.p, c.K,
         c.src64.p, str, c.mv_active, T.leaf_sys.p, mom.p);
  for (int d = T.ndepth - 2; d >= T.m2m_min_depth; --d) {  // depths above are in no far list
    const int first = T.h_depth_begin[d], cnt = T.h_depth_begin[d + 1] - first;
    launch(m2m_kernel<P, Real>, cnt, TB, 0, s, first, T.child0.p, T.nchild.p, T.center.p, mom.p);
  }
  const int S = T.near_splits;
  const size_t need = (size_t)(S + 1) * 4 * c.n;
  if (c.part.n < need) c.part.alloc(need);
  const Real kappa = (Real)c.par.kappa;
  const Real nk = (Real)(-c.par.kappa * 1.4426950408889634);
  Ctx::Timed tm;
  c.time_begin(0, s, tm);
  c.stat_pairs += T.pairs_per_matvec;
  launch(near_kernel<Real>, dim3(T.nblk32, S), NTB, 0, s, T.blk32.p, c.tgt64.p, T.leaf_cell.p, T.center.p,
         T.begin.p, T.end.p, T.near_ptr.p, T.near_list.p, c.K, c.src64.p, str, kappa, nk, c.n, T.src_rel32.p,
         c.mv_active, T.leaf_sys.p, c.part.p);
  c.time_end(s, tm);
  Ctx::Timed tf;
  c.time_begin(1, s, tf);
  c.stat_far += T.far_per_matvec;
  double* far_out = c.part.p + (size_t)S * 4 * c.n;
  const int* lp = T.farL_same ? T.far_ptr.p : T.farL_ptr.p;
  const int* ll = T.farL_same ? T.far_list.p : T.farL_list.p;
  launch(far_kernel<P, Real, 0>, T.nblk, TBT, 0, s, T.blk.p, c.tgt64.p, T.leaf_cell.p, T.center.p, lp, ll, mom.p,
         kappa, c.n, c.mv_active, T.leaf_sys.p, far_out);
  launch(far_kernel<P, Real, 1>, T.nblk, TBT, 0, s, T.blk.p, c.tgt64.p, T.leaf_cell.p, T.center.p, T.far_ptr.p,
         T.far_list.p, mom.p, kappa, c.n, c.mv_active, T.leaf_sys.p, far_out);
  c.time_end(s, tf);
  c.part_splits = S + 1;
}

template <typename Real>
void dispatch(Ctx& c, DBuf<Real>& mom, cudaStream_t s) {
  switch (c.par.order) {
    case 1: run_tree<1, Real>(c, mom, s); break;
    case 2: run_tree<2, Real>(c, mom, s); break;
    case 3: run_tree<3, Real>(c, mom, s); break;
    case 4: run_tree<4, Real>(c, mom, s); break;
    case 5: run_tree<5, Real>(c, mom, s); break;
    case 6: run_tree<6, Real>(c, mom, s); break;
    default: fail(BEMPOL_ERR_ARG, "treecode order must be in 1..6");
  }
}

template <typename Real>
DBuf<Real>& momT(Tree& T, int w);
template <>
DBuf<float>& momT<float>(Tree& T, int w) {
  return T.momT32[w];
}
template <>
DBuf<double>& momT<double>(Tree& T, int w) {
  return T.momT64[w];
}

template <int P, typename Real>
void runT_tree(Ctx& c, const double* u, cudaStream_t s) {
  Tree& T = c.tree;
  constexpr int NC = MI<P>::NC;
  typedef typename Vec4<Real>::T R4;
  DBuf<Real>& mL = momT<Real>(T, 0);
  DBuf<Real>& mY = momT<Real>(T, 1);
  if (mL.n < (size_t)T.ncell * 2 * NC) mL.alloc((size_t)T.ncell * 2 * NC);
  if (mY.n < (size_t)T.ncell * 2 * NC) mY.alloc((size_t)T.ncell * 2 * NC);
  DBuf<R4> sL, sY;
  sL.alloc(c.n);
  sY.alloc(c.n);
  launch(centroid_charges_kernel<R4>, cdiv(c.n, 256), 256, 0, s, u, c.n, sL.p, sY.p);
  for (int w = 0; w < 2; ++w) {
    DBuf<Real>& m = w ? mY : mL;
    launch(leaf_moments_kernel<P, Real>, T.nleaf, TB, 0, s, T.leaf_cell.p, T.begin.p, T.end.p, T.center.p, 1,
           c.tgt64.p, (const R4*)(w ? sY.p : sL.p), c.mv_active, T.leaf_sys.p, m.p);
    for (int d = T.ndepth - 2; d >= T.m2m_min_depth; --d) {
      const int first = T.h_depth_begin[d], cnt = T.h_depth_begin[d + 1] - first;
      launch(m2m_kernel<P, Real>, cnt, TB, 0, s, first, T.child0.p, T.nchild.p, T.center.p, m.p);
    }
  }
  const int S = T.near_splits;
  const size_t need = (size_t)(S + 1) * 4 * c.n;
  if (c.part.n < need) c.part.alloc(need);
  const Real kappa = (Real)c.par.kappa;
  Ctx::Timed tm;
  c.time_begin(0, s, tm);
  launch(nearT_kernel<Real>, dim3(T.nblk32, S), NTB, 0, s, T.blk32.p, T.src_rel32.p, c.src64.p, c.nrm64.p, c.K,
         T.leaf_cell.p, T.center.p, T.begin.p, T.end.p, T.near_ptr.p, T.near_list.p, T.cen_rel32.p, c.tgt64.p, u,
         kappa, c.n, c.mv_active, T.leaf_sys.p, c.part.p);
  c.time_end(s, tm);
  Ctx::Timed tf;
  c.time_begin(1, s, tf);
  double* far_out = c.part.p + (size_t)S * 4 * c.n;
  const int* lp = T.farL_same ? T.far_ptr.p : T.farL_ptr.p;
  const int* ll = T.farL_same ? T.far_list.p : T.farL_list.p;
  launch(farT_kernel<P, Real, 0>, T.nblk, TBT, 0, s, T.blk.p, T.src_rel32.p, c.src64.p, c.nrm64.p, c.K,
         T.leaf_cell.p, T.center.p, lp, ll, mL.p, kappa, c.n, c.mv_active, T.leaf_sys.p, far_out);
  launch(farT_kernel<P, Real, 1>, T.nblk, TBT, 0, s, T.blk.p, T.src_rel32.p, c.src64.p, c.nrm64.p, c.K,
         T.leaf_cell.p, T.center.p, T.far_ptr.p, T.far_list.p, mY.p, kappa, c.n, c.mv_active, T.leaf_sys.p,
         far_out);
  c.time_end(s, tf);
  c.part_splits = S + 1;
  BP_CUDA(cudaStreamSynchronize(s));  // the strength buffers are released on return
}

template <typename Real>
void dispatchT(Ctx& c, const double* u, cudaStream_t s) {
  switch (c.par.order) {
    case 1: runT_tree<1, Real>(c, u, s); break;
    case 2: runT_tree<2, Real>(c, u, s); break;
    case 3: runT_tree<3, Real>(c, u, s); break;
    case 4: runT_tree<4, Real>(c, u, s); break;
    case 5: runT_tree<5, Real>(c, u, s); break;
    case 6: runT_tree<6, Real>(c, u, s); break;
    default: fail(BEMPOL_ERR_ARG, "treecode order must be in 1..6");
  }
}

}  // namespace

// Leaves of the same system that may hold a panel centroid within `rmax` of a centroid of leaf l: every
// centroid lies inside its leaf's Gauss-node sphere, so a cell whose sphere is at
// least rmax from the target leaf's sphere is pruned.  Candidates of each leaf are
// sorted by their first panel, so scanning them in order visits panels in order.
void tree_near_candidates(Ctx& c, double rmax, std::vector<int>& ptr, std::vector<int>& cells) {
  Tree& T = c.tree;
  ptr.assign(T.nleaf + 1, 0);
  cells.clear();
  std::vector<int> stack, found;
  for (int l = 0; l < T.nleaf; ++l) {
    const int ct = T.h_leaf_cell[l];
    const int sy = c.h_grp_sys[T.h_cell_grp[ct]];
    const double4 a = T.h_center[ct];
    found.clear();
    stack.assign(1, 0);
    while (!stack.empty()) {
      const int q = stack.back();
      stack.pop_back();
      const int cg = T.h_cell_grp[q];
      if (cg < 0) {
        for (int k = 0; k < T.h_nchild[q]; ++k) stack.push_back(T.h_child0[q] + k);
        continue;
      }
      if (c.h_grp_sys[cg] != sy) continue;  // other systems never interact
      const double4 b = T.h_center[q];
      const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
      if (std::sqrt(dx * dx + dy * dy + dz * dz) - a.w - b.w >= rmax) continue;
      if (T.h_nchild[q] == 0)
        found.push_back(q);
      else
        for (int k = 0; k < T.h_nchild[q]; ++k) stack.push_back(T.h_child0[q] + k);
    }
    std::sort(found.begin(), found.end(), [&](int u, int v) { return T.h_begin[u] < T.h_begin[v]; });
    cells.insert(cells.end(), found.begin(), found.end());
    ptr[l + 1] = (int)cells.size();
  }
}

void build_tree(Ctx& c, cudaStream_t s) {
  Tree& T = c.tree;
  build_topology(c);
  upload(T.begin, T.h_begin, s);
  upload(T.end, T.h_end, s);
  upload(T.child0, T.h_child0, s);
  upload(T.nchild, T.h_nchild, s);
  upload(T.leaf_cell, T.h_leaf_cell, s);
  T.center.alloc(T.ncell);
  launch(cell_geometry_kernel, T.ncell, 256, 0, s, T.begin.p, T.end.p, c.K, c.src64.p, T.center.p);
  T.h_center.resize(T.ncell);
  BP_CUDA(cudaMemcpyAsync(T.h_center.data(), T.center.p, sizeof(double4) * T.ncell, cudaMemcpyDeviceToHost, s));
  T.src_rel32.alloc((size_t)c.K * c.n);
  launch(src_rel_kernel, T.nleaf, 128, 0, s, T.leaf_cell.p, T.nleaf, T.begin.p, T.end.p, T.center.p, c.K, c.src64.p,
         T.src_rel32.p);
  T.cen_rel32.alloc(c.n);
  launch(src_rel_kernel, T.nleaf, 128, 0, s, T.leaf_cell.p, T.nleaf, T.begin.p, T.end.p, T.center.p, 1, c.tgt64.p,
         T.cen_rel32.p);
  BP_CUDA(cudaStreamSynchronize(s));
  build_lists(c, s);
  BP_CUDA(cudaStreamSynchronize(s));
  T.mom_order = -1;
  c.tree_ready = true;
}

// Partial sums of the transposed product (rows V_L, K_L, V_Y, K_Y per panel, part_splits
// pieces in c.part) by the treecode; combineT assembles A^T u from them.
void tree_matvec_T_sums(Ctx& c, const double* u, bool fp32, cudaStream_t s) {
  if (!c.tree_ready) build_tree(c, s);
  if (fp32)
    dispatchT<float>(c, u, s);
  else
    dispatchT<double>(c, u, s);
}

void tree_matvec_sums(Ctx& c, bool fp32, cudaStream_t s) {
  if (!c.tree_ready) build_tree(c, s);
  if (fp32)
    dispatch<float>(c, c.tree.mom32, s);
  else
    dispatch<double>(c, c.tree.mom64, s);
}

}  // namespace bp
