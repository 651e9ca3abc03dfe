// Shared pieces of the treecode (tree.cu: the matrix-vector product; treeT.cu: its
// transpose; sitetree.cu: the fields at the sites): launch constants, the multi-index
// tables of the Taylor expansions, FP32 approximate rsqrt/exp2, the cell-geometry and
// leaf-relative position kernels, the moment kernels (leaf moments from sources, exact
// M2M shifts), and the far-field coefficients of the cells (their index table, the
// host-built table of their terms, the kernel that forms them from two moment sets, and
// the staging shape and 16-byte reads of the far-field kernels).
#pragma once

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
  int p1[NC][3];  // index of k + e_j, or -1 above order P
  int idx[P + 1][P + 1][P + 1];
  constexpr MI() : k{}, ord{}, m1{}, m2{}, p1{}, idx{} {
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
        p1[u][j] = -1;
        if (ord[u] < P) {
          q[j] += 1;
          p1[u][j] = idx[q[0]][q[1]][q[2]];
          q[j] -= 1;
        }
      }
  }
};

__host__ __device__ constexpr int ncoef(int P) { return (P + 1) * (P + 2) * (P + 3) / 6; }

// constant-memory copy of the tables for set-up code that indexes them at run time
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
// Leaf moments from the sources: one block of 2 * MT threads per leaf, tiles of MT
// sources.  Thread j < MT forms, for source j of the tile, the single-layer terms
// m h^k of every k (the monomials h^k built in registers, each from h^(k - e_j) times
// one coordinate, in the order of the multi-index table); thread MT + j forms the
// double-layer terms sum_i k_i d_i h^(k - e_i).  The terms go to a shared [source][moment]
// table, and thread o then adds column o over the tile's sources (one conflict-free
// shared load per source and moment).
constexpr int MT = 64;  // sources per tile
template <int P>
struct MomShape {
  static constexpr int NC = (P + 1) * (P + 2) * (P + 3) / 6;
  static constexpr int TPB = 2 * MT;
};

template <int P, typename Real>
__global__ void __launch_bounds__(2 * MT) leaf_moments_kernel(const int* __restrict__ leaf_cell,
                                                              const int* __restrict__ begin,
                                                              const int* __restrict__ end,
                                                              const double4* __restrict__ center, int K,
                                                              const double4* __restrict__ src64,
                                                              const typename Vec4<Real>::T* __restrict__ str,
                                                              const int* __restrict__ active,
                                                              const int* __restrict__ leaf_sys,
                                                              Real* __restrict__ mom) {
  constexpr MI<P> mi{};
  constexpr int NC = MI<P>::NC;
  constexpr int NO = (2 * NC + 2 * MT - 1) / (2 * MT);  // moments per thread in the column sums
  __shared__ Real term[MT][2 * NC + 1];
  if (active && !active[leaf_sys[blockIdx.x]]) return;  // system not being solved
  const int cidx = leaf_cell[blockIdx.x];
  const double4 c = center[cidx];
  const int s0 = begin[cidx] * K, s1 = end[cidx] * K;
  const int j = threadIdx.x % MT;
  const bool dbl = threadIdx.x >= MT;
  Real acc[NO];
#pragma unroll
  for (int u = 0; u < NO; ++u) acc[u] = 0;
  for (int t0 = s0; t0 < s1; t0 += MT) {
    const int q = t0 + j;
    Real mono[NC];
    Real w[4] = {0, 0, 0, 0};
    mono[0] = 1;
    if (q < s1) {
      const double4 y = src64[q];
      const Real h[3] = {(Real)(y.x - c.x), (Real)(y.y - c.y), (Real)(y.z - c.z)};
#pragma unroll
      for (int t = 1; t < NC; ++t) {
        const int jj = mi.m1[t][0] >= 0 ? 0 : (mi.m1[t][1] >= 0 ? 1 : 2);
        mono[t] = mono[mi.m1[t][jj]] * h[jj];
      }
      const auto sv = str[q];
      w[0] = sv.x;
      w[1] = sv.y;
      w[2] = sv.z;
      w[3] = sv.w;
    }
    if (!dbl) {
#pragma unroll
      for (int t = 0; t < NC; ++t) term[j][t] = w[0] * mono[t];
    } else {
#pragma unroll
      for (int t = 0; t < NC; ++t) {
        Real v = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          if (mi.m1[t][i] >= 0) v += (Real)mi.k[t][i] * w[1 + i] * mono[mi.m1[t][i]];
        term[j][NC + t] = v;
      }
    }
    __syncthreads();
    const int lim = min(MT, s1 - t0);
#pragma unroll
    for (int u = 0; u < NO; ++u) {
      const int o = threadIdx.x + u * 2 * MT;
      if (o < 2 * NC)
        for (int r = 0; r < lim; ++r) acc[u] += term[r][o];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < NO; ++u) {
    const int o = threadIdx.x + u * 2 * MT;
    if (o < 2 * NC) mom[(size_t)cidx * 2 * NC + o] = acc[u];
  }
}

// Parent moments by shifting the children's: one block per parent cell of one depth,
// one thread per (moment, child) shift; the children's shifted moments are then
// added in child order.  The multi-index of a lower index l comes from its closed
// form (orders below n, then a descending, then b descending) and the binomial
// factors from a shared-memory copy, so threads of one warp may take different
// moments without serialising on constant-memory reads.
constexpr int M2M_TPB = 256;
__device__ __forceinline__ int mi_index(int a, int b, int c) {
  const int n = a + b + c;
  return n * (n + 1) * (n + 2) / 6 + (n - a) * (n - a + 1) / 2 + (n - a - b);
}
template <int P, typename Real>
__global__ void __launch_bounds__(M2M_TPB) m2m_kernel(int first_cell, const int* __restrict__ child0,
                                                      const int* __restrict__ nchild,
                                                      const double4* __restrict__ center, Real* __restrict__ mom) {
  constexpr int NC = MI<P>::NC;
  __shared__ Real dp[8][3][P + 1];
  __shared__ Real cm[8][2 * NC];
  __shared__ Real red[8][2 * NC];
  __shared__ int sk[NC][3];
  __shared__ Real sb[P + 1][P + 1];
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
  for (int q = threadIdx.x; q < NC * 3; q += M2M_TPB) sk[q / 3][q % 3] = c_mi<P>.k[q / 3][q % 3];
  for (int q = threadIdx.x; q < (P + 1) * (P + 1); q += M2M_TPB)
    sb[q / (P + 1)][q % (P + 1)] = (Real)c_binom.b[q / (P + 1)][q % (P + 1)];
  for (int q = threadIdx.x; q < nch * 2 * NC; q += M2M_TPB)
    cm[q / (2 * NC)][q % (2 * NC)] = mom[(size_t)(c0 + q / (2 * NC)) * 2 * NC + q % (2 * NC)];
  __syncthreads();
  for (int w = threadIdx.x; w < nch * 2 * NC; w += M2M_TPB) {
    const int ch = w / (2 * NC), o = w - ch * 2 * NC;
    const int t = o < NC ? o : o - NC;
    const int off = o < NC ? 0 : NC;
    const int kx = sk[t][0], ky = sk[t][1], kz = sk[t][2];
    Real a = 0;
    for (int lx = 0; lx <= kx; ++lx) {
      const Real bx = sb[kx][lx] * dp[ch][0][kx - lx];
      for (int ly = 0; ly <= ky; ++ly) {
        const Real bxy = bx * sb[ky][ly] * dp[ch][1][ky - ly];
        for (int lz = 0; lz <= kz; ++lz)
          a += bxy * sb[kz][lz] * dp[ch][2][kz - lz] * cm[ch][off + mi_index(lx, ly, lz)];
      }
    }
    red[ch][o] = a;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 2 * NC; o += M2M_TPB) {
    Real a = 0;
    for (int ch = 0; ch < nch; ++ch) a += red[ch][o];
    mom[(size_t)pc * 2 * NC + o] = a;
  }
}

// asynchronous global -> shared copies of 16 bytes (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ---------------------------------------------------------------- far-field coefficients
// Entries of one cell's far-field coefficients at order P: one per pair (m, e) of a
// radial index m and a monomial exponent e with |e| <= m and 2m - |e| <= P.
constexpr int nb_of(int P) {
  int t = 0;
  for (int d = 0; d <= P; ++d) t += (d + 1) * (d + 2) / 2 * ((P - d) / 2 + 1);
  return t;
}

// Position of the first entry of monomial e = (a, b, c) in a cell's coefficient array
// (monomials in the order a, then b, then c ascending; within one, m ascending).
template <int P>
struct BIdx {
  static constexpr int NB = nb_of(P);
  int t[P + 1][P + 1][P + 1];
  constexpr BIdx() : t{} {
    int q = 0;
    for (int a = 0; a <= P; ++a)
      for (int b = 0; b <= P; ++b)
        for (int c = 0; c <= P; ++c) {
          t[a][b][c] = -1;
          if (a + b + c > P) continue;
          t[a][b][c] = q;
          const int d = a + b + c;
          q += (P - d) / 2 + 1;  // m = d .. floor((P + d) / 2)
        }
  }
};

// Far-field coefficients of a cell from two of its moment sets X and Y (read at the moment
// layout [cell][2][NC]: the product's single and double layers, or the transposed
// product's Laplace and Yukawa charges): B[m, e](X) = sum over j with |j| = m - |e| and
// |e + 2j| <= P of prod_i c(e_i + 2 j_i, j_i) X_{e + 2j}, stored as interleaved pairs
// (B(X), B(Y)).  One thread per (cell, entry) of the cells [c0, ncell); the entry's terms
// come from a table built on the host (ptr, moment index, coefficient).
template <int P, typename Real>
__global__ void bcoef_kernel(int c0, int ncell, const int* __restrict__ tptr, const int* __restrict__ tk,
                             const double* __restrict__ tc, const Real* __restrict__ xa, const Real* __restrict__ xb,
                             Real* __restrict__ bco) {
  constexpr int NC = MI<P>::NC, NB = nb_of(P);
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)(ncell - c0) * NB) return;
  const int cell = c0 + (int)(g / NB), q = (int)(g - (long long)(cell - c0) * NB);
  const Real* __restrict__ X = xa + (size_t)cell * 2 * NC;
  const Real* __restrict__ Y = xb + (size_t)cell * 2 * NC;
  Real bm = 0, bd = 0;
  for (int u = tptr[q]; u < tptr[q + 1]; ++u) {
    const Real cf = (Real)tc[u];
    bm += cf * X[tk[u]];
    bd += cf * Y[tk[u]];
  }
  Real* o = bco + ((size_t)cell * NB + q) * 2;
  o[0] = bm;
  o[1] = bd;
}

// Entry t of a cell's staged coefficients, the pair (B(X), B(Y)).  When a cell's row is a
// whole number of 16-byte pieces (VEC) the row is read 16 bytes at a time (FP32: entries
// t and t + 1 together, so an unrolled pass issues one shared-memory load per two
// entries); otherwise element by element.
template <typename Real, bool VEC>
__device__ __forceinline__ void ld_entry(const Real* __restrict__ Bc, int t, Real& bx, Real& by) {
  if constexpr (VEC && sizeof(Real) == 4) {
    const float4 q = reinterpret_cast<const float4*>(Bc)[t >> 1];
    bx = (t & 1) ? q.z : q.x;
    by = (t & 1) ? q.w : q.y;
  } else if constexpr (VEC) {
    const double2 q = reinterpret_cast<const double2*>(Bc)[t];
    bx = q.x;
    by = q.y;
  } else {
    bx = Bc[2 * t];
    by = Bc[2 * t + 1];
  }
}

// Staging of the far-field kernels: one cell's coefficients are 2 NB values; groups of
// FW cells (even, 2..8) keep two staging buffers near 8 KB.
template <int P, typename Real>
struct FarShape {
  static constexpr int NB = nb_of(P);
  static constexpr int BYTES = 2 * NB * (int)sizeof(Real);  // one cell's coefficients
  static constexpr int FW0 = 8192 / (2 * BYTES);
  // cells per staged group: even, 2..8
  static constexpr int FW = FW0 >= 8 ? 8 : (FW0 < 2 ? 2 : (FW0 & ~1));
};

template <typename V>
void upload(DBuf<V>& d, const std::vector<V>& h, cudaStream_t s) {
  d.alloc(std::max<size_t>(1, h.size()));
  if (!h.empty()) BP_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, s));
}

// Terms of every far-field coefficient at order P (see bcoef_kernel), in the entry order
// of BIdx: for entry (m, e), the moments X_{e + 2j} with |j| = m - |e| and |e + 2j| <= P,
// each with the constant prod_i (-1)^{k_i} / (2^{j_i} j_i! (k_i - 2 j_i)!), k = e + 2j.
// CSR over the entries: ptr (NB + 1), moment index in the MI<P> order, constant.
template <int P>
void btab_terms(std::vector<int>& ptr, std::vector<int>& kk, std::vector<double>& cf) {
  constexpr MI<P> mi{};
  auto cu = [](int k, int j) {
    double d = 1.0;
    for (int q = 0; q < j; ++q) d *= 2.0 * (q + 1);  // 2^j j!
    for (int q = 2; q <= k - 2 * j; ++q) d *= q;     // (k - 2j)!
    return ((k & 1) ? -1.0 : 1.0) / d;
  };
  ptr.assign(1, 0);
  kk.clear();
  cf.clear();
  for (int a = 0; a <= P; ++a)
    for (int b = 0; b <= P; ++b)
      for (int c = 0; c <= P; ++c) {
        const int d = a + b + c;
        if (d > P) continue;
        for (int m = d; 2 * m - d <= P; ++m) {
          const int J = m - d;
          for (int j0 = 0; j0 <= J; ++j0)
            for (int j1 = 0; j0 + j1 <= J; ++j1) {
              const int j2 = J - j0 - j1;
              const int k0 = a + 2 * j0, k1 = b + 2 * j1, k2 = c + 2 * j2;
              if (k0 + k1 + k2 > P) continue;
              kk.push_back(mi.idx[k0][k1][k2]);
              cf.push_back(cu(k0, j0) * cu(k1, j1) * cu(k2, j2));
            }
          ptr.push_back((int)kk.size());
        }
      }
}

// The same table on the device, built once per order.
template <int P>
void build_btab(Tree::BTab& T, cudaStream_t s) {
  if (T.order == P) return;
  std::vector<int> ptr, kk;
  std::vector<double> cf;
  btab_terms<P>(ptr, kk, cf);
  if ((int)ptr.size() != nb_of(P) + 1) fail(BEMPOL_ERR_ARG, "far-field coefficient table has the wrong size");
  upload(T.ptr, ptr, s);
  upload(T.k, kk, s);
  upload(T.c, cf, s);
  T.order = P;
}

constexpr int NTB = 32;  // targets (one warp) per near-field block

}  // namespace

}  // namespace bp
