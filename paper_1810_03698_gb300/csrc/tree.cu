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
// Coefficients of a radial kernel G(r) = g(r^2/2) (Laplace 1/r; Yukawa e^{-kappa r}/r) in
// closed form: since d/dx_i acts on g(s), s = |Delta|^2/2, through s alone, each factor
// splits as a one-dimensional Hermite-type sum,
//     a_k = sum_{j <= k/2} prod_i u(k_i, j_i; Delta_i) g_{|k| - |j|},
//     u(k, j; x) = (-1)^k x^(k - 2j) / (2^j j! (k - 2j)!),   g_m = (1/r d/dr)^m G,
// with the radial sequences  Laplace  g_m = -(2m - 1) g_{m-1} / r^2,  g_0 = 1/r;
//                            Yukawa   g_0 = e^{-kappa r}/r,  g_1 = -(1 + kappa r) g_0 / r^2,
//                                     g_{m+1} = (kappa^2 g_{m-1} - (2m + 1) g_m) / r^2.
// Hence  V = sum_m g_m S_m(M),  K = sum_m g_m S_m(D),  S_m(M) = sum_{|k|-|j| = m} prod_i u M_k:
// the polynomial sums S_m do not depend on the kernel, so one pass over a cell's data
// serves the Laplace and the Yukawa single and double layers together.  Writing
// e = k - 2j, S_m is a polynomial in Delta with coefficients fixed per cell,
//     S_m(M) = sum_{|e| <= m, 2m - |e| <= P} Delta^e B_{m,e}(M),
//     B_{m,e}(M) = sum_{|j| = m - |e|, |e + 2j| <= P} prod_i c(e_i + 2j_i, j_i) M_{e + 2j},
// c(k, j) = (-1)^k / (2^j j! (k - 2j)!), so each product forms the B of every cell once
// from its moments and a (target, cell) term costs one product per monomial Delta^e and
// two FMAs per coefficient (80 coefficients per layer at P = 5).
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
#include <thread>
#include <vector>

#include "internal.h"

#include "tree_common.h"

namespace bp {

namespace {


// ---------------------------------------------------------------- far field
// One (target, cell) interaction, both kernels and both layers: the kernel-independent
// sums S_m = sum_e Delta^e B[m, e] of the cell's coefficients (B interleaved as
// (single layer, double layer) pairs), then the Laplace and Yukawa radial sequences.
// Fully unrolled for a compile-time order, so every table index is a constant.  lw = 1
// adds the Laplace terms (0: a cell of another body).
template <int P, typename Real>
__device__ __forceinline__ void far_eval(const Real D[3], const Real* __restrict__ Bc, Real kappa, Real kappa2,
                                         Real lw, Real& vl, Real& kl, Real& vy, Real& ky) {
  constexpr BIdx<P> bi{};
  Real SM[P + 1], SD[P + 1], py[P + 1], pz[P + 1];
#pragma unroll
  for (int m = 0; m <= P; ++m) SM[m] = SD[m] = (Real)0;
  py[0] = pz[0] = (Real)1;
#pragma unroll
  for (int e = 1; e <= P; ++e) {
    py[e] = py[e - 1] * D[1];
    pz[e] = pz[e - 1] * D[2];
  }
  Real px = (Real)1;
#pragma unroll
  for (int a = 0; a <= P; ++a) {
#pragma unroll
    for (int b = 0; b <= P; ++b) {  // fixed trip counts, so every index is a constant
      if (a + b > P) continue;
      const Real pab = px * py[b];
#pragma unroll
      for (int c = 0; c <= P; ++c) {
        if (a + b + c > P) continue;
        const Real w = pab * pz[c];
        const int d = a + b + c, t0 = bi.t[a][b][c];
#pragma unroll
        for (int m = 0; m <= P; ++m) {
          if (m < d || 2 * m - d > P) continue;
          const int t = t0 + (m - d);
          Real bm, bd;
          ld_entry<Real, (2 * nb_of(P) * sizeof(Real)) % 16 == 0>(Bc, t, bm, bd);
          SM[m] = fma(w, bm, SM[m]);
          SD[m] = fma(w, bd, SD[m]);
        }
      }
    }
    px *= D[0];
  }
  const Real r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
  const Real rinv = inv_sqrt(r2);
  const Real ir2 = rinv * rinv;
  // Laplace
  Real g = rinv, sV = g * SM[0], sK = g * SD[0];
#pragma unroll
  for (int m = 1; m <= P; ++m) {
    g *= (Real)(-(2.0 * m - 1.0)) * ir2;
    sV += g * SM[m];
    sK += g * SD[m];
  }
  vl += lw * sV;
  kl += lw * sK;
  // Yukawa
  const Real kr = kappa * (r2 * rinv);
  Real g0 = exp_neg(kr) * rinv;
  Real yV = g0 * SM[0], yK = g0 * SD[0];
  if constexpr (P >= 1) {
    Real g1 = -((Real)1 + kr) * g0 * ir2;
    yV += g1 * SM[1];
    yK += g1 * SD[1];
#pragma unroll
    for (int m = 1; m < P; ++m) {
      const Real g2 = (kappa2 * g0 - (Real)(2.0 * m + 1.0) * g1) * ir2;
      yV += g2 * SM[m + 1];
      yK += g2 * SD[m + 1];
      g0 = g1;
      g1 = g2;
    }
  }
  vy += yV;
  ky += yK;
}

// Far field, one warp per block of <= 16 targets of one leaf.  Lane l serves target
// (l & 15); the two half-warps take alternate cells of the batch's far list (half h the
// cells h, h + 2, ... of every staged group) and their sums are added at the end.  Each
// warp stages its own groups of cells' coefficients (2 NB values per cell) with
// cp.async, double-buffered, and waits only for its own copies (no block-wide barrier:
// a warp never waits for another).  The group size keeps the two buffers near 8 KB.
// lap (NULL: every cell) marks the far-list entries whose cell lies in the target's own
// body, the only ones with Laplace terms.
template <int P, typename Real>
__global__ void __launch_bounds__(32) far16_kernel(const int4* __restrict__ blk, const double4* __restrict__ tgt64,
                                                   const int* __restrict__ leaf_cell,
                                                   const double4* __restrict__ center,
                                                   const int* __restrict__ far_ptr, const int* __restrict__ far_list,
                                                   const int* __restrict__ lap, const Real* __restrict__ bco,
                                                   Real kappa, int n, const int* __restrict__ active,
                                                   const int* __restrict__ leaf_sys, double* __restrict__ out) {
  constexpr int NB = FarShape<P, Real>::NB, FW = FarShape<P, Real>::FW;
  // cp.async when a cell's coefficients are a whole number of 16-byte pieces
  constexpr bool ASYNC = (2 * NB * sizeof(Real)) % 16 == 0;
  constexpr int CH = (int)(2 * NB * sizeof(Real) / 16);  // 16-byte pieces per cell
  __shared__ __align__(16) Real sm[2][FW][2 * NB];
  __shared__ Real so[2][FW][4];
  const int lane = threadIdx.x, h = lane >> 4, tl = lane & 15;
  const int4 B = blk[blockIdx.x];
  const int leaf = B.x;
  if (active && !active[leaf_sys[leaf]]) return;
  const double4 ct = center[leaf_cell[leaf]];
  const int i = B.y + tl;
  const bool act = tl < B.z;
  Real xr[3] = {0, 0, 0};
  if (act) {
    const double4 x = tgt64[i];
    xr[0] = (Real)(x.x - ct.x);
    xr[1] = (Real)(x.y - ct.y);
    xr[2] = (Real)(x.z - ct.z);
  }
  const Real kappa2 = kappa * kappa;
  double aVL = 0, aKL = 0, aVY = 0, aKY = 0;
  const int f0 = far_ptr[B.w], f1 = far_ptr[B.w + 1];  // the batch's own far list
  auto stage = [&](int b, int fb) {
    const int cnt = min(FW, f1 - fb);
    if constexpr (ASYNC) {
      for (int q = lane; q < cnt * CH; q += 32) {
        const int cell = q / CH, piece = q - cell * CH;
        const char* g = reinterpret_cast<const char*>(bco + (size_t)far_list[fb + cell] * 2 * NB) + 16 * piece;
        cp_async16(reinterpret_cast<char*>(&sm[b][cell][0]) + 16 * piece, g);
      }
      cp_async_commit();
    } else {
      for (int q = lane; q < cnt * 2 * NB; q += 32)
        sm[b][q / (2 * NB)][q % (2 * NB)] = bco[(size_t)far_list[fb + q / (2 * NB)] * 2 * NB + q % (2 * NB)];
    }
    if (lane < cnt) {
      const double4 cc = center[far_list[fb + lane]];
      so[b][lane][0] = (Real)(ct.x - cc.x);
      so[b][lane][1] = (Real)(ct.y - cc.y);
      so[b][lane][2] = (Real)(ct.z - cc.z);
      so[b][lane][3] = lap ? (Real)lap[fb + lane] : (Real)1;
    }
  };
  if (f0 < f1) stage(0, f0);
  int b = 0;
  for (int fb = f0; fb < f1; fb += FW, b ^= 1) {
    const int cnt = min(FW, f1 - fb);
    if constexpr (ASYNC) cp_async_wait_all();  // this lane's pieces of group b
    __syncwarp();  // every lane's pieces and offsets of group b; all done with the other buffer
    if (fb + FW < f1) stage(b ^ 1, fb + FW);
    Real vl = 0, kl = 0, vy = 0, ky = 0;
    for (int q = h; q < cnt; q += 2) {
      const Real D[3] = {xr[0] + so[b][q][0], xr[1] + so[b][q][1], xr[2] + so[b][q][2]};
      far_eval<P, Real>(D, sm[b][q], kappa, kappa2, so[b][q][3], vl, kl, vy, ky);
    }
    aVL += (double)vl;
    aKL += (double)kl;
    aVY += (double)vy;
    aKY += (double)ky;
  }
  aVL += __shfl_down_sync(0xffffffffu, aVL, 16);
  aKL += __shfl_down_sync(0xffffffffu, aKL, 16);
  aVY += __shfl_down_sync(0xffffffffu, aVY, 16);
  aKY += __shfl_down_sync(0xffffffffu, aKY, 16);
  if (h == 0 && act) {
    out[i] = aVL;
    out[(size_t)n + i] = aKL;
    out[2 * (size_t)n + i] = aVY;
    out[3 * (size_t)n + i] = aKY;
  }
}

// ---------------------------------------------------------------- near field
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

// ---------------------------------------------------------------- FP32 near field
// Sixteen targets per warp, paired FP32 arithmetic, sources staged by 1-D bulk copies.
//
// Source records: the Gauss nodes of every leaf, taken two at a time (a leaf with an odd
// count gets a padding node far away with zero strength), stored side by side in every
// component: positions relative to the node's own leaf centre PA = (x0, x1, y0, y1),
// PB = (z0, z1, 0, 0) (once per mesh), strengths SA = (m0, m1, d0x, d1x),
// SB = (d0y, d1y, d0z, d1z) (once per product).  Leaf L owns the pairs
// [pair_ptr[L], pair_ptr[L+1]).
//
// Lane l serves target (l & 15) of a block of <= 16 targets of one leaf; the two
// half-warps take alternate pairs of every staged chunk and their sums are added at the
// end, so a leaf's last, partly filled block leaves at most 15 of 32 lanes idle (with 32
// targets per warp the idle share at leaf size 256 is about twice as large).  For each
// near leaf the target is put in that leaf's frame once (x - c_L, formed in FP64), so the
// loop over its sources is the pair formula alone: every FP32 operation runs as one
// f32x2 instruction for the two nodes of a pair (sm_100 family), only the reciprocal
// square root and 2^x stay one per node.  Chunks of CP pairs are copied into shared
// memory by lane 0 with cp.async.bulk (completion on an mbarrier), double-buffered, so
// the next chunk is in flight while the current one is summed.  Every wait on an
// mbarrier is bounded: past MBAR_SPIN polls the kernel sets *err, waits (bounded) for
// its other copy in flight and returns without writing.
//
// The leaf itself is the only near leaf whose nodes can coincide with a target (the
// centroid node of the target's own panel), so only its sums carry the r = 0 test (a
// coincident pair of different panels is rejected when the near table is built).  Block
// (leaf, first, count, batch) takes the near list of its batch, cut into gridDim.y
// consecutive pieces; piece s writes its partial sums to out + s * 4n (the combine
// kernel adds the pieces in order).
// Registers are bounded for 24 resident one-warp blocks per SM (80 per thread, six warps
// per scheduler), which hides more of the pair formula's dependent latencies.
constexpr int CP = 64;             // source pairs per staged chunk
constexpr float FAR_PAD = 1.0e4f;  // leaf-relative position of a padding node (zero strength)
constexpr int MBAR_SPIN = 1 << 20; // polls of an mbarrier before a wait is declared failed

typedef unsigned long long f2;  // two FP32 values in one 64-bit register (low = first)

__device__ __forceinline__ f2 pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// mbarrier and 1-D bulk copy (global -> this CTA's shared memory), sm_90 and later
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (int it = 0; it < MBAR_SPIN; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

struct NearChunk {
  float4 PA[CP], PB[CP], SA[CP], SB[CP];
};

template <bool SELF>
__device__ __forceinline__ void pair_x2(f2 X, f2 Y, f2 Z, const NearChunk& T, int m, f2 PW, f2 K2, f2 NK2,
                                        f2 ONE2, f2* a) {
  const float4 va = T.PA[m], vb = T.PB[m], vc = T.SA[m], vd = T.SB[m];
  const f2 dx = sub2(X, pk(va.x, va.y)), dy = sub2(Y, pk(va.z, va.w)), dz = sub2(Z, pk(vb.x, vb.y));
  const f2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
  float r2a, r2b;
  upk(r2, r2a, r2b);
  float ra = rsqrt_approx(r2a), rb = rsqrt_approx(r2b);
  if (SELF) {
    ra = r2a > 0.f ? ra : 0.f;
    rb = r2b > 0.f ? rb : 0.f;
  }
  const f2 rinv = pk(ra, rb);
  const f2 r = mul2(r2, rinv);
  float ea, eb;
  upk(mul2(r, NK2), ea, eb);
  const f2 e = pk(exp2_approx(ea), exp2_approx(eb));
  const f2 mr = mul2(pk(vc.x, vc.y), rinv);
  a[0] = fma2(mr, PW, a[0]);
  a[2] = fma2(mr, e, a[2]);
  const f2 dR = fma2(pk(vc.z, vc.w), dx, fma2(pk(vd.x, vd.y), dy, mul2(pk(vd.z, vd.w), dz)));
  const f2 t = mul2(mul2(dR, mul2(rinv, rinv)), rinv);
  a[1] = fma2(t, PW, a[1]);
  a[3] = fma2(mul2(t, fma2(K2, r, ONE2)), e, a[3]);
}

// pairs h, h + 2, h + 4, ... of a staged chunk of `cnt` pairs
template <bool SELF>
__device__ __forceinline__ void chunk_x2(f2 X, f2 Y, f2 Z, const NearChunk& T, int h, int cnt, f2 PW, f2 K2, f2 NK2,
                                         f2 ONE2, f2* a) {
  if (cnt == CP) {
#pragma unroll 4
    for (int m = h; m < CP; m += 2) pair_x2<SELF>(X, Y, Z, T, m, PW, K2, NK2, ONE2, a);
  } else {
    for (int m = h; m < cnt; m += 2) pair_x2<SELF>(X, Y, Z, T, m, PW, K2, NK2, ONE2, a);
  }
}

__global__ void __launch_bounds__(32, 24) near16_kernel(const int4* __restrict__ blk, const double4* __restrict__ tgt64,
                                                    const int* __restrict__ leaf_cell,
                                                    const double4* __restrict__ center,
                                                    const int* __restrict__ near_ptr,
                                                    const int* __restrict__ near_list,
                                                    const int* __restrict__ pair_ptr, const float4* __restrict__ PA,
                                                    const float4* __restrict__ PB, const float4* __restrict__ SA,
                                                    const float4* __restrict__ SB, float kappa, float nk_log2e, int n,
                                                    const int* __restrict__ active, const int* __restrict__ leaf_sys,
                                                    double* __restrict__ out, int* __restrict__ err) {
  __shared__ __align__(128) NearChunk st[2];
  __shared__ __align__(8) unsigned long long bar[2];
  const int lane = threadIdx.x, h = lane >> 4, tl = lane & 15;
  const int4 B = blk[blockIdx.x];
  const int leaf = B.x;
  if (active && !active[leaf_sys[leaf]]) return;
  const int i = B.y + tl;
  const bool act = tl < B.z;
  const double4 x = tgt64[act ? i : B.y];
  const f2 K2 = pk(kappa, kappa), NK2 = pk(nk_log2e, nk_log2e), ONE2 = pk(1.f, 1.f);
  const unsigned b0 = smem_addr(&bar[0]), b1 = smem_addr(&bar[1]);
  if (lane == 0) {
    mbar_init(b0, 1);
    mbar_init(b1, 1);
    mbar_init_fence();
  }
  __syncwarp();
  const int base = near_ptr[B.w];  // the batch's own near list
  const int nl = near_ptr[B.w + 1] - base;
  const int e0 = base + (int)(((long long)nl * blockIdx.y) / gridDim.y);
  const int e1 = base + (int)(((long long)nl * (blockIdx.y + 1)) / gridDim.y);
  // lane 0 copies chunk (pairs [p, p + cnt)) into buffer b
  auto issue = [&](int b, int p, int cnt) {
    if (lane == 0) {
      const unsigned bb = b ? b1 : b0;
      const unsigned bytes = (unsigned)cnt * 16u;
      fence_proxy_async_smem();  // earlier generic reads of this buffer before the async writes
      mbar_expect_tx(bb, 4u * bytes);
      bulk_copy_g2s(smem_addr(st[b].PA), PA + p, bytes, bb);
      bulk_copy_g2s(smem_addr(st[b].PB), PB + p, bytes, bb);
      bulk_copy_g2s(smem_addr(st[b].SA), SA + p, bytes, bb);
      bulk_copy_g2s(smem_addr(st[b].SB), SB + p, bytes, bb);
    }
  };
  // items: chunks (entry e, pairs [p, min(p + CP, pe))) of the near leaves of this piece
  int ce = e0, cp_ = 0, cpe = 0;  // current entry, chunk start, end of its leaf's pairs
  if (ce < e1) {
    const int L = near_list[ce] & ~NEAR_CROSS;
    cp_ = pair_ptr[L];
    cpe = pair_ptr[L + 1];
    issue(0, cp_, min(CP, cpe - cp_));
  }
  double acc[4] = {0, 0, 0, 0};
  f2 f[4] = {0ull, 0ull, 0ull, 0ull};
  unsigned ph0 = 0u, ph1 = 0u;  // parity of the next completion of each buffer's barrier
  int b = 0, cur_e = -1, nsum = 0;
  bool self = false;
  f2 X = 0ull, Y = 0ull, Z = 0ull, PW = 0ull;
  auto flush = [&]() {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float lo_, hi_;
      upk(f[c], lo_, hi_);
      acc[c] += (double)lo_ + (double)hi_;
      f[c] = 0ull;
    }
    nsum = 0;
  };
  while (ce < e1) {
    const int ccnt = min(CP, cpe - cp_);
    // the next chunk: the rest of this leaf, else the next entry's leaf
    int ne = ce, np = cp_ + CP, npe = cpe;
    if (np >= cpe) {
      ++ne;
      if (ne < e1) {
        const int L = near_list[ne] & ~NEAR_CROSS;
        np = pair_ptr[L];
        npe = pair_ptr[L + 1];
      }
    }
    if (ne < e1) issue(b ^ 1, np, min(CP, npe - np));
    if (ce != cur_e) {  // a new near leaf: the target in its frame, its Laplace weight
      flush();
      cur_e = ce;
      const int ent = near_list[ce];
      const int L = ent & ~NEAR_CROSS;
      const double4 cs = center[leaf_cell[L]];
      const float xl = (float)(x.x - cs.x), yl = (float)(x.y - cs.y), zl = (float)(x.z - cs.z);
      X = pk(xl, xl);
      Y = pk(yl, yl);
      Z = pk(zl, zl);
      const float w = (ent & NEAR_CROSS) ? 0.f : 1.f;
      PW = pk(w, w);
      self = L == leaf;
    }
    if (!mbar_wait(b ? b1 : b0, b ? ph1 : ph0)) {
      atomicExch(err, 1);
      if (ne < e1) mbar_wait(b ? b0 : b1, b ? ph0 : ph1);  // the other copy in flight
      return;
    }
    if (b)
      ph1 ^= 1u;
    else
      ph0 ^= 1u;
    if (self)
      chunk_x2<true>(X, Y, Z, st[b], h, ccnt, PW, K2, NK2, ONE2, f);
    else
      chunk_x2<false>(X, Y, Z, st[b], h, ccnt, PW, K2, NK2, ONE2, f);
    if (++nsum == 2) flush();  // FP32 sums over at most 64 nodes per slot and lane, then FP64
    __syncwarp();              // every lane is done with buffer b before it is refilled
    ce = ne;
    cp_ = np;
    cpe = npe;
    b ^= 1;
  }
  flush();
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], 16);
  if (h == 0 && act) {
    double* o = out + (size_t)blockIdx.y * 4 * n;
    o[i] = acc[0];
    o[n + i] = acc[1];
    o[2 * n + i] = acc[2];
    o[3 * n + i] = acc[3];
  }
}

// FP64 near field of the forward product over the same 16-target batches and near
// lists as the FP32 kernel: lane l serves target (l & 15), the two half-warps take
// alternate nodes of every staged tile of 64 nodes of one near leaf, FP64 pair terms and
// sums, the r = 0 test everywhere (FP64 throughput, not issue, bounds this kernel).
__global__ void __launch_bounds__(32) near16d_kernel(const int4* __restrict__ blk, const double4* __restrict__ tgt64,
                                                     const int* __restrict__ leaf_cell,
                                                     const int* __restrict__ begin, const int* __restrict__ end,
                                                     const int* __restrict__ near_ptr,
                                                     const int* __restrict__ near_list, int K,
                                                     const double4* __restrict__ src64,
                                                     const double4* __restrict__ str, double kappa, int n,
                                                     const int* __restrict__ active, const int* __restrict__ leaf_sys,
                                                     double* __restrict__ out) {
  __shared__ double4 sp[64];
  __shared__ double4 ss[64];
  const int lane = threadIdx.x, h = lane >> 4, tl = lane & 15;
  const int4 B = blk[blockIdx.x];
  if (active && !active[leaf_sys[B.x]]) return;
  const int i = B.y + tl;
  const bool act = tl < B.z;
  const double4 xt = tgt64[act ? i : B.y];
  const double x[3] = {xt.x, xt.y, xt.z};
  double acc[4] = {0, 0, 0, 0};
  const int base = near_ptr[B.w];
  const int nl = near_ptr[B.w + 1] - base;
  const int e0 = base + (int)(((long long)nl * blockIdx.y) / gridDim.y);
  const int e1 = base + (int)(((long long)nl * (blockIdx.y + 1)) / gridDim.y);
  for (int e = e0; e < e1; ++e) {
    const int ent = near_list[e];
    const int cl = leaf_cell[ent & ~NEAR_CROSS];
    const double w = (ent & NEAR_CROSS) ? 0.0 : 1.0;
    const int s0 = begin[cl] * K, s1 = end[cl] * K;
    for (int t0 = s0; t0 < s1; t0 += 64) {
      __syncwarp();  // the previous tile is done
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = t0 + 32 * u + lane;
        if (j < s1) {
          double4 y = src64[j];
          y.w = w;
          sp[32 * u + lane] = y;
          ss[32 * u + lane] = str[j];
        }
      }
      __syncwarp();
      const int lim = min(64, s1 - t0);
      for (int k = h; k < lim; k += 2)
        pair_accum(x, sp[k], ss[k], kappa, 0.0, acc[0], acc[1], acc[2], acc[3]);
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], 16);
  if (h == 0 && act) {
    double* o = out + (size_t)blockIdx.y * 4 * n;
    o[i] = acc[0];
    o[n + i] = acc[1];
    o[2 * n + i] = acc[2];
    o[3 * n + i] = acc[3];
  }
}

// source-pair records of the FP32 near field: positions once per mesh, strengths per
// product (pair_src[p] = first node of pair p, negative (~node) when the second is padding)
__global__ void pair_pos_kernel(const int* __restrict__ pair_src, int npair, const float4* __restrict__ rel,
                                float4* __restrict__ PA, float4* __restrict__ PB) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npair) return;
  const int q = pair_src[p];
  const float4 a = rel[q < 0 ? ~q : q];
  const float4 b = q < 0 ? make_float4(FAR_PAD, FAR_PAD, FAR_PAD, 0.f) : rel[q + 1];
  PA[p] = make_float4(a.x, b.x, a.y, b.y);
  PB[p] = make_float4(a.z, b.z, 0.f, 0.f);
}

__global__ void pair_str_kernel(const int* __restrict__ pair_src, int npair, const float4* __restrict__ str,
                                float4* __restrict__ SA, float4* __restrict__ SB) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npair) return;
  const int q = pair_src[p];
  const float4 a = str[q < 0 ? ~q : q];
  const float4 b = q < 0 ? make_float4(0.f, 0.f, 0.f, 0.f) : str[q + 1];
  SA[p] = make_float4(a.x, b.x, a.y, b.y);
  SB[p] = make_float4(a.z, b.z, a.w, b.w);
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


// Interaction lists of the forward product's target batches (the 16-target blocks of
// the FP32 and FP64 near and far kernels): batch b holds the targets [first, first +
// count) of one leaf, and a cell C is accepted for it when R_C < theta (|c_b - c_C| - R_b)
// with (c_b, R_b) the bounding sphere of the batch's own collocation points, so every
// target satisfies the paper's criterion theta > R_C / r and a small batch accepts
// cells closer to its targets than its whole leaf could (fewer near pairs and far
// terms).  Cells of another system are skipped, cells of another body of the same
// system enter the Yukawa lists only, the multi-group root and any cell holding the
// batch are opened; the leaf of the batch comes first in its near list.  Built on
// several host threads, each over a contiguous range of batches.
struct BatchLists {
  std::vector<int> fptr, fl, lptr, ll, nptr, nl;
  long long pairs = 0, fars = 0, farsL = 0;
};

static void batch_lists(const Ctx& c, const std::vector<int4>& batches, const std::vector<double4>& h_tgt,
                        const std::vector<int>& leaf_of, BatchLists& out) {
  const Tree& T = c.tree;
  const double theta = c.par.theta;
  const int nb = (int)batches.size();
  unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  nth = std::min<unsigned>(nth, (unsigned)std::max(1, nb / 64));
  std::vector<BatchLists> part(nth);
  auto work = [&](unsigned w) {
    BatchLists& o = part[w];
    const int b0 = (int)((long long)nb * w / nth), b1 = (int)((long long)nb * (w + 1) / nth);
    std::vector<int> stack;
    o.fptr.push_back(0);
    o.lptr.push_back(0);
    o.nptr.push_back(0);
    for (int bi = b0; bi < b1; ++bi) {
      const int4 B = batches[bi];
      const int leaf = B.x, first = B.y, cnt = B.z;
      const int ct = T.h_leaf_cell[leaf];
      const int g = T.h_cell_grp[ct];
      const int sy = c.h_grp_sys[g];
      double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
      for (int i = first; i < first + cnt; ++i) {
        const double v[3] = {h_tgt[i].x, h_tgt[i].y, h_tgt[i].z};
        for (int d = 0; d < 3; ++d) {
          lo[d] = std::min(lo[d], v[d]);
          hi[d] = std::max(hi[d], v[d]);
        }
      }
      const double ax = 0.5 * (lo[0] + hi[0]), ay = 0.5 * (lo[1] + hi[1]), az = 0.5 * (lo[2] + hi[2]);
      double rb = 0.0;
      for (int i = first; i < first + cnt; ++i) {
        const double dx = h_tgt[i].x - ax, dy = h_tgt[i].y - ay, dz = h_tgt[i].z - az;
        rb = std::max(rb, std::sqrt(dx * dx + dy * dy + dz * dz));
      }
      const size_t nl0 = o.nl.size();
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
        const double4 cc = T.h_center[q];
        const double dx = ax - cc.x, dy = ay - cc.y, dz = az - cc.z;
        const double gap = std::sqrt(dx * dx + dy * dy + dz * dz) - rb;
        const bool holds = T.h_begin[q] <= first && first + cnt <= T.h_end[q];
        if (!holds && gap > 0.0 && cc.w < theta * gap) {
          o.fl.push_back(q);
          o.fars += cnt;
          if (cg == g) {
            o.ll.push_back(q);
            o.farsL += cnt;
          }
        } else if (T.h_nchild[q] == 0) {
          o.nl.push_back(leaf_of[q] | (cg == g ? 0 : NEAR_CROSS));
          o.pairs += (long long)cnt * (T.h_end[q] - T.h_begin[q]) * c.K;
        } else {
          for (int k = T.h_nchild[q] - 1; k >= 0; --k) stack.push_back(T.h_child0[q] + k);
        }
      }
      for (size_t e = nl0; e < o.nl.size(); ++e)
        if (o.nl[e] == leaf) {
          std::rotate(o.nl.begin() + nl0, o.nl.begin() + e, o.nl.begin() + e + 1);
          break;
        }
      o.fptr.push_back((int)o.fl.size());
      o.lptr.push_back((int)o.ll.size());
      o.nptr.push_back((int)o.nl.size());
    }
  };
  std::vector<std::thread> th;
  for (unsigned w = 1; w < nth; ++w) th.emplace_back(work, w);
  work(0);
  for (auto& t : th) t.join();
  out = BatchLists();
  out.fptr.assign(1, 0);
  out.lptr.assign(1, 0);
  out.nptr.assign(1, 0);
  for (const BatchLists& o : part) {
    const int f0 = (int)out.fl.size(), l0 = (int)out.ll.size(), n0 = (int)out.nl.size();
    for (size_t k = 1; k < o.fptr.size(); ++k) {
      out.fptr.push_back(f0 + o.fptr[k]);
      out.lptr.push_back(l0 + o.lptr[k]);
      out.nptr.push_back(n0 + o.nptr[k]);
    }
    out.fl.insert(out.fl.end(), o.fl.begin(), o.fl.end());
    out.ll.insert(out.ll.end(), o.ll.begin(), o.ll.end());
    out.nl.insert(out.nl.end(), o.nl.begin(), o.nl.end());
    out.pairs += o.pairs;
    out.fars += o.fars;
    out.farsL += o.farsL;
  }
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
  std::vector<int4> blk, blk32, blk16;
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
      // a cell holding the target leaf is never accepted (possible only for theta >= 1)
      const bool holds = T.h_begin[q] <= T.h_begin[ct] && T.h_end[ct] <= T.h_end[q];
      if (!holds && gap > 0.0 && b.w < theta * gap) {
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
    // the leaf itself first in its near list (the FP32 near kernel sums it in a pass of its own)
    for (size_t e = (size_t)nptr[l]; e < nlist.size(); ++e)
      if (nlist[e] == l) {
        std::rotate(nlist.begin() + nptr[l], nlist.begin() + e, nlist.begin() + e + 1);
        break;
      }
    fptr[l + 1] = (int)flist.size();
    lptr[l + 1] = (int)llist.size();
    nptr[l + 1] = (int)nlist.size();
    for (int off = 0; off < ntgt; off += TBT)
      blk.push_back(make_int4(l, T.h_begin[ct] + off, std::min(TBT, ntgt - off), 0));
    for (int off = 0; off < ntgt; off += 32)
      blk32.push_back(make_int4(l, T.h_begin[ct] + off, std::min(32, ntgt - off), 0));
    for (int off = 0; off < ntgt; off += 16)
      blk16.push_back(make_int4(l, T.h_begin[ct] + off, std::min(16, ntgt - off), 0));
  }
  // lists of the 16-target batches of the forward product (batch id = blk16[.].w)
  {
    std::vector<double4> h_tgt(c.n);
    BP_CUDA(cudaMemcpyAsync(h_tgt.data(), c.tgt64.p, sizeof(double4) * c.n, cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaStreamSynchronize(s));
    for (size_t b = 0; b < blk16.size(); ++b) blk16[b].w = (int)b;
    BatchLists BL;
    batch_lists(c, blk16, h_tgt, leaf_of, BL);
    std::vector<long long> bnear(blk16.size(), 0), bfar(blk16.size(), 0);
    for (size_t b = 0; b < blk16.size(); ++b) {
      bfar[b] = BL.fptr[b + 1] - BL.fptr[b];
      for (int e = BL.nptr[b]; e < BL.nptr[b + 1]; ++e) {
        const int q = T.h_leaf_cell[BL.nl[e] & ~NEAR_CROSS];
        bnear[b] += T.h_end[q] - T.h_begin[q];
      }
    }
    T.h_batch = blk16;
    T.h_batch_cost.assign(blk16.size(), 0.0);
    T.h_batch_pairs.assign(blk16.size(), 0);
    T.h_batch_far.assign(blk16.size(), 0);
    for (size_t b = 0; b < blk16.size(); ++b) {
      T.h_batch_pairs[b] = bnear[b] * c.K * blk16[b].z;
      T.h_batch_far[b] = bfar[b] * blk16[b].z;
      // a far term costs about 16 pair terms (464 against 30 flops at order 5)
      T.h_batch_cost[b] = (double)T.h_batch_pairs[b] + 16.0 * (double)T.h_batch_far[b];
    }
    std::vector<int4> bf = blk16;
    // largest blocks first: the grids are a few waves deep, so launching the long blocks
    // early shortens the tail (a block's result does not depend on the order)
    std::stable_sort(blk16.begin(), blk16.end(), [&](const int4& u, const int4& v) { return bnear[u.w] > bnear[v.w]; });
    std::stable_sort(bf.begin(), bf.end(), [&](const int4& u, const int4& v) { return bfar[u.w] > bfar[v.w]; });
    T.h_blk16 = blk16;
    T.h_blk16f = bf;
    T.nblk16 = (int)blk16.size();
    T.nblk16f = (int)bf.size();
    T.near_splits16 = std::max(1, std::min(4, cdiv((long long)num_sms(c.device) * 56, std::max(1, T.nblk16))));
    upload(T.blk16, blk16, s);
    upload(T.blk16f, bf, s);
    upload(T.bfar_ptr, BL.fptr, s);
    upload(T.bfar_list, BL.fl, s);
    T.bfarL_same = BL.ll.size() == BL.fl.size();
    if (!T.bfarL_same) {
      // Laplace flag of every far-list entry: the cell lies in the batch's own body
      std::vector<int> lapf(BL.fl.size());
      for (size_t bb = 0; bb < blk16.size(); ++bb) {
        const int gb = T.h_cell_grp[T.h_leaf_cell[blk16[bb].x]];
        const int w = blk16[bb].w;
        for (int e = BL.fptr[w]; e < BL.fptr[w + 1]; ++e) lapf[e] = T.h_cell_grp[BL.fl[e]] == gb ? 1 : 0;
      }
      upload(T.bfar_lap, lapf, s);
    }
    upload(T.bnear_ptr, BL.nptr, s);
    upload(T.bnear_list, BL.nl, s);
    T.bpairs_per_matvec = BL.pairs;
    T.bfar_per_matvec = BL.fars;
    // shallowest tree depth that holds a cell of a batch far list
    T.bm2m_min_depth = T.ndepth;
    for (int q : BL.fl) {
      int d = 0;
      while (d + 1 < T.ndepth && T.h_depth_begin[d + 1] <= q) ++d;
      T.bm2m_min_depth = std::min(T.bm2m_min_depth, d);
    }
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
  if (!T.farL_same) {  // Laplace flag of every far-list entry: the cell lies in the leaf's own body
    std::vector<int> lapf(flist.size());
    for (int l = 0; l < T.nleaf; ++l) {
      const int gl = T.h_cell_grp[T.h_leaf_cell[l]];
      for (int e = fptr[l]; e < fptr[l + 1]; ++e) lapf[e] = T.h_cell_grp[flist[e]] == gl ? 1 : 0;
    }
    upload(T.far_lap, lapf, s);
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
  constexpr bool F64 = sizeof(Real) == 8;
  constexpr int NC = MI<P>::NC, NB = nb_of(P);
  if (T.mom_order != P || mom.n < (size_t)T.ncell * 2 * NC) {
    mom.alloc((size_t)T.ncell * 2 * NC);
    T.mom_order = P;
  }
  DBuf<Real>* bco;
  if constexpr (F64)
    bco = &T.bco64;
  else
    bco = &T.bco32;
  if (bco->n < (size_t)T.ncell * 2 * NB) bco->alloc((size_t)T.ncell * 2 * NB);
  build_btab<P>(T.btab, s);
  typedef typename Vec4<Real>::T R4;
  const R4* str = nullptr;
  if (sizeof(Real) == 4)
    str = reinterpret_cast<const R4*>(c.str32.p);
  else
    str = reinterpret_cast<const R4*>(c.str64.p);
  // this rank's blocks when the rows are sharded over several GPUs
  const bool sh = c.sh_world > 1;
  if (sh && !c.sh_ready) build_shard(c, s);
  const int4* b16 = sh ? c.sh_blk16.p : T.blk16.p;
  const int4* b16f = sh ? c.sh_blk16f.p : T.blk16f.p;
  const int nb16 = sh ? c.sh_nblk16 : T.nblk16, nb16f = sh ? c.sh_nblk16f : T.nblk16f;
  const int S = T.near_splits16;
  const size_t need = (size_t)(S + 1) * 4 * c.n;
  if (c.part.n < need) c.part.alloc(need);
  const Real kappa = (Real)c.par.kappa;
  const float nk = (float)(-c.par.kappa * 1.4426950408889634);
  // Fork: the far-field chain (moments, M2M shifts, far kernels) on the context's
  // high-priority side stream, the near field on `s`; the near kernel needs no moments,
  // so its blocks fill the SMs that the small M2M grids and the far kernels' last wave
  // leave idle.  The two write disjoint pieces of c.part.  Both precisions use the
  // interaction lists of the 16-target batches.
  c.ensure_aux();
  const cudaStream_t sf = c.aux;
  // accounting: FP32 products per kernel (pair, far) and whole; FP64 products (the
  // refinement residuals) whole only, under their own kind
  Ctx::Timed tp;
  c.time_begin(F64 ? 6 : 2, s, tp);
  BP_CUDA(cudaEventRecord(c.ev_fork, s));
  BP_CUDA(cudaStreamWaitEvent(sf, c.ev_fork, 0));
  launch(leaf_moments_kernel<P, Real>, T.nleaf, MomShape<P>::TPB, 0, sf, T.leaf_cell.p, T.begin.p, T.end.p,
         T.center.p, c.K, c.src64.p, str, c.mv_active, T.leaf_sys.p, mom.p);
  for (int d = T.ndepth - 2; d >= T.bm2m_min_depth; --d) {  // depths above are in no far list
    const int first = T.h_depth_begin[d], cnt = T.h_depth_begin[d + 1] - first;
    launch(m2m_kernel<P, Real>, cnt, M2M_TPB, 0, sf, first, T.child0.p, T.nchild.p, T.center.p, mom.p);
  }
  {  // far-field coefficients of the cells that far lists can hold
    const int cb = T.h_depth_begin[T.bm2m_min_depth];
    if (cb < T.ncell)
      launch(bcoef_kernel<P, Real>, cdiv((long long)(T.ncell - cb) * NB, 256), 256, 0, sf, cb, T.ncell,
             T.btab.ptr.p, T.btab.k.p, T.btab.c.p, mom.p, mom.p + NC, bco->p);
  }
  Ctx::Timed tf;
  if (!F64) {
    c.time_begin(1, sf, tf);
    c.stat_far += sh ? c.sh_far : T.bfar_per_matvec;
  }
  double* far_out = c.part.p + (size_t)S * 4 * c.n;
  {  // one-warp blocks: the largest shared-memory carveout, so that shared memory does not
     // cap the resident blocks below the register limit (once per device and instantiation)
    static bool carve[64] = {};
    if (c.device >= 0 && c.device < 64 && !carve[c.device]) {
      BP_CUDA(cudaFuncSetAttribute(far16_kernel<P, Real>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared));
      carve[c.device] = true;
    }
  }
  launch(far16_kernel<P, Real>, nb16f, 32, 0, sf, b16f, c.tgt64.p, T.leaf_cell.p, T.center.p, T.bfar_ptr.p,
         T.bfar_list.p, T.bfarL_same ? nullptr : T.bfar_lap.p, bco->p, kappa, c.n, c.mv_active, T.leaf_sys.p,
         far_out);
  if (!F64) c.time_end(sf, tf);
  Ctx::Timed tm;
  if (!F64) {
    c.time_begin(0, s, tm);
    c.stat_pairs += sh ? c.sh_pairs : T.bpairs_per_matvec;
  }
  if constexpr (F64) {
    launch(near16d_kernel, dim3(nb16, S), 32, 0, s, b16, c.tgt64.p, T.leaf_cell.p, T.begin.p, T.end.p,
           T.bnear_ptr.p, T.bnear_list.p, c.K, c.src64.p, str, (double)kappa, c.n, c.mv_active, T.leaf_sys.p,
           c.part.p);
  } else {
    launch(pair_str_kernel, cdiv(T.npair, 256), 256, 0, s, T.pair_src.p, T.npair, c.str32.p, T.pairSA.p,
           T.pairSB.p);
    static bool carve[64] = {};  // as for the far kernel: shared memory must not cap the resident blocks
    if (c.device >= 0 && c.device < 64 && !carve[c.device]) {
      BP_CUDA(cudaFuncSetAttribute(near16_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   (int)cudaSharedmemCarveoutMaxShared));
      carve[c.device] = true;
    }
    launch(near16_kernel, dim3(nb16, S), 32, 0, s, b16, c.tgt64.p, T.leaf_cell.p, T.center.p,
           T.bnear_ptr.p, T.bnear_list.p, T.pair_ptr.p, T.pairPA.p, T.pairPB.p, T.pairSA.p, T.pairSB.p,
           (float)kappa, nk, c.n, c.mv_active, T.leaf_sys.p, c.part.p, c.dev_err.p);
  }
  if (!F64) c.time_end(s, tm);
  BP_CUDA(cudaEventRecord(c.ev_join, sf));  // join
  BP_CUDA(cudaStreamWaitEvent(s, c.ev_join, 0));
  c.time_end(s, tp);
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

std::vector<int64_t> shard_cuts(const std::vector<double>& cost, int world) {
  const int64_t n = (int64_t)cost.size();
  std::vector<int64_t> b(world + 1, 0);
  double total = 0.0;
  for (double v : cost) total += v;
  b[world] = n;
  if (!(total > 0.0)) {  // no cost anywhere: equal unit counts
    for (int r = 1; r < world; ++r) b[r] = n * r / world;
    return b;
  }
  // cut r at the unit boundary whose cost prefix is nearest to r/world of the total
  // (ties to the earlier boundary); cuts never move backwards
  double prefix = 0.0;
  int64_t i = 0;
  for (int r = 1; r < world; ++r) {
    const double want = total * r / world;
    while (i < n && prefix + cost[i] <= want) prefix += cost[i++];
    if (i < n && prefix + cost[i] - want < want - prefix) prefix += cost[i++];
    b[r] = i;
  }
  return b;
}

void build_shard(Ctx& c, cudaStream_t s) {
  Tree& T = c.tree;
  c.sh_ready = true;
  c.sh_bounds.assign(2, 0);
  c.sh_bounds[1] = c.n;
  if (c.sh_world <= 1) return;
  // batches in panel order; cuts at batch boundaries
  std::vector<int> ord(T.h_batch.size());
  for (size_t k = 0; k < ord.size(); ++k) ord[k] = (int)k;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return T.h_batch[a].y < T.h_batch[b].y; });
  std::vector<double> cost(ord.size());
  for (size_t k = 0; k < ord.size(); ++k) cost[k] = T.h_batch_cost[ord[k]];
  const std::vector<int64_t> cut = shard_cuts(cost, c.sh_world);
  c.sh_bounds.assign(c.sh_world + 1, 0);
  for (int r = 0; r <= c.sh_world; ++r)
    c.sh_bounds[r] = cut[r] < (int64_t)ord.size() ? T.h_batch[ord[cut[r]]].y : c.n;
  std::vector<char> own(T.h_batch.size(), 0);
  c.sh_pairs = c.sh_far = 0;
  for (int64_t k = cut[c.sh_rank]; k < cut[c.sh_rank + 1]; ++k) {
    own[ord[k]] = 1;
    c.sh_pairs += T.h_batch_pairs[ord[k]];
    c.sh_far += T.h_batch_far[ord[k]];
  }
  std::vector<int4> b16, b16f;
  for (const int4& q : T.h_blk16)
    if (own[q.w]) b16.push_back(q);
  for (const int4& q : T.h_blk16f)
    if (own[q.w]) b16f.push_back(q);
  c.sh_nblk16 = (int)b16.size();
  c.sh_nblk16f = (int)b16f.size();
  c.sh_blk16.alloc(std::max<size_t>(1, b16.size()));
  c.sh_blk16f.alloc(std::max<size_t>(1, b16f.size()));
  if (!b16.empty())
    BP_CUDA(cudaMemcpyAsync(c.sh_blk16.p, b16.data(), sizeof(int4) * b16.size(), cudaMemcpyHostToDevice, s));
  if (!b16f.empty())
    BP_CUDA(cudaMemcpyAsync(c.sh_blk16f.p, b16f.data(), sizeof(int4) * b16f.size(), cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaStreamSynchronize(s));
}

void build_tree(Ctx& c, cudaStream_t s) {
  Tree& T = c.tree;
  c.ensure_aux();  // the products' side stream, created here rather than inside a product
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
  {  // source pairs of every leaf for the FP32 near field
    std::vector<int> pptr(T.nleaf + 1, 0), psrc;
    for (int l = 0; l < T.nleaf; ++l) {
      const int cl = T.h_leaf_cell[l];
      const int a = T.h_begin[cl] * c.K, e = T.h_end[cl] * c.K;
      for (int q = a; q < e; q += 2) psrc.push_back(q + 1 < e ? q : ~q);
      pptr[l + 1] = (int)psrc.size();
    }
    T.npair = (int)psrc.size();
    upload(T.pair_ptr, pptr, s);
    upload(T.pair_src, psrc, s);
    for (DBuf<float4>* d : {&T.pairPA, &T.pairPB, &T.pairSA, &T.pairSB}) d->alloc(std::max(1, T.npair));
    launch(pair_pos_kernel, cdiv(T.npair, 256), 256, 0, s, T.pair_src.p, T.npair, T.src_rel32.p, T.pairPA.p,
           T.pairPB.p);
  }
  BP_CUDA(cudaStreamSynchronize(s));
  build_lists(c, s);
  BP_CUDA(cudaStreamSynchronize(s));
  T.mom_order = -1;
  c.tree_ready = true;
  c.sh_ready = false;  // the shard tables follow the tree
  c.stree.ready = false;  // so do the sites' lists
}


void tree_matvec_sums(Ctx& c, bool fp32, cudaStream_t s) {
  if (!c.tree_ready) build_tree(c, s);
  if (fp32)
    dispatch<float>(c, c.tree.mom32, s);
  else
    dispatch<double>(c, c.tree.mom64, s);
}

}  // namespace bp

namespace {

template <int P>
bempol_status far_coefficients_copy(int64_t* n_entries, int64_t* n_terms, int32_t* ptr, int32_t* moment,
                                    double* coef) {
  std::vector<int> p, k;
  std::vector<double> c;
  bp::btab_terms<P>(p, k, c);
  *n_entries = (int64_t)p.size() - 1;
  *n_terms = (int64_t)k.size();
  if (ptr) std::copy(p.begin(), p.end(), ptr);
  if (moment) std::copy(k.begin(), k.end(), moment);
  if (coef) std::copy(c.begin(), c.end(), coef);
  return BEMPOL_OK;
}

}  // namespace

extern "C" bempol_status bempol_far_coefficients(int order, int64_t* n_entries, int64_t* n_terms, int32_t* ptr,
                                                 int32_t* moment, double* coef) {
  if (!n_entries || !n_terms) return BEMPOL_ERR_ARG;
  try {
    switch (order) {
      case 1: return far_coefficients_copy<1>(n_entries, n_terms, ptr, moment, coef);
      case 2: return far_coefficients_copy<2>(n_entries, n_terms, ptr, moment, coef);
      case 3: return far_coefficients_copy<3>(n_entries, n_terms, ptr, moment, coef);
      case 4: return far_coefficients_copy<4>(n_entries, n_terms, ptr, moment, coef);
      case 5: return far_coefficients_copy<5>(n_entries, n_terms, ptr, moment, coef);
      case 6: return far_coefficients_copy<6>(n_entries, n_terms, ptr, moment, coef);
      default: return BEMPOL_ERR_ARG;
    }
  } catch (...) {
    return BEMPOL_ERR_ARG;
  }
}
