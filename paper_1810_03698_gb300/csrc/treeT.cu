// Transposed treecode product A^T u (used by the adjoint): charges u at the
// collocation points, potentials and their normal derivatives at the Gauss nodes,
// with the octree, interaction lists and near lists of the forward product (tree.cu).
#include "tree_common.h"

namespace bp {

namespace {

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
    const Real m = M[t];
    v += A[t] * m;
    g0 -= (Real)(mi.k[t][0] + 1) * A[mi.p1[t][0]] * m;
    g1 -= (Real)(mi.k[t][1] + 1) * A[mi.p1[t][1]] * m;
    g2 -= (Real)(mi.k[t][2] + 1) * A[mi.p1[t][2]] * m;
  }
  V = v;
  G[0] = g0;
  G[1] = g1;
  G[2] = g2;
}

// Four threads per panel (one per Gauss node, K <= 4) of a target block of <= 32
// panels of one leaf; loops over the leaf's far cells (Laplace list for YUK = 0,
// Yukawa list for 1) with the charge moments `mom` ([cell][2][NC], first NC used),
// then adds the nodes of each panel with shuffles.  Writes rows (2 YUK, 2 YUK + 1) =
// (sum_g W V, sum_g W n . grad V) of `out` ([4][n]).
template <int P, typename Real, int YUK>
__global__ void __launch_bounds__(128) farT_kernel(const int4* __restrict__ blk, const float4* __restrict__ node_rel,
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
  const int pl = threadIdx.x >> 2, g = threadIdx.x & 3;
  const int i = B.y + pl;
  const bool act = pl < B.z && g < K;
  Real yr[3] = {0, 0, 0}, w = 0, nv[3] = {0, 0, 0};
  if (act) {
    const size_t q = (size_t)K * i + g;
    if (sizeof(Real) == 4) {
      const float4 r = node_rel[q];
      yr[0] = r.x;
      yr[1] = r.y;
      yr[2] = r.z;
    } else {
      const double4 y = node64[q];
      yr[0] = (Real)(y.x - ct.x);
      yr[1] = (Real)(y.y - ct.y);
      yr[2] = (Real)(y.z - ct.z);
    }
    w = (Real)node64[q].w;
    const double4 nn = nrm[i];
    nv[0] = (Real)nn.x;
    nv[1] = (Real)nn.y;
    nv[2] = (Real)nn.z;
  }
  double aV = 0, aK = 0;
  const int f0 = far_ptr[leaf], f1 = far_ptr[leaf + 1];
  for (int fb = f0; fb < f1; fb += FCH) {
    const int cnt = min(FCH, f1 - fb);
    for (int q = threadIdx.x; q < cnt * NC; q += 128)
      sm[q / NC][q % NC] = mom[(size_t)far_list[fb + q / NC] * 2 * NC + q % NC];
    if ((int)threadIdx.x < cnt) {
      const double4 cc = center[far_list[fb + threadIdx.x]];
      so[threadIdx.x][0] = (Real)(ct.x - cc.x);
      so[threadIdx.x][1] = (Real)(ct.y - cc.y);
      so[threadIdx.x][2] = (Real)(ct.z - cc.z);
    }
    __syncthreads();
    Real v = 0, k = 0;
    if ((int)(threadIdx.x >> 5) * 8 < B.z) {  // warp holds at least one panel
      for (int q = 0; q < cnt; ++q) {
        const Real D[3] = {yr[0] + so[q][0], yr[1] + so[q][1], yr[2] + so[q][2]};
        Real V, G[3];
        farT_eval<P, Real, YUK>(D, sm[q], kappa, V, G);
        v += w * V;
        k += w * (nv[0] * G[0] + nv[1] * G[1] + nv[2] * G[2]);
      }
    }
    aV += (double)v;
    aK += (double)k;
    __syncthreads();
  }
  // the nodes of a panel are four consecutive lanes
  for (int o = 1; o < 4; o <<= 1) {
    aV += __shfl_xor_sync(0xffffffffu, aV, o);
    aK += __shfl_xor_sync(0xffffffffu, aK, o);
  }
  if (g == 0 && pl < B.z) {
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
    int lo = 0;  // leaf of this lane's source (j only grows)
    for (int t0 = 0; t0 < total; t0 += NTB) {
      const int j = t0 + threadIdx.x;
      R4 pz;
      pz.x = pz.y = pz.z = pz.w = 0;
      Real a1 = 0;
      if (j < total) {
        while (lc[lo + 1] <= j) ++lo;
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


template <typename R4>
DBuf<R4>& chgT(Tree& T, int w);
template <>
DBuf<float4>& chgT<float4>(Tree& T, int w) {
  return T.chgT32[w];
}
template <>
DBuf<double4>& chgT<double4>(Tree& T, int w) {
  return T.chgT64[w];
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
  DBuf<R4>& sL = chgT<R4>(T, 0);
  DBuf<R4>& sY = chgT<R4>(T, 1);
  if (sL.n < (size_t)c.n) sL.alloc(c.n);
  if (sY.n < (size_t)c.n) sY.alloc(c.n);
  const int S = T.near_splits;
  const size_t need = (size_t)(S + 1) * 4 * c.n;
  if (c.part.n < need) c.part.alloc(need);
  const Real kappa = (Real)c.par.kappa;
  // Fork as in the forward product: charges, moments, M2M shifts and far kernels on the
  // high-priority side stream, the near field (which reads u directly) on `s`.
  c.ensure_aux();
  const cudaStream_t sf = c.aux;
  Ctx::Timed tp;
  c.time_begin(2, s, tp);
  BP_CUDA(cudaEventRecord(c.ev_fork, s));
  BP_CUDA(cudaStreamWaitEvent(sf, c.ev_fork, 0));
  launch(centroid_charges_kernel<R4>, cdiv(c.n, 256), 256, 0, sf, u, c.n, sL.p, sY.p);
  for (int w = 0; w < 2; ++w) {
    DBuf<Real>& m = w ? mY : mL;
    launch(leaf_moments_kernel<P, Real>, T.nleaf, MomShape<P>::TPB, 0, sf, T.leaf_cell.p, T.begin.p, T.end.p, T.center.p, 1,
           c.tgt64.p, (const R4*)(w ? sY.p : sL.p), c.mv_active, T.leaf_sys.p, m.p);
    for (int d = T.ndepth - 2; d >= T.m2m_min_depth; --d) {
      const int first = T.h_depth_begin[d], cnt = T.h_depth_begin[d + 1] - first;
      launch(m2m_kernel<P, Real>, cnt, M2M_TPB, 0, sf, first, T.child0.p, T.nchild.p, T.center.p, m.p);
    }
  }
  Ctx::Timed tf;
  c.time_begin(1, sf, tf);
  double* far_out = c.part.p + (size_t)S * 4 * c.n;
  const int* lp = T.farL_same ? T.far_ptr.p : T.farL_ptr.p;
  const int* ll = T.farL_same ? T.far_list.p : T.farL_list.p;
  launch(farT_kernel<P, Real, 0>, T.nblk32, 128, 0, sf, T.blk32.p, T.src_rel32.p, c.src64.p, c.nrm64.p, c.K,
         T.leaf_cell.p, T.center.p, lp, ll, mL.p, kappa, c.n, c.mv_active, T.leaf_sys.p, far_out);
  launch(farT_kernel<P, Real, 1>, T.nblk32, 128, 0, sf, T.blk32.p, T.src_rel32.p, c.src64.p, c.nrm64.p, c.K,
         T.leaf_cell.p, T.center.p, T.far_ptr.p, T.far_list.p, mY.p, kappa, c.n, c.mv_active, T.leaf_sys.p,
         far_out);
  c.time_end(sf, tf);
  Ctx::Timed tm;
  c.time_begin(0, s, tm);
  launch(nearT_kernel<Real>, dim3(T.nblk32, S), NTB, 0, s, T.blk32.p, T.src_rel32.p, c.src64.p, c.nrm64.p, c.K,
         T.leaf_cell.p, T.center.p, T.begin.p, T.end.p, T.near_ptr.p, T.near_list.p, T.cen_rel32.p, c.tgt64.p, u,
         kappa, c.n, c.mv_active, T.leaf_sys.p, c.part.p);
  c.time_end(s, tm);
  BP_CUDA(cudaEventRecord(c.ev_join, sf));  // join
  BP_CUDA(cudaStreamWaitEvent(s, c.ev_join, 0));
  c.time_end(s, tp);
  c.part_splits = S + 1;
}

// The transposed far field runs in FP32 at order 4 whatever the forward order: the
// adjoint needs A^T only to about the accuracy of the forward treecode (theta^(P+1)
// bounds both), the order-P transposed kernel carries coefficients to order P + 1 at
// four Gauss nodes per panel, and one compiled order keeps the build short.
void dispatchT(Ctx& c, const double* u, cudaStream_t s) { runT_tree<4, float>(c, u, s); }

}  // namespace

// Partial sums of the transposed product (rows V_L, K_L, V_Y, K_Y per panel, part_splits
// pieces in c.part) by the FP32 treecode; combineT assembles A^T u from them.
void tree_matvec_T_sums(Ctx& c, const double* u, cudaStream_t s) {
  if (!c.tree_ready) build_tree(c, s);
  dispatchT(c, u, s);
}

}  // namespace bp
