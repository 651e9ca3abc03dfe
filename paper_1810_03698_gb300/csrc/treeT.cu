// Transposed treecode product A^T u (used by the adjoint): charges u at the
// collocation points, potentials and their normal derivatives at the Gauss nodes,
// with the octree, interaction lists and near lists of the forward product (tree.cu).
#include "tree_common.h"

namespace bp {

namespace {

// ---------------------------------------------------------------- transposed product
// A^T puts charges at the collocation points and evaluates at the Gauss nodes: per
// panel j, sum_g W_g V(y_g) and sum_g W_g n_j . grad V(y_g) with V the potential of the
// charges u (u1 for the Laplace kernel, u2 for Yukawa).  Far field: with D = y - c_C the
// potential of a cell's charges is V = sum_m g_m(|D|) S_m(D), S_m = sum_e D^e B[m, e]
// (the cell's far-field coefficients, as in the product), and since grad g_m = D g_{m+1},
//     n . grad V = (n . D) sum_m g_{m+1} S_m + sum_m g_m (n . grad S_m).
// The monomials D^e are carried together with their derivatives along n (first-order
// dual numbers), so one pass over a cell's interleaved (Laplace, Yukawa) coefficients
// gives all four rows; the radial sequences run to order P + 1.  lw = 1 adds the
// Laplace terms (0: a cell of another body).
template <int P, typename Real>
__device__ __forceinline__ void farT_eval(const Real D[3], const Real nv[3], const Real* __restrict__ Bc, Real kappa,
                                          Real kappa2, Real lw, Real& vl, Real& kl, Real& vy, Real& ky) {
  constexpr BIdx<P> bi{};
  Real SL[P + 1], TL[P + 1], SY[P + 1], TY[P + 1];  // S_m and n . grad S_m, both charge sets
  Real py[P + 1], dy[P + 1], pz[P + 1], dz[P + 1];   // powers of D_y, D_z and their n-derivatives
#pragma unroll
  for (int m = 0; m <= P; ++m) SL[m] = TL[m] = SY[m] = TY[m] = (Real)0;
  py[0] = pz[0] = (Real)1;
  dy[0] = dz[0] = (Real)0;
#pragma unroll
  for (int e = 1; e <= P; ++e) {
    dy[e] = dy[e - 1] * D[1] + py[e - 1] * nv[1];
    py[e] = py[e - 1] * D[1];
    dz[e] = dz[e - 1] * D[2] + pz[e - 1] * nv[2];
    pz[e] = pz[e - 1] * D[2];
  }
  Real px = (Real)1, dx = (Real)0;
#pragma unroll
  for (int a = 0; a <= P; ++a) {
#pragma unroll
    for (int b = 0; b <= P; ++b) {  // fixed trip counts, so every index is a constant
      if (a + b > P) continue;
      const Real pab = px * py[b], dab = dx * py[b] + px * dy[b];
#pragma unroll
      for (int c = 0; c <= P; ++c) {
        if (a + b + c > P) continue;
        const Real w = pab * pz[c], dw = dab * pz[c] + pab * dz[c];
        const int d = a + b + c, t0 = bi.t[a][b][c];
#pragma unroll
        for (int m = 0; m <= P; ++m) {
          if (m < d || 2 * m - d > P) continue;
          const int t = t0 + (m - d);
          Real bl, by;
          ld_entry<Real, (2 * nb_of(P) * sizeof(Real)) % 16 == 0>(Bc, t, bl, by);
          SL[m] = fma(w, bl, SL[m]);
          TL[m] = fma(dw, bl, TL[m]);
          SY[m] = fma(w, by, SY[m]);
          TY[m] = fma(dw, by, TY[m]);
        }
      }
    }
    dx = dx * D[0] + px * nv[0];
    px *= D[0];
  }
  const Real r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
  const Real rinv = inv_sqrt(r2);
  const Real ir2 = rinv * rinv;
  const Real nD = nv[0] * D[0] + nv[1] * D[1] + nv[2] * D[2];
  // Laplace: g_0 = 1/r, g_{m+1} = -(2m + 1) g_m / r^2
  Real g = rinv, V = 0, K1 = 0, K2 = 0;
#pragma unroll
  for (int m = 0; m <= P; ++m) {
    const Real gn = g * (Real)(-(2.0 * m + 1.0)) * ir2;
    V += g * SL[m];
    K2 += g * TL[m];
    K1 += gn * SL[m];
    g = gn;
  }
  vl += lw * V;
  kl += lw * (nD * K1 + K2);
  // Yukawa: g_0 = e^{-kappa r}/r, g_1 = -(1 + kappa r) g_0 / r^2,
  // g_{m+1} = (kappa^2 g_{m-1} - (2m + 1) g_m) / r^2
  const Real kr = kappa * (r2 * rinv);
  Real g0 = exp_neg(kr) * rinv;
  Real g1 = -((Real)1 + kr) * g0 * ir2;
  V = g0 * SY[0];
  K2 = g0 * TY[0];
  K1 = g1 * SY[0];
#pragma unroll
  for (int m = 1; m <= P; ++m) {
    const Real g2 = (kappa2 * g0 - (Real)(2.0 * m + 1.0) * g1) * ir2;
    V += g1 * SY[m];
    K2 += g1 * TY[m];
    K1 += g2 * SY[m];
    g0 = g1;
    g1 = g2;
  }
  vy += V;
  ky += nD * K1 + K2;
}

// Far field of the transposed product, one warp per 8 panels of one leaf (half of a
// 16-panel block; blockIdx.x = 2 * block + half): lane 4p + g serves Gauss node g of
// panel p.  Every lane takes every cell of the leaf's far list (the acceptance test of
// the list holds for the leaf's nodes); the warp stages its own groups of cells'
// coefficients with cp.async, double-buffered, with no block-wide barrier.  The four
// nodes of a panel are summed with shuffles; rows (V_L, K_L, V_Y, K_Y) go to out
// ([4][n]).  lap (NULL: every cell) marks the entries with Laplace terms.
template <int P, typename Real>
__global__ void __launch_bounds__(32) farT16_kernel(const int4* __restrict__ blk, const float4* __restrict__ node_rel,
                                                    const double4* __restrict__ node64,
                                                    const double4* __restrict__ nrm, int K,
                                                    const int* __restrict__ leaf_cell,
                                                    const double4* __restrict__ center,
                                                    const int* __restrict__ far_ptr, const int* __restrict__ far_list,
                                                    const int* __restrict__ lap, const Real* __restrict__ bco,
                                                    Real kappa, int n, const int* __restrict__ active,
                                                    const int* __restrict__ leaf_sys, double* __restrict__ out) {
  constexpr int NB = FarShape<P, Real>::NB, FW = FarShape<P, Real>::FW;
  constexpr bool ASYNC = (2 * NB * sizeof(Real)) % 16 == 0;
  constexpr int CH = (int)(2 * NB * sizeof(Real) / 16);  // 16-byte pieces per cell
  __shared__ __align__(16) Real sm[2][FW][2 * NB];
  __shared__ Real so[2][FW][4];
  const int lane = threadIdx.x;
  const int4 B = blk[blockIdx.x >> 1];
  const int leaf = B.x;
  if (active && !active[leaf_sys[leaf]]) return;
  const int first = B.y + 8 * (int)(blockIdx.x & 1), cnt = min(8, B.z - 8 * (int)(blockIdx.x & 1));
  if (cnt <= 0) return;
  const double4 ct = center[leaf_cell[leaf]];
  const int pl = lane >> 2, g = lane & 3;
  const int i = first + pl;
  const bool act = pl < cnt && g < K;
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
  const Real kappa2 = kappa * kappa;
  double aVL = 0, aKL = 0, aVY = 0, aKY = 0;
  const int f0 = far_ptr[leaf], f1 = far_ptr[leaf + 1];
  auto stage = [&](int b, int fb) {
    const int c = min(FW, f1 - fb);
    if constexpr (ASYNC) {
      for (int q = lane; q < c * CH; q += 32) {
        const int cell = q / CH, piece = q - cell * CH;
        const char* gp = reinterpret_cast<const char*>(bco + (size_t)far_list[fb + cell] * 2 * NB) + 16 * piece;
        cp_async16(reinterpret_cast<char*>(&sm[b][cell][0]) + 16 * piece, gp);
      }
      cp_async_commit();
    } else {
      for (int q = lane; q < c * 2 * NB; q += 32)
        sm[b][q / (2 * NB)][q % (2 * NB)] = bco[(size_t)far_list[fb + q / (2 * NB)] * 2 * NB + q % (2 * NB)];
    }
    if (lane < c) {
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
    const int c = min(FW, f1 - fb);
    if constexpr (ASYNC) cp_async_wait_all();  // this lane's pieces of group b
    __syncwarp();  // every lane's pieces and offsets of group b; all done with the other buffer
    if (fb + FW < f1) stage(b ^ 1, fb + FW);
    Real vl = 0, kl = 0, vy = 0, ky = 0;
    for (int q = 0; q < c; ++q) {
      const Real D[3] = {yr[0] + so[b][q][0], yr[1] + so[b][q][1], yr[2] + so[b][q][2]};
      farT_eval<P, Real>(D, nv, sm[b][q], kappa, kappa2, so[b][q][3], vl, kl, vy, ky);
    }
    aVL += (double)(w * vl);
    aKL += (double)(w * kl);
    aVY += (double)(w * vy);
    aKY += (double)(w * ky);
  }
  // the nodes of a panel are four consecutive lanes
  for (int o = 1; o < 4; o <<= 1) {
    aVL += __shfl_xor_sync(0xffffffffu, aVL, o);
    aKL += __shfl_xor_sync(0xffffffffu, aKL, o);
    aVY += __shfl_xor_sync(0xffffffffu, aVY, o);
    aKY += __shfl_xor_sync(0xffffffffu, aKY, o);
  }
  if (g == 0 && pl < cnt) {
    out[i] = aVL;
    out[(size_t)n + i] = aKL;
    out[2 * (size_t)n + i] = aVY;
    out[3 * (size_t)n + i] = aKY;
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

template <typename Real>
DBuf<Real>& bcoT(Tree& T);
template <>
DBuf<float>& bcoT<float>(Tree& T) {
  return T.bcoT32;
}
template <>
DBuf<double>& bcoT<double>(Tree& T) {
  return T.bcoT64;
}

template <int P, typename Real>
void runT_tree(Ctx& c, const double* u, cudaStream_t s) {
  Tree& T = c.tree;
  constexpr int NC = MI<P>::NC, NB = nb_of(P);
  typedef typename Vec4<Real>::T R4;
  DBuf<Real>& mL = momT<Real>(T, 0);
  DBuf<Real>& mY = momT<Real>(T, 1);
  if (mL.n < (size_t)T.ncell * 2 * NC) mL.alloc((size_t)T.ncell * 2 * NC);
  if (mY.n < (size_t)T.ncell * 2 * NC) mY.alloc((size_t)T.ncell * 2 * NC);
  DBuf<Real>& bco = bcoT<Real>(T);
  if (bco.n < (size_t)T.ncell * 2 * NB) bco.alloc((size_t)T.ncell * 2 * NB);
  build_btab<P>(T.btabT, s);
  DBuf<R4>& sL = chgT<R4>(T, 0);
  DBuf<R4>& sY = chgT<R4>(T, 1);
  if (sL.n < (size_t)c.n) sL.alloc(c.n);
  if (sY.n < (size_t)c.n) sY.alloc(c.n);
  const int S = T.near_splits;
  const size_t need = (size_t)(S + 1) * 4 * c.n;
  if (c.part.n < need) c.part.alloc(need);
  const Real kappa = (Real)c.par.kappa;
  // Fork as in the forward product: charges, moments, M2M shifts, coefficients and the
  // far kernel on the high-priority side stream, the near field (which reads u
  // directly) on `s`.
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
  {  // far-field coefficients (Laplace, Yukawa) of the cells that the leaves' far lists can hold
    const int cb = T.h_depth_begin[T.m2m_min_depth];
    if (cb < T.ncell)
      launch(bcoef_kernel<P, Real>, cdiv((long long)(T.ncell - cb) * NB, 256), 256, 0, sf, cb, T.ncell,
             T.btabT.ptr.p, T.btabT.k.p, T.btabT.c.p, mL.p, mY.p, bco.p);
  }
  Ctx::Timed tf;
  c.time_begin(1, sf, tf);
  double* far_out = c.part.p + (size_t)S * 4 * c.n;
  launch(farT16_kernel<P, Real>, 2 * T.nblk16f, 32, 0, sf, T.blk16f.p, T.src_rel32.p, c.src64.p, c.nrm64.p, c.K,
         T.leaf_cell.p, T.center.p, T.far_ptr.p, T.far_list.p, T.farL_same ? nullptr : T.far_lap.p, bco.p, kappa,
         c.n, c.mv_active, T.leaf_sys.p, far_out);
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
// bounds both), the order-P transposed kernel evaluates four times as many targets (the
// Gauss nodes) with derivatives along the normal, and one compiled order keeps the build
// short.
void dispatchT(Ctx& c, const double* u, cudaStream_t s) { runT_tree<4, float>(c, u, s); }

}  // namespace

// Partial sums of the transposed product (rows V_L, K_L, V_Y, K_Y per panel, part_splits
// pieces in c.part) by the FP32 treecode; combineT assembles A^T u from them.
void tree_matvec_T_sums(Ctx& c, const double* u, cudaStream_t s) {
  if (!c.tree_ready) build_tree(c, s);
  dispatchT(c, u, s);
}

}  // namespace bp
