// Adjoint of the solvation energy: gradient of Delta G_solv with respect to the
// sites' permanent moments (q, d, Q) and positions, through the BEM solve (Eq.
// integral_eq) and the self-consistent induced dipoles (Sec. "Self-consistent
// induced field").
//
// Forward (dissolved state, per body): b = B(q, d + mu, Q) (Eq. rhs_multipole),
// A x = [b; 0], reaction fields F_s = R x at the sites (Eqs. pot_solvent,
// Efield_solv, ddphi), mu = a (-grad phi_s + E_perm + T mu) with a = 4 pi alpha,
// T the damped dipole field tensor, E_perm the group-masked permanent field, and
// G_diss = 1/2 sum_l <m_l, F_s + F_mult>, <m, F> = q phi + d . grad phi + Q : H / 6
// (Eq. energy_multipole_polarizable).  With Lagrange multipliers lambda (BEM) and
// nu (induced dipoles), nu~ = a nu, the stationarity conditions are
//     A^T lambda = R^T (q/2, d/2 - nu~, Q/2)                         (transposed BEM)
//     nu~ = a (c_mu + B_p^T lambda_1 + T nu~)                        (transposed SCF)
// with c_mu = -1/2 (damped, unmasked field of the permanent moments) the derivative
// of the energy's induced terms, and B_p^T lambda_1 = grad Psi, Psi the potential
// of charges lambda_1 / eps_in at the collocation points.  T is symmetric, so the
// transposed SCF is relaxed like the forward one (same omega, same RMS test), each
// step with one transposed BEM solve.  Then, per site,
//     dG_diss/dq = phi_s/2 + (P(mu) + P(0))/2 + Psi - phi_nu
//     dG_diss/dd = the same with gradients,  dG_diss/dQ = (the same with Hessians)/6
// where P(mu) is the energy-form multipole potential (permanent unmasked plus
// induced damped) and phi_nu the group-masked undamped potential of dipoles nu~.
// The vacuum state has no BEM: nu~_v = a (c_mu,v + T_v nu~_v) over the whole system
// and dG_vac/dq = (P_v(mu_v) + P_v(0))/2 - phi_nu,v (and so on).  The quadrupole
// gradient is returned projected on symmetric traceless matrices.
//
// Positions (the mesh held fixed): the derivative of the Lagrangian at the converged
// state, taken with dual numbers seeded on the site coordinates -- the gradient of
// <(q/2, d/2 - nu~, Q/2), F_s> (third derivatives of the reaction potential), of
// <(q, d + mu, Q), F_Psi> (the right-hand side's site dependence), and of every
// site-site term (permanent-permanent, Thole-damped induced, masked adjoint field
// and damped adjoint-induced couplings, with the damping factors differentiated).
//
// The transposed BEM product: with u = [u1; u2],
//     (A^T u)_phi = (u1 + u2)/2 + K_L^T u1 - K_Y^T u2,   (A^T u)_psi = -V_L^T u1 + (eps_in/eps_out) V_Y^T u2,
// i.e. charges u1, u2 at the collocation points evaluated at every panel's Gauss
// nodes (potential, and normal derivative for K), weighted by w_g A_j, plus the
// near-field corrections taken by columns.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "dual.h"
#include "internal.h"

namespace bp {

namespace {

constexpr int TPB = 128;
constexpr double INV4PI = 0.07957747154594767;

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

// One thread per target panel j (blocks of the direct block table: panels of one
// body), looping over the source collocation points of the block's system; the
// Laplace strength u1 of a source outside the block's body is staged as 0.
// Per (node g of j, source i), R = x_i - y_jg:
//   VL += W u1 / r, KL += W u1 (n.R) / r^3, VY += W u2 e / r, KY += W u2 (n.R)(1 + k r) e / r^3.
template <bool F32>
__global__ void __launch_bounds__(TPB) p2pT_kernel(const double4* __restrict__ cen, const double4* __restrict__ node,
                                                   const double4* __restrict__ nrm, int K, int n,
                                                   const int4* __restrict__ blk, const int4* __restrict__ rng,
                                                   const double4* __restrict__ blk_center,
                                                   const double* __restrict__ u, double kappa,
                                                   const int* __restrict__ active, const int* __restrict__ grp_sys,
                                                   double* __restrict__ part) {
  typedef typename std::conditional<F32, float, double>::type Real;
  __shared__ Real sx[TPB], sy[TPB], sz[TPB], s1[TPB], s2[TPB];
  const int4 B = blk[blockIdx.x], Rg = rng[blockIdx.x];
  if (active && !active[grp_sys[B.z]]) return;
  const int j = B.x + threadIdx.x;
  const bool act = (int)threadIdx.x < B.y;
  // source ranges in panels (the table holds Gauss-node ranges, K per panel)
  const int y0 = Rg.x / K, y1 = Rg.y / K, l0 = Rg.z / K, l1 = Rg.w / K;
  const int per = ((y1 - y0 + (int)gridDim.y - 1) / (int)gridDim.y + TPB - 1) / TPB * TPB;
  const int s0 = y0 + blockIdx.y * per, s1e = min(y1, s0 + per);
  const double4 c = F32 ? blk_center[blockIdx.x] : make_double4(0, 0, 0, 0);
  Real gx[4] = {0, 0, 0, 0}, gy[4] = {0, 0, 0, 0}, gz[4] = {0, 0, 0, 0}, gw[4] = {0, 0, 0, 0};
  Real nx = 0, ny = 0, nz = 0;
  if (act) {
    for (int g = 0; g < K; ++g) {
      const double4 y = node[(size_t)K * j + g];
      gx[g] = (Real)(y.x - c.x);
      gy[g] = (Real)(y.y - c.y);
      gz[g] = (Real)(y.z - c.z);
      gw[g] = (Real)y.w;
    }
    const double4 nn = nrm[j];
    nx = (Real)nn.x;
    ny = (Real)nn.y;
    nz = (Real)nn.z;
  }
  const Real kap = (Real)kappa;
  double aVL = 0, aKL = 0, aVY = 0, aKY = 0;
  for (int t0 = s0; t0 < s1e; t0 += TPB) {
    const int i = t0 + threadIdx.x;
    if (i < s1e) {
      const double4 x = cen[i];
      sx[threadIdx.x] = (Real)(x.x - c.x);
      sy[threadIdx.x] = (Real)(x.y - c.y);
      sz[threadIdx.x] = (Real)(x.z - c.z);
      s1[threadIdx.x] = (i >= l0 && i < l1) ? (Real)u[i] : (Real)0;
      s2[threadIdx.x] = (Real)u[n + i];
    }
    __syncthreads();
    const int lim = min(TPB, s1e - t0);
    Real vl = 0, kl = 0, vy = 0, ky = 0;
    if (act) {
      for (int k = 0; k < lim; ++k) {
        const Real X = sx[k], Y = sy[k], Z = sz[k], a1 = s1[k], a2 = s2[k];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          if (g >= K) break;
          const Real dx = X - gx[g], dy = Y - gy[g], dz = Z - gz[g];
          const Real r2 = dx * dx + dy * dy + dz * dz;
          if (F32) {
            const float ri = r2 > 0.f ? rsqrt_approx((float)r2) : 0.f;
            const float r = (float)r2 * ri;
            const float e = exp2_approx(-1.4426950408889634f * (float)kap * r);
            const float w = (float)gw[g] * ri;
            const float nR = (float)(nx * dx + ny * dy + nz * dz) * ri * ri;
            vl += (Real)(w * (float)a1);
            vy += (Real)(w * (float)a2 * e);
            kl += (Real)(w * nR * (float)a1);
            ky += (Real)(w * nR * (float)a2 * fmaf((float)kap, r, 1.f) * e);
          } else {
            if (r2 == 0.0) continue;
            const double r = sqrt((double)r2);
            const double ri = 1.0 / r;
            const double e = exp(-(double)kap * r);
            const double w = (double)gw[g] * ri;
            const double nR = (double)(nx * dx + ny * dy + nz * dz) * ri * ri;
            vl += (Real)(w * (double)a1);
            vy += (Real)(w * (double)a2 * e);
            kl += (Real)(w * nR * (double)a1);
            ky += (Real)(w * nR * (double)a2 * (1.0 + (double)kap * r) * e);
          }
        }
      }
    }
    aVL += (double)vl;
    aKL += (double)kl;
    aVY += (double)vy;
    aKY += (double)ky;
    __syncthreads();
  }
  if (act) {
    double* o = part + (size_t)blockIdx.y * 4 * n;
    o[j] = aVL;
    o[n + j] = aKL;
    o[2 * n + j] = aVY;
    o[3 * n + j] = aKY;
  }
}

// (A^T u) from the split sums plus the near corrections taken by columns.
__global__ void combineT_kernel(const double* __restrict__ part, int S, int n, const int* __restrict__ ptrT,
                                const int* __restrict__ rowT, const int* __restrict__ eT,
                                const double4* __restrict__ corr, const double* __restrict__ u, double eps_ratio,
                                double* __restrict__ y) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double vl = 0, kl = 0, vy = 0, ky = 0;
  for (int q = 0; q < S; ++q) {
    const double* o = part + (size_t)q * 4 * n;
    vl += o[j];
    kl += o[n + j];
    vy += o[2 * n + j];
    ky += o[3 * n + j];
  }
  vl *= INV4PI;
  kl *= INV4PI;
  vy *= INV4PI;
  ky *= INV4PI;
  for (int e = ptrT[j]; e < ptrT[j + 1]; ++e) {
    const int i = rowT[e];
    const double4 cc = corr[eT[e]];
    const double u1 = u[i], u2 = u[n + i];
    vl += cc.x * u1;
    kl += cc.y * u1;
    vy += cc.z * u2;
    ky += cc.w * u2;
  }
  y[j] = 0.5 * (u[j] + u[n + j]) + kl - ky;
  y[n + j] = -vl + eps_ratio * vy;
}

// R^T w: per panel j, the potential U and its gradient at the Gauss nodes of point
// multipoles (charge wq, dipole wd, traceless quadrupole wQ in the convention of
// Eq. pot_multipole) at the sites of j's body; out[j] = -(1/4 pi) sum_g W_g n_j . grad U,
// out[n + j] = (1/4 pi) sum_g W_g U.  Real = float: pair arithmetic in FP32 with
// coordinates relative to the block's centre, per-tile sums added in FP64.
template <typename Real>
__global__ void __launch_bounds__(TPB) adj_reaction_kernel(const double4* __restrict__ node,
                                                           const double4* __restrict__ nrm, int K, int n,
                                                           const int4* __restrict__ blk,
                                                           const double4* __restrict__ blk_center,
                                                           const int* __restrict__ gsite,
                                                           const double4* __restrict__ spos,
                                                           const double* __restrict__ wq, const double* __restrict__ wd,
                                                           const double* __restrict__ wQ, double* __restrict__ out) {
  __shared__ Real sh[13][TPB];
  const int4 B = blk[blockIdx.x];
  const int j = B.x + threadIdx.x;
  const bool act = (int)threadIdx.x < B.y;
  const int k0 = gsite[B.z], k1 = gsite[B.z + 1];
  const double4 c = blk_center[blockIdx.x];
  Real ny[4][4];
  Real nj[3] = {0, 0, 0};
  for (int g = 0; g < 4; ++g) ny[g][0] = ny[g][1] = ny[g][2] = ny[g][3] = 0;
  if (act) {
    for (int g = 0; g < K; ++g) {
      const double4 y = node[(size_t)K * j + g];
      ny[g][0] = (Real)(y.x - c.x);
      ny[g][1] = (Real)(y.y - c.y);
      ny[g][2] = (Real)(y.z - c.z);
      ny[g][3] = (Real)y.w;
    }
    const double4 nn = nrm[j];
    nj[0] = (Real)nn.x;
    nj[1] = (Real)nn.y;
    nj[2] = (Real)nn.z;
  }
  double aU = 0.0, aG = 0.0;
  for (int t0 = k0; t0 < k1; t0 += TPB) {
    const int k = t0 + threadIdx.x;
    if (k < k1) {
      const double4 p = spos[k];
      sh[0][threadIdx.x] = (Real)(p.x - c.x);
      sh[1][threadIdx.x] = (Real)(p.y - c.y);
      sh[2][threadIdx.x] = (Real)(p.z - c.z);
      sh[3][threadIdx.x] = (Real)wq[k];
      for (int a = 0; a < 3; ++a) sh[4 + a][threadIdx.x] = (Real)wd[3 * k + a];
      for (int a = 0; a < 6; ++a) sh[7 + a][threadIdx.x] = (Real)wQ[6 * k + a];
    }
    __syncthreads();
    const int lim = min(TPB, k1 - t0);
    Real tU = 0, tG = 0;
    if (act) {
      for (int kk = 0; kk < lim; ++kk) {
        const Real q = sh[3][kk], px = sh[4][kk], py = sh[5][kk], pz = sh[6][kk];
        const Real Qxx = sh[7][kk], Qxy = sh[8][kk], Qxz = sh[9][kk], Qyy = sh[10][kk], Qyz = sh[11][kk],
                   Qzz = sh[12][kk];
        for (int g = 0; g < K; ++g) {
          const Real Rx = ny[g][0] - sh[0][kk], Ry = ny[g][1] - sh[1][kk], Rz = ny[g][2] - sh[2][kk];
          const Real r2 = Rx * Rx + Ry * Ry + Rz * Rz;
          const Real ri = (Real)1 / sqrt(r2);
          const Real i2 = ri * ri, i3 = i2 * ri, i5 = i3 * i2, i7 = i5 * i2;
          const Real pR = px * Rx + py * Ry + pz * Rz;
          const Real QRx = Qxx * Rx + Qxy * Ry + Qxz * Rz;
          const Real QRy = Qxy * Rx + Qyy * Ry + Qyz * Rz;
          const Real QRz = Qxz * Rx + Qyz * Ry + Qzz * Rz;
          const Real RQR = QRx * Rx + QRy * Ry + QRz * Rz;
          const Real U = q * ri + pR * i3 + (Real)0.5 * RQR * i5;
          const Real cR = -q * i3 - (Real)3 * pR * i5 - (Real)2.5 * RQR * i7;  // coefficient of R in grad U
          const Real gx = cR * Rx + px * i3 + QRx * i5;
          const Real gy = cR * Ry + py * i3 + QRy * i5;
          const Real gz = cR * Rz + pz * i3 + QRz * i5;
          tU += ny[g][3] * U;
          tG += ny[g][3] * (nj[0] * gx + nj[1] * gy + nj[2] * gz);
        }
      }
    }
    aU += (double)tU;
    aG += (double)tG;
    __syncthreads();
  }
  if (act) {
    out[j] = -aG * INV4PI;
    out[n + j] = aU * INV4PI;
  }
}

// Site-site terms of the adjoint, warp per site l, over the sites of l's body
// (whole = 0) or of its system (whole = 1):
//   mode 0: out[3l..] = damped field at l of the other sites' permanent moments,
//           unmasked (q: lambda3, d: lambda3/lambda5, Q: lambda5/lambda7);
//   mode 1: out[10l..] = potential, gradient, Hessian at l of undamped dipoles
//           nu at the other sites outside l's polarisation group.
__global__ void __launch_bounds__(256) site_adjoint_kernel(const double4* __restrict__ pos,
                                                           const double* __restrict__ q, const double* __restrict__ d,
                                                           const double* __restrict__ Q, const double* __restrict__ nu,
                                                           const int* __restrict__ group, const int* __restrict__ stag,
                                                           const int* __restrict__ gsite,
                                                           const int* __restrict__ grp_sys,
                                                           const int* __restrict__ sys_site, int ns, int mode,
                                                           int whole, double thole_a, double scale,
                                                           double* __restrict__ out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * 8 + warp;
  if (l >= ns) return;
  const double4 pl = pos[l];
  const int gl = group[l];
  const int tg = stag[l];
  const int m0 = whole ? sys_site[grp_sys[tg]] : gsite[tg];
  const int m1 = whole ? sys_site[grp_sys[tg] + 1] : gsite[tg + 1];
  double acc[10];
  for (int c = 0; c < 10; ++c) acc[c] = 0.0;
  for (int m = m0 + lane; m < m1; m += 32) {
    if (m == l) continue;
    const double4 pm = pos[m];
    // R from source m to field point l
    const double R[3] = {pl.x - pm.x, pl.y - pm.y, pl.z - pm.z};
    const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    const double ri = 1.0 / sqrt(r2);
    const double i2 = ri * ri, i3 = i2 * ri, i5 = i3 * i2, i7 = i5 * i2;
    if (mode == 0) {
      double l3 = 1.0, l5 = 1.0, l7 = 1.0;
      const double aa = pl.w * pm.w;
      if (aa > 0.0) {
        const double au3 = thole_a * r2 * sqrt(r2) / sqrt(aa);
        const double e = exp(-au3);
        l3 = 1.0 - e;
        l5 = 1.0 - (1.0 + au3) * e;
        l7 = 1.0 - (1.0 + au3 + 0.6 * au3 * au3) * e;
      }
      const double qm = q[m];
      const double pv[3] = {d[3 * m], d[3 * m + 1], d[3 * m + 2]};
      const double* Qm = Q + 6 * m;
      const double QM[3][3] = {{Qm[0], Qm[1], Qm[2]}, {Qm[1], Qm[3], Qm[4]}, {Qm[2], Qm[4], Qm[5]}};
      double QR[3];
      for (int a = 0; a < 3; ++a) QR[a] = QM[a][0] * R[0] + QM[a][1] * R[1] + QM[a][2] * R[2];
      const double RQR = QR[0] * R[0] + QR[1] * R[1] + QR[2] * R[2];
      const double pR = pv[0] * R[0] + pv[1] * R[1] + pv[2] * R[2];
      // E = -grad phi with the damped kernels
      for (int a = 0; a < 3; ++a)
        acc[a] += qm * l3 * R[a] * i3 - l3 * pv[a] * i3 + 3.0 * l5 * pR * R[a] * i5 - l5 * QR[a] * i5 +
                  2.5 * l7 * RQR * R[a] * i7;
    } else {
      if (group[m] == gl) continue;
      const double mv[3] = {nu[3 * m], nu[3 * m + 1], nu[3 * m + 2]};
      const double mR = mv[0] * R[0] + mv[1] * R[1] + mv[2] * R[2];
      acc[0] += mR * i3;
      for (int a = 0; a < 3; ++a) acc[1 + a] += mv[a] * i3 - 3.0 * mR * R[a] * i5;
      int k = 0;
      for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b, ++k) {
          const double dab = a == b ? 1.0 : 0.0;
          acc[4 + k] += 15.0 * mR * R[a] * R[b] * i7 - 3.0 * (mR * dab + mv[a] * R[b] + mv[b] * R[a]) * i5;
        }
    }
  }
  const int nc = mode == 0 ? 3 : 10;
  for (int c = 0; c < nc; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    acc[c] = v;
  }
  if (lane == 0)
    for (int c = 0; c < nc; ++c) out[(size_t)nc * l + c] = acc[c] * scale;
}

// out[3l..] = scale * sum over the S splits of part (site forces)
__global__ void force_reduce_kernel(const double* __restrict__ part, int S, int ns, double scale,
                                    double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * 3) return;
  double v = 0.0;
  for (int q = 0; q < S; ++q) v += part[(size_t)q * ns * 3 + t];
  out[t] = v * scale;
}

// position gradient = fA + fB + pd - pv (3 per site)
__global__ void add4_kernel(int len, const double* __restrict__ a, const double* __restrict__ b,
                            const double* __restrict__ c, const double* __restrict__ d, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < len) out[t] = a[t] + b[t] + c[t] - d[t];
}

// site weights (q, d + mu, Q) of the right-hand side's multipoles
__global__ void rhs_weights_kernel(int ns, const double* __restrict__ q, const double* __restrict__ d,
                                   const double* __restrict__ mu, const double* __restrict__ Q,
                                   double* __restrict__ wq, double* __restrict__ wd, double* __restrict__ wQ) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= ns) return;
  wq[l] = q[l];
  for (int a = 0; a < 3; ++a) wd[3 * l + a] = d[3 * l + a] + mu[3 * l + a];
  for (int a = 0; a < 6; ++a) wQ[6 * l + a] = Q[6 * l + a];
}

// g10[l] = sum_k coef_k * f_k[l] (10 components), NULL inputs skipped
__global__ void combine10_kernel(int ns, double c0, const double* __restrict__ f0, double c1,
                                 const double* __restrict__ f1, double c2, const double* __restrict__ f2, double c3,
                                 const double* __restrict__ f3, double c4, const double* __restrict__ f4,
                                 double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * 10) return;
  double v = 0.0;
  if (f0) v += c0 * f0[t];
  if (f1) v += c1 * f1[t];
  if (f2) v += c2 * f2[t];
  if (f3) v += c3 * f3[t];
  if (f4) v += c4 * f4[t];
  out[t] = v;
}

// nu~ <- (1 - w) nu~ + w a (c + f + Tn) for the active systems; out_sq[s] = sum of squared changes
__global__ void adj_sor_kernel(double* __restrict__ nu, const double4* __restrict__ pos, const double* __restrict__ c3,
                               const double* __restrict__ f10, const double* __restrict__ t3,
                               const int* __restrict__ sys_site, const int* __restrict__ active, double omega,
                               double* __restrict__ out_sq) {
  __shared__ double sh[256];
  const int l0 = sys_site[blockIdx.x], l1 = sys_site[blockIdx.x + 1];
  const bool on = !active || active[blockIdx.x];
  double v = 0.0;
  for (int l = l0 + threadIdx.x; on && l < l1; l += 256) {
    const double fa = 4.0 * M_PI * pos[l].w;
    for (int a = 0; a < 3; ++a) {
      const double src = c3[3 * l + a] + (f10 ? f10[10 * l + 1 + a] : 0.0) + t3[3 * l + a];
      const double old = nu[3 * l + a];
      const double nw = (1.0 - omega) * old + omega * fa * src;
      nu[3 * l + a] = nw;
      v += (nw - old) * (nw - old);
    }
  }
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out_sq[blockIdx.x] = sh[0];
}

// adjoint weights of the transposed BEM right-hand side: (q/2, d/2 - nu~, Q/2)
__global__ void adj_weights_kernel(int ns, const double* __restrict__ q, const double* __restrict__ d,
                                   const double* __restrict__ Q, const double* __restrict__ nu,
                                   double* __restrict__ wq, double* __restrict__ wd, double* __restrict__ wQ) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= ns) return;
  wq[l] = 0.5 * q[l];
  for (int a = 0; a < 3; ++a) wd[3 * l + a] = 0.5 * d[3 * l + a] - nu[3 * l + a];
  for (int a = 0; a < 6; ++a) wQ[6 * l + a] = 0.5 * Q[6 * l + a];
}

// charges lambda_1 / eps_in at the collocation points, as (x, 0, 0, 0) strengths
__global__ void lam_strength_kernel(const double* __restrict__ lam, int n, double inv_eps, double4* __restrict__ str,
                                    float4* __restrict__ str32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  str[i] = make_double4(lam[i] * inv_eps, 0.0, 0.0, 0.0);
  str32[i] = make_float4((float)(lam[i] * inv_eps), 0.f, 0.f, 0.f);
}

// gradient from the combined 10-vectors: g_q = f[0], g_d = f[1..3], g_Q = traceless(H) / 6
__global__ void gradient_out_kernel(int ns, const double* __restrict__ f, double* __restrict__ gq,
                                    double* __restrict__ gd, double* __restrict__ gQ) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= ns) return;
  const double* v = f + 10 * l;
  if (gq) gq[l] = v[0];
  if (gd)
    for (int a = 0; a < 3; ++a) gd[3 * l + a] = v[1 + a];
  if (gQ) {
    const double tr = (v[4] + v[7] + v[9]) / 3.0;
    const double H[3][3] = {{v[4] - tr, v[5], v[6]}, {v[5], v[7] - tr, v[8]}, {v[6], v[8], v[9] - tr}};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) gQ[9 * l + 3 * a + b] = H[a][b] / 6.0;
  }
}

// ---------------------------------------------------------------- position derivatives
// Field triple (potential, gradient, Hessian xx xy xz yy yz zz) at R = field point -
// source of an undamped multipole (q, p, Q6) (Eq. pot_multipole and its derivatives).
template <typename T>
__device__ void field_und(double q, const double* p, const double* Q6, const T R[3], T& P, T g[3], T H[6]) {
  const T r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  const T ri = inv(sqrt(r2));
  const T i2 = ri * ri, i3 = i2 * ri, i5 = i3 * i2, i7 = i5 * i2, i9 = i7 * i2;
  const double QM[3][3] = {{Q6[0], Q6[1], Q6[2]}, {Q6[1], Q6[3], Q6[4]}, {Q6[2], Q6[4], Q6[5]}};
  T QR[3];
  for (int a = 0; a < 3; ++a) QR[a] = R[0] * QM[a][0] + R[1] * QM[a][1] + R[2] * QM[a][2];
  const T RQR = QR[0] * R[0] + QR[1] * R[1] + QR[2] * R[2];
  const T pR = R[0] * p[0] + R[1] * p[1] + R[2] * p[2];
  P = q * ri + pR * i3 + 0.5 * RQR * i5;
  for (int a = 0; a < 3; ++a)
    g[a] = (-q) * R[a] * i3 + p[a] * i3 - 3.0 * pR * R[a] * i5 + QR[a] * i5 - 2.5 * RQR * R[a] * i7;
  int k = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b, ++k) {
      const double dab = a == b ? 1.0 : 0.0;
      H[k] = q * (3.0 * R[a] * R[b] * i5 - dab * i3) + 15.0 * pR * R[a] * R[b] * i7 -
             3.0 * (pR * dab + p[a] * R[b] + p[b] * R[a]) * i5 + 17.5 * RQR * R[a] * R[b] * i9 -
             2.5 * (RQR * dab + 2.0 * QR[a] * R[b] + 2.0 * QR[b] * R[a]) * i7 + QM[a][b] * i5;
    }
}

// Field triple of a Thole-damped point dipole mu (alpha product aa of the pair).
template <typename T>
__device__ void field_damp(const double* mu, const T R[3], double aa, double thole_a, T& P, T g[3], T H[6]) {
  const T r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  const T r = sqrt(r2);
  const T ri = inv(r);
  const T i2 = ri * ri, i3 = i2 * ri, i5 = i3 * i2, i7 = i5 * i2;
  T l3 = dual(1.0), l5 = dual(1.0), l7 = dual(1.0);
  if (aa > 0.0) {
    const T au3 = (thole_a / ::sqrt(aa)) * r2 * r;
    const T e = exp(-au3);
    l3 = 1.0 - e;
    l5 = 1.0 - (1.0 + au3) * e;
    l7 = 1.0 - (1.0 + au3 + 0.6 * au3 * au3) * e;
  }
  const T mR = R[0] * mu[0] + R[1] * mu[1] + R[2] * mu[2];
  P = l3 * mR * i3;
  for (int a = 0; a < 3; ++a) g[a] = l3 * mu[a] * i3 - 3.0 * l5 * mR * R[a] * i5;
  int k = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b, ++k) {
      const double dab = a == b ? 1.0 : 0.0;
      H[k] = 15.0 * l7 * mR * R[a] * R[b] * i7 - 3.0 * l5 * (mR * dab + mu[a] * R[b] + mu[b] * R[a]) * i5;
    }
}

// Field triple of a point charge q and dipole p (no quadrupole).
template <typename T>
__device__ void field_cd(double q, double px, double py, double pz, const T R[3], T& P, T g[3], T H[6]) {
  const T r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  const T ri = inv(sqrt(r2));
  const T i2 = ri * ri, i3 = i2 * ri, i5 = i3 * i2, i7 = i5 * i2;
  const double p[3] = {px, py, pz};
  const T pR = R[0] * px + R[1] * py + R[2] * pz;
  P = q * ri + pR * i3;
  for (int a = 0; a < 3; ++a) g[a] = (-q) * R[a] * i3 + p[a] * i3 - 3.0 * pR * R[a] * i5;
  int k = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b, ++k) {
      const double dab = a == b ? 1.0 : 0.0;
      H[k] = q * (3.0 * R[a] * R[b] * i5 - dab * i3) + 15.0 * pR * R[a] * R[b] * i7 -
             3.0 * (pR * dab + p[a] * R[b] + p[b] * R[a]) * i5;
    }
}

// <m, F> = q P + d . g + Q : H / 6 (energy weights of Eq. energy_multipole_polarizable)
template <typename T>
__device__ T contract(double q, const double* d, const double* Q6, const T& P, const T g[3], const T H[6]) {
  return q * P + d[0] * g[0] + d[1] * g[1] + d[2] * g[2] +
         (1.0 / 6.0) * (Q6[0] * H[0] + Q6[3] * H[3] + Q6[5] * H[5] +
                        2.0 * (Q6[1] * H[1] + Q6[2] * H[2] + Q6[4] * H[4]));
}

// d/dr_l of the site-site part of the Lagrangian, warp per site l, over l's body
// (whole = 0) or system (whole = 1).  Per pair (l, m), with E(a <- b) = <a, F_b>:
//   W = E(m_l <- m_m) + [E(m_l <- mu_m) + E(m_m <- mu_l)]/2 (damped)
//       - [E(nu_l <- m_m) + E(nu_m <- m_l)] (undamped, only across polarisation groups)
//       - [E(nu_l <- mu_m) + E(nu_m <- mu_l)] (damped),
// nu the adjoint dipoles; the permanent-permanent, induced-energy, masked-field and
// T-coupling terms of the energy and of the induced-dipole constraint.  R = r_l - r_m
// carries the derivative.  out[3l..] = sign * scale * dW/dr_l summed over m.
__global__ void __launch_bounds__(256) pair_force_kernel(const double4* __restrict__ pos,
                                                         const double* __restrict__ q, const double* __restrict__ d,
                                                         const double* __restrict__ Q, const double* __restrict__ mu,
                                                         const double* __restrict__ nu, const int* __restrict__ group,
                                                         const int* __restrict__ stag, const int* __restrict__ gsite,
                                                         const int* __restrict__ grp_sys,
                                                         const int* __restrict__ sys_site, int ns, int whole,
                                                         double thole_a, double scale, double* __restrict__ out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * 8 + warp;
  if (l >= ns) return;
  const double4 pl = pos[l];
  const int tg = stag[l];
  const int m0 = whole ? sys_site[grp_sys[tg]] : gsite[tg];
  const int m1 = whole ? sys_site[grp_sys[tg] + 1] : gsite[tg + 1];
  const double ql = q[l];
  const double dl[3] = {d[3 * l], d[3 * l + 1], d[3 * l + 2]};
  const double* Ql = Q + 6 * l;
  const double mul[3] = {mu[3 * l], mu[3 * l + 1], mu[3 * l + 2]};
  const double nul[3] = {nu[3 * l], nu[3 * l + 1], nu[3 * l + 2]};
  const double zero6[6] = {0, 0, 0, 0, 0, 0};
  double acc[3] = {0, 0, 0};
  for (int m = m0 + lane; m < m1; m += 32) {
    if (m == l) continue;
    const double4 pm = pos[m];
    const Dual3 R[3] = {seed(pl.x - pm.x, 0), seed(pl.y - pm.y, 1), seed(pl.z - pm.z, 2)};
    const Dual3 Rn[3] = {-R[0], -R[1], -R[2]};
    const double qm = q[m];
    const double dm[3] = {d[3 * m], d[3 * m + 1], d[3 * m + 2]};
    const double* Qm = Q + 6 * m;
    const double mum[3] = {mu[3 * m], mu[3 * m + 1], mu[3 * m + 2]};
    const double num[3] = {nu[3 * m], nu[3 * m + 1], nu[3 * m + 2]};
    const double aa = pl.w * pm.w;
    const bool masked = group[m] != group[l];
    Dual3 P, g[3], H[6];
    // sources at m seen from l
    field_und(qm, dm, Qm, R, P, g, H);
    Dual3 W = contract(ql, dl, Ql, P, g, H);
    if (masked) W = W - contract(0.0, nul, zero6, P, g, H);
    field_damp(mum, R, aa, thole_a, P, g, H);
    W = W + 0.5 * contract(ql, dl, Ql, P, g, H) - contract(0.0, nul, zero6, P, g, H);
    // sources at l seen from m
    if (masked) {
      field_und(ql, dl, Ql, Rn, P, g, H);
      W = W - contract(0.0, num, zero6, P, g, H);
    }
    field_damp(mul, Rn, aa, thole_a, P, g, H);
    W = W + 0.5 * contract(qm, dm, Qm, P, g, H) - contract(0.0, num, zero6, P, g, H);
    acc[0] += W.d0;
    acc[1] += W.d1;
    acc[2] += W.d2;
  }
  for (int c = 0; c < 3; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    acc[c] = v;
  }
  if (lane == 0)
    for (int c = 0; c < 3; ++c) out[3 * l + c] = acc[c] * scale;
}

// d/dr_l <w_l, F(r_l)> of the field F of surface sources (charge s.x, dipole s.y..w,
// at K positions per panel of l's body), warp per site, sources staged in shared
// memory; blockIdx.y takes an equal share; part[(y * ns + l) * 3 ..] (x 4 pi).
// S = float: dual arithmetic in FP32 (sites are at least a near radius from every
// panel), per-lane sums in FP64.
template <typename S>
__global__ void __launch_bounds__(256) site_force_kernel(const double4* __restrict__ spos, int ns,
                                                         const int4* __restrict__ sblk, const int* __restrict__ gpan,
                                                         int K, const double4* __restrict__ src,
                                                         const double4* __restrict__ str,
                                                         const double* __restrict__ wq, const double* __restrict__ wd,
                                                         const double* __restrict__ wQ, double* __restrict__ part) {
  constexpr int T = 256;
  __shared__ double4 tp[T];
  __shared__ double4 ts[T];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 B = sblk[blockIdx.x];
  const bool act = warp < B.y;
  const int site = B.x + warp;
  const int r0 = K * gpan[B.z], r1 = K * gpan[B.z + 1];
  const int per = ((r1 - r0 + (int)gridDim.y - 1) / (int)gridDim.y + T - 1) / T * T;
  const int s0 = r0 + blockIdx.y * per, s1 = min(r1, s0 + per);
  const double4 sd = act ? spos[site] : make_double4(0, 0, 0, 0);
  double w0 = 0, w1[3] = {0, 0, 0}, w2[6] = {0, 0, 0, 0, 0, 0};
  if (act) {
    w0 = wq[site];
    for (int a = 0; a < 3; ++a) w1[a] = wd[3 * site + a];
    for (int a = 0; a < 6; ++a) w2[a] = wQ[6 * site + a];
  }
  const Dual3T<S> X[3] = {seed_of<S>((S)sd.x, 0), seed_of<S>((S)sd.y, 1), seed_of<S>((S)sd.z, 2)};
  double acc[3] = {0, 0, 0};
  for (int t0 = s0; t0 < s1; t0 += T) {
    const int j = t0 + threadIdx.x;
    if (j < s1) {
      tp[threadIdx.x] = src[j];
      ts[threadIdx.x] = str[j];
    }
    __syncthreads();
    const int lim = min(T, s1 - t0);
    if (act) {
      for (int k = lane; k < lim; k += 32) {
        const double4 p = tp[k], sv = ts[k];
        const Dual3T<S> R[3] = {X[0] - (S)p.x, X[1] - (S)p.y, X[2] - (S)p.z};
        Dual3T<S> P, g[3], H[6];
        field_cd(sv.x, -sv.y, -sv.z, -sv.w, R, P, g, H);
        const Dual3T<S> e = contract(w0, w1, w2, P, g, H);
        acc[0] += (double)e.d0;
        acc[1] += (double)e.d1;
        acc[2] += (double)e.d2;
      }
    }
    __syncthreads();
  }
  for (int c = 0; c < 3; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    acc[c] = v;
  }
  if (lane == 0 && act) {
    double* o = part + ((size_t)blockIdx.y * ns + site) * 3;
    for (int c = 0; c < 3; ++c) o[c] = acc[c];
  }
}

}  // namespace

void ensure_near_transpose(Ctx& c, cudaStream_t s) {
  if (c.nearT_ready) return;
  const int n = c.n;
  std::vector<int> ptr(n + 1), col(std::max<int64_t>(1, c.nnz));
  BP_CUDA(cudaMemcpyAsync(ptr.data(), c.near_ptr.p, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s));
  if (c.nnz)
    BP_CUDA(cudaMemcpyAsync(col.data(), c.near_col.p, sizeof(int) * c.nnz, cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  std::vector<int> pT(n + 1, 0), rT(std::max<int64_t>(1, c.nnz)), eT(std::max<int64_t>(1, c.nnz));
  for (int64_t e = 0; e < c.nnz; ++e) ++pT[col[e] + 1];
  for (int j = 0; j < n; ++j) pT[j + 1] += pT[j];
  std::vector<int> fill(pT.begin(), pT.end() - 1);
  for (int i = 0; i < n; ++i)
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
      const int k = fill[col[e]]++;
      rT[k] = i;
      eT[k] = e;
    }
  c.near_ptrT.alloc(n + 1);
  c.near_rowT.alloc(rT.size());
  c.near_eT.alloc(eT.size());
  BP_CUDA(cudaMemcpyAsync(c.near_ptrT.p, pT.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaMemcpyAsync(c.near_rowT.p, rT.data(), sizeof(int) * rT.size(), cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaMemcpyAsync(c.near_eT.p, eT.data(), sizeof(int) * eT.size(), cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaStreamSynchronize(s));
  c.nearT_ready = true;
}

void matvec_T_internal(Ctx& c, const double* u, double* y, int op, cudaStream_t s) {
  const int n = c.n;
  ensure_near_transpose(c, s);
  const bool fp32 = (op == BEMPOL_OP_FP32_DIRECT || op == BEMPOL_OP_FP32_TREE);
  if (op == BEMPOL_OP_FP32_TREE) {
    tree_matvec_T_sums(c, u, s);
  } else {  // the direct forms; the FP64 tree form is applied as the FP64 direct product
    int maxr = 1;
    for (int g = 0; g < c.ngroup; ++g) {
      const int sy = c.h_grp_sys[g];
      maxr = std::max(maxr, c.h_sys_pan[sy + 1] - c.h_sys_pan[sy]);
    }
    int S = std::max(1, cdiv((long long)num_sms(c.device) * 8, std::max(1, c.ndblk)));
    S = std::min(S, std::max(1, maxr / (2 * TPB)));
    S = std::min(S, 64);
    const int per = cdiv(cdiv(maxr, S), TPB) * TPB;
    S = std::max(1, cdiv(maxr, per));
    if (c.part.n < (size_t)S * 4 * n) c.part.alloc((size_t)S * 4 * n);
    c.part_splits = S;
    dim3 grid(c.ndblk, S);
    Ctx::Timed tm;
    c.time_begin(0, s, tm);
    if (fp32)
      launch(p2pT_kernel<true>, grid, TPB, 0, s, c.tgt64.p, c.src64.p, c.nrm64.p, c.K, n, c.dblk.p, c.dblk_rng.p,
             c.blk_center.p, u, c.par.kappa, c.mv_active, c.grp_sys.p, c.part.p);
    else
      launch(p2pT_kernel<false>, grid, TPB, 0, s, c.tgt64.p, c.src64.p, c.nrm64.p, c.K, n, c.dblk.p, c.dblk_rng.p,
             c.blk_center.p, u, c.par.kappa, c.mv_active, c.grp_sys.p, c.part.p);
    c.time_end(s, tm);
  }
  launch(combineT_kernel, cdiv(n, 256), 256, 0, s, c.part.p, c.part_splits, n, c.near_ptrT.p, c.near_rowT.p,
         c.near_eT.p, c.near_corr.p, u, c.par.eps_in / c.par.eps_out, y);
  BP_CHECK_LAUNCH();
}

namespace {

struct TransposeScope {
  Ctx& c;
  explicit TransposeScope(Ctx& cc) : c(cc) { c.transposed = true; }
  ~TransposeScope() { c.transposed = false; }
};

}  // namespace

namespace {

// d/dr_l <w_l, F(r_l)> / (4 pi) for surface sources (src, str, K per panel) of l's body
void site_force(Ctx& c, const double4* src, const double4* str, int K, const double* wq, const double* wd,
                const double* wQ, double* out3, bool f32, cudaStream_t s) {
  int mr = 1;
  for (int g = 0; g < c.ngroup; ++g) mr = std::max(mr, K * (c.h_gpan[g + 1] - c.h_gpan[g]));
  int S = std::max(1, cdiv((long long)num_sms(c.device) * 6, std::max(1, c.nsblk)));
  S = std::min(S, std::max(1, mr / 1024));
  S = std::min(S, 256);
  const int per = cdiv(cdiv(mr, S), 256) * 256;
  S = std::max(1, cdiv(mr, per));
  DBuf<double> part;
  part.alloc((size_t)S * c.ns * 3);
  if (f32)
    launch(site_force_kernel<float>, dim3(c.nsblk, S), 256, 0, s, c.site_pos.p, c.ns, c.sblk.p, c.gpan.p, K, src,
           str, wq, wd, wQ, part.p);
  else
    launch(site_force_kernel<double>, dim3(c.nsblk, S), 256, 0, s, c.site_pos.p, c.ns, c.sblk.p, c.gpan.p, K, src,
           str, wq, wd, wQ, part.p);
  launch(force_reduce_kernel, cdiv(c.ns * 3, 256), 256, 0, s, part.p, S, c.ns, INV4PI, out3);
  BP_CHECK_LAUNCH();
  BP_CUDA(cudaStreamSynchronize(s));  // `part` is released on return
}

}  // namespace

AdjointOut gradient_internal(Ctx& c, double* g_q, double* g_d, double* g_Q, double* g_pos, cudaStream_t s) {
  const int n = c.n, ns = c.ns, S = c.nsys, len = 2 * n;
  const bempol_params& P = c.par;
  const double scale = INV4PI / P.eps_in;
  // Site-side sums in FP32 pairs (FP64 sums) when the solves' residual is an FP32 form.
  // When the forward solve refined only its final solve, the transposed solves run
  // with `op` alone and the site-side sums take op's precision.
  const bool final_only = P.residual_op != P.op && P.refine_scope == BEMPOL_REFINE_FINAL;
  const int prec_op = final_only ? P.op : P.residual_op;
  const bool f32 = (prec_op == BEMPOL_OP_FP32_DIRECT || prec_op == BEMPOL_OP_FP32_TREE);
  AdjointOut ao;
  DBuf<double> F_s, P_mu, P_0, Pv_mu, Pv_0, cmu, cmuv, nu, nuv, tn, psi, phinu, phinuv, g10, gv10, wq, wd, wQ, rT,
      lam;
  DBuf<double4> lstr;
  DBuf<float4> lstr32;
  DBuf<int> d_act;
  for (auto* b : {&F_s, &P_mu, &P_0, &Pv_mu, &Pv_0, &psi, &phinu, &phinuv, &g10, &gv10}) b->alloc(10 * (size_t)ns);
  for (auto* b : {&cmu, &cmuv, &nu, &nuv, &tn, &wd}) b->alloc(3 * (size_t)ns);
  wq.alloc(ns);
  wQ.alloc(6 * (size_t)ns);
  rT.alloc(len);
  lam.alloc(len);
  lstr.alloc(n);
  lstr32.alloc(n);
  d_act.alloc(S);
  nu.zero(s);
  nuv.zero(s);
  lam.zero(s);
  DBuf<double> zero3;
  zero3.alloc(3 * (size_t)ns);
  zero3.zero(s);
  // forward quantities at the solution: reaction fields (FP64) and energy-form multipole potentials
  site_reaction_form(c, c.sol_x.p, F_s.p, P.residual_op, true, s);  // as the forward energy's
  multipole_internal(c, c.sol_mu.p, 1, P_mu.p, s, f32);
  multipole_internal(c, zero3.p, 1, P_0.p, s, f32);
  multipole_internal(c, c.sol_mu_v.p, 3, Pv_mu.p, s, f32);
  multipole_internal(c, zero3.p, 3, Pv_0.p, s, f32);
  // c_mu = -1/2 (damped unmasked field of the permanent moments), dissolved (body) and vacuum (system)
  launch(site_adjoint_kernel, cdiv(ns, 8), 256, 0, s, c.site_pos.p, c.site_q.p, c.site_d.p, c.site_Q.p, zero3.p,
         c.site_group.p, c.stag.p, c.gsite.p, c.grp_sys.p, c.sys_site.p, ns, 0, 0, P.thole_a, -0.5 * scale, cmu.p);
  launch(site_adjoint_kernel, cdiv(ns, 8), 256, 0, s, c.site_pos.p, c.site_q.p, c.site_d.p, c.site_Q.p, zero3.p,
         c.site_group.p, c.stag.p, c.gsite.p, c.grp_sys.p, c.sys_site.p, ns, 0, 1, P.thole_a, -0.5 * scale,
         cmuv.p);
  BP_CHECK_LAUNCH();

  auto upload_act = [&](const std::vector<int>& act) {
    int* hp = reinterpret_cast<int*>(c.h_pinned + 2 * S);
    std::copy(act.begin(), act.end(), hp);
    BP_CUDA(cudaMemcpyAsync(d_act.p, hp, sizeof(int) * S, cudaMemcpyHostToDevice, s));
    BP_CUDA(cudaStreamSynchronize(s));
  };
  auto read_sq = [&]() {
    BP_CUDA(cudaMemcpyAsync(c.h_pinned, c.scal.p, sizeof(double) * S, cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaStreamSynchronize(s));
    std::vector<double> r(S);
    for (int q = 0; q < S; ++q)
      r[q] = std::sqrt(c.h_pinned[q] / std::max(1, c.h_sys_site[q + 1] - c.h_sys_site[q]));
    return r;
  };
  // transposed BEM solve for the current nu~: lambda = A^-T R^T (q/2, d/2 - nu~, Q/2), warm-started
  auto adj_bem = [&](const std::vector<char>& want) {
    launch(adj_weights_kernel, cdiv(ns, 128), 128, 0, s, ns, c.site_q.p, c.site_d.p, c.site_Q.p, nu.p, wq.p, wd.p,
           wQ.p);
    if (f32)
      launch(adj_reaction_kernel<float>, c.ndblk, TPB, 0, s, c.src64.p, c.nrm64.p, c.K, n, c.dblk.p, c.blk_center.p,
             c.gsite.p, c.site_pos.p, wq.p, wd.p, wQ.p, rT.p);
    else
      launch(adj_reaction_kernel<double>, c.ndblk, TPB, 0, s, c.src64.p, c.nrm64.p, c.K, n, c.dblk.p,
             c.blk_center.p, c.gsite.p, c.site_pos.p, wq.p, wd.p, wQ.p, rT.p);
    BP_CHECK_LAUNCH();
    GmresOut g;
    {
      TransposeScope ts(c);
      g = solve_bem(c, rT.p, lam.p, want, s, !final_only);
    }
    ao.gmres_iters += g.iters;
    ++ao.solves;
    if (!g.converged) ao.converged = false;
    launch(lam_strength_kernel, cdiv(n, 256), 256, 0, s, lam.p, n, 1.0 / P.eps_in, lstr.p, lstr32.p);
    site_field_of_charges(c, c.tgt64.p, lstr.p, c.tgt32.p, lstr32.p, 1, f32, psi.p, s);
  };
  // dissolved: relaxed transposed SCF
  {
    std::vector<int> act(S, 1);
    std::vector<char> want(S, 1);
    for (int it = 1; it <= P.scf_maxit; ++it) {
      for (int q = 0; q < S; ++q) want[q] = (char)act[q];
      adj_bem(want);
      multipole_internal(c, nu.p, 0 | 4, tn.p, s, f32);  // T nu~: damped field of the dipoles nu~ alone
      upload_act(act);
      launch(adj_sor_kernel, S, 256, 0, s, nu.p, c.site_pos.p, cmu.p, psi.p, tn.p, c.sys_site.p, d_act.p,
             P.sor_omega, c.scal.p);
      std::vector<double> rms = read_sq();
      int left = 0;
      for (int q = 0; q < S; ++q) {
        if (!act[q]) continue;
        ao.iters_diss = std::max(ao.iters_diss, it);
        if (rms[q] < P.scf_tol || !std::isfinite(rms[q])) {
          if (!std::isfinite(rms[q])) ao.converged = false;
          act[q] = 0;
        } else {
          ++left;
        }
      }
      if (!left) break;
      if (it == P.scf_maxit) ao.converged = false;
    }
    std::vector<char> all(S, 1);
    adj_bem(all);  // lambda and Psi for the converged nu~
  }
  // vacuum: relaxed transposed SCF without BEM
  {
    std::vector<int> act(S, 1);
    for (int it = 1; it <= P.scf_maxit; ++it) {
      multipole_internal(c, nuv.p, 2 | 4, tn.p, s, f32);
      upload_act(act);
      launch(adj_sor_kernel, S, 256, 0, s, nuv.p, c.site_pos.p, cmuv.p, (const double*)nullptr, tn.p, c.sys_site.p,
             d_act.p, P.sor_omega, c.scal.p);
      std::vector<double> rms = read_sq();
      int left = 0;
      for (int q = 0; q < S; ++q) {
        if (!act[q]) continue;
        ao.iters_vac = std::max(ao.iters_vac, it);
        if (rms[q] < P.scf_tol || !std::isfinite(rms[q])) {
          if (!std::isfinite(rms[q])) ao.converged = false;
          act[q] = 0;
        } else {
          ++left;
        }
      }
      if (!left) break;
      if (it == P.scf_maxit) ao.converged = false;
    }
  }
  // masked undamped potentials of the adjoint dipoles
  launch(site_adjoint_kernel, cdiv(ns, 8), 256, 0, s, c.site_pos.p, c.site_q.p, c.site_d.p, c.site_Q.p, nu.p,
         c.site_group.p, c.stag.p, c.gsite.p, c.grp_sys.p, c.sys_site.p, ns, 1, 0, P.thole_a, scale, phinu.p);
  launch(site_adjoint_kernel, cdiv(ns, 8), 256, 0, s, c.site_pos.p, c.site_q.p, c.site_d.p, c.site_Q.p, nuv.p,
         c.site_group.p, c.stag.p, c.gsite.p, c.grp_sys.p, c.sys_site.p, ns, 1, 1, P.thole_a, scale, phinuv.p);
  // dG_diss = F_s/2 + (P(mu) + P(0))/2 + Psi - phi_nu ;  dG_vac = (P_v(mu_v) + P_v(0))/2 - phi_nu,v
  launch(combine10_kernel, cdiv(ns * 10, 256), 256, 0, s, ns, 0.5, F_s.p, 0.5, P_mu.p, 0.5, P_0.p, 1.0, psi.p, -1.0,
         phinu.p, g10.p);
  launch(combine10_kernel, cdiv(ns * 10, 256), 256, 0, s, ns, 0.5, Pv_mu.p, 0.5, Pv_0.p, -1.0, phinuv.p, 0.0,
         (const double*)nullptr, 0.0, (const double*)nullptr, gv10.p);
  launch(combine10_kernel, cdiv(ns * 10, 256), 256, 0, s, ns, 1.0, g10.p, -1.0, gv10.p, 0.0, (const double*)nullptr,
         0.0, (const double*)nullptr, 0.0, (const double*)nullptr, g10.p);
  launch(gradient_out_kernel, cdiv(ns, 128), 128, 0, s, ns, g10.p, g_q, g_d, g_Q);
  BP_CHECK_LAUNCH();
  if (g_pos) {
    // Position derivatives of the Lagrangian at the converged state (x, mu, lambda, nu):
    // (A) the surface solution's fields at the sites with weights (q/2, d/2 - nu~, Q/2)
    //     (still in wq, wd, wQ from the last transposed solve),
    // (B) the fields of the charges lambda_1 / eps_in at the collocation points with
    //     weights (q, d + mu, Q) (the right-hand side's dependence on the sites),
    // (C) the site-site terms, dissolved minus vacuum.
    DBuf<double> fA, fB, pd, pv, wq2, wd2, wQ2;
    for (auto* b : {&fA, &fB, &pd, &pv, &wd2}) b->alloc(3 * (size_t)ns);
    wq2.alloc(ns);
    wQ2.alloc(6 * (size_t)ns);
    strengths(c, c.sol_x.p, false, s);
    site_force(c, c.src64.p, c.str64.p, c.K, wq.p, wd.p, wQ.p, fA.p, f32, s);
    launch(rhs_weights_kernel, cdiv(ns, 128), 128, 0, s, ns, c.site_q.p, c.site_d.p, c.sol_mu.p, c.site_Q.p, wq2.p,
           wd2.p, wQ2.p);
    site_force(c, c.tgt64.p, lstr.p, 1, wq2.p, wd2.p, wQ2.p, fB.p, f32, s);
    launch(pair_force_kernel, cdiv(ns, 8), 256, 0, s, c.site_pos.p, c.site_q.p, c.site_d.p, c.site_Q.p, c.sol_mu.p,
           nu.p, c.site_group.p, c.stag.p, c.gsite.p, c.grp_sys.p, c.sys_site.p, ns, 0, P.thole_a, scale, pd.p);
    launch(pair_force_kernel, cdiv(ns, 8), 256, 0, s, c.site_pos.p, c.site_q.p, c.site_d.p, c.site_Q.p,
           c.sol_mu_v.p, nuv.p, c.site_group.p, c.stag.p, c.gsite.p, c.grp_sys.p, c.sys_site.p, ns, 1, P.thole_a,
           scale, pv.p);
    launch(add4_kernel, cdiv(3 * ns, 256), 256, 0, s, 3 * ns, fA.p, fB.p, pd.p, pv.p, g_pos);
    BP_CHECK_LAUNCH();
  }
  BP_CUDA(cudaStreamSynchronize(s));
  return ao;
}

}  // namespace bp
