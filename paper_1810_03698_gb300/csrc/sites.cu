// Site-side kernels: multipole right-hand side (Eq. rhs_multipole), reaction
// potential/field/Hessian at the sites (Eqs. pot_solvent, Efield_solv, ddphi),
// multipole-multipole fields with Thole damping (Eqs. Efield_mult,
// derivatives_Emult, second_derivative), the SOR update of the induced dipoles
// (Sec. "Self-consistent induced field") and the energy of Eq.
// energy_multipole_polarizable.
//
// Tensor conventions: R = r_field - r_source, r = |R|.  A site with charge q,
// dipole p and traceless quadrupole Q (Eq. pot_multipole) has potential
//   q/r + p.R/r^3 + R.Q.R/(2 r^5)        (times 1/(4 pi eps_in))
// gradient
//   -q R/r^3 + p/r^3 - 3 (p.R) R/r^5 + Q R/r^5 - (5/2)(R.Q.R) R/r^7
// and Hessian
//   q (3 R R/r^5 - I/r^3) + 15 (p.R) R R/r^7 - 3 ((p.R) I + p R + R p)/r^5
//   + (35/2)(R.Q.R) R R/r^9 - (5/2)((R.Q.R) I + 2 (Q R) R + 2 R (Q R))/r^7 + Q/r^5.
// Induced dipoles mu use the Thole-damped forms (AMOEBA reading of the paper's
// "Thole-like" damping): u^3 = r^3 / sqrt(alpha_l alpha_m), e = exp(-a u^3),
// lambda3 = 1 - e, lambda5 = 1 - (1 + a u^3) e, lambda7 = 1 - (1 + a u^3 + 0.6 (a u^3)^2) e:
//   potential lambda3 mu.R/r^3, gradient lambda3 mu/r^3 - 3 lambda5 (mu.R) R/r^5,
//   Hessian 15 lambda7 (mu.R) R R/r^7 - 3 lambda5 ((mu.R) I + mu R + R mu)/r^5.
// Induced dipoles: mu = 4 pi alpha E (alpha a polarizability volume, potentials
// in units with vacuum permittivity 1).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace bp {

namespace {

constexpr double INV4PI = 0.07957747154594767;  // 1/(4 pi)

struct SiteSrc {   // one multipole, 13 values
  double x, y, z, q, px, py, pz, qxx, qxy, qxz, qyy, qyz, qzz;
};

// ---------------------------------------------------------------- RHS
// One block per direct target block (<= 128 panels of one body): the panels see the
// sites of their own body only.
template <typename Real>
__global__ void rhs_kernel(const double4* __restrict__ tgt, const int4* __restrict__ blk,
                           const int* __restrict__ gsite, const double4* __restrict__ spos,
                           const double* __restrict__ sq, const double* __restrict__ sp,
                           const double* __restrict__ sQ, double scale, double* __restrict__ b) {
  constexpr int T = 128;
  __shared__ Real sh[13][T];
  const int4 B = blk[blockIdx.x];
  const int i = B.x + threadIdx.x;
  const bool act = (int)threadIdx.x < B.y;
  const int k0 = gsite[B.z], k1 = gsite[B.z + 1];
  double4 xd = act ? tgt[i] : make_double4(0, 0, 0, 0);
  Real x = (Real)xd.x, y = (Real)xd.y, z = (Real)xd.z;
  double acc = 0.0;
  for (int t0 = k0; t0 < k1; t0 += T) {
    int k = t0 + threadIdx.x;
    if (k < k1) {
      double4 p = spos[k];
      sh[0][threadIdx.x] = (Real)p.x;
      sh[1][threadIdx.x] = (Real)p.y;
      sh[2][threadIdx.x] = (Real)p.z;
      sh[3][threadIdx.x] = (Real)sq[k];
      sh[4][threadIdx.x] = (Real)sp[3 * k];
      sh[5][threadIdx.x] = (Real)sp[3 * k + 1];
      sh[6][threadIdx.x] = (Real)sp[3 * k + 2];
      for (int c = 0; c < 6; ++c) sh[7 + c][threadIdx.x] = (Real)sQ[6 * k + c];
    }
    __syncthreads();
    int lim = min(T, k1 - t0);
    Real a = 0;
    for (int kk = 0; kk < lim; ++kk) {
      Real Rx = x - sh[0][kk], Ry = y - sh[1][kk], Rz = z - sh[2][kk];
      Real r2 = Rx * Rx + Ry * Ry + Rz * Rz;
      Real rinv = (Real)1 / sqrt(r2);
      Real rinv2 = rinv * rinv;
      Real rinv3 = rinv2 * rinv;
      Real pR = sh[4][kk] * Rx + sh[5][kk] * Ry + sh[6][kk] * Rz;
      Real RQR = sh[7][kk] * Rx * Rx + sh[10][kk] * Ry * Ry + sh[12][kk] * Rz * Rz +
                 (Real)2 * (sh[8][kk] * Rx * Ry + sh[9][kk] * Rx * Rz + sh[11][kk] * Ry * Rz);
      a += sh[3][kk] * rinv + pR * rinv3 + (Real)0.5 * RQR * rinv3 * rinv2;
    }
    acc += (double)a;
    __syncthreads();
  }
  if (act) b[i] = acc * scale;
}

// ---------------------------------------------------------------- reaction at sites
// warp per site; the block's (up to 8) sites belong to one body, whose Gauss nodes
// (its own surface: the Laplace layers) are the sources, staged in shared memory.
// blockIdx.y takes an equal share of them.
template <typename Real, typename R4, bool HESS>
__global__ void __launch_bounds__(256) site_reaction_kernel(const double4* __restrict__ spos_site, int ns,
                                                            const int4* __restrict__ sblk,
                                                            const int* __restrict__ gpan, int K,
                                                            const R4* __restrict__ src, const R4* __restrict__ str,
                                                            double* __restrict__ part) {
  constexpr int T = 256;
  __shared__ R4 tp[T];
  __shared__ R4 ts[T];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 B = sblk[blockIdx.x];
  const bool act = warp < B.y;
  const int site = B.x + warp;
  const int r0 = K * gpan[B.z], r1 = K * gpan[B.z + 1];
  const int per = ((r1 - r0 + (int)gridDim.y - 1) / (int)gridDim.y + T - 1) / T * T;
  const int s0 = r0 + blockIdx.y * per, s1 = min(r1, s0 + per);
  double4 sd = act ? spos_site[site] : make_double4(0, 0, 0, 0);
  const Real X = (Real)sd.x, Y = (Real)sd.y, Z = (Real)sd.z;
  double acc[10];
#pragma unroll
  for (int c = 0; c < 10; ++c) acc[c] = 0.0;
  for (int t0 = s0; t0 < s1; t0 += T) {
    int j = t0 + threadIdx.x;
    if (j < s1) {
      tp[threadIdx.x] = src[j];
      ts[threadIdx.x] = str[j];
    }
    __syncthreads();
    int lim = min(T, s1 - t0);
    Real a[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) a[c] = 0;
    for (int k = lane; k < lim; k += 32) {
      R4 p = tp[k], s = ts[k];
      Real Rx = X - p.x, Ry = Y - p.y, Rz = Z - p.z;
      Real r2 = Rx * Rx + Ry * Ry + Rz * Rz;
      Real rinv = (Real)1 / sqrt(r2);
      Real rinv2 = rinv * rinv;
      Real A3 = rinv2 * rinv;             // 1/r^3
      Real B5 = (Real)3 * A3 * rinv2;      // 3/r^5
      Real m = s.x;
      Real dR = s.y * Rx + s.z * Ry + s.w * Rz;
      a[0] += m * rinv - dR * A3;
      Real gc = -m * A3 + dR * B5;
      a[1] += gc * Rx - s.y * A3;
      a[2] += gc * Ry - s.z * A3;
      a[3] += gc * Rz - s.w * A3;
      if (HESS) {
        Real C7 = (Real)5 * B5 * rinv2;    // 15/r^7
        Real hc = m * B5 - dR * C7;
        Real hd = dR * B5 - m * A3;
        a[4] += hc * Rx * Rx + hd + (Real)2 * B5 * Rx * s.y;
        a[5] += hc * Rx * Ry + B5 * (Rx * s.z + Ry * s.y);
        a[6] += hc * Rx * Rz + B5 * (Rx * s.w + Rz * s.y);
        a[7] += hc * Ry * Ry + hd + (Real)2 * B5 * Ry * s.z;
        a[8] += hc * Ry * Rz + B5 * (Ry * s.w + Rz * s.z);
        a[9] += hc * Rz * Rz + hd + (Real)2 * B5 * Rz * s.w;
      }
    }
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[c] += (double)a[c];
    __syncthreads();
  }
  const int nc = HESS ? 10 : 4;
#pragma unroll
  for (int c = 0; c < 10; ++c) {
    if (c >= nc) break;
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    acc[c] = v;
  }
  if (lane == 0 && act) {
    double* o = part + ((size_t)blockIdx.y * ns + site) * 10;
    for (int c = 0; c < 10; ++c) o[c] = c < nc ? acc[c] : 0.0;
  }
}

__global__ void site_reduce_kernel(const double* __restrict__ part, int S, int ns, double* __restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ns * 10) return;
  double v = 0;
  for (int s = 0; s < S; ++s) v += part[(size_t)s * ns * 10 + t];
  out[t] = v * INV4PI;
}

// ---------------------------------------------------------------- multipole-multipole
// mode 0: polarising field E (3 per site): permanent masked by group, induced damped.
// mode 1: energy potentials (10 per site): permanent unmasked, induced damped.
// Modes 0 and 1 sum over the sites of the site's own body (dissolved state: each
// cavity holds its own multipoles), modes 2 and 3 are the same over every site of
// its system (vacuum state).  Adding 4 to the mode drops the permanent moments
// (the damped field of the dipoles `mu` alone).
template <typename Real>
__global__ void __launch_bounds__(256) multipole_kernel(const double4* __restrict__ pos, const double* __restrict__ q,
                                                        const double* __restrict__ d, const double* __restrict__ Q,
                                                        const double* __restrict__ mu, const int* __restrict__ group,
                                                        const int* __restrict__ stag, const int* __restrict__ gsite,
                                                        const int* __restrict__ grp_sys,
                                                        const int* __restrict__ sys_site, int ns, int mode,
                                                        double thole_a, int damp_perm, double scale,
                                                        double* __restrict__ out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * 8 + warp;
  if (l >= ns) return;
  const double4 pl = pos[l];
  const int gl = group[l];
  const int tg = stag[l];
  const bool ind_only = (mode & 4) != 0;  // induced dipoles only (no permanent moments)
  mode &= 3;
  const bool whole = mode >= 2;
  const int m0 = whole ? sys_site[grp_sys[tg]] : gsite[tg];
  const int m1 = whole ? sys_site[grp_sys[tg] + 1] : gsite[tg + 1];
  mode &= 1;
  const Real ta = (Real)thole_a;
  // pair terms in Real, summed per lane in Real over up to 32 pairs, then into FP64
  double acc[10];
  Real part[10];
  for (int c = 0; c < 10; ++c) acc[c] = 0.0, part[c] = 0;
  int npart = 0;
  for (int m = m0 + lane; m < m1; m += 32) {
    if (m == l) continue;
    double4 pm = pos[m];
    const Real Rx = (Real)(pl.x - pm.x), Ry = (Real)(pl.y - pm.y), Rz = (Real)(pl.z - pm.z);
    const Real r2 = Rx * Rx + Ry * Ry + Rz * Rz;
    const Real rinv = (Real)1 / sqrt(r2);
    const Real i2 = rinv * rinv, i3 = i2 * rinv, i5 = i3 * i2, i7 = i5 * i2, i9 = i7 * i2;
    const Real R[3] = {Rx, Ry, Rz};
    Real g[3] = {0, 0, 0}, H[6] = {0, 0, 0, 0, 0, 0}, P = 0;
    // Thole factors of the pair (the induced dipoles' damping, and the permanent moments'
    // polarising field when damp_perm is set)
    const double aa = pl.w * pm.w;
    Real l3 = 1, l5 = 1, l7 = 1;
    if (aa > 0.0) {
      const Real au3 = ta * r2 * sqrt(r2) / (Real)sqrt(aa);
      const Real e = exp(-au3);
      l3 = (Real)1 - e;
      l5 = (Real)1 - ((Real)1 + au3) * e;
      l7 = (Real)1 - ((Real)1 + au3 + (Real)0.6 * au3 * au3) * e;
    }
    bool perm = !ind_only && ((mode == 1) || (group[m] != gl));
    if (perm) {
      const Real qm = (Real)q[m];
      const Real pv[3] = {(Real)d[3 * m], (Real)d[3 * m + 1], (Real)d[3 * m + 2]};
      const double* Qm = Q + 6 * m;
      const Real QM[3][3] = {{(Real)Qm[0], (Real)Qm[1], (Real)Qm[2]},
                             {(Real)Qm[1], (Real)Qm[3], (Real)Qm[4]},
                             {(Real)Qm[2], (Real)Qm[4], (Real)Qm[5]}};
      Real QR[3];
      for (int a = 0; a < 3; ++a) QR[a] = QM[a][0] * Rx + QM[a][1] * Ry + QM[a][2] * Rz;
      const Real RQR = QR[0] * Rx + QR[1] * Ry + QR[2] * Rz;
      const Real pR = pv[0] * Rx + pv[1] * Ry + pv[2] * Rz;
      P = qm * rinv + pR * i3 + (Real)0.5 * RQR * i5;
      // the polarising field (mode 0) optionally with the damped tensors: the 1/r^3 terms
      // take lambda3, the 1/r^5 terms lambda5, the 1/r^7 term lambda7
      const bool dp = damp_perm && mode == 0;
      const Real d3 = dp ? l3 : (Real)1, d5 = dp ? l5 : (Real)1, d7 = dp ? l7 : (Real)1;
      for (int a = 0; a < 3; ++a)
        g[a] = d3 * (-qm * R[a] * i3 + pv[a] * i3) + d5 * (-(Real)3 * pR * R[a] * i5 + QR[a] * i5) -
               d7 * (Real)2.5 * RQR * R[a] * i7;
      if (mode == 1) {
        int k = 0;
        for (int a = 0; a < 3; ++a)
          for (int b = a; b < 3; ++b, ++k) {
            const Real dab = a == b ? (Real)1 : (Real)0;
            H[k] = qm * ((Real)3 * R[a] * R[b] * i5 - dab * i3) + (Real)15 * pR * R[a] * R[b] * i7 -
                   (Real)3 * (pR * dab + pv[a] * R[b] + pv[b] * R[a]) * i5 + (Real)17.5 * RQR * R[a] * R[b] * i9 -
                   (Real)2.5 * (RQR * dab + (Real)2 * QR[a] * R[b] + (Real)2 * QR[b] * R[a]) * i7 + QM[a][b] * i5;
          }
      }
    }
    // induced dipole, Thole damped
    const Real mv[3] = {(Real)mu[3 * m], (Real)mu[3 * m + 1], (Real)mu[3 * m + 2]};
    const Real mR = mv[0] * Rx + mv[1] * Ry + mv[2] * Rz;
    P += l3 * mR * i3;
    for (int a = 0; a < 3; ++a) g[a] += l3 * mv[a] * i3 - (Real)3 * l5 * mR * R[a] * i5;
    if (mode == 1) {
      int k = 0;
      for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b, ++k) {
          const Real dab = a == b ? (Real)1 : (Real)0;
          H[k] += (Real)15 * l7 * mR * R[a] * R[b] * i7 - (Real)3 * l5 * (mR * dab + mv[a] * R[b] + mv[b] * R[a]) * i5;
        }
    }
    part[0] += P;
    for (int a = 0; a < 3; ++a) part[1 + a] += g[a];
    for (int k = 0; k < 6; ++k) part[4 + k] += H[k];
    if (++npart == 32) {
      for (int c = 0; c < 10; ++c) acc[c] += (double)part[c], part[c] = 0;
      npart = 0;
    }
  }
  for (int c = 0; c < 10; ++c) acc[c] += (double)part[c];
  for (int c = 0; c < 10; ++c) {
    double v = acc[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    acc[c] = v;
  }
  if (lane == 0) {
    if (mode == 0) {
      for (int a = 0; a < 3; ++a) out[3 * l + a] = -acc[1 + a] * scale;
    } else {
      for (int c = 0; c < 10; ++c) out[10 * l + c] = acc[c] * scale;
    }
  }
}

// ---------------------------------------------------------------- energy and SOR
// one block per system: outE[s] = 1/2 sum over the system's sites
__global__ void energy_kernel(const double* __restrict__ q, const double* __restrict__ d,
                              const double* __restrict__ Q, const double* __restrict__ r10,
                              const double* __restrict__ m10, const int* __restrict__ sys_site,
                              double* __restrict__ outE) {
  __shared__ double sh[256];
  const int l0 = sys_site[blockIdx.x], l1 = sys_site[blockIdx.x + 1];
  double v = 0.0;
  for (int l = l0 + threadIdx.x; l < l1; l += 256) {
    double f[10];
    for (int c = 0; c < 10; ++c) f[c] = (r10 ? r10[10 * l + c] : 0.0) + (m10 ? m10[10 * l + c] : 0.0);
    const double* Ql = Q + 6 * l;
    double QH = Ql[0] * f[4] + Ql[3] * f[7] + Ql[5] * f[9] + 2.0 * (Ql[1] * f[5] + Ql[2] * f[6] + Ql[4] * f[8]);
    v += q[l] * f[0] + d[3 * l] * f[1] + d[3 * l + 1] * f[2] + d[3 * l + 2] * f[3] + QH / 6.0;
  }
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) outE[blockIdx.x] = 0.5 * sh[0];
}

// One block per system: mu_new = (1 - w) mu + w 4 pi alpha (E_solv + E_mult) for the
// system's sites when active[s] (NULL = every system); out_sq[s] = sum |mu_new - mu|^2.
__global__ void sor_kernel(double* __restrict__ mu, const double4* __restrict__ pos,
                           const double* __restrict__ react10, const double* __restrict__ emult,
                           const int* __restrict__ sys_site, const int* __restrict__ active, double omega,
                           double* __restrict__ out_sq) {
  __shared__ double sh[256];
  const int l0 = sys_site[blockIdx.x], l1 = sys_site[blockIdx.x + 1];
  const bool on = !active || active[blockIdx.x];
  double v = 0.0;
  for (int l = l0 + threadIdx.x; on && l < l1; l += 256) {
    double fa = 4.0 * M_PI * pos[l].w;
    for (int a = 0; a < 3; ++a) {
      double E = emult[3 * l + a] - (react10 ? react10[10 * l + 1 + a] : 0.0);
      double old = mu[3 * l + a];
      double nw = (1.0 - omega) * old + omega * fa * E;
      mu[3 * l + a] = nw;
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

// ---------------------------------------------------------------- validation
// flag[l] = 1 if site l is within the near radius of a panel centroid of its
// system, 2 if outside its own body's surface, 3 if inside another body's surface
__global__ void site_check_kernel(const double4* __restrict__ spos, int ns, const int* __restrict__ stag,
                                  const int* __restrict__ grp_sys, const int* __restrict__ sys_pan,
                                  const int* __restrict__ ptag, const double4* __restrict__ tgt64,
                                  const float4* __restrict__ src32, const double4* __restrict__ nrm64, int K,
                                  double nf2, int* __restrict__ flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = blockIdx.x * 8 + warp;
  if (l >= ns) return;
  double4 p = spos[l];
  const int g = stag[l];
  const int j0 = sys_pan[grp_sys[g]], j1 = sys_pan[grp_sys[g] + 1];
  int near = 0;
  double dl = 0.0, dother = 0.0;
  for (int j = j0 + lane; j < j1; j += 32) {
    double4 c = tgt64[j];
    double dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
    if (dx * dx + dy * dy + dz * dz < nf2 * c.w) near = 1;
    // inside test in FP32: -K_L[1] is 1 inside a closed surface and 0 outside, compared with 1/2
    double4 nj = nrm64[j];
    const float nx = (float)nj.x, ny = (float)nj.y, nz = (float)nj.z;
    float part = 0.f;
    for (int q = 0; q < K; ++q) {
      float4 y = src32[(size_t)K * j + q];
      float rx = (float)p.x - y.x, ry = (float)p.y - y.y, rz = (float)p.z - y.z;
      float r2 = rx * rx + ry * ry + rz * rz;
      float ri = rsqrtf(r2);
      part += y.w * (nx * rx + ny * ry + nz * rz) * ri * ri * ri;
    }
    if (ptag[j] == g)
      dl += (double)part;
    else
      dother += (double)part;
  }
  for (int o = 16; o > 0; o >>= 1) {
    dl += __shfl_down_sync(0xffffffffu, dl, o);
    dother += __shfl_down_sync(0xffffffffu, dother, o);
    near |= __shfl_down_sync(0xffffffffu, near, o);
  }
  if (lane == 0) {
    const double inside = -dl * INV4PI, inside_other = -dother * INV4PI;
    flag[l] = near ? 1 : (inside > 0.5 ? (inside_other > 0.5 ? 3 : 0) : 2);
  }
}

int site_splits(Ctx& c, int max_range) {
  int want = num_sms(c.device) * 6;
  int S = std::max(1, cdiv(want, std::max(1, c.nsblk)));
  S = std::min(S, std::max(1, max_range / 1024));
  S = std::min(S, 256);
  int per = cdiv(cdiv(max_range, S), 256) * 256;
  return std::max(1, cdiv(max_range, per));
}

int max_group_sources(const Ctx& c) {
  int m = 1;
  for (int g = 0; g < c.ngroup; ++g) m = std::max(m, c.K * (c.h_gpan[g + 1] - c.h_gpan[g]));
  return m;
}

template <typename Real, typename R4, bool HESS>
void launch_site_reaction(Ctx& c, int S, const R4* src, const R4* str, double* part, cudaStream_t s) {
  launch(site_reaction_kernel<Real, R4, HESS>, dim3(c.nsblk, S), 256, 0, s, c.site_pos.p, c.ns, c.sblk.p, c.gpan.p,
         c.K, src, str, part);
}

void site_reaction_launch(Ctx& c, int S, bool fp32, bool hessian, double* part, cudaStream_t s) {
  if (fp32) {
    if (hessian)
      launch_site_reaction<float, float4, true>(c, S, c.src32.p, c.str32.p, part, s);
    else
      launch_site_reaction<float, float4, false>(c, S, c.src32.p, c.str32.p, part, s);
  } else {
    if (hessian)
      launch_site_reaction<double, double4, true>(c, S, c.src64.p, c.str64.p, part, s);
    else
      launch_site_reaction<double, double4, false>(c, S, c.src64.p, c.str64.p, part, s);
  }
}

}  // namespace

// Potential, gradient and Hessian (10 per site, x 1/(4 pi)) at every site of the
// field of point charges str[j].x at positions src[j] (K per panel), over the
// panels of the site's own body; FP64, or FP32 pairs with FP64 sums (src32, str32).
void site_field_of_charges(Ctx& c, const double4* src, const double4* str, const float4* src32, const float4* str32,
                           int K, bool fp32, double* out10, cudaStream_t s) {
  int mr = 1;
  for (int g = 0; g < c.ngroup; ++g) mr = std::max(mr, K * (c.h_gpan[g + 1] - c.h_gpan[g]));
  const int S = site_splits(c, mr);
  size_t need = (size_t)S * c.ns * 10;
  if (c.site_part.n < need) c.site_part.alloc(need);
  if (fp32)
    launch(site_reaction_kernel<float, float4, true>, dim3(c.nsblk, S), 256, 0, s, c.site_pos.p, c.ns, c.sblk.p,
           c.gpan.p, K, src32, str32, c.site_part.p);
  else
    launch(site_reaction_kernel<double, double4, true>, dim3(c.nsblk, S), 256, 0, s, c.site_pos.p, c.ns, c.sblk.p,
           c.gpan.p, K, src, str, c.site_part.p);
  launch(site_reduce_kernel, cdiv(c.ns * 10, 256), 256, 0, s, c.site_part.p, S, c.ns, out10);
  BP_CHECK_LAUNCH();
}

void rhs_internal(Ctx& c, const double* p, double* b, bool fp32, cudaStream_t s) {
  const double* pp = p ? p : c.site_d.p;
  double scale = INV4PI / c.par.eps_in;
  if (fp32)
    launch(rhs_kernel<float>, c.ndblk, 128, 0, s, c.tgt64.p, c.dblk.p, c.gsite.p, c.site_pos.p, c.site_q.p, pp,
           c.site_Q.p, scale, b);
  else
    launch(rhs_kernel<double>, c.ndblk, 128, 0, s, c.tgt64.p, c.dblk.p, c.gsite.p, c.site_pos.p, c.site_q.p, pp,
           c.site_Q.p, scale, b);
  BP_CHECK_LAUNCH();
}

void site_reaction_form(Ctx& c, const double* x, double* out, int op, bool hessian, cudaStream_t s) {
  const bool fp32 = op == BEMPOL_OP_FP32_DIRECT || op == BEMPOL_OP_FP32_TREE;
  if (op == BEMPOL_OP_FP32_TREE || op == BEMPOL_OP_FP64_TREE)
    site_reaction_tree(c, x, out, fp32, s);
  else
    site_reaction_internal(c, x, out, fp32, hessian, s);
}

void site_reaction_internal(Ctx& c, const double* x, double* out, bool fp32, bool hessian, cudaStream_t s) {
  strengths(c, x, fp32, s);
  const int S = site_splits(c, max_group_sources(c));
  size_t need = (size_t)S * c.ns * 10;
  if (c.site_part.n < need) c.site_part.alloc(need);
  site_reaction_launch(c, S, fp32, hessian, c.site_part.p, s);
  BP_CHECK_LAUNCH();
  launch(site_reduce_kernel, cdiv(c.ns * 10, 256), 256, 0, s, c.site_part.p, S, c.ns, out);
  BP_CHECK_LAUNCH();
}

void multipole_internal(Ctx& c, const double* mu, int mode, double* out, cudaStream_t s, bool fp32) {
  if (fp32)
    launch(multipole_kernel<float>, cdiv(c.ns, 8), 256, 0, s, c.site_pos.p, c.site_q.p, c.site_d.p, c.site_Q.p, mu,
           c.site_group.p, c.stag.p, c.gsite.p, c.grp_sys.p, c.sys_site.p, c.ns, mode, c.par.thole_a,
           c.par.thole_perm, INV4PI / c.par.eps_in, out);
  else
    launch(multipole_kernel<double>, cdiv(c.ns, 8), 256, 0, s, c.site_pos.p, c.site_q.p, c.site_d.p, c.site_Q.p, mu,
           c.site_group.p, c.stag.p, c.gsite.p, c.grp_sys.p, c.sys_site.p, c.ns, mode, c.par.thole_a,
           c.par.thole_perm, INV4PI / c.par.eps_in, out);
  BP_CHECK_LAUNCH();
}

std::vector<double> energy_internal(Ctx& c, const double* react10, const double* mult10, cudaStream_t s) {
  launch(energy_kernel, c.nsys, 256, 0, s, c.site_q.p, c.site_d.p, c.site_Q.p, react10, mult10, c.sys_site.p,
         c.scal.p);
  BP_CHECK_LAUNCH();
  std::vector<double> e(c.nsys);
  BP_CUDA(cudaMemcpyAsync(c.h_pinned, c.scal.p, sizeof(double) * c.nsys, cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  for (int q = 0; q < c.nsys; ++q) e[q] = c.h_pinned[q];
  return e;
}

std::vector<double> sor_update(Ctx& c, double* mu, const double* react10, const double* emult3, bool vacuum,
                               const int* d_active, cudaStream_t s) {
  launch(sor_kernel, c.nsys, 256, 0, s, mu, c.site_pos.p, vacuum ? nullptr : react10, emult3, c.sys_site.p, d_active,
         c.par.sor_omega, c.scal.p + c.nsys);
  BP_CHECK_LAUNCH();
  BP_CUDA(cudaMemcpyAsync(c.h_pinned + c.nsys, c.scal.p + c.nsys, sizeof(double) * c.nsys, cudaMemcpyDeviceToHost,
                          s));
  BP_CUDA(cudaStreamSynchronize(s));
  std::vector<double> r(c.nsys);
  for (int q = 0; q < c.nsys; ++q)
    r[q] = std::sqrt(c.h_pinned[c.nsys + q] / std::max(1, c.h_sys_site[q + 1] - c.h_sys_site[q]));
  return r;
}

void site_validation(Ctx& c, cudaStream_t s) {
  DBuf<int> flag;
  flag.alloc(c.ns);
  double nf2 = c.par.near_factor * c.par.near_factor;
  launch(site_check_kernel, cdiv(c.ns, 8), 256, 0, s, c.site_pos.p, c.ns, c.stag.p, c.grp_sys.p, c.sys_pan.p,
         c.ptag.p, c.tgt64.p, c.src32.p, c.nrm64.p, c.K, nf2, flag.p);
  BP_CHECK_LAUNCH();
  std::vector<int> h(c.ns);
  BP_CUDA(cudaMemcpyAsync(h.data(), flag.p, sizeof(int) * c.ns, cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  for (int l = 0; l < c.ns; ++l) {
    if (h[l] == 1)
      fail(BEMPOL_ERR_SITES, "site " + std::to_string(l) + " lies within the near-singular radius of a panel");
    if (h[l] == 2) fail(BEMPOL_ERR_SITES, "site " + std::to_string(l) + " lies outside the surface");
    // with a Stern layer the sites lie inside both surfaces; otherwise inside their own only
    if (h[l] == 3 && !c.stern)
      fail(BEMPOL_ERR_SITES, "site " + std::to_string(l) + " lies inside the surface of another body");
    if (h[l] == 0 && c.stern)
      fail(BEMPOL_ERR_SITES, "site " + std::to_string(l) + " lies outside the ion-exclusion surface");
  }
}

// The reaction-field kernels with partial sums written to a caller-provided
// scratch of `cap` doubles instead of the context's own buffer.  The number of
// source splits is reduced until S * ns * 10 <= cap; every scratch entry the
// reduction reads is written first by the partial kernel.  Returns false (and
// launches nothing) when even one split does not fit.
bool site_reaction_scratch(Ctx& c, const double* x, double* out, bool fp32, bool hessian, double* scratch,
                           size_t cap, cudaStream_t s) {
  if ((size_t)c.ns * 10 > cap) return false;
  const int mr = max_group_sources(c);
  int S = site_splits(c, mr);
  S = std::max(1, std::min<int>(S, (int)(cap / ((size_t)c.ns * 10))));
  int per = cdiv(cdiv(mr, S), 256) * 256;
  S = cdiv(mr, per);
  strengths(c, x, fp32, s);
  site_reaction_launch(c, S, fp32, hessian, scratch, s);
  BP_CHECK_LAUNCH();
  launch(site_reduce_kernel, cdiv(c.ns * 10, 256), 256, 0, s, scratch, S, c.ns, out);
  BP_CHECK_LAUNCH();
  return true;
}

}  // namespace bp
