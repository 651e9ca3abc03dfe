// Near-singular and singular panel integrals (Sec. "The boundary element method").
//
// Near pairs: panel j is near collocation point i when |x_i - c_j|^2 < nf^2 * A_i
// (nf = near_factor, A_i the area of the collocation point's own panel).  The
// decision is taken in FP64 with explicitly rounded operations in the order
// ((dx*dx + dy*dy) + dz*dz) < (nf*nf)*A_i; the octree only narrows the candidates
// (leaves whose bounding spheres come within the largest threshold radius).
//
// For every near pair the FP64 correction (accurate integral - K-node sum) of the
// four kernels V_L, K_L, V_Y, K_Y is stored, so that a matvec over all Gauss
// nodes plus this sparse correction equals the discrete operator.
//
// Accurate integrals (semi-analytical; the paper cites Hess-Smith and Zhu et al.
// without formulas, this is the reading used):
//   * foot point p of x on the panel plane, signed height h = n.(x - v0)
//     (h = 0 exactly when x is the centroid of the same panel);
//   * three signed sub-triangles (p, v_a, v_b), sign = orientation along n;
//   * radial integrals in closed form with s = sqrt(rho^2 + h^2):
//       G_L: s - |h|;  G_Y: (e^{-k|h|} - e^{-k s})/k;
//       dG_L/dn_y: sgn(h)(1 - |h|/s);  dG_Y/dn_y: sgn(h)(e^{-k|h|} - |h| e^{-k s}/s)
//     (all over 4 pi), written without cancellation (s - |h| = rho^2/(s + |h|),
//     expm1 for the exponential differences);
//   * angular integral along each edge in the variable u with t = d sinh(u)
//     (d = distance from p to the edge line, t = position along it), so
//     dpsi = du/cosh(u) and rho_max = d cosh(u); every singularity of the
//     integrand then lies at |Im u| >= pi/2, and composite 10-node
//     Gauss-Legendre on pieces of length <= 1 converges to ~1e-16.
//
// Optional 19-node rule (near_rule = BEMPOL_NEAR_GAUSS19): near pairs off the self panel
// take the sums over the fully symmetric 19-node rule of degree 9 instead, as the paper's
// production runs do ("finer quadrature rules with 19 Gauss nodes" within 1.25 sqrt(A),
// Sec. "Comparison with Tinker-APBS").  Its 12 orbit parameters (centroid weight; four
// (a, a, 1-2a) orbits; one (b, c, 1-b-c) orbit) meet the 12 independent moment
// conditions of degree <= 9 of a symmetric rule, which fix them; they are computed on the
// host by Gauss-Newton on the monomial moments from Dunavant's table (Int. J. Numer.
// Meth. Eng. 21, 1985) rounded to 3 digits.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace bp {

namespace {

constexpr int GL_N = 10;
__constant__ double c_gl_x[GL_N];
__constant__ double c_gl_w[GL_N];
constexpr int R19 = 19;
__constant__ double4 c_r19[R19];  // barycentric (l1, l2, l3) and weight (sum 1); node 0 = centroid

double factorial(int n) {
  double f = 1.0;
  for (int k = 2; k <= n; ++k) f *= k;
  return f;
}

double ipow(double x, int e) {
  double r = 1.0;
  for (int k = 0; k < e; ++k) r *= x;
  return r;
}

// x = {w0, a1..a4, W1..W4, b, c, W5} (W = an orbit's total weight) -> the 19 nodes
void rule19_nodes(const double* x, double4* out) {
  const double t = 1.0 / 3.0;
  int n = 0;
  out[n++] = make_double4(t, t, t, x[0]);
  for (int o = 0; o < 4; ++o) {
    const double a = x[1 + o], z = 1.0 - 2.0 * a, w = x[5 + o] / 3.0;
    out[n++] = make_double4(a, a, z, w);
    out[n++] = make_double4(a, z, a, w);
    out[n++] = make_double4(z, a, a, w);
  }
  const double b = x[9], c = x[10], d = 1.0 - b - c, w = x[11] / 6.0;
  const double perm[6][3] = {{b, c, d}, {b, d, c}, {c, b, d}, {c, d, b}, {d, b, c}, {d, c, b}};
  for (int k = 0; k < 6; ++k) out[n++] = make_double4(perm[k][0], perm[k][1], perm[k][2], w);
}

// Gauss-Newton on the relative moment residuals of the monomials l1^i l2^j l3^k
// (i >= j >= k, i + j + k <= 9; the rule is symmetric, so these cover every monomial),
// F_m(x) = sum_g w_g l1^i l2^j l3^k / mean_ijk - 1 with mean_ijk = 2 i! j! k! / (i+j+k+2)!.
// The Jacobian is taken by central differences and each step is solved by Householder
// QR.  Returns the largest |F_m| at the end.
double solve_rule19(double* x) {
  constexpr int NM = 53, NX = 12;
  int I[NM], Jx[NM], Kx[NM], m = 0;
  for (int i = 0; i <= 9; ++i)
    for (int j = 0; j <= i; ++j)
      for (int k = 0; k <= j; ++k)
        if (i + j + k <= 9) I[m] = i, Jx[m] = j, Kx[m] = k, ++m;
  if (m != NM) return 1.0;
  double mean[NM];
  for (int t = 0; t < NM; ++t)
    mean[t] = 2.0 * factorial(I[t]) * factorial(Jx[t]) * factorial(Kx[t]) / factorial(I[t] + Jx[t] + Kx[t] + 2);
  auto resid = [&](const double* xv, double* r) {
    double4 nd[R19];
    rule19_nodes(xv, nd);
    for (int t = 0; t < NM; ++t) {
      double f = 0.0;
      for (int g = 0; g < R19; ++g) f += nd[g].w * ipow(nd[g].x, I[t]) * ipow(nd[g].y, Jx[t]) * ipow(nd[g].z, Kx[t]);
      r[t] = f / mean[t] - 1.0;
    }
  };
  double fmax = 1.0;
  int polish = 0;  // steps taken after the residual reached rounding level
  for (int it = 0; it < 60 && polish < 3; ++it) {
    double A[NM][NX], b[NM], rp[NM], rm[NM];
    resid(x, b);
    fmax = 0.0;
    for (int t = 0; t < NM; ++t) fmax = std::max(fmax, std::fabs(b[t]));
    if (fmax < 1e-15) ++polish;
    for (int c = 0; c < NX; ++c) {
      double xp[NX], xm[NX];
      const double h = 1e-7;
      for (int q = 0; q < NX; ++q) xp[q] = xm[q] = x[q];
      xp[c] += h;
      xm[c] -= h;
      resid(xp, rp);
      resid(xm, rm);
      for (int t = 0; t < NM; ++t) A[t][c] = (rp[t] - rm[t]) / (2.0 * h);
    }
    // Householder QR of A applied to b; then R dx = (Q^T b)[0:NX]
    for (int c = 0; c < NX; ++c) {
      double nrm = 0.0;
      for (int t = c; t < NM; ++t) nrm += A[t][c] * A[t][c];
      nrm = std::sqrt(nrm);
      if (nrm == 0.0) return 1.0;
      const double alpha = A[c][c] > 0 ? -nrm : nrm;
      double v[NM];
      for (int t = 0; t < NM; ++t) v[t] = t < c ? 0.0 : A[t][c];
      v[c] -= alpha;
      double vv = 0.0;
      for (int t = c; t < NM; ++t) vv += v[t] * v[t];
      if (vv == 0.0) continue;
      for (int q = c; q < NX; ++q) {
        double d = 0.0;
        for (int t = c; t < NM; ++t) d += v[t] * A[t][q];
        d = 2.0 * d / vv;
        for (int t = c; t < NM; ++t) A[t][q] -= d * v[t];
      }
      double d = 0.0;
      for (int t = c; t < NM; ++t) d += v[t] * b[t];
      d = 2.0 * d / vv;
      for (int t = c; t < NM; ++t) b[t] -= d * v[t];
    }
    double dx[NX];
    for (int r = NX - 1; r >= 0; --r) {
      double v = b[r];
      for (int q = r + 1; q < NX; ++q) v -= A[r][q] * dx[q];
      dx[r] = v / A[r][r];
    }
    for (int q = 0; q < NX; ++q) x[q] -= dx[q];
  }
  return fmax;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n (host).
void gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

__device__ __forceinline__ double dsq3(double dx, double dy, double dz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// pass 1/2: count, then fill, the near columns of every target (ascending j).
// One thread per target of a tree target block; it scans the panels of the
// candidate leaves of its leaf (sorted by first panel, so j comes out ascending).
template <bool FILL>
__global__ void near_list_kernel(const int4* __restrict__ blk, const double4* __restrict__ tgt64,
                                 const int* __restrict__ cand_ptr, const int* __restrict__ cand,
                                 const int* __restrict__ begin, const int* __restrict__ end, double nf2,
                                 const int* __restrict__ ptr, int* __restrict__ out) {
  const int4 B = blk[blockIdx.x];
  if ((int)threadIdx.x >= B.z) return;
  const int i = B.y + threadIdx.x;
  const double4 xi = tgt64[i];
  const double thr = __dmul_rn(nf2, xi.w);
  int cnt = 0;
  const int base = FILL ? ptr[i] : 0;
  for (int e = cand_ptr[B.x]; e < cand_ptr[B.x + 1]; ++e) {
    const int cl = cand[e];
    for (int j = begin[cl]; j < end[cl]; ++j) {
      const double4 cj = tgt64[j];
      const double e2 = dsq3(__dsub_rn(xi.x, cj.x), __dsub_rn(xi.y, cj.y), __dsub_rn(xi.z, cj.z));
      if (e2 < thr) {
        if (FILL) out[base + cnt] = j;
        ++cnt;
      }
    }
  }
  if (!FILL) out[i] = cnt;
}

__device__ void panel_exact(double xx, double xy, double xz, const double* __restrict__ v, bool self,
                            double kappa, double out[4]) {
  const double v0x = v[0], v0y = v[1], v0z = v[2];
  double e1x = v[3] - v0x, e1y = v[4] - v0y, e1z = v[5] - v0z;
  double e2x = v[6] - v0x, e2y = v[7] - v0y, e2z = v[8] - v0z;
  double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
  double nn = sqrt(nx * nx + ny * ny + nz * nz);
  nx /= nn;
  ny /= nn;
  nz /= nn;
  double h = self ? 0.0 : nx * (xx - v0x) + ny * (xy - v0y) + nz * (xz - v0z);
  double px = xx - h * nx, py = xy - h * ny, pz = xz - h * nz;
  double ah = fabs(h);
  double sh = h > 0.0 ? 1.0 : (h < 0.0 ? -1.0 : 0.0);
  double eh = exp(-kappa * ah);
  double acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
  for (int e = 0; e < 3; ++e) {
    const double* A = v + 3 * e;
    const double* B = v + 3 * ((e + 1) % 3);
    double apx = A[0] - px, apy = A[1] - py, apz = A[2] - pz;
    double bpx = B[0] - px, bpy = B[1] - py, bpz = B[2] - pz;
    double abx = B[0] - A[0], aby = B[1] - A[1], abz = B[2] - A[2];
    double L = sqrt(abx * abx + aby * aby + abz * abz);
    double ux = abx / L, uy = aby / L, uz = abz / L;
    double cx = apy * bpz - apz * bpy, cy = apz * bpx - apx * bpz, cz = apx * bpy - apy * bpx;
    double nc = nx * cx + ny * cy + nz * cz;
    double d = fabs(nc) / L;
    if (!(d > 1e-14 * L)) continue;
    double sig = nc > 0.0 ? 1.0 : -1.0;
    double ta = apx * ux + apy * uy + apz * uz;
    double tb = bpx * ux + bpy * uy + bpz * uz;
    double ua = asinh(ta / d), ub = asinh(tb / d);
    int np = max(1, (int)ceil(ub - ua));
    double du = (ub - ua) / np;
    for (int pc = 0; pc < np; ++pc) {
      double u0 = ua + pc * du;
      for (int q = 0; q < GL_N; ++q) {
        double u = u0 + 0.5 * du * (c_gl_x[q] + 1.0);
        double wq = 0.5 * du * c_gl_w[q];
        double ch = cosh(u);
        double rho = d * ch;
        double s = sqrt(rho * rho + h * h);
        double sm = rho * rho / (s + ah);
        double fvl = sm, fkl = sh * sm / s, fvy, fky;
        if (kappa > 0.0) {
          double em = -expm1(-kappa * sm);
          fvy = eh * em / kappa;
          fky = sh * (eh * sm / s + (ah / s) * eh * em);
        } else {
          fvy = fvl;
          fky = fkl;
        }
        double wt = sig * wq / ch;
        acc0 += wt * fvl;
        acc1 += wt * fkl;
        acc2 += wt * fvy;
        acc3 += wt * fky;
      }
    }
  }
  const double inv4pi = 0.25 / M_PI;
  out[0] = acc0 * inv4pi;
  out[1] = acc1 * inv4pi;
  out[2] = acc2 * inv4pi;
  out[3] = acc3 * inv4pi;
}

// Sums of the four kernels over the 19-node rule on panel j (vertices v, centroid and area
// cj, normal nj) for the target x, over 4 pi.  Node 0 is the panel's centroid as computed
// for its collocation point.
__device__ void rule19_sums(double xx, double xy, double xz, const double* __restrict__ v, double4 cj, double4 nj,
                            double kappa, double out[4], int* __restrict__ coincide) {
  double vl = 0, kl = 0, vy = 0, ky = 0;
  for (int g = 0; g < R19; ++g) {
    const double4 L = c_r19[g];
    double y0 = cj.x, y1 = cj.y, y2 = cj.z;
    if (g > 0) {
      y0 = (L.x * v[0] + L.y * v[3]) + L.z * v[6];
      y1 = (L.x * v[1] + L.y * v[4]) + L.z * v[7];
      y2 = (L.x * v[2] + L.y * v[5]) + L.z * v[8];
    }
    const double w = L.w * cj.w;
    const double rx = xx - y0, ry = xy - y1, rz = xz - y2;
    const double r2 = rx * rx + ry * ry + rz * rz;
    if (r2 == 0.0) {  // a node of another panel on the collocation point: overlapping panels
      atomicExch(coincide, 1);
      continue;
    }
    const double R = sqrt(r2), inv = 1.0 / R, inv3 = inv * inv * inv;
    const double nr = nj.x * rx + nj.y * ry + nj.z * rz;
    const double ek = exp(-kappa * R);
    vl += w * inv;
    kl += w * nr * inv3;
    vy += w * ek * inv;
    ky += w * nr * (1.0 + kappa * R) * ek * inv3;
  }
  const double inv4pi = 0.25 / M_PI;
  out[0] = vl * inv4pi;
  out[1] = kl * inv4pi;
  out[2] = vy * inv4pi;
  out[3] = ky * inv4pi;
}

// one thread per near pair k (row found by binary search in the CSR pointers)
__global__ void near_corr_kernel(const int* __restrict__ ptr, const int* __restrict__ col, int n, int nnz,
                                 const double4* __restrict__ tgt64, const double* __restrict__ vert9,
                                 const double4* __restrict__ src64, const double4* __restrict__ nrm64, int K,
                                 double kappa, int rule19, int stern, const int* __restrict__ ptag,
                                 double4* __restrict__ corr, int* __restrict__ coincide) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  int lo = 0, hi = n - 1;  // largest row i with ptr[i] <= k
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ptr[mid] <= k)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int i = lo;
  const double4 x = tgt64[i];
  {
    int j = col[k];
    double ex[4];
    double4 nj = nrm64[j];
    if (rule19 && i != j)
      rule19_sums(x.x, x.y, x.z, vert9 + 9 * (size_t)j, tgt64[j], nj, kappa, ex, coincide);
    else
      panel_exact(x.x, x.y, x.z, vert9 + 9 * (size_t)j, i == j, kappa, ex);
    double vl = 0, kl = 0, vy = 0, ky = 0;
    for (int g = 0; g < K; ++g) {
      double4 y = src64[(size_t)K * j + g];
      double rx = x.x - y.x, ry = x.y - y.y, rz = x.z - y.z;
      double r2 = rx * rx + ry * ry + rz * rz;
      if (r2 == 0.0) {
        if (i != j) atomicExch(coincide, 1);  // only the own panel's centroid node may sit on x_i
        continue;
      }
      double R = sqrt(r2);
      double inv = 1.0 / R;
      double nr = nj.x * rx + nj.y * ry + nj.z * rz;
      double ek = exp(-kappa * R);
      double inv3 = inv * inv * inv;
      vl += y.w * inv;
      kl += y.w * nr * inv3;
      vy += y.w * ek * inv;
      ky += y.w * nr * (1.0 + kappa * R) * ek * inv3;
    }
    const double inv4pi = 0.25 / M_PI;
    if (ptag[i] == ptag[j])
      corr[k] = make_double4(ex[0] - vl * inv4pi, ex[1] - kl * inv4pi, ex[2] - vy * inv4pi, ex[3] - ky * inv4pi);
    else if (stern)  // the other surface of a Stern layer: the Laplace layers of the ion-free region
      corr[k] = make_double4(ex[0] - vl * inv4pi, ex[1] - kl * inv4pi, 0.0, 0.0);
    else  // another body: its Laplace layers do not reach this target
      corr[k] = make_double4(0.0, 0.0, ex[2] - vy * inv4pi, ex[3] - ky * inv4pi);
  }
}

}  // namespace

namespace {

// the 19-node rule, solved once per process (host only)
struct R19Table {
  double4 node[R19];
  bool ok;
  R19Table() {
    // Dunavant's degree-9 table to 3 digits: centroid weight, the four a's, their orbit
    // weights, b, c and the six-node orbit's weight
    double x[12] = {0.0971, 0.490, 0.437, 0.188, 0.0447, 0.094, 0.233, 0.239, 0.0767, 0.0368, 0.222, 0.260};
    const double f = solve_rule19(x);
    rule19_nodes(x, node);
    ok = f < 1e-13;
    for (int g = 0; g < R19; ++g) ok = ok && node[g].w > 0 && node[g].x > 0 && node[g].y > 0 && node[g].z > 0;
  }
};

const R19Table& rule19() {
  static const R19Table tab;
  return tab;
}

}  // namespace

void init_near_rules() {
  double x[GL_N], w[GL_N];
  gauss_legendre(GL_N, x, w);
  BP_CUDA(cudaMemcpyToSymbol(c_gl_x, x, sizeof(x)));
  BP_CUDA(cudaMemcpyToSymbol(c_gl_w, w, sizeof(w)));
  const R19Table& tab = rule19();
  if (!tab.ok) fail(BEMPOL_ERR_NOT_CONVERGED, "the 19-node triangle rule did not converge");
  BP_CUDA(cudaMemcpyToSymbol(c_r19, tab.node, sizeof(tab.node)));
}

void build_near(Ctx& c, cudaStream_t s) {
  const int n = c.n;
  const double nf2 = c.par.near_factor * c.par.near_factor;
  // candidate leaves from the tree: radius above every threshold near_factor*sqrt(A_i)
  const double rmax = std::sqrt(nf2 * c.max_area) * (1.0 + 1e-9) + 1e-12;
  std::vector<int> cptr, ccell;
  tree_near_candidates(c, rmax, cptr, ccell);
  DBuf<int> d_cptr, d_ccell;
  d_cptr.alloc(cptr.size());
  d_ccell.alloc(std::max<size_t>(1, ccell.size()));
  BP_CUDA(cudaMemcpyAsync(d_cptr.p, cptr.data(), sizeof(int) * cptr.size(), cudaMemcpyHostToDevice, s));
  if (!ccell.empty())
    BP_CUDA(cudaMemcpyAsync(d_ccell.p, ccell.data(), sizeof(int) * ccell.size(), cudaMemcpyHostToDevice, s));
  const Tree& T = c.tree;
  DBuf<int> cnt;
  cnt.alloc(n);
  launch(near_list_kernel<false>, T.nblk, 128, 0, s, T.blk.p, c.tgt64.p, d_cptr.p, d_ccell.p, T.begin.p, T.end.p,
         nf2, nullptr, cnt.p);
  std::vector<int> h(n);
  BP_CUDA(cudaMemcpyAsync(h.data(), cnt.p, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  std::vector<int> ptr(n + 1, 0);
  for (int i = 0; i < n; ++i) ptr[i + 1] = ptr[i] + h[i];
  c.nnz = ptr[n];
  c.near_ptr.alloc(n + 1);
  c.near_col.alloc(std::max<int64_t>(1, c.nnz));
  c.near_corr.alloc(std::max<int64_t>(1, c.nnz));
  BP_CUDA(cudaMemcpyAsync(c.near_ptr.p, ptr.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
  launch(near_list_kernel<true>, T.nblk, 128, 0, s, T.blk.p, c.tgt64.p, d_cptr.p, d_ccell.p, T.begin.p, T.end.p,
         nf2, c.near_ptr.p, c.near_col.p);
  DBuf<int> coincide;
  coincide.alloc(1);
  coincide.zero(s);
  launch(near_corr_kernel, cdiv(c.nnz, 128), 128, 0, s, c.near_ptr.p, c.near_col.p, n, (int)c.nnz, c.tgt64.p,
         c.vert9.p, c.src64.p, c.nrm64.p, c.K, c.par.kappa, c.par.near_rule == BEMPOL_NEAR_GAUSS19 ? 1 : 0,
         c.stern ? 1 : 0, c.ptag.p, c.near_corr.p, coincide.p);
  BP_CHECK_LAUNCH();
  c.nearT_ready = false;  // the table by columns is built on the first transposed product
  int bad = 0;
  BP_CUDA(cudaMemcpyAsync(&bad, coincide.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  // Two different panels at distance 0 overlap: an invalid surface.  Those within the near
  // radius are caught here (the FP32 treecode near field sums the sources of other panels
  // without an r = 0 test).
  if (bad)
    fail(BEMPOL_ERR_MESH, "a Gauss node of one panel coincides with the centroid of another (overlapping panels)");
}

}  // namespace bp

extern "C" bempol_status bempol_near_rule19(double* nodes) {
  if (!nodes) return BEMPOL_ERR_ARG;
  try {
    const bp::R19Table& tab = bp::rule19();
    if (!tab.ok) return BEMPOL_ERR_NOT_CONVERGED;
    for (int g = 0; g < bp::R19; ++g) {
      nodes[4 * g] = tab.node[g].x;
      nodes[4 * g + 1] = tab.node[g].y;
      nodes[4 * g + 2] = tab.node[g].z;
      nodes[4 * g + 3] = tab.node[g].w;
    }
    return BEMPOL_OK;
  } catch (...) {
    return BEMPOL_ERR_ARG;
  }
}
