// Stern (ion-exclusion) layer: three regions bounded by two closed surfaces (Sec.
// "Spherical cavity": a layer free of ions between the solute's dielectric boundary
// Gamma_1 and the surface Gamma_2 where the salt begins).  The paper does not write the
// boundary integral equations of this case; they follow from Green's representation in
// each region, as Eq. integral_eq does for one surface:
//   region 1 (inside Gamma_1): Laplace, eps_in, the sites;
//   region 2 (between):        Laplace, eps_out, no ions;
//   region 3 (outside Gamma_2): Yukawa (kappa), eps_out.
// Unknowns per panel: phi and psi = dphi/dn, on Gamma_1 as seen from region 1, on
// Gamma_2 the same from both sides (eps_out on both).  Normals point out of the enclosed
// volume on both surfaces; with r = eps_in / eps_out the rows are
//   Gamma_1, region 1: phi1/2 + K11 phi1 - V11 psi1
//   Gamma_1, region 2: phi1/2 - K11 phi1 + r V11 psi1 + K12 phi2 - V12 psi2
//   Gamma_2, region 2: phi2/2 + K22 phi2 - V22 psi2 - K21 phi1 + r V21 psi1
//   Gamma_2, region 3: phi2/2 - KY22 phi2 + VY22 psi2
// (Kij, Vij the Laplace layers at targets on Gamma_i from panels of Gamma_j; KY, VY the
// Yukawa ones), laid out like the one-surface system: x = [phi; psi] over the panels of
// both surfaces, the first row of each pair in the first half.  The right-hand side is
// the one-surface one on Gamma_1 and zero on Gamma_2; the reaction field at the sites is
// region 1's representation over Gamma_1 alone.
//
// The product reuses the direct pair kernels twice with different source ranges per
// target block: pass A over the target's own surface (Laplace and Yukawa sums), pass B
// over the other surface (its Laplace sums are used).  Near pairs across the surfaces
// carry Laplace corrections in the near table; the combine kernel below assigns each
// near pair to pass A or B by the source's surface.
#include <algorithm>

#include "internal.h"

namespace bp {

namespace {

__global__ void stern_combine_kernel(const double* __restrict__ partA, const double* __restrict__ partB, int S,
                                     int n, const int* __restrict__ ptag, const int* __restrict__ nptr,
                                     const int* __restrict__ ncol, const double4* __restrict__ ncorr,
                                     const double* __restrict__ x, double r, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double vlA = 0, klA = 0, vyA = 0, kyA = 0, vlB = 0, klB = 0;
  for (int s = 0; s < S; ++s) {
    const double* a = partA + (size_t)s * 4 * n;
    const double* b = partB + (size_t)s * 4 * n;
    vlA += a[i];
    klA += a[n + i];
    vyA += a[2 * n + i];
    kyA += a[3 * n + i];
    vlB += b[i];
    klB += b[n + i];
  }
  const double inv4pi = 0.25 / M_PI;
  vlA *= inv4pi;
  klA *= inv4pi;
  vyA *= inv4pi;
  kyA *= inv4pi;
  vlB *= inv4pi;
  klB *= inv4pi;
  const int gi = ptag[i];
  for (int e = nptr[i]; e < nptr[i + 1]; ++e) {
    const int j = ncol[e];
    const double4 c = ncorr[e];
    const double phj = x[j], psj = x[n + j];
    if (ptag[j] == gi) {
      vlA += c.x * psj;
      klA += c.y * phj;
      vyA += c.z * psj;
      kyA += c.w * phj;
    } else {
      vlB += c.x * psj;
      klB += c.y * phj;
    }
  }
  const double ph = x[i];
  if (gi == 0) {  // Gamma_1: regions 1 and 2
    y[i] = 0.5 * ph + klA - vlA;
    y[n + i] = 0.5 * ph - klA + r * vlA + klB - vlB;
  } else {  // Gamma_2: regions 2 and 3
    y[i] = 0.5 * ph + klA - vlA - klB + r * vlB;
    y[n + i] = 0.5 * ph - kyA + vyA;
  }
}

// flag[i] = 1 for a panel of Gamma_1 whose centroid is not inside Gamma_2 (the solid
// angle of Gamma_2 seen from it, -K_L[1] summed over Gamma_2's Gauss nodes in FP64, is
// 1 inside a closed surface and 0 outside; compared with 1/2).  One warp per panel.
__global__ void nested_kernel(const double4* __restrict__ tgt64, const double4* __restrict__ src64,
                              const double4* __restrict__ nrm64, int K, int n1, int j0, int j1,
                              int* __restrict__ flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + warp;
  if (i >= n1) return;
  const double4 p = tgt64[i];
  double acc = 0.0;
  for (int j = j0 + lane; j < j1; j += 32) {
    const double4 nj = nrm64[j];
    for (int q = 0; q < K; ++q) {
      const double4 y = src64[(size_t)K * j + q];
      const double rx = p.x - y.x, ry = p.y - y.y, rz = p.z - y.z;
      const double r2 = rx * rx + ry * ry + rz * rz;
      const double ri = 1.0 / sqrt(r2);
      acc += y.w * (nj.x * rx + nj.y * ry + nj.z * rz) * ri * ri * ri;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) flag[i] = (-acc * (0.25 / M_PI) > 0.5) ? 0 : 1;
}

}  // namespace

void build_stern_blocks(Ctx& c, cudaStream_t s) {
  if (c.ngroup != 2 || c.nsys != 1) fail(BEMPOL_ERR_ARG, "a Stern layer needs exactly two surfaces in one system");
  const int K = c.K;
  std::vector<int4> blk(c.ndblk);
  BP_CUDA(cudaMemcpyAsync(blk.data(), c.dblk.p, sizeof(int4) * c.ndblk, cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  std::vector<int4> ra(c.ndblk), rb(c.ndblk);
  int maxr = 0;
  for (int b = 0; b < c.ndblk; ++b) {
    const int g = blk[b].z, o = 1 - g;
    const int a0 = K * c.h_gpan[g], a1 = K * c.h_gpan[g + 1];
    const int b0 = K * c.h_gpan[o], b1 = K * c.h_gpan[o + 1];
    ra[b] = make_int4(a0, a1, a0, a1);
    rb[b] = make_int4(b0, b1, b0, b1);
    maxr = std::max(maxr, std::max(a1 - a0, b1 - b0));
  }
  c.stern_rngA.alloc(c.ndblk);
  c.stern_rngB.alloc(c.ndblk);
  BP_CUDA(cudaMemcpyAsync(c.stern_rngA.p, ra.data(), sizeof(int4) * c.ndblk, cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaMemcpyAsync(c.stern_rngB.p, rb.data(), sizeof(int4) * c.ndblk, cudaMemcpyHostToDevice, s));
  c.stern_splits = p2p_splits(c, maxr);
  const size_t len = (size_t)c.stern_splits * 4 * c.n;
  if (c.part.n < len) c.part.alloc(len);
  c.stern_part.alloc(len);
  BP_CUDA(cudaStreamSynchronize(s));
}

void stern_check_nested(Ctx& c, cudaStream_t s) {
  const int n1 = c.h_gpan[1];
  DBuf<int> flag;
  flag.alloc(n1);
  launch(nested_kernel, cdiv(n1, 8), 256, 0, s, c.tgt64.p, c.src64.p, c.nrm64.p, c.K, n1, c.h_gpan[1], c.h_gpan[2],
         flag.p);
  BP_CHECK_LAUNCH();
  std::vector<int> h(n1);
  BP_CUDA(cudaMemcpyAsync(h.data(), flag.p, sizeof(int) * n1, cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n1; ++i)
    if (h[i]) fail(BEMPOL_ERR_MESH, "the dielectric boundary is not inside the ion-exclusion surface");
}

void stern_matvec(Ctx& c, const double* x, double* y, bool fp32, cudaStream_t s) {
  const int S = c.stern_splits;
  long long pairs = 0;
  for (int g = 0; g < 2; ++g) pairs += (long long)(c.h_gpan[g + 1] - c.h_gpan[g]) * c.K * c.n;
  Ctx::Timed tm;
  c.time_begin(0, s, tm);
  c.stat_pairs += pairs;
  p2p_direct_ranges(c, fp32, c.stern_rngA.p, c.part.p, S, s);
  p2p_direct_ranges(c, fp32, c.stern_rngB.p, c.stern_part.p, S, s);
  c.time_end(s, tm);
  launch(stern_combine_kernel, cdiv(c.n, 256), 256, 0, s, c.part.p, c.stern_part.p, S, c.n, c.ptag.p,
         c.near_ptr.p, c.near_col.p, c.near_corr.p, x, c.par.eps_in / c.par.eps_out, y);
  BP_CHECK_LAUNCH();
}

}  // namespace bp
