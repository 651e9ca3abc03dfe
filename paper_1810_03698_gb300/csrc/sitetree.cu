// Reaction potential, field and Hessian at the sites by the treecode (Eqs. pot_solvent,
// Efield_solv, ddphi, evaluated as in Sec. "The treecode algorithm").
//
// At a site x of body B the reaction potential is phi(x) = V_L[psi](x) - K_L[phi](x)
// over the panels of B, i.e. the field of the Gauss-node charges m and dipoles d of the
// current strengths.  With the cell moments of the matrix-vector product (single layer
// M_k, dipole layer D_k about the cell centre c) and W_k = M_k - D_k, a cell far from x
// contributes sum_k a_k(Delta) W_k with Delta = x - c and a_k the Laplace Taylor
// coefficients (the recurrence of the product's far field).  Since
//     d/dx_j a_k(Delta) = -(k_j + 1) a_{k + e_j}(Delta),
// the field and Hessian need the same coefficients two orders higher:
//     d_j phi   = - sum_t t_j a_t W_{t - e_j},
//     d_i d_j phi =  sum_t t_i t_j a_t W_{t - e_i - e_j}   (i != j),
//     d_i d_i phi =  sum_t t_i (t_i - 1) a_t W_{t - 2 e_i},
// each coefficient a_t (order <= P + 2) added to every output it reaches as soon as it
// is formed.  Cells that fail the acceptance test are opened down to leaves, whose
// Gauss nodes are summed directly (sites are validated to lie outside every panel's
// near-singular radius, so the K-node rule holds for all of them).
//
// Sites are grouped per body into batches of <= 8 in Morton order; a cell C is accepted
// for a batch when R_C < theta_s (|c_b - c_C| - R_b) with (c_b, R_b) the batch's bounding
// sphere and theta_s = theta / 2 (below), so every site satisfies the paper's criterion.
// Only cells of the site's own body are visited (Laplace layers act within a body).
// Each batch's lists are cut into pieces over the grid's y dimension; one warp per
// (batch, piece) in both kernels: lane l serves site (l & 7) of the batch, the four
// groups of eight lanes split the cells (far) or the nodes of every staged tile (near),
// FP32 (or FP64) terms with FP64 per-site sums; the pieces' partial sums are added in
// order.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "internal.h"

#include "tree_common.h"

namespace bp {

namespace {

// Multi-index tables to order Q for the site far field: for coefficient t, the index of
// t - e_j (m1), t - 2 e_j (m2) and t - e_i - e_j for (i, j) = (0, 1), (0, 2), (1, 2) (mx),
// or -1.  Indices of orders <= P coincide with those of MI<P>.
template <int Q>
struct SiteMI {
  static constexpr int NC = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  int k[NC][3];
  int ord[NC];
  int m1[NC][3];
  int m2[NC][3];
  int mx[NC][3];
  constexpr SiteMI() : k{}, ord{}, m1{}, m2{}, mx{} {
    constexpr MI<Q> b{};
    for (int t = 0; t < NC; ++t) {
      ord[t] = b.ord[t];
      for (int j = 0; j < 3; ++j) {
        k[t][j] = b.k[t][j];
        m1[t][j] = b.m1[t][j];
        m2[t][j] = b.m2[t][j];
      }
      const int a = b.k[t][0], bb = b.k[t][1], c = b.k[t][2];
      mx[t][0] = (a >= 1 && bb >= 1) ? b.idx[a - 1][bb - 1][c] : -1;
      mx[t][1] = (a >= 1 && c >= 1) ? b.idx[a - 1][bb][c - 1] : -1;
      mx[t][2] = (bb >= 1 && c >= 1) ? b.idx[a][bb - 1][c - 1] : -1;
    }
  }
};

// f[10] += potential, gradient and Hessian (xx, xy, xz, yy, yz, zz) at Delta of a cell
// with combined moments W (order P)
template <int P, typename Real>
__device__ __forceinline__ void site_far_eval(const Real D[3], const Real* __restrict__ W, Real* f) {
  constexpr int Q = P + 2;
  constexpr SiteMI<Q> mi{};
  constexpr int NQ = SiteMI<Q>::NC;
  const Real r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
  const Real rinv = inv_sqrt(r2);
  const Real ir2 = rinv * rinv;
  Real q1[Q + 1], q2[Q + 1];
#pragma unroll
  for (int n = 1; n <= Q; ++n) {
    q1[n] = ir2 * (Real)((2.0 * n - 1.0) / n);
    q2[n] = ir2 * (Real)((n - 1.0) / n);
  }
  Real a[NQ];
  a[0] = rinv;
  f[0] += a[0] * W[0];
#pragma unroll
  for (int t = 1; t < NQ; ++t) {
    const int n = mi.ord[t];
    Real s1 = 0, s2 = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (mi.m1[t][j] >= 0) s1 += D[j] * a[mi.m1[t][j]];
      if (mi.m2[t][j] >= 0) s2 += a[mi.m2[t][j]];
    }
    const Real at = q1[n] * s1 - q2[n] * s2;
    a[t] = at;
    if (n <= P) f[0] += at * W[t];
    if (n - 1 <= P) {
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (mi.k[t][j] >= 1) f[1 + j] -= (Real)mi.k[t][j] * at * W[mi.m1[t][j]];
    }
    if (n - 2 <= P) {
      const int kx = mi.k[t][0], ky = mi.k[t][1], kz = mi.k[t][2];
      if (kx >= 2) f[4] += (Real)(kx * (kx - 1)) * at * W[mi.m2[t][0]];
      if (kx >= 1 && ky >= 1) f[5] += (Real)(kx * ky) * at * W[mi.mx[t][0]];
      if (kx >= 1 && kz >= 1) f[6] += (Real)(kx * kz) * at * W[mi.mx[t][1]];
      if (ky >= 2) f[7] += (Real)(ky * (ky - 1)) * at * W[mi.m2[t][1]];
      if (ky >= 1 && kz >= 1) f[8] += (Real)(ky * kz) * at * W[mi.mx[t][2]];
      if (kz >= 2) f[9] += (Real)(kz * (kz - 1)) * at * W[mi.m2[t][2]];
    }
  }
}

// W = M - D of every cell (order P), from the product's moment layout [cell][2][NC]
template <int P, typename Real>
__global__ void wmom_kernel(const Real* __restrict__ mom, int ncell, Real* __restrict__ w) {
  constexpr int NC = MI<P>::NC;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ncell * NC) return;
  const int cell = q / NC, t = q - cell * NC;
  w[q] = mom[(size_t)cell * 2 * NC + t] - mom[(size_t)cell * 2 * NC + NC + t];
}

constexpr int SFW = 8;  // cells per staged batch of the site far kernel (two per lane group)

// batch b = (first position in site_perm, count <= 8, group, 0); batch centre bcen[b]
template <int P, typename Real>
__global__ void __launch_bounds__(32) site_far_kernel(const int4* __restrict__ bat, const int* __restrict__ perm,
                                                      const double4* __restrict__ site_pos,
                                                      const double4* __restrict__ bcen,
                                                      const double4* __restrict__ center,
                                                      const int* __restrict__ far_ptr,
                                                      const int* __restrict__ far_list, const Real* __restrict__ wm,
                                                      int nsites, double* __restrict__ out) {
  constexpr int NC = MI<P>::NC;
  constexpr bool ASYNC = (NC * sizeof(Real)) % 16 == 0;
  constexpr int CH = (int)(NC * sizeof(Real) / 16);
  __shared__ __align__(16) Real sm[2][SFW][NC];
  __shared__ Real so[2][SFW][3];
  const int lane = threadIdx.x, h = lane >> 3, tl = lane & 7;  // site tl, stream h of 4
  const int4 B = bat[blockIdx.x];
  const double4 cb = bcen[blockIdx.x];
  const bool act = tl < B.y;
  const int site = perm[B.x + (act ? tl : 0)];
  const double4 x = site_pos[site];
  const Real xr[3] = {(Real)(x.x - cb.x), (Real)(x.y - cb.y), (Real)(x.z - cb.z)};
  double acc[10];
#pragma unroll
  for (int c = 0; c < 10; ++c) acc[c] = 0.0;
  // this block's piece of the batch's far list (the list is cut into gridDim.y pieces)
  const int fa = far_ptr[blockIdx.x], fz = far_ptr[blockIdx.x + 1];
  const int f0 = fa + (int)(((long long)(fz - fa) * blockIdx.y) / gridDim.y);
  const int f1 = fa + (int)(((long long)(fz - fa) * (blockIdx.y + 1)) / gridDim.y);
  auto stage = [&](int b, int fb) {
    const int cnt = min(SFW, f1 - fb);
    if constexpr (ASYNC) {
      for (int q = lane; q < cnt * CH; q += 32) {
        const int cell = q / CH, piece = q - cell * CH;
        const unsigned sa = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char*>(&sm[b][cell][0]) + 16 * piece);
        const char* g = reinterpret_cast<const char*>(wm + (size_t)far_list[fb + cell] * NC) + 16 * piece;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    } else {
      for (int q = lane; q < cnt * NC; q += 32) sm[b][q / NC][q % NC] = wm[(size_t)far_list[fb + q / NC] * NC + q % NC];
    }
    if (lane < cnt) {
      const double4 cc = center[far_list[fb + lane]];
      so[b][lane][0] = (Real)(cb.x - cc.x);
      so[b][lane][1] = (Real)(cb.y - cc.y);
      so[b][lane][2] = (Real)(cb.z - cc.z);
    }
  };
  if (f0 < f1) stage(0, f0);
  int b = 0;
  for (int fb = f0; fb < f1; fb += SFW, b ^= 1) {
    const int cnt = min(SFW, f1 - fb);
    if constexpr (ASYNC) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();  // batch b complete for every lane; all done with the other buffer
    if (fb + SFW < f1) stage(b ^ 1, fb + SFW);
    Real f[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) f[c] = 0;
    for (int q = h; q < cnt; q += 4) {
      const Real D[3] = {xr[0] + so[b][q][0], xr[1] + so[b][q][1], xr[2] + so[b][q][2]};
      site_far_eval<P, Real>(D, sm[b][q], f);
    }
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[c] += (double)f[c];
  }
#pragma unroll
  for (int c = 0; c < 10; ++c) {
    acc[c] += __shfl_down_sync(0xffffffffu, acc[c], 16);
    acc[c] += __shfl_down_sync(0xffffffffu, acc[c], 8);
  }
  if (h == 0 && act) {
#pragma unroll
    for (int c = 0; c < 10; ++c) out[((size_t)blockIdx.y * nsites + site) * 10 + c] = acc[c];
  }
}

// Direct K-node sums over the batch's near leaves: FP32 with positions relative to
// each leaf's centre (the site put in the leaf's frame in FP64), or FP64 absolute.
template <typename Real, typename R4>
__global__ void __launch_bounds__(32) site_near_kernel(const int4* __restrict__ bat, const int* __restrict__ perm,
                                                       const double4* __restrict__ site_pos,
                                                       const int* __restrict__ leaf_cell,
                                                       const double4* __restrict__ center,
                                                       const int* __restrict__ begin, const int* __restrict__ end,
                                                       const int* __restrict__ near_ptr,
                                                       const int* __restrict__ near_list, int K,
                                                       const R4* __restrict__ pos, const R4* __restrict__ str,
                                                       int nsites, double* __restrict__ out) {
  constexpr bool REL = sizeof(Real) == 4;  // FP32: positions relative to the node's leaf centre
  __shared__ R4 sp[64];
  __shared__ R4 ss[64];
  const int lane = threadIdx.x, h = lane >> 3, tl = lane & 7;  // site tl, stream h of 4
  const int4 B = bat[blockIdx.x];
  const bool act = tl < B.y;
  const int site = perm[B.x + (act ? tl : 0)];
  const double4 x = site_pos[site];
  double acc[10];
#pragma unroll
  for (int c = 0; c < 10; ++c) acc[c] = 0.0;
  // this block's piece of the batch's near list (cut into gridDim.y pieces)
  const int ea = near_ptr[blockIdx.x], ez = near_ptr[blockIdx.x + 1];
  const int e0 = ea + (int)(((long long)(ez - ea) * blockIdx.y) / gridDim.y);
  const int e1 = ea + (int)(((long long)(ez - ea) * (blockIdx.y + 1)) / gridDim.y);
  for (int e = e0; e < e1; ++e) {
    const int cl = leaf_cell[near_list[e]];
    const double4 cc = center[cl];
    const Real X = REL ? (Real)(x.x - cc.x) : (Real)x.x;
    const Real Y = REL ? (Real)(x.y - cc.y) : (Real)x.y;
    const Real Z = REL ? (Real)(x.z - cc.z) : (Real)x.z;
    const int s0 = begin[cl] * K, s1 = end[cl] * K;
    Real a[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) a[c] = 0;
    for (int t0 = s0; t0 < s1; t0 += 64) {
      __syncwarp();  // the previous tile is done
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = t0 + 32 * u + lane;
        if (j < s1) {
          sp[32 * u + lane] = pos[j];
          ss[32 * u + lane] = str[j];
        }
      }
      __syncwarp();
      const int lim = min(64, s1 - t0);
      for (int k = h; k < lim; k += 4) {
        const R4 p = sp[k], sg = ss[k];
        const Real Rx = X - p.x, Ry = Y - p.y, Rz = Z - p.z;
        const Real r2 = Rx * Rx + Ry * Ry + Rz * Rz;
        const Real rinv = inv_sqrt(r2);
        const Real rinv2 = rinv * rinv;
        const Real A3 = rinv2 * rinv;          // 1/r^3
        const Real B5 = (Real)3 * A3 * rinv2;  // 3/r^5
        const Real m = sg.x;
        const Real dR = sg.y * Rx + sg.z * Ry + sg.w * Rz;
        a[0] += m * rinv - dR * A3;
        const Real gc = -m * A3 + dR * B5;
        a[1] += gc * Rx - sg.y * A3;
        a[2] += gc * Ry - sg.z * A3;
        a[3] += gc * Rz - sg.w * A3;
        const Real C7 = (Real)5 * B5 * rinv2;  // 15/r^7
        const Real hc = m * B5 - dR * C7;
        const Real hd = dR * B5 - m * A3;
        a[4] += hc * Rx * Rx + hd + (Real)2 * B5 * Rx * sg.y;
        a[5] += hc * Rx * Ry + B5 * (Rx * sg.z + Ry * sg.y);
        a[6] += hc * Rx * Rz + B5 * (Rx * sg.w + Rz * sg.y);
        a[7] += hc * Ry * Ry + hd + (Real)2 * B5 * Ry * sg.z;
        a[8] += hc * Ry * Rz + B5 * (Ry * sg.w + Rz * sg.z);
        a[9] += hc * Rz * Rz + hd + (Real)2 * B5 * Rz * sg.w;
      }
    }
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[c] += (double)a[c];
  }
#pragma unroll
  for (int c = 0; c < 10; ++c) {
    acc[c] += __shfl_down_sync(0xffffffffu, acc[c], 16);
    acc[c] += __shfl_down_sync(0xffffffffu, acc[c], 8);
  }
  if (h == 0 && act) {
#pragma unroll
    for (int c = 0; c < 10; ++c) out[((size_t)blockIdx.y * nsites + site) * 10 + c] = acc[c];
  }
}

// out = (sum of the np partial layers [np][n10]) / (4 pi), layers added in order
__global__ void site_tree_reduce_kernel(const double* __restrict__ part, int np, int n10, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n10) return;
  double v = 0.0;
  for (int q = 0; q < np; ++q) v += part[(size_t)q * n10 + t];
  out[t] = v * (0.25 / M_PI);
}

template <typename V>
void upload_vec(DBuf<V>& d, const std::vector<V>& h, cudaStream_t s) {
  d.alloc(std::max<size_t>(1, h.size()));
  if (!h.empty()) BP_CUDA(cudaMemcpyAsync(d.p, h.data(), sizeof(V) * h.size(), cudaMemcpyHostToDevice, s));
}

// Sites per batch, and the acceptance parameter of the site fields relative to the
// product's theta: the field and Hessian are derivatives of the truncated expansion and
// converge more slowly than the potential, so the sites accept a cell only at half the
// product's theta (errors about 2^-(P+1) smaller at the same order).
constexpr int SB = 8;
constexpr double SITE_THETA_SCALE = 0.5;

// Site batches of every body (Morton order of the sites within the body's bounding box)
// and their interaction lists with the panel octree, built on several host threads.
void build_site_tree(Ctx& c, cudaStream_t s) {
  Tree& T = c.tree;
  SiteTree& ST = c.stree;
  const int ns = c.ns;
  std::vector<double4> hp(ns);
  BP_CUDA(cudaMemcpyAsync(hp.data(), c.site_pos.p, sizeof(double4) * ns, cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  std::vector<int> perm(ns);
  std::vector<int4> bat;
  std::vector<double4> bcen;
  for (int g = 0; g < c.ngroup; ++g) {
    const int a = c.h_gsite[g], e = c.h_gsite[g + 1];
    if (a == e) continue;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int l = a; l < e; ++l) {
      const double v[3] = {hp[l].x, hp[l].y, hp[l].z};
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], v[d]);
        hi[d] = std::max(hi[d], v[d]);
      }
    }
    const double ext = std::max(1e-12, std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2])));
    std::vector<std::pair<unsigned, int>> key;
    for (int l = a; l < e; ++l) {
      auto q = [&](double v, double l0) { return (unsigned)std::min(1023.0, std::max(0.0, (v - l0) / ext * 1024.0)); };
      auto spread = [](unsigned u) {
        u &= 0x3ffu;
        u = (u | (u << 16)) & 0x030000FFu;
        u = (u | (u << 8)) & 0x0300F00Fu;
        u = (u | (u << 4)) & 0x030C30C3u;
        u = (u | (u << 2)) & 0x09249249u;
        return u;
      };
      key.push_back({(spread(q(hp[l].x, lo[0])) << 2) | (spread(q(hp[l].y, lo[1])) << 1) | spread(q(hp[l].z, lo[2])),
                     l});
    }
    std::sort(key.begin(), key.end());
    for (int k = 0; k < e - a; ++k) perm[a + k] = key[k].second;
    for (int k = a; k < e; k += SB) {
      const int cnt = std::min(SB, e - k);
      double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
      for (int q = k; q < k + cnt; ++q) {
        const double4 p = hp[perm[q]];
        const double v[3] = {p.x, p.y, p.z};
        for (int d = 0; d < 3; ++d) {
          blo[d] = std::min(blo[d], v[d]);
          bhi[d] = std::max(bhi[d], v[d]);
        }
      }
      double4 cb = make_double4(0.5 * (blo[0] + bhi[0]), 0.5 * (blo[1] + bhi[1]), 0.5 * (blo[2] + bhi[2]), 0.0);
      for (int q = k; q < k + cnt; ++q) {
        const double4 p = hp[perm[q]];
        const double dx = p.x - cb.x, dy = p.y - cb.y, dz = p.z - cb.z;
        cb.w = std::max(cb.w, std::sqrt(dx * dx + dy * dy + dz * dz));
      }
      bat.push_back(make_int4(k, cnt, g, 0));
      bcen.push_back(cb);
    }
  }
  const int nb = (int)bat.size();
  std::vector<int> leaf_of(T.ncell, -1);
  for (int l = 0; l < T.nleaf; ++l) leaf_of[T.h_leaf_cell[l]] = l;
  const double theta = SITE_THETA_SCALE * c.par.theta;
  unsigned nth = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  nth = std::min<unsigned>(nth, (unsigned)std::max(1, nb / 16));
  struct Part {
    std::vector<int> fptr, fl, nptr, nl;
    long long far = 0, pairs = 0;
    int dmin = 1 << 30;
  };
  std::vector<Part> part(nth);
  auto work = [&](unsigned w) {
    Part& o = part[w];
    const int b0 = (int)((long long)nb * w / nth), b1 = (int)((long long)nb * (w + 1) / nth);
    std::vector<std::pair<int, int>> stack;  // (cell, depth)
    o.fptr.push_back(0);
    o.nptr.push_back(0);
    for (int bi = b0; bi < b1; ++bi) {
      const int g = bat[bi].z, cnt = bat[bi].y;
      const double4 cb = bcen[bi];
      stack.assign(1, {0, 0});
      while (!stack.empty()) {
        const int q = stack.back().first, dq = stack.back().second;
        stack.pop_back();
        const int cg = T.h_cell_grp[q];
        if (cg < 0) {
          for (int k = T.h_nchild[q] - 1; k >= 0; --k) stack.push_back({T.h_child0[q] + k, dq + 1});
          continue;
        }
        if (cg != g) continue;  // the reaction field of a site comes from its own body
        const double4 cc = T.h_center[q];
        const double dx = cb.x - cc.x, dy = cb.y - cc.y, dz = cb.z - cc.z;
        const double gap = std::sqrt(dx * dx + dy * dy + dz * dz) - cb.w;
        if (gap > 0.0 && cc.w < theta * gap) {
          o.fl.push_back(q);
          o.far += cnt;
          o.dmin = std::min(o.dmin, dq);
        } else if (T.h_nchild[q] == 0) {
          o.nl.push_back(leaf_of[q]);
          o.pairs += (long long)cnt * (T.h_end[q] - T.h_begin[q]) * c.K;
        } else {
          for (int k = T.h_nchild[q] - 1; k >= 0; --k) stack.push_back({T.h_child0[q] + k, dq + 1});
        }
      }
      o.fptr.push_back((int)o.fl.size());
      o.nptr.push_back((int)o.nl.size());
    }
  };
  std::vector<std::thread> th;
  for (unsigned w = 1; w < nth; ++w) th.emplace_back(work, w);
  work(0);
  for (auto& t : th) t.join();
  std::vector<int> fptr(1, 0), fl, nptr(1, 0), nl;
  ST.far_evals = ST.pairs = 0;
  ST.min_depth = T.ndepth;
  for (const Part& o : part) {
    const int f0 = (int)fl.size(), n0 = (int)nl.size();
    for (size_t k = 1; k < o.fptr.size(); ++k) {
      fptr.push_back(f0 + o.fptr[k]);
      nptr.push_back(n0 + o.nptr[k]);
    }
    fl.insert(fl.end(), o.fl.begin(), o.fl.end());
    nl.insert(nl.end(), o.nl.begin(), o.nl.end());
    ST.far_evals += o.far;
    ST.pairs += o.pairs;
    ST.min_depth = std::min(ST.min_depth, o.dmin);
  }
  ST.nbat = nb;
  upload_vec(ST.bat, bat, s);
  upload_vec(ST.bcen, bcen, s);
  upload_vec(ST.perm, perm, s);
  upload_vec(ST.far_ptr, fptr, s);
  upload_vec(ST.far_list, fl, s);
  upload_vec(ST.near_ptr, nptr, s);
  upload_vec(ST.near_list, nl, s);
  BP_CUDA(cudaStreamSynchronize(s));
  ST.ready = true;
}

// the moment buffers of one precision
template <typename Real>
struct SiteBufs;
template <>
struct SiteBufs<float> {
  static DBuf<float>& mom(Ctx& c) { return c.tree.mom32; }
  static DBuf<float>& w(Ctx& c) { return c.stree.w32; }
  static const float4* pos(Ctx& c) { return c.tree.src_rel32.p; }
  static const float4* str(Ctx& c) { return c.str32.p; }
};
template <>
struct SiteBufs<double> {
  static DBuf<double>& mom(Ctx& c) { return c.tree.mom64; }
  static DBuf<double>& w(Ctx& c) { return c.stree.w64; }
  static const double4* pos(Ctx& c) { return c.src64.p; }
  static const double4* str(Ctx& c) { return c.str64.p; }
};

template <int P, typename Real>
void site_tree_eval(Ctx& c, double* out, cudaStream_t s) {
  Tree& T = c.tree;
  SiteTree& ST = c.stree;
  constexpr int NC = MI<P>::NC;
  DBuf<Real>& mom = SiteBufs<Real>::mom(c);
  if (T.mom_order != P || mom.n < (size_t)T.ncell * 2 * NC) {
    mom.alloc((size_t)T.ncell * 2 * NC);
    T.mom_order = P;
  }
  DBuf<Real>& wm = SiteBufs<Real>::w(c);
  if (wm.n < (size_t)T.ncell * NC) wm.alloc((size_t)T.ncell * NC);
  typedef typename Vec4<Real>::T R4;
  const R4* str = SiteBufs<Real>::str(c);
  const R4* pos = SiteBufs<Real>::pos(c);
  launch(leaf_moments_kernel<P, Real>, T.nleaf, MomShape<P>::TPB, 0, s, T.leaf_cell.p, T.begin.p, T.end.p,
         T.center.p, c.K, c.src64.p, str, (const int*)nullptr, T.leaf_sys.p, mom.p);
  for (int d = T.ndepth - 2; d >= ST.min_depth; --d) {
    const int first = T.h_depth_begin[d], cnt = T.h_depth_begin[d + 1] - first;
    launch(m2m_kernel<P, Real>, cnt, M2M_TPB, 0, s, first, T.child0.p, T.nchild.p, T.center.p, mom.p);
  }
  launch(wmom_kernel<P, Real>, cdiv((long long)T.ncell * NC, 256), 256, 0, s, mom.p, T.ncell, wm.p);
  // each batch's far and near lists cut into Y pieces (grid y), so the grids hold about
  // 24 warps per SM whatever the number of sites; partial sums per piece
  const int Y = std::max(1, std::min(64, cdiv((long long)num_sms(c.device) * 24, std::max(1, ST.nbat))));
  const size_t need = 2 * (size_t)Y * c.ns * 10;
  if (c.site_part.n < need) c.site_part.alloc(need);
  double* far = c.site_part.p;
  double* near = c.site_part.p + (size_t)Y * c.ns * 10;
  launch(site_far_kernel<P, Real>, dim3(ST.nbat, Y), 32, 0, s, ST.bat.p, ST.perm.p, c.site_pos.p, ST.bcen.p,
         T.center.p, ST.far_ptr.p, ST.far_list.p, wm.p, c.ns, far);
  launch(site_near_kernel<Real, R4>, dim3(ST.nbat, Y), 32, 0, s, ST.bat.p, ST.perm.p, c.site_pos.p,
         T.leaf_cell.p, T.center.p, T.begin.p, T.end.p, ST.near_ptr.p, ST.near_list.p, c.K, pos, str, c.ns,
         near);
  launch(site_tree_reduce_kernel, cdiv((long long)c.ns * 10, 256), 256, 0, s, c.site_part.p, 2 * Y, c.ns * 10,
         out);
  BP_CHECK_LAUNCH();
}

template <typename Real>
void site_tree_dispatch(Ctx& c, double* out, cudaStream_t s) {
  switch (c.par.order) {
    case 1: site_tree_eval<1, Real>(c, out, s); break;
    case 2: site_tree_eval<2, Real>(c, out, s); break;
    case 3: site_tree_eval<3, Real>(c, out, s); break;
    case 4: site_tree_eval<4, Real>(c, out, s); break;
    case 5: site_tree_eval<5, Real>(c, out, s); break;
    case 6: site_tree_eval<6, Real>(c, out, s); break;
    default: fail(BEMPOL_ERR_ARG, "treecode order must be in 1..6");
  }
}

}  // namespace

void site_reaction_tree(Ctx& c, const double* x, double* out, bool fp32, cudaStream_t s) {
  if (c.ns == 0) return;
  if (!c.tree_ready) build_tree(c, s);
  if (!c.stree.ready) build_site_tree(c, s);
  strengths(c, x, fp32, s);
  c.stat_site_far += c.stree.far_evals;
  c.stat_site_pairs += c.stree.pairs;
  if (fp32)
    site_tree_dispatch<float>(c, out, s);
  else
    site_tree_dispatch<double>(c, out, s);
}

}  // namespace bp
