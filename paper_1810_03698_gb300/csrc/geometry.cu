// Panel geometry, Morton ordering and Gauss nodes (Sec. "The boundary element method":
// flat triangles, piecewise-constant unknowns collocated at centroids, 1/3/4-node
// Gauss rules for far-away panels).
//
// This file is compiled with -fmad=false: centroids, normals and areas are formed
// with separately rounded products and sums in a fixed order, so they are
// reproducible bit for bit by any FP64 implementation that follows the same order
// (centroid = ((v0 + v1) + v2) / 3, cross = (v1 - v0) x (v2 - v0), area = |cross| / 2).
#include <algorithm>
#include <cstring>
#include <climits>
#include <unordered_map>

#include "internal.h"

namespace bp {

namespace {

__global__ void panel_geom_kernel(const double* __restrict__ verts, const int* __restrict__ tris, int n,
                                  double4* __restrict__ cen_area, double4* __restrict__ nrm,
                                  double* __restrict__ vert9) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
  double ax = verts[3 * a], ay = verts[3 * a + 1], az = verts[3 * a + 2];
  double bx = verts[3 * b], by = verts[3 * b + 1], bz = verts[3 * b + 2];
  double cx = verts[3 * c], cy = verts[3 * c + 1], cz = verts[3 * c + 2];
  double e1x = bx - ax, e1y = by - ay, e1z = bz - az;
  double e2x = cx - ax, e2y = cy - ay, e2z = cz - az;
  double crx = e1y * e2z - e1z * e2y;
  double cry = e1z * e2x - e1x * e2z;
  double crz = e1x * e2y - e1y * e2x;
  double nn = sqrt(crx * crx + cry * cry + crz * crz);
  double area = 0.5 * nn;
  cen_area[t] = make_double4((ax + bx + cx) / 3.0, (ay + by + cy) / 3.0, (az + bz + cz) / 3.0, area);
  nrm[t] = make_double4(crx / nn, cry / nn, crz / nn, 0.0);
  double* v = vert9 + 9 * (size_t)t;
  v[0] = ax; v[1] = ay; v[2] = az;
  v[3] = bx; v[4] = by; v[5] = bz;
  v[6] = cx; v[7] = cy; v[8] = cz;
}

// Sort key of panel t: group (10 bits) | Morton code of the centroid in the group's
// bounding box (30 bits) | caller index (24 bits).
__global__ void morton_kernel(const double4* __restrict__ cen, int n, int npad, const int* __restrict__ grp,
                              const double4* __restrict__ gbox, unsigned long long* __restrict__ keys) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= npad) return;
  if (t >= n) {
    keys[t] = ~0ull;
    return;
  }
  double4 c = cen[t];
  const int g = grp ? grp[t] : 0;
  const double4 b = gbox[g];  // lo x, y, z and 1 / extent
  auto q = [&](double v, double lo) {
    double s = (v - lo) * b.w;
    int iv = (int)(s * 1024.0);
    return (unsigned)min(1023, max(0, iv));
  };
  auto spread = [](unsigned x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
  };
  unsigned m = (spread(q(c.x, b.x)) << 2) | (spread(q(c.y, b.y)) << 1) | spread(q(c.z, b.z));
  keys[t] = ((unsigned long long)g << 54) | ((unsigned long long)m << 24) | (unsigned)t;
}

// one compare-exchange stage of a bitonic sort (ascending)
__global__ void bitonic_step(unsigned long long* __restrict__ keys, int npad, int j, int k) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  int l = i ^ j;
  if (l > i) {
    unsigned long long a = keys[i], b = keys[l];
    bool up = (i & k) == 0;
    if ((a > b) == up) {
      keys[i] = b;
      keys[l] = a;
    }
  }
}

__global__ void perm_from_keys(const unsigned long long* __restrict__ keys, int n, int* __restrict__ perm,
                               int* __restrict__ iperm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int p = (int)(keys[i] & 0xffffffu);
  perm[i] = p;
  iperm[p] = i;
}

__global__ void gather_geometry(const int* __restrict__ perm, int n, int K, const double4* __restrict__ cen_c,
                                const double4* __restrict__ nrm_c, const double* __restrict__ v9_c,
                                double4* __restrict__ tgt64, float4* __restrict__ tgt32,
                                double4* __restrict__ nrm64, double* __restrict__ v9,
                                double4* __restrict__ src64, float4* __restrict__ src32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int p = perm[i];
  double4 c = cen_c[p];
  tgt64[i] = c;
  tgt32[i] = make_float4((float)c.x, (float)c.y, (float)c.z, 0.f);
  nrm64[i] = nrm_c[p];
  const double* a = v9_c + 9 * (size_t)p;
  double* o = v9 + 9 * (size_t)i;
  for (int k = 0; k < 9; ++k) o[k] = a[k];
  // barycentric nodes and weights of the K-node rule
  double lam[4][3], w[4];
  if (K == 1) {
    lam[0][0] = lam[0][1] = lam[0][2] = 1.0 / 3.0;
    w[0] = 1.0;
  } else if (K == 3) {
    const double hi = 2.0 / 3.0, lo = 1.0 / 6.0;
    for (int g = 0; g < 3; ++g) {
      for (int d = 0; d < 3; ++d) lam[g][d] = (g == d) ? hi : lo;
      w[g] = 1.0 / 3.0;
    }
  } else {
    lam[0][0] = lam[0][1] = lam[0][2] = 1.0 / 3.0;
    w[0] = -27.0 / 48.0;
    for (int g = 1; g < 4; ++g) {
      for (int d = 0; d < 3; ++d) lam[g][d] = (g - 1 == d) ? 0.6 : 0.2;
      w[g] = 25.0 / 48.0;
    }
  }
  for (int g = 0; g < K; ++g) {
    double x = lam[g][0] * a[0] + lam[g][1] * a[3] + lam[g][2] * a[6];
    double y = lam[g][0] * a[1] + lam[g][1] * a[4] + lam[g][2] * a[7];
    double z = lam[g][0] * a[2] + lam[g][1] * a[5] + lam[g][2] * a[8];
    if (K != 3 && g == 0) {
      // the centroid node is the collocation point itself (bit for bit), so the
      // self pair has r = 0 and drops out instead of leaving a rounding-sized r
      x = c.x;
      y = c.y;
      z = c.z;
    }
    double W = w[g] * c.w;
    src64[(size_t)K * i + g] = make_double4(x, y, z, W);
    src32[(size_t)K * i + g] = make_float4((float)x, (float)y, (float)z, (float)W);
  }
}

}  // namespace

// Every directed edge a->b of the mesh must be used once and have its opposite b->a,
// on a triangle of the same body.  The outgoing edges of each vertex are bucketed by a
// counting sort and sorted by their end vertex (buckets are small), so duplicates are
// adjacent and each opposite edge is a binary search in its start vertex's bucket.
void validate_closed(const int* tris, int n, int nv, const std::vector<int>& grp) {
  std::vector<int> ptr((size_t)nv + 1, 0);
  for (int t = 0; t < n; ++t) {
    for (int k = 0; k < 3; ++k) {
      const int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
      if (a < 0 || a >= nv || b < 0 || b >= nv)
        fail(BEMPOL_ERR_MESH, "triangle " + std::to_string(t) + " has a vertex index out of range");
      if (a == b) fail(BEMPOL_ERR_MESH, "triangle " + std::to_string(t) + " repeats a vertex");
      ++ptr[a + 1];
    }
  }
  for (int v = 0; v < nv; ++v) ptr[v + 1] += ptr[v];
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  std::vector<std::pair<int, int>> out(3 * (size_t)n);  // (end vertex, body group)
  for (int t = 0; t < n; ++t)
    for (int k = 0; k < 3; ++k) {
      const int a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
      out[fill[a]++] = {b, grp.empty() ? 0 : grp[t]};
    }
  for (int v = 0; v < nv; ++v) {
    std::sort(out.begin() + ptr[v], out.begin() + ptr[v + 1]);
    for (int q = ptr[v] + 1; q < ptr[v + 1]; ++q)
      if (out[q].first == out[q - 1].first)
        fail(BEMPOL_ERR_MESH, "a directed edge is used twice (inconsistent orientation or non-manifold mesh)");
  }
  for (int a = 0; a < nv; ++a)
    for (int q = ptr[a]; q < ptr[a + 1]; ++q) {
      const int b = out[q].first;
      auto lo = out.begin() + ptr[b], hi = out.begin() + ptr[b + 1];
      auto it = std::lower_bound(lo, hi, std::make_pair(a, INT_MIN));
      if (it == hi || it->first != a) fail(BEMPOL_ERR_MESH, "the mesh is not closed: an edge has no opposite neighbour");
      if (it->second != out[q].second) fail(BEMPOL_ERR_MESH, "two bodies share an edge: each body must be closed");
    }
}

void build_geometry(Ctx& c, const double* d_verts, const int* h_tris_for_check, const std::vector<int>& h_group,
                    cudaStream_t s) {
  const int n = c.n;
  const int G = c.ngroup;
  DBuf<int> d_tris;
  d_tris.alloc(3 * (size_t)n);
  BP_CUDA(cudaMemcpyAsync(d_tris.p, h_tris_for_check, 3 * sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s));
  DBuf<double4> cen_c, nrm_c;
  DBuf<double> v9_c;
  cen_c.alloc(n);
  nrm_c.alloc(n);
  v9_c.alloc(9 * (size_t)n);
  launch(panel_geom_kernel, cdiv(n, 256), 256, 0, s, d_verts, d_tris.p, n, cen_c.p, nrm_c.p, v9_c.p);
  BP_CHECK_LAUNCH();
  // areas and the centroid bounding box of each group on the host (validation, Morton normalisation)
  std::vector<double4> h(n);
  BP_CUDA(cudaMemcpyAsync(h.data(), cen_c.p, sizeof(double4) * (size_t)n, cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  std::vector<double> lo(3 * (size_t)G, 1e300), hi(3 * (size_t)G, -1e300);
  c.max_area = 0.0;
  for (int t = 0; t < n; ++t) {
    if (!(h[t].w > 0.0)) fail(BEMPOL_ERR_MESH, "triangle " + std::to_string(t) + " has zero or invalid area");
    c.max_area = std::max(c.max_area, h[t].w);
    const int g = h_group.empty() ? 0 : h_group[t];
    double v[3] = {h[t].x, h[t].y, h[t].z};
    for (int d = 0; d < 3; ++d) {
      lo[3 * g + d] = std::min(lo[3 * g + d], v[d]);
      hi[3 * g + d] = std::max(hi[3 * g + d], v[d]);
    }
  }
  std::vector<double4> gbox(G);
  for (int g = 0; g < G; ++g) {
    double ext = std::max(hi[3 * g] - lo[3 * g], std::max(hi[3 * g + 1] - lo[3 * g + 1], hi[3 * g + 2] - lo[3 * g + 2]));
    if (!(ext > 0.0)) ext = 1.0;
    gbox[g] = make_double4(lo[3 * g], lo[3 * g + 1], lo[3 * g + 2], 1.0 / ext);
  }
  for (int d = 0; d < 3; ++d) {
    c.bbox_lo[d] = 1e300;
    c.bbox_hi[d] = -1e300;
    for (int g = 0; g < G; ++g) {
      c.bbox_lo[d] = std::min(c.bbox_lo[d], lo[3 * g + d]);
      c.bbox_hi[d] = std::max(c.bbox_hi[d], hi[3 * g + d]);
    }
  }
  DBuf<double4> d_gbox;
  d_gbox.alloc(G);
  BP_CUDA(cudaMemcpyAsync(d_gbox.p, gbox.data(), sizeof(double4) * G, cudaMemcpyHostToDevice, s));
  DBuf<int> d_grp;
  if (!h_group.empty()) {
    d_grp.alloc(n);
    BP_CUDA(cudaMemcpyAsync(d_grp.p, h_group.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, s));
  }
  int npad = 1;
  while (npad < n) npad <<= 1;
  DBuf<unsigned long long> keys;
  keys.alloc(npad);
  launch(morton_kernel, cdiv(npad, 256), 256, 0, s, cen_c.p, n, npad, d_grp.p, d_gbox.p, keys.p);
  BP_CHECK_LAUNCH();
  for (int k = 2; k <= npad; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) launch(bitonic_step, cdiv(npad, 256), 256, 0, s, keys.p, npad, j, k);
  BP_CHECK_LAUNCH();
  c.perm.alloc(n);
  c.iperm.alloc(n);
  launch(perm_from_keys, cdiv(n, 256), 256, 0, s, keys.p, n, c.perm.p, c.iperm.p);
  BP_CHECK_LAUNCH();
  {
    // sorted Morton codes for the host-side tree topology; group ranges and tags
    std::vector<unsigned long long> hk(n);
    BP_CUDA(cudaMemcpyAsync(hk.data(), keys.p, sizeof(unsigned long long) * (size_t)n, cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaStreamSynchronize(s));
    c.h_morton.resize(n);
    std::vector<int> tag(n), sys(n);
    c.h_gpan.assign(G + 1, 0);
    for (int i = 0; i < n; ++i) {
      c.h_morton[i] = (unsigned)((hk[i] >> 24) & 0x3fffffffu);
      tag[i] = (int)(hk[i] >> 54);
      sys[i] = c.h_grp_sys[tag[i]];
      ++c.h_gpan[tag[i] + 1];
    }
    for (int g = 0; g < G; ++g) c.h_gpan[g + 1] += c.h_gpan[g];
    c.h_sys_pan.assign(c.nsys + 1, 0);
    for (int q = 0; q <= c.nsys; ++q) c.h_sys_pan[q] = c.h_gpan[c.h_sys_grp[q]];
    auto up = [&](DBuf<int>& d, const std::vector<int>& v) {
      d.alloc(v.size());
      BP_CUDA(cudaMemcpyAsync(d.p, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice, s));
    };
    up(c.ptag, tag);
    up(c.psys, sys);
    up(c.gpan, c.h_gpan);
    up(c.sys_pan, c.h_sys_pan);
    up(c.grp_sys, c.h_grp_sys);
    BP_CUDA(cudaStreamSynchronize(s));
  }
  c.tgt64.alloc(n);
  c.tgt32.alloc(n);
  c.nrm64.alloc(n);
  c.vert9.alloc(9 * (size_t)n);
  c.src64.alloc((size_t)c.K * n);
  c.src32.alloc((size_t)c.K * n);
  c.str64.alloc((size_t)c.K * n);
  c.str32.alloc((size_t)c.K * n);
  launch(gather_geometry, cdiv(n, 128), 128, 0, s, c.perm.p, n, c.K, cen_c.p, nrm_c.p, v9_c.p, c.tgt64.p,
                                                c.tgt32.p, c.nrm64.p, c.vert9.p, c.src64.p, c.src32.p);
  BP_CHECK_LAUNCH();
  BP_CUDA(cudaStreamSynchronize(s));
}

}  // namespace bp
