// Direct matrix-vector product of Eq. integral_eq over Gauss nodes (Sec. "The
// treecode algorithm": the product is an N-body sum with Gauss nodes as sources
// and collocation points as targets).
//
// Source g of panel j carries a charge m = w_g A_j psi_j and a dipole
// d = w_g A_j phi_j n_j, so that per target x
//   V_L psi = sum m / (4 pi r),            K_L phi = sum d.(x - y) / (4 pi r^3),
//   V_Y psi = sum m e^{-k r} / (4 pi r),    K_Y phi = sum d.(x - y)(1 + k r) e^{-k r} / (4 pi r^3),
// with coincident node/target pairs (r = 0, the centroid node of the target's own
// panel) contributing zero.  Near pairs are then corrected with the FP64 table of
// near.cu, and the rows assembled as
//   y1 = phi/2 + K_L phi - V_L psi,   y2 = phi/2 - K_Y phi + (eps_in/eps_out) V_Y psi.
//
// FP32 form: pair arithmetic in FP32 (rsqrt and 2^x on the SFU), sums over a
// 128-source tile in FP32, tile sums added into FP64 per-target accumulators.
// Sources are split across blockIdx.y so the grid fills every SM; each split
// writes its own FP64 partial sums (no atomics, deterministic), and the combine
// kernel adds the splits in a fixed order.
#include <algorithm>

#include "internal.h"

namespace bp {

namespace {

constexpr int P2P_TPB = 128;

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

__global__ void strength_kernel(const double* __restrict__ x, int n, int K, const double4* __restrict__ src64,
                                const double4* __restrict__ nrm64, double4* __restrict__ str64,
                                float4* __restrict__ str32, bool fp32) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  int j = t / K;
  double W = src64[t].w;
  double phi = x[j], psi = x[n + j];
  double4 nj = nrm64[j];
  double m = W * psi, dd = W * phi;
  if (fp32)
    str32[t] = make_float4((float)m, (float)(dd * nj.x), (float)(dd * nj.y), (float)(dd * nj.z));
  else
    str64[t] = make_double4(m, dd * nj.x, dd * nj.y, dd * nj.z);
}

// Target blocks come from the block table (first target, count, group); every
// target of a block belongs to one body, so its sources are one range of Gauss
// nodes: the block's system (Yukawa terms), of which the block's own body
// (Laplace terms) is a sub-range.  The staged source carries that Laplace weight
// (1 or 0) in its fourth component.  blockIdx.y takes an equal share of the range.
__global__ void __launch_bounds__(P2P_TPB) p2p_f32_kernel(const double4* __restrict__ tgt, int n,
                                                          const int4* __restrict__ blk, const int4* __restrict__ rng,
                                                          const double4* __restrict__ blk_center,
                                                          const double4* __restrict__ spos,
                                                          const float4* __restrict__ sstr, float kappa,
                                                          float nk_log2e, const int* __restrict__ active,
                                                          const int* __restrict__ grp_sys, double* __restrict__ part) {
  // Coordinates enter the FP32 arithmetic relative to this block's centre c (the
  // subtraction done in FP64), so the rounding of a position is that of a number
  // of the block's size instead of the molecule's: pair distances keep ~1e-7
  // relative accuracy down to the closest (same-panel) pairs.
  __shared__ float4 sp[P2P_TPB];
  __shared__ float4 ss[P2P_TPB];
  const int4 B = blk[blockIdx.x], Rg = rng[blockIdx.x];
  if (active && !active[grp_sys[B.z]]) return;  // system not being solved
  const int i = B.x + threadIdx.x;
  const bool act = (int)threadIdx.x < B.y;
  const int per = ((Rg.y - Rg.x + (int)gridDim.y - 1) / (int)gridDim.y + P2P_TPB - 1) / P2P_TPB * P2P_TPB;
  const int s0 = Rg.x + blockIdx.y * per;
  const int s1 = min(Rg.y, s0 + per);
  const double4 c = blk_center[blockIdx.x];
  float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
  if (act) {
    double4 xd = tgt[i];
    x = make_float4((float)(xd.x - c.x), (float)(xd.y - c.y), (float)(xd.z - c.z), 0.f);
  }
  double aVL = 0, aKL = 0, aVY = 0, aKY = 0;
  for (int t0 = s0; t0 < s1; t0 += P2P_TPB) {
    int j = t0 + threadIdx.x;
    if (j < s1) {
      double4 yd = spos[j];
      const float wl = (j >= Rg.z && j < Rg.w) ? 1.f : 0.f;
      sp[threadIdx.x] = make_float4((float)(yd.x - c.x), (float)(yd.y - c.y), (float)(yd.z - c.z), wl);
      ss[threadIdx.x] = sstr[j];
    } else {
      sp[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
      ss[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    float vl = 0.f, kl = 0.f, vy = 0.f, ky = 0.f;
#pragma unroll 8
    for (int k = 0; k < P2P_TPB; ++k) {
      float4 p = sp[k];
      float4 s = ss[k];
      float dx = x.x - p.x, dy = x.y - p.y, dz = x.z - p.z;
      float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      float rinv = r2 > 0.f ? rsqrt_approx(r2) : 0.f;
      float r = r2 * rinv;
      float e = exp2_approx(r * nk_log2e);
      float mr = s.x * rinv;
      vl = fmaf(mr, p.w, vl);
      vy = fmaf(mr, e, vy);
      float dR = fmaf(s.y, dx, fmaf(s.z, dy, s.w * dz));
      float t = dR * (rinv * rinv) * rinv;
      kl = fmaf(t, p.w, kl);
      ky = fmaf(t * fmaf(kappa, r, 1.f), e, ky);
    }
    aVL += vl;
    aKL += kl;
    aVY += vy;
    aKY += ky;
    __syncthreads();
  }
  if (act) {
    double* o = part + (size_t)blockIdx.y * 4 * n;
    o[i] = aVL;
    o[n + i] = aKL;
    o[2 * n + i] = aVY;
    o[3 * n + i] = aKY;
  }
}

__global__ void __launch_bounds__(P2P_TPB) p2p_f64_kernel(const double4* __restrict__ tgt, int n,
                                                          const int4* __restrict__ blk, const int4* __restrict__ rng,
                                                          const double4* __restrict__ spos,
                                                          const double4* __restrict__ sstr, double kappa,
                                                          const int* __restrict__ active,
                                                          const int* __restrict__ grp_sys, double* __restrict__ part) {
  __shared__ double4 sp[P2P_TPB];
  __shared__ double4 ss[P2P_TPB];
  const int4 B = blk[blockIdx.x], Rg = rng[blockIdx.x];
  if (active && !active[grp_sys[B.z]]) return;  // system not being solved
  const int i = B.x + threadIdx.x;
  const bool act = (int)threadIdx.x < B.y;
  const int per = ((Rg.y - Rg.x + (int)gridDim.y - 1) / (int)gridDim.y + P2P_TPB - 1) / P2P_TPB * P2P_TPB;
  const int s0 = Rg.x + blockIdx.y * per;
  const int s1 = min(Rg.y, s0 + per);
  double4 x = act ? tgt[i] : make_double4(0, 0, 0, 0);
  double aVL = 0, aKL = 0, aVY = 0, aKY = 0;
  for (int t0 = s0; t0 < s1; t0 += P2P_TPB) {
    int j = t0 + threadIdx.x;
    if (j < s1) {
      const double4 y = spos[j];
      sp[threadIdx.x] = make_double4(y.x, y.y, y.z, (j >= Rg.z && j < Rg.w) ? 1.0 : 0.0);
      ss[threadIdx.x] = sstr[j];
    } else {
      sp[threadIdx.x] = make_double4(0, 0, 0, 0);
      ss[threadIdx.x] = make_double4(0, 0, 0, 0);
    }
    __syncthreads();
    int lim = min(P2P_TPB, s1 - t0);
    for (int k = 0; k < lim; ++k) {
      double4 p = sp[k];
      double4 s = ss[k];
      double dx = x.x - p.x, dy = x.y - p.y, dz = x.z - p.z;
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 == 0.0) continue;
      double R = sqrt(r2);
      double rinv = 1.0 / R;
      double e = exp(-kappa * R);
      double mr = s.x * rinv;
      aVL = fma(mr, p.w, aVL);
      aVY += mr * e;
      double t = (s.y * dx + s.z * dy + s.w * dz) * rinv * rinv * rinv;
      aKL = fma(t, p.w, aKL);
      aKY += t * (1.0 + kappa * R) * e;
    }
    __syncthreads();
  }
  if (act) {
    double* o = part + (size_t)blockIdx.y * 4 * n;
    o[i] = aVL;
    o[n + i] = aKL;
    o[2 * n + i] = aVY;
    o[3 * n + i] = aKY;
  }
}

// y = rows of Eq. integral_eq from the partial pair sums (S splits) + near corrections.
__global__ void combine_kernel(const double* __restrict__ part, int S, int n, const int* __restrict__ nptr,
                               const int* __restrict__ ncol, const double4* __restrict__ ncorr,
                               const double* __restrict__ x, double eps_ratio, double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double vl = 0, kl = 0, vy = 0, ky = 0;
  for (int s = 0; s < S; ++s) {
    const double* o = part + (size_t)s * 4 * n;
    vl += o[i];
    kl += o[n + i];
    vy += o[2 * n + i];
    ky += o[3 * n + i];
  }
  const double inv4pi = 0.25 / M_PI;
  vl *= inv4pi;
  kl *= inv4pi;
  vy *= inv4pi;
  ky *= inv4pi;
  for (int e = nptr[i]; e < nptr[i + 1]; ++e) {
    int j = ncol[e];
    double4 c = ncorr[e];
    double phj = x[j], psj = x[n + j];
    vl += c.x * psj;
    kl += c.y * phj;
    vy += c.z * psj;
    ky += c.w * phj;
  }
  double ph = x[i];
  y[i] = 0.5 * ph + kl - vl;
  y[n + i] = 0.5 * ph - ky + eps_ratio * vy;
}

// centre of each target block: midpoint of its targets' bounding box (FP64)
__global__ void block_center_kernel(const double4* __restrict__ tgt, const int4* __restrict__ blk, int nb,
                                    double4* __restrict__ out) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int4 B = blk[b];
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = B.x; i < B.x + B.y; ++i) {
    double4 t = tgt[i];
    lo[0] = fmin(lo[0], t.x); hi[0] = fmax(hi[0], t.x);
    lo[1] = fmin(lo[1], t.y); hi[1] = fmax(hi[1], t.y);
    lo[2] = fmin(lo[2], t.z); hi[2] = fmax(hi[2], t.z);
  }
  out[b] = make_double4(0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2]), 0.0);
}

// splits of the source range so the grid holds about eight resident blocks per SM
int choose_splits(int nblk, int max_range, int device) {
  int want = num_sms(device) * 8;
  int S = std::max(1, cdiv(want, std::max(1, nblk)));
  S = std::min(S, std::max(1, max_range / (4 * P2P_TPB)));
  S = std::min(S, 64);
  // no split may be empty for the longest range (equal shares rounded up to tiles)
  int per = cdiv(cdiv(max_range, S), P2P_TPB) * P2P_TPB;
  return std::max(1, cdiv(max_range, per));
}

}  // namespace

// Direct-kernel target blocks (<= 128 consecutive targets of one group) with their
// source ranges, and the chunks of the GMRES vectors (per system and half).
void build_blocks(Ctx& c, cudaStream_t s) {
  const int K = c.K;
  std::vector<int4> blk, rng;
  for (int g = 0; g < c.ngroup; ++g) {
    const int sy = c.h_grp_sys[g];
    for (int off = c.h_gpan[g]; off < c.h_gpan[g + 1]; off += P2P_TPB) {
      blk.push_back(make_int4(off, std::min(P2P_TPB, c.h_gpan[g + 1] - off), g, 0));
      rng.push_back(make_int4(K * c.h_sys_pan[sy], K * c.h_sys_pan[sy + 1], K * c.h_gpan[g], K * c.h_gpan[g + 1]));
    }
  }
  c.ndblk = (int)blk.size();
  c.dblk.alloc(blk.size());
  c.dblk_rng.alloc(rng.size());
  BP_CUDA(cudaMemcpyAsync(c.dblk.p, blk.data(), sizeof(int4) * blk.size(), cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaMemcpyAsync(c.dblk_rng.p, rng.data(), sizeof(int4) * rng.size(), cudaMemcpyHostToDevice, s));
  c.blk_center.alloc(c.ndblk);
  launch(block_center_kernel, cdiv(c.ndblk, 128), 128, 0, s, c.tgt64.p, c.dblk.p, c.ndblk, c.blk_center.p);
  BP_CHECK_LAUNCH();
  // GMRES chunks: about 512 in all, each within one system and one half of [phi; psi]
  const int n = c.n;
  const int ch = std::max(512, cdiv(cdiv(2 * (long long)n, 512), 256) * 256);
  std::vector<int4> chunks;
  std::vector<int> cptr(c.nsys + 1, 0);
  for (int sy = 0; sy < c.nsys; ++sy) {
    for (int half = 0; half < 2; ++half)
      for (int b = c.h_sys_pan[sy]; b < c.h_sys_pan[sy + 1]; b += ch)
        chunks.push_back(make_int4(sy, half * n + b, half * n + std::min(b + ch, c.h_sys_pan[sy + 1]), 0));
    cptr[sy + 1] = (int)chunks.size();
  }
  c.nchunk = (int)chunks.size();
  c.chunks.alloc(chunks.size());
  c.chunk_ptr.alloc(cptr.size());
  BP_CUDA(cudaMemcpyAsync(c.chunks.p, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaMemcpyAsync(c.chunk_ptr.p, cptr.data(), sizeof(int) * cptr.size(), cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaStreamSynchronize(s));
}

void strengths(Ctx& c, const double* x, bool fp32, cudaStream_t s) {
  int tot = c.n * c.K;
  launch(strength_kernel, cdiv(tot, 256), 256, 0, s, x, c.n, c.K, c.src64.p, c.nrm64.p, c.str64.p, c.str32.p, fp32);
  BP_CHECK_LAUNCH();
}

int p2p_splits(Ctx& c, int max_range) { return choose_splits(c.ndblk, max_range, c.device); }

void p2p_direct_ranges(Ctx& c, bool fp32, const int4* rng, double* part, int S, cudaStream_t s) {
  dim3 grid(c.ndblk, S);
  if (fp32) {
    const float k = (float)c.par.kappa;
    launch(p2p_f32_kernel, grid, P2P_TPB, 0, s, c.tgt64.p, c.n, c.dblk.p, rng, c.blk_center.p, c.src64.p,
           c.str32.p, k, (float)(-c.par.kappa * 1.4426950408889634), c.mv_active, c.grp_sys.p, part);
  } else {
    launch(p2p_f64_kernel, grid, P2P_TPB, 0, s, c.tgt64.p, c.n, c.dblk.p, rng, c.src64.p, c.str64.p, c.par.kappa,
           c.mv_active, c.grp_sys.p, part);
  }
  BP_CHECK_LAUNCH();
}

void p2p_direct(Ctx& c, bool fp32, cudaStream_t s) {
  const int n = c.n;
  int maxr = 0;
  long long pairs = 0;
  for (int g = 0; g < c.ngroup; ++g) {
    const int sy = c.h_grp_sys[g];
    const int r = c.K * (c.h_sys_pan[sy + 1] - c.h_sys_pan[sy]);
    maxr = std::max(maxr, r);
    pairs += (long long)(c.h_gpan[g + 1] - c.h_gpan[g]) * r;
  }
  const int S = choose_splits(c.ndblk, maxr, c.device);
  if (c.part.n < (size_t)S * 4 * n) c.part.alloc((size_t)S * 4 * n);
  c.part_splits = S;
  Ctx::Timed tm;
  c.time_begin(0, s, tm);
  c.stat_pairs += pairs;
  p2p_direct_ranges(c, fp32, c.dblk_rng.p, c.part.p, S, s);
  c.time_end(s, tm);
}

void combine(Ctx& c, const double* x, double* y, cudaStream_t s) {
  launch(combine_kernel, cdiv(c.n, 256), 256, 0, s, c.part.p, c.part_splits, c.n, c.near_ptr.p, c.near_col.p,
                                                c.near_corr.p, x, c.par.eps_in / c.par.eps_out, y);
  BP_CHECK_LAUNCH();
}

void matvec_internal(Ctx& c, const double* x, double* y, int op, cudaStream_t s) {
  bool fp32 = (op == BEMPOL_OP_FP32_DIRECT || op == BEMPOL_OP_FP32_TREE);
  const bool tree = op == BEMPOL_OP_FP32_TREE || op == BEMPOL_OP_FP64_TREE;
  if (c.stern) {
    if (tree || c.transposed) fail(BEMPOL_ERR_ARG, "a Stern-layer mesh takes the direct operator forms only");
    strengths(c, x, fp32, s);
    stern_matvec(c, x, y, fp32, s);
    return;
  }
  if (c.transposed) {
    matvec_T_internal(c, x, y, op, s);
    return;
  }
  strengths(c, x, fp32, s);
  if (tree)
    tree_matvec_sums(c, fp32, s);
  else
    p2p_direct(c, fp32, s);
  combine(c, x, y, s);
  if (tree && c.sh_world > 1) {
    // this rank's treecode rows are valid; the caller's all-gather supplies the rest
    const size_t bytes = sizeof(double) * 2 * (size_t)c.n;
    BP_CUDA(cudaMemcpyAsync(c.sh_buf, y, bytes, cudaMemcpyDeviceToDevice, s));
    c.sh_fn(c.sh_user, c.sh_bounds.data(), c.sh_world, (void*)s);
    BP_CUDA(cudaMemcpyAsync(y, c.sh_buf, bytes, cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace bp
