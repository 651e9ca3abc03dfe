// FP64 restarted GMRES (Saad and Schultz; Sec. "The boundary element method")
// with optional FP64 iterative refinement around a lower-precision operator.
//
// Arnoldi: classical Gram-Schmidt applied twice (CGS2) with every inner product
// formed by a deterministic two-stage reduction (per-block partials, then a
// fixed-order sum), so reruns are bit-identical.  Givens rotations, the residual
// estimate and the triangular solve run in single-thread device kernels; the
// host reads one scalar per iteration to decide convergence.
//
// Refinement (when params.residual_op != params.op): x <- x + A_op^{-1} (b - A_res x),
// the residual formed in FP64 with the more accurate operator, each inner solve
// run to params.inner_tol, until ||b - A_res x|| / ||b|| < params.gmres_tol.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace bp {

namespace {

constexpr int DOT_BLOCKS = 256;
constexpr int DOT_TPB = 256;
constexpr int MAXV = 16;  // basis vectors handled per multi-dot pass

// out[k] = V_k . w for k < nv, in one launch.  Each block writes its partial sums
// partial[b][k] (chunks of MAXV vectors per pass over its slice); the last block to
// finish (atomic ticket) adds the partials in block order, so the result does not
// depend on scheduling, and resets the ticket for the next call.
__global__ void __launch_bounds__(DOT_TPB) multidot_kernel(const double* __restrict__ V, size_t ld, int nv,
                                                           const double* __restrict__ w, int len,
                                                           double* __restrict__ partial, int ldp,
                                                           unsigned* __restrict__ ticket, double* __restrict__ out,
                                                           int accumulate) {
  __shared__ double sh[MAXV][DOT_TPB / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k0 = 0; k0 < nv; k0 += MAXV) {
    const int cnt = min(MAXV, nv - k0);
    double acc[MAXV];
#pragma unroll
    for (int k = 0; k < MAXV; ++k) acc[k] = 0.0;
    for (int i = blockIdx.x * DOT_TPB + threadIdx.x; i < len; i += gridDim.x * DOT_TPB) {
      const double wi = w[i];
#pragma unroll
      for (int k = 0; k < MAXV; ++k)
        if (k < cnt) acc[k] += V[(size_t)(k0 + k) * ld + i] * wi;
    }
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
      double v = acc[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < cnt) {
      double v = 0.0;
      for (int wv = 0; wv < DOT_TPB / 32; ++wv) v += sh[threadIdx.x][wv];
      partial[(size_t)blockIdx.x * ldp + k0 + threadIdx.x] = v;
    }
    __syncthreads();
  }
  __threadfence();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  for (int k = threadIdx.x; k < nv; k += DOT_TPB) {
    double v = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) v += __ldcg(partial + (size_t)b * ldp + k);
    out[k] = accumulate ? out[k] + v : v;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

// w -= sum_k V_k h_k   (k < nv)
__global__ void subtract_proj(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ h,
                              double* __restrict__ w, int len) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  double v = w[i];
  for (int k = 0; k < nv; ++k) v -= V[(size_t)k * ld + i] * h[k];
  w[i] = v;
}

__global__ void axpby(double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                      double* __restrict__ out, int len) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[i] = a * x[i] + b * y[i];
}

// v_out = w / sqrt(*nrm2)  (the norm read on the device)
__global__ void normalize_kernel(const double* __restrict__ w, const double* __restrict__ nrm2,
                                 double* __restrict__ out, int len) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[i] = w[i] / sqrt(*nrm2);
}

// Givens step for column j of the Hessenberg matrix.  hcol[0..j] = projections,
// *nrm2 = |w|^2 gives h_{j+1,j}.  State: cs, sn [m], g [m+1].  Writes |g_{j+1}| to *res.
__global__ void givens_kernel(double* __restrict__ H, int ldh, int j, const double* __restrict__ hcol,
                              const double* __restrict__ nrm2, double* __restrict__ cs, double* __restrict__ sn,
                              double* __restrict__ g, double* __restrict__ res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* col = H + (size_t)j * ldh;
  for (int k = 0; k <= j; ++k) col[k] = hcol[k];
  col[j + 1] = sqrt(*nrm2);
  for (int k = 0; k < j; ++k) {
    double t = cs[k] * col[k] + sn[k] * col[k + 1];
    col[k + 1] = -sn[k] * col[k] + cs[k] * col[k + 1];
    col[k] = t;
  }
  double a = col[j], b = col[j + 1];
  double r = hypot(a, b);
  double c = r > 0 ? a / r : 1.0, s = r > 0 ? b / r : 0.0;
  cs[j] = c;
  sn[j] = s;
  col[j] = r;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  *res = fabs(g[j + 1]);
}

// solve the k x k upper-triangular system R y = g
__global__ void backsolve_kernel(const double* __restrict__ H, int ldh, int k, const double* __restrict__ g,
                                 double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double v = g[i];
    for (int c = i + 1; c < k; ++c) v -= H[(size_t)c * ldh + i] * y[c];
    y[i] = v / H[(size_t)i * ldh + i];
  }
}

__global__ void set_g0(double* __restrict__ g, const double* __restrict__ nrm2, int m) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    g[0] = sqrt(*nrm2);
    for (int i = 1; i <= m; ++i) g[i] = 0.0;
  }
}

__global__ void permute_kernel(const int* __restrict__ perm, int n, int nb, const double* __restrict__ src,
                               double* __restrict__ dst, int to_internal) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * nb) return;
  int b = t / n, i = t - b * n;
  int p = perm[i];
  if (to_internal)
    dst[(size_t)b * n + i] = src[(size_t)b * n + p];
  else
    dst[(size_t)b * n + p] = src[(size_t)b * n + i];
}

struct Work {
  double* V;
  size_t ld;
  double* H;
  int ldh;
  double *cs, *sn, *g, *y, *hcol, *nrm2, *res, *partial;
  int ldp;
  unsigned* ticket;
};

void multidot(Ctx& c, const Work& w, const double* V, int nv, const double* vec, int len, double* out,
              bool accumulate, cudaStream_t s) {
  launch(multidot_kernel, DOT_BLOCKS, DOT_TPB, 0, s, V, w.ld, nv, vec, len, w.partial, w.ldp, w.ticket, out,
         accumulate ? 1 : 0);
  (void)c;
}

double read_scalar(Ctx& c, const double* d, cudaStream_t s) {
  BP_CUDA(cudaMemcpyAsync(c.h_pinned + 2, d, sizeof(double), cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  return c.h_pinned[2];
}

Work workspace(Ctx& c) {
  const int len = 2 * c.n;
  int m = std::max(1, c.par.gmres_restart);
  if (c.gm_m != m || c.gm_V.n < (size_t)(m + 1) * len) {
    c.gm_V.alloc((size_t)(m + 1) * len);
    c.gm_H.alloc((size_t)(m + 1) * m);
    c.gm_small.alloc(4 * (size_t)(m + 2) + 8);
    c.gm_m = m;
  }
  const size_t ndots = (size_t)DOT_BLOCKS * (m + 2) + m + 2;
  if (c.gm_dots.n < ndots) c.gm_dots.alloc(ndots);
  if (!c.gm_ticket.p) {
    c.gm_ticket.alloc(1);
    BP_CUDA(cudaMemset(c.gm_ticket.p, 0, sizeof(unsigned)));
  }
  Work w;
  w.V = c.gm_V.p;
  w.ld = len;
  w.H = c.gm_H.p;
  w.ldh = m + 1;
  double* sm = c.gm_small.p;
  w.cs = sm;
  w.sn = sm + (m + 2);
  w.g = sm + 2 * (m + 2);
  w.y = sm + 3 * (m + 2);
  w.nrm2 = sm + 4 * (m + 2);
  w.res = w.nrm2 + 1;
  w.partial = c.gm_dots.p;
  w.ldp = m + 2;
  w.ticket = c.gm_ticket.p;
  w.hcol = c.gm_dots.p + (size_t)DOT_BLOCKS * (m + 2);
  return w;
}

// GMRES on A_op x = b from the initial x; stops when ||b - A x|| <= tol_abs (true
// residual at restarts and on exit, the Givens estimate inside a cycle).
GmresOut gmres(Ctx& c, int op, const double* b, double* x, double tol_abs, int maxit, cudaStream_t s) {
  const int len = 2 * c.n;
  Work w = workspace(c);
  const int m = c.gm_m;
  const int tb = 256, nb = cdiv(len, tb);
  double* r = c.vec_a.p;
  GmresOut out;
  int total = 0;
  while (true) {
    // r = b - A x
    matvec_internal(c, x, r, op, s);
    ++out.matvecs;
    launch(axpby, nb, tb, 0, s, 1.0, b, -1.0, r, r, len);
    multidot(c, w, r, 1, r, len, w.nrm2, false, s);
    double beta = std::sqrt(read_scalar(c, w.nrm2, s));
    out.rel_res = beta;
    if (beta <= tol_abs) {
      out.converged = true;
      break;
    }
    if (total >= maxit) break;
    launch(normalize_kernel, nb, tb, 0, s, r, w.nrm2, w.V, len);
    launch(set_g0, 1, 1, 0, s, w.g, w.nrm2, m);
    BP_CHECK_LAUNCH();
    int k = 0;
    for (int j = 0; j < m && total < maxit; ++j) {
      double* vj = w.V + (size_t)j * w.ld;
      double* wv = w.V + (size_t)(j + 1) * w.ld;
      matvec_internal(c, vj, wv, op, s);
      ++out.matvecs;
      // CGS2
      multidot(c, w, w.V, j + 1, wv, len, w.hcol, false, s);
      launch(subtract_proj, nb, tb, 0, s, w.V, w.ld, j + 1, w.hcol, wv, len);
      double* h2 = w.y;  // scratch for the second pass
      multidot(c, w, w.V, j + 1, wv, len, h2, false, s);
      launch(subtract_proj, nb, tb, 0, s, w.V, w.ld, j + 1, h2, wv, len);
      launch(axpby, cdiv(j + 1, 64), 64, 0, s, 1.0, w.hcol, 1.0, h2, w.hcol, j + 1);
      multidot(c, w, wv, 1, wv, len, w.nrm2, false, s);
      launch(givens_kernel, 1, 1, 0, s, w.H, w.ldh, j, w.hcol, w.nrm2, w.cs, w.sn, w.g, w.res);
      launch(normalize_kernel, nb, tb, 0, s, wv, w.nrm2, wv, len);
      BP_CHECK_LAUNCH();
      ++total;
      ++out.iters;
      k = j + 1;
      double est = read_scalar(c, w.res, s);
      if (!(est > tol_abs)) break;
    }
    launch(backsolve_kernel, 1, 1, 0, s, w.H, w.ldh, k, w.g, w.y);
    // x += V y   (subtract_proj with -y)
    launch(axpby, cdiv(k, 64), 64, 0, s, -1.0, w.y, 0.0, w.y, w.y, k);
    launch(subtract_proj, nb, tb, 0, s, w.V, w.ld, k, w.y, x, len);
    BP_CHECK_LAUNCH();
  }
  return out;
}

}  // namespace

double dot_dev(Ctx& c, const double* a, const double* b, int len, cudaStream_t s) {
  Work w = workspace(c);
  multidot(c, w, a, 1, b, len, w.nrm2, false, s);
  return read_scalar(c, w.nrm2, s);
}

void permute_to_internal(const Ctx& c, const double* src, double* dst, int nb, cudaStream_t s) {
  launch(permute_kernel, cdiv((long long)c.n * nb, 256), 256, 0, s, c.perm.p, c.n, nb, src, dst, 1);
  BP_CHECK_LAUNCH();
}

void permute_to_caller(const Ctx& c, const double* src, double* dst, int nb, cudaStream_t s) {
  launch(permute_kernel, cdiv((long long)c.n * nb, 256), 256, 0, s, c.perm.p, c.n, nb, src, dst, 0);
  BP_CHECK_LAUNCH();
}

GmresOut solve_bem(Ctx& c, const double* b, double* x, cudaStream_t s) {
  const int len = 2 * c.n;
  double bn = std::sqrt(dot_dev(c, b, b, len, s));
  if (bn == 0.0) {
    BP_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * len, s));
    GmresOut o;
    o.converged = true;
    return o;
  }
  const double tol = c.par.gmres_tol * bn;
  if (c.par.residual_op == c.par.op) {
    GmresOut o = gmres(c, c.par.op, b, x, tol, c.par.gmres_maxit, s);
    o.rel_res /= bn;
    return o;
  }
  // iterative refinement
  GmresOut tot;
  double* r = c.vec_b.p;
  double* e = c.vec_c.p;
  const int tb = 256, nb = cdiv(len, tb);
  for (int it = 0; it <= c.par.refine_maxit; ++it) {
    matvec_internal(c, x, r, c.par.residual_op, s);
    ++tot.matvecs;
    launch(axpby, nb, tb, 0, s, 1.0, b, -1.0, r, r, len);
    BP_CHECK_LAUNCH();
    double rn = std::sqrt(dot_dev(c, r, r, len, s));
    tot.rel_res = rn / bn;
    if (rn <= tol) {
      tot.converged = true;
      break;
    }
    if (it == c.par.refine_maxit) break;
    BP_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * len, s));
    double itol = std::max(c.par.inner_tol * rn, 0.5 * tol);
    GmresOut o = gmres(c, c.par.op, r, e, itol, c.par.gmres_maxit, s);
    tot.iters += o.iters;
    tot.matvecs += o.matvecs;
    launch(axpby, nb, tb, 0, s, 1.0, x, 1.0, e, x, len);
    BP_CHECK_LAUNCH();
  }
  return tot;
}

}  // namespace bp
