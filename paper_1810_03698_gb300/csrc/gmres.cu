// FP64 restarted GMRES (Saad and Schultz; Sec. "The boundary element method")
// with optional FP64 iterative refinement around a lower-precision operator.
//
// Every system of the context (independent surfaces sharing one set of launches)
// runs its own Arnoldi process in lockstep: one matrix-vector product serves all
// systems, inner products are segmented by system, and each system has its own
// Hessenberg matrix, Givens rotations, residual estimate and stopping test.  A
// system that has converged stops updating while the others go on.
//
// Arnoldi: classical Gram-Schmidt applied twice (CGS2) with every inner product
// formed by a deterministic two-stage reduction (per-chunk partials, then a
// fixed-order sum per system), so reruns are bit-identical.  Givens rotations,
// the residual estimates and the triangular solves run in one device thread per
// system; the host reads one scalar per system and iteration.
//
// Refinement (when params.residual_op != params.op): x <- x + A_op^{-1} (b - A_res x),
// the residual formed in FP64 with the more accurate operator, each inner solve
// run to params.inner_tol, until ||b - A_res x|| / ||b|| < params.gmres_tol (per system).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace bp {

namespace {

constexpr int DOT_TPB = 256;

// out[s * ldo + k] = sum over the elements of system s of V_k . w, for k < nv, in one
// launch.  Work items are (chunk, vector) pairs, one warp each (grid-stride over the
// items): the lanes sum the chunk's products with a fixed stride and a shuffle tree
// gives partial[chunk][k]; the last block to finish (atomic ticket) adds, for every
// system, its chunks' partials in a fixed order (a warp per sum: strided lane sums,
// then a shuffle tree) -- so the result does not depend on scheduling -- and resets
// the ticket for the next call.  Systems with active[s] == 0 are skipped (NULL = all
// active).
__global__ void __launch_bounds__(DOT_TPB) multidot_kernel(const double* __restrict__ V, size_t ld, int nv,
                                                           const double* __restrict__ w,
                                                           const int4* __restrict__ chunks, int nchunk,
                                                           const int* __restrict__ chunk_ptr, int nsys,
                                                           const int* __restrict__ active,
                                                           double* __restrict__ partial, int ldp,
                                                           unsigned* __restrict__ ticket, double* __restrict__ out,
                                                           int ldo, int accumulate) {
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long items = (long long)nchunk * nv;
  const long long nwarps = (long long)gridDim.x * (DOT_TPB / 32);
  for (long long it = (long long)blockIdx.x * (DOT_TPB / 32) + warp; it < items; it += nwarps) {
    const int ci = (int)(it / nv), k = (int)(it - (long long)ci * nv);
    const int4 C = chunks[ci];
    if (active && !active[C.x]) continue;  // uniform across the warp
    const double* __restrict__ vk = V + (size_t)k * ld;
    double a0 = 0.0, a1 = 0.0;
    int i = C.y + lane;
    for (; i + 32 < C.z; i += 64) {
      a0 += vk[i] * w[i];
      a1 += vk[i + 32] * w[i + 32];
    }
    if (i < C.z) a0 += vk[i] * w[i];
    double v = a0 + a1;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) partial[(size_t)ci * ldp + k] = v;
  }
  // every writer makes its partials visible device-wide, and the whole block has done
  // so, before the block takes its ticket
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  // one warp per (system, vector): lanes take every 32nd chunk, then a fixed shuffle tree
  for (int t = warp; t < nsys * nv; t += DOT_TPB / 32) {
    const int sy = t / nv, k = t - sy * nv;
    if (active && !active[sy]) continue;
    double v = 0.0;
    for (int ci = chunk_ptr[sy] + lane; ci < chunk_ptr[sy + 1]; ci += 32) v += __ldcg(partial + (size_t)ci * ldp + k);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) {
      double* o = out + (size_t)sy * ldo + k;
      *o = accumulate ? *o + v : v;
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
}

__device__ __forceinline__ int sys_of(const int* __restrict__ psys, int i, int n) {
  return psys[i < n ? i : i - n];
}

// w -= sum_k V_k h[s][k]   (k < nv, s the system of the element; active systems only)
__global__ void subtract_proj(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ h, int ldh,
                              const int* __restrict__ psys, const int* __restrict__ active, double* __restrict__ w,
                              int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  const int sy = sys_of(psys, i, n);
  if (active && !active[sy]) return;
  const double* hs = h + (size_t)sy * ldh;
  double v = w[i];
  for (int k = 0; k < nv; ++k) v -= V[(size_t)k * ld + i] * hs[k];
  w[i] = v;
}

// x += sum_{k < kk[s]} V_k y[s][k]
__global__ void add_basis(const double* __restrict__ V, size_t ld, const double* __restrict__ y, int ldy,
                          const int* __restrict__ kk, const int* __restrict__ psys, double* __restrict__ x, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  const int sy = sys_of(psys, i, n);
  const int k = kk[sy];
  if (k == 0) return;
  const double* ys = y + (size_t)sy * ldy;
  double v = x[i];
  for (int q = 0; q < k; ++q) v += V[(size_t)q * ld + i] * ys[q];
  x[i] = v;
}

__global__ void axpby(double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                      double* __restrict__ out, int len) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < len) out[i] = a * x[i] + b * y[i];
}

// Second Gram-Schmidt pass and normalisation in one sweep, for the active systems:
// w = (w - sum_k V_k h[s][k]) / sqrt(nrm2[s * ldn]), k < nv.
__global__ void subtract_normalize(const double* __restrict__ V, size_t ld, int nv, const double* __restrict__ h,
                                   int ldh, const double* __restrict__ nrm2, int ldn, const int* __restrict__ psys,
                                   const int* __restrict__ active, double* __restrict__ w, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  const int sy = sys_of(psys, i, n);
  if (active && !active[sy]) return;
  const double* hs = h + (size_t)sy * ldh;
  double v = w[i];
  for (int k = 0; k < nv; ++k) v -= V[(size_t)k * ld + i] * hs[k];
  w[i] = v / sqrt(nrm2[(size_t)sy * ldn]);
}

// v_out = w / sqrt(nrm2[s * ldn]) for the active systems (the norm read on the device)
__global__ void normalize_kernel(const double* __restrict__ w, const double* __restrict__ nrm2, int ldn,
                                 const int* __restrict__ psys, const int* __restrict__ active,
                                 double* __restrict__ out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  const int sy = sys_of(psys, i, n);
  if (active && !active[sy]) return;
  out[i] = w[i] / sqrt(nrm2[(size_t)sy * ldn]);
}

// Givens step for column j of system s's Hessenberg matrix (one thread per active
// system).  Column j = hcol[s][0..j] + h2[s][0..j] (the two Gram-Schmidt passes);
// h2[s][j + 1] = |w'|^2 of the vector after the first pass, so the vector after the
// second pass has |w''|^2 = |w'|^2 - sum_k h2[s][k]^2 (Pythagoras: the columns of V
// are orthonormal), stored to nrm2[s * ldc]; h_{j+1,j} = |w''|.  State cs, sn [m],
// g [m+1] per system.  Writes |g_{j+1}| to res[s] and clears active[s] when it is no
// longer above tol[s] (the system stops; later launches skip it).
__global__ void givens_kernel(double* __restrict__ H, int ldh, size_t sH, int j, const double* __restrict__ hcol,
                              const double* __restrict__ h2, int ldc, double* __restrict__ nrm2,
                              double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g, int ldg,
                              double* __restrict__ res, const double* __restrict__ tol, int* __restrict__ active,
                              int nsys) {
  const int sy = blockIdx.x * blockDim.x + threadIdx.x;
  if (sy >= nsys || !active[sy]) return;
  double* col = H + sy * sH + (size_t)j * ldh;
  const double* hc = hcol + (size_t)sy * ldc;
  const double* hd = h2 + (size_t)sy * ldc;
  double* c_ = cs + (size_t)sy * ldg;
  double* s_ = sn + (size_t)sy * ldg;
  double* g_ = g + (size_t)sy * ldg;
  double q2 = 0.0;
  for (int k = 0; k <= j; ++k) {
    col[k] = hc[k] + hd[k];
    q2 += hd[k] * hd[k];
  }
  const double nn = fmax(hd[j + 1] - q2, 0.0);
  nrm2[(size_t)sy * ldc] = nn;
  col[j + 1] = sqrt(nn);
  for (int k = 0; k < j; ++k) {
    double t = c_[k] * col[k] + s_[k] * col[k + 1];
    col[k + 1] = -s_[k] * col[k] + c_[k] * col[k + 1];
    col[k] = t;
  }
  double a = col[j], b = col[j + 1];
  double r = hypot(a, b);
  double c = r > 0 ? a / r : 1.0, s = r > 0 ? b / r : 0.0;
  c_[j] = c;
  s_[j] = s;
  col[j] = r;
  col[j + 1] = 0.0;
  g_[j + 1] = -s * g_[j];
  g_[j] = c * g_[j];
  const double rj = fabs(g_[j + 1]);
  res[sy] = rj;
  if (!(rj > tol[sy])) active[sy] = 0;
}

// solve the k[s] x k[s] upper-triangular system R y = g of every system
__global__ void backsolve_kernel(const double* __restrict__ H, int ldh, size_t sH, const int* __restrict__ kk,
                                 const double* __restrict__ g, int ldg, double* __restrict__ y, int nsys) {
  const int sy = blockIdx.x * blockDim.x + threadIdx.x;
  if (sy >= nsys) return;
  const int k = kk[sy];
  const double* Hs = H + sy * sH;
  const double* gs = g + (size_t)sy * ldg;
  double* ys = y + (size_t)sy * ldg;
  for (int i = k - 1; i >= 0; --i) {
    double v = gs[i];
    for (int c = i + 1; c < k; ++c) v -= Hs[(size_t)c * ldh + i] * ys[c];
    ys[i] = v / Hs[(size_t)i * ldh + i];
  }
}

__global__ void set_g0(double* __restrict__ g, int ldg, const double* __restrict__ nrm2, int ldn, int m,
                       const int* __restrict__ active, int nsys) {
  const int sy = blockIdx.x * blockDim.x + threadIdx.x;
  if (sy >= nsys || (active && !active[sy])) return;
  double* gs = g + (size_t)sy * ldg;
  gs[0] = sqrt(nrm2[(size_t)sy * ldn]);
  for (int i = 1; i <= m; ++i) gs[i] = 0.0;
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
  size_t sH;               // stride between systems' Hessenberg matrices
  int lds;                 // stride between systems' small vectors (m + 2)
  double *cs, *sn, *g, *y, *hcol, *h2, *nrm2, *res, *partial;
  int ldp;
  unsigned* ticket;
  int *active, *kk;        // device [S] flags and Krylov sizes
};

void multidot(Ctx& c, const Work& w, const double* V, int nv, const double* vec, double* out, const int* active,
              cudaStream_t s) {
  const long long items = (long long)c.nchunk * nv;
  const int blocks = (int)std::min<long long>(2048, std::max<long long>(1, (items + DOT_TPB / 32 - 1) / (DOT_TPB / 32)));
  launch(multidot_kernel, blocks, DOT_TPB, 0, s, V, w.ld, nv, vec, c.chunks.p, c.nchunk,
         c.chunk_ptr.p, c.nsys, active, w.partial, w.ldp, w.ticket, out, w.lds, 0);
}

Work workspace(Ctx& c) {
  const int len = 2 * c.n;
  const int S = c.nsys;
  int m = std::max(1, c.par.gmres_restart);
  const int lds = m + 2;
  if (c.gm_m != m || c.gm_V.n < (size_t)(m + 1) * len || c.gm_H.n < (size_t)S * (m + 1) * m) {
    c.gm_V.alloc((size_t)(m + 1) * len);
    BP_CUDA(cudaMemset(c.gm_V.p, 0, sizeof(double) * c.gm_V.n));  // finite values in every slot
    c.gm_H.alloc((size_t)S * (m + 1) * m);
    c.gm_small.alloc((size_t)S * 8 * lds);
    c.gm_m = m;
  }
  const size_t ndots = (size_t)c.nchunk * lds;
  if (c.gm_dots.n < ndots) c.gm_dots.alloc(ndots);
  if (!c.gm_ticket.p) {
    c.gm_ticket.alloc(1);
    BP_CUDA(cudaMemset(c.gm_ticket.p, 0, sizeof(unsigned)));
  }
  if (c.gm_flags.n < 2 * (size_t)S) c.gm_flags.alloc(2 * (size_t)S);
  Work w;
  w.V = c.gm_V.p;
  w.ld = len;
  w.H = c.gm_H.p;
  w.ldh = m + 1;
  w.sH = (size_t)(m + 1) * m;
  w.lds = lds;
  double* sm = c.gm_small.p;
  const size_t blk = (size_t)S * lds;
  w.cs = sm;
  w.sn = sm + blk;
  w.g = sm + 2 * blk;
  w.y = sm + 3 * blk;
  w.hcol = sm + 4 * blk;
  w.h2 = sm + 5 * blk;
  w.nrm2 = sm + 6 * blk;   // nrm2[s * lds]
  w.res = sm + 7 * blk;    // res[s]
  w.partial = c.gm_dots.p;
  w.ldp = lds;
  w.ticket = c.gm_ticket.p;
  w.active = c.gm_flags.p;
  w.kk = c.gm_flags.p + S;
  return w;
}

// per-system squared norms of v (device; host copy returned)
std::vector<double> sys_norm2(Ctx& c, const Work& w, const double* v, const int* active, cudaStream_t s) {
  multidot(c, w, v, 1, v, w.nrm2, active, s);
  BP_CUDA(cudaMemcpy2DAsync(c.h_pinned, sizeof(double), w.nrm2, sizeof(double) * w.lds, sizeof(double), c.nsys,
                            cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  return std::vector<double>(c.h_pinned, c.h_pinned + c.nsys);
}

void put_flags(Ctx& c, int* d, const std::vector<int>& h, cudaStream_t s) {
  int* hp = reinterpret_cast<int*>(c.h_pinned + 2 * c.nsys);
  std::copy(h.begin(), h.end(), hp);
  BP_CUDA(cudaMemcpyAsync(d, hp, sizeof(int) * h.size(), cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaStreamSynchronize(s));  // the pinned staging area is reused right away
}

// GMRES on A_op x = b from the initial x for the systems with tol_abs[s] >= 0 (the
// others are left alone); system s stops when ||b - A x||_s <= tol_abs[s] (true
// residual at restarts and on exit, the Givens estimate inside a cycle).
// rres[s] receives the final true residual norm of each solved system.
GmresOut gmres(Ctx& c, int op, const double* b, double* x, const std::vector<double>& tol_abs, int maxit,
               std::vector<double>& rres, cudaStream_t s) {
  const int n = c.n, len = 2 * n, S = c.nsys;
  Work w = workspace(c);
  const int m = c.gm_m;
  const int tb = 256, nb = cdiv(len, tb);
  double* r = c.vec_a.p;
  GmresOut out;
  out.sys_iters.assign(S, 0);
  out.sys_conv.assign(S, 0);
  std::vector<int> todo(S, 0), act(S, 0), kk(S, 0);
  for (int q = 0; q < S; ++q) todo[q] = tol_abs[q] >= 0.0;
  rres.assign(S, 0.0);
  if (c.gm_tol.n < (size_t)S) c.gm_tol.alloc(S);
  for (cudaEvent_t& e : c.gm_ev)
    if (!e) BP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  std::copy(tol_abs.begin(), tol_abs.end(), c.h_pinned);
  BP_CUDA(cudaMemcpyAsync(c.gm_tol.p, c.h_pinned, sizeof(double) * S, cudaMemcpyHostToDevice, s));
  BP_CUDA(cudaStreamSynchronize(s));  // the pinned staging area is reused right away
  int total = 0;
  while (true) {
    // r = b - A x, per-system norms
    put_flags(c, w.active, todo, s);
    c.mv_active = w.active;
    matvec_internal(c, x, r, op, s);
    c.mv_active = nullptr;
    ++out.matvecs;
    launch(axpby, nb, tb, 0, s, 1.0, b, -1.0, r, r, len);
    std::vector<double> nr = sys_norm2(c, w, r, w.active, s);
    int nact = 0;
    for (int q = 0; q < S; ++q) {
      if (!todo[q]) continue;
      rres[q] = std::sqrt(nr[q]);
      if (rres[q] <= tol_abs[q]) {
        out.sys_conv[q] = 1;
        todo[q] = 0;
      } else {
        ++nact;
      }
    }
    if (nact == 0 || total >= maxit) break;
    act = todo;
    put_flags(c, w.active, act, s);
    launch(normalize_kernel, nb, tb, 0, s, r, w.nrm2, w.lds, c.psys.p, w.active, w.V, n);
    launch(set_g0, cdiv(S, 64), 64, 0, s, w.g, w.lds, w.nrm2, w.lds, m, w.active, S);
    BP_CHECK_LAUNCH();
    std::fill(kk.begin(), kk.end(), 0);
    // Arnoldi steps, pipelined one deep: step j is enqueued before the host waits for
    // the residual estimates of step j - 1.  The Givens kernel clears a converged
    // system's device flag itself, so step j already skips it; the host's flags follow
    // the same test one step later.  After the last system stops, the step enqueued
    // behind it finds every flag clear and does no work.
    int pending = -1;
    for (int j = 0;; ++j) {
      const bool more = j < m && total + (pending >= 0 ? 1 : 0) < maxit;
      const Ctx::StatMark mark = c.stat_mark();
      if (more) {
        double* vj = w.V + (size_t)j * w.ld;
        double* wv = w.V + (size_t)(j + 1) * w.ld;
        c.mv_active = w.active;
        matvec_internal(c, vj, wv, op, s);
        c.mv_active = nullptr;
        // CGS2 per system; the second inner product also gives |w'|^2 (V_{j+1} = w')
        multidot(c, w, w.V, j + 1, wv, w.hcol, w.active, s);
        launch(subtract_proj, nb, tb, 0, s, w.V, w.ld, j + 1, w.hcol, w.lds, c.psys.p, w.active, wv, n);
        multidot(c, w, w.V, j + 2, wv, w.h2, w.active, s);
        launch(givens_kernel, cdiv(S, 64), 64, 0, s, w.H, w.ldh, w.sH, j, w.hcol, w.h2, w.lds, w.nrm2, w.cs, w.sn,
               w.g, w.lds, w.res, c.gm_tol.p, w.active, S);
        launch(subtract_normalize, nb, tb, 0, s, w.V, w.ld, j + 1, w.h2, w.lds, w.nrm2, w.lds, c.psys.p, w.active, wv,
               n);
        BP_CHECK_LAUNCH();
        BP_CUDA(cudaMemcpyAsync(c.h_pinned + (size_t)(j & 1) * S, w.res, sizeof(double) * S, cudaMemcpyDeviceToHost,
                                s));
        BP_CUDA(cudaEventRecord(c.gm_ev[j & 1], s));
      }
      bool any = pending >= 0;
      if (pending >= 0) {
        BP_CUDA(cudaEventSynchronize(c.gm_ev[pending & 1]));
        const double* hr = c.h_pinned + (size_t)(pending & 1) * S;
        ++total;
        ++out.iters;
        ++out.matvecs;
        any = false;
        for (int q = 0; q < S; ++q) {
          if (!act[q]) continue;
          kk[q] = pending + 1;
          ++out.sys_iters[q];
          if (!(hr[q] > tol_abs[q]))
            act[q] = 0;
          else
            any = true;
        }
      }
      if (pending >= 0 && !any) {
        if (more) c.stat_rewind(mark);  // step j found every system stopped
        break;
      }
      if (!more) break;
      pending = j;
    }
    // x += V y per system
    put_flags(c, w.kk, kk, s);
    launch(backsolve_kernel, cdiv(S, 64), 64, 0, s, w.H, w.ldh, w.sH, w.kk, w.g, w.lds, w.y, S);
    launch(add_basis, nb, tb, 0, s, w.V, w.ld, w.y, w.lds, w.kk, c.psys.p, x, n);
    BP_CHECK_LAUNCH();
  }
  out.converged = true;
  for (int q = 0; q < S; ++q)
    if (tol_abs[q] >= 0.0 && !out.sys_conv[q]) out.converged = false;
  return out;
}

}  // namespace

double dot_dev(Ctx& c, const double* a, const double* b, int len, cudaStream_t s) {
  // plain FP64 dot over the whole vector (a single-system segmentation is not needed)
  (void)len;
  Work w = workspace(c);
  multidot(c, w, a, 1, b, w.nrm2, nullptr, s);
  BP_CUDA(cudaMemcpy2DAsync(c.h_pinned, sizeof(double), w.nrm2, sizeof(double) * w.lds, sizeof(double), c.nsys,
                            cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  double v = 0.0;
  for (int q = 0; q < c.nsys; ++q) v += c.h_pinned[q];
  return v;
}

void permute_to_internal(const Ctx& c, const double* src, double* dst, int nb, cudaStream_t s) {
  launch(permute_kernel, cdiv((long long)c.n * nb, 256), 256, 0, s, c.perm.p, c.n, nb, src, dst, 1);
  BP_CHECK_LAUNCH();
}

void permute_to_caller(const Ctx& c, const double* src, double* dst, int nb, cudaStream_t s) {
  launch(permute_kernel, cdiv((long long)c.n * nb, 256), 256, 0, s, c.perm.p, c.n, nb, src, dst, 0);
  BP_CHECK_LAUNCH();
}

GmresOut solve_bem(Ctx& c, const double* b, double* x, const std::vector<char>& want, cudaStream_t s,
                   bool refine, double rel_tol) {
  if (!(rel_tol > 0.0)) rel_tol = c.par.gmres_tol;
  const int n = c.n, len = 2 * n, S = c.nsys;
  Work w = workspace(c);
  std::vector<int> all(S, 1);
  for (int q = 0; q < S; ++q) all[q] = want.empty() ? 1 : (want[q] ? 1 : 0);
  put_flags(c, w.active, all, s);
  std::vector<double> bn2 = sys_norm2(c, w, b, w.active, s);
  std::vector<double> bn(S, 0.0), tol(S, -1.0);
  GmresOut tot;
  tot.sys_iters.assign(S, 0);
  tot.sys_res.assign(S, 0.0);
  tot.sys_conv.assign(S, 1);
  std::vector<int> zero_sys(S, 0);
  bool any_zero = false;
  for (int q = 0; q < S; ++q) {
    if (!all[q]) continue;
    bn[q] = std::sqrt(bn2[q]);
    if (bn[q] == 0.0) {
      zero_sys[q] = 1;  // b = 0: x = 0 exactly
      any_zero = true;
    } else {
      tol[q] = rel_tol * bn[q];
      tot.sys_conv[q] = 0;
    }
  }
  if (any_zero) {
    for (int q = 0; q < S; ++q)
      if (zero_sys[q]) {
        BP_CUDA(cudaMemsetAsync(x + c.h_sys_pan[q], 0, sizeof(double) * (c.h_sys_pan[q + 1] - c.h_sys_pan[q]), s));
        BP_CUDA(cudaMemsetAsync(x + n + c.h_sys_pan[q], 0,
                                sizeof(double) * (c.h_sys_pan[q + 1] - c.h_sys_pan[q]), s));
      }
  }
  auto finish = [&](const std::vector<double>& rn) {
    tot.converged = true;
    tot.rel_res = 0.0;
    for (int q = 0; q < S; ++q) {
      if (tol[q] < 0.0) continue;
      tot.sys_res[q] = rn[q] / bn[q];
      tot.rel_res = std::max(tot.rel_res, tot.sys_res[q]);
      if (!tot.sys_conv[q]) tot.converged = false;
    }
  };
  if (!refine || c.par.residual_op == c.par.op) {
    std::vector<double> rn;
    GmresOut o = gmres(c, c.par.op, b, x, tol, c.par.gmres_maxit, rn, s);
    tot.iters = o.iters;
    tot.matvecs = o.matvecs;
    for (int q = 0; q < S; ++q) {
      tot.sys_iters[q] = o.sys_iters[q];
      if (tol[q] >= 0.0) tot.sys_conv[q] = o.sys_conv[q];
    }
    finish(rn);
    return tot;
  }
  // iterative refinement, per system
  double* r = c.vec_b.p;
  double* e = c.vec_c.p;
  const int tb = 256, nb = cdiv(len, tb);
  std::vector<double> rn(S, 0.0), itol(S, -1.0);
  std::vector<int> todo(S, 0);
  for (int q = 0; q < S; ++q) todo[q] = tol[q] >= 0.0;
  for (int it = 0; it <= c.par.refine_maxit; ++it) {
    put_flags(c, w.active, todo, s);
    c.mv_active = w.active;
    matvec_internal(c, x, r, c.par.residual_op, s);
    c.mv_active = nullptr;
    ++tot.matvecs;
    ++tot.residual_matvecs;
    launch(axpby, nb, tb, 0, s, 1.0, b, -1.0, r, r, len);
    BP_CHECK_LAUNCH();
    std::vector<double> r2 = sys_norm2(c, w, r, w.active, s);
    int nact = 0;
    for (int q = 0; q < S; ++q) {
      itol[q] = -1.0;
      if (!todo[q]) continue;
      rn[q] = std::sqrt(r2[q]);
      if (rn[q] <= tol[q]) {
        tot.sys_conv[q] = 1;
        todo[q] = 0;
        continue;
      }
      itol[q] = std::max(c.par.inner_tol * rn[q], 0.5 * tol[q]);
      ++nact;
    }
    if (nact == 0 || it == c.par.refine_maxit) break;
    BP_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * len, s));
    std::vector<double> ir;
    GmresOut o = gmres(c, c.par.op, r, e, itol, c.par.gmres_maxit, ir, s);
    tot.iters += o.iters;
    tot.matvecs += o.matvecs;
    for (int q = 0; q < S; ++q) tot.sys_iters[q] += o.sys_iters[q];
    launch(axpby, nb, tb, 0, s, 1.0, x, 1.0, e, x, len);  // e = 0 outside the refined systems
    BP_CHECK_LAUNCH();
  }
  finish(rn);
  return tot;
}

}  // namespace bp
