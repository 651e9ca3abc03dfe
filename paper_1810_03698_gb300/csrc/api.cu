// C ABI of the library (declared in include/bempol.h): context lifecycle,
// validation, data marshalling and the self-consistent solvation driver.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

struct bempol_ctx : public bp::Ctx {};

namespace bp {

static std::atomic<long long> g_launches{0};

void note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  BP_CUDA(cudaGetLastError());
}

void Ctx::time_begin(int kind, cudaStream_t s, Timed& t) {
  t.kind = kind;
  ++stat_launches[kind];
  if (!stats_on) return;
  BP_CUDA(cudaEventCreate(&t.a));
  BP_CUDA(cudaEventCreate(&t.b));
  BP_CUDA(cudaEventRecord(t.a, s));
}

void Ctx::time_end(cudaStream_t s, Timed& t) {
  if (!stats_on) return;
  BP_CUDA(cudaEventRecord(t.b, s));
  timed.push_back(t);
}

void Ctx::stat_rewind(const StatMark& m) {
  for (size_t k = m.ntimed; k < timed.size(); ++k) {
    cudaEventSynchronize(timed[k].b);
    cudaEventDestroy(timed[k].a);
    cudaEventDestroy(timed[k].b);
  }
  if (timed.size() > m.ntimed) timed.resize(m.ntimed);
  for (int k = 0; k < NKIND; ++k) stat_launches[k] = m.launches[k];
  stat_pairs = m.pairs;
  stat_far = m.far;
}

void Ctx::collect_timers() {
  for (auto& t : timed) {
    float ms = 0;
    cudaEventSynchronize(t.b);
    cudaEventElapsedTime(&ms, t.a, t.b);
    stat_ms[t.kind] += ms;
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  timed.clear();
}

void Ctx::ensure_aux() {
  if (aux) return;
  int lo = 0, hi = 0;
  BP_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  BP_CUDA(cudaStreamCreateWithPriority(&aux, cudaStreamNonBlocking, hi));
  BP_CUDA(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
  BP_CUDA(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
}

Ctx::~Ctx() {
  collect_timers();
  if (h_pinned) cudaFreeHost(h_pinned);
  for (cudaEvent_t e : gm_ev)
    if (e) cudaEventDestroy(e);
  if (aux) {
    cudaStreamSynchronize(aux);
    cudaStreamDestroy(aux);
    cudaEventDestroy(ev_fork);
    cudaEventDestroy(ev_join);
  }
}

void check_device_error(Ctx& c, cudaStream_t s) {
  if (!c.dev_err.p) return;
  int v = 0;
  BP_CUDA(cudaMemcpyAsync(&v, c.dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  BP_CUDA(cudaStreamSynchronize(s));
  if (v) {
    c.dev_err.zero(s);
    BP_CUDA(cudaStreamSynchronize(s));
    fail(BEMPOL_ERR_TIMEOUT, "a device-side wait of the FP32 near-field kernel exceeded its limit; results invalid");
  }
}

int num_sms(int device) {
  static int cache[64] = {0};
  if (device < 0 || device >= 64) device = 0;
  if (!cache[device]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 148;
    cache[device] = v;
  }
  return cache[device];
}

namespace {

// e^2/(4 pi eps0 A) per mole in kcal/mol from the SI-defined e, eps0 (CODATA 2018), N_A and 4184 J/kcal
constexpr double COULOMB_KCAL = 332.0637132991921;
constexpr double KCAL_PER_UNIT = 4.0 * M_PI * COULOMB_KCAL;

void check_params(const bempol_params* p) {
  if (!p) fail(BEMPOL_ERR_ARG, "params is NULL");
  auto bad = [](const char* m) { fail(BEMPOL_ERR_ARG, m); };
  if (!(p->eps_in > 0) || !(p->eps_out > 0)) bad("eps_in and eps_out must be > 0");
  if (!(p->kappa >= 0)) bad("kappa must be >= 0");
  if (p->gauss_k != 1 && p->gauss_k != 3 && p->gauss_k != 4) bad("gauss_k must be 1, 3 or 4");
  if (!(p->near_factor >= 0)) bad("near_factor must be >= 0");
  if (!(p->theta > 0 && p->theta < 1.5)) bad("theta must be in (0, 1.5)");
  if (p->order < 1 || p->order > 6) bad("order must be in 1..6");
  if (p->leaf < 8 || p->leaf > 4096) bad("leaf must be in 8..4096");
  if (!(p->gmres_tol > 0)) bad("gmres_tol must be > 0");
  if (p->gmres_restart < 1 || p->gmres_restart > 1000) bad("gmres_restart must be in 1..1000");
  if (p->gmres_maxit < 1) bad("gmres_maxit must be >= 1");
  if (!(p->scf_tol > 0)) bad("scf_tol must be > 0");
  if (!(p->sor_omega > 0 && p->sor_omega <= 1.0)) bad("sor_omega must be in (0, 1]");
  if (p->scf_maxit < 1) bad("scf_maxit must be >= 1");
  if (p->op < 0 || p->op > 3 || p->residual_op < 0 || p->residual_op > 3) bad("op/residual_op out of range");
  if (!(p->inner_tol > 0 && p->inner_tol < 1)) bad("inner_tol must be in (0, 1)");
  if (p->refine_maxit < 0) bad("refine_maxit must be >= 0");
  if (!(p->thole_a >= 0)) bad("thole_a must be >= 0");
  if (p->refine_scope != BEMPOL_REFINE_EVERY && p->refine_scope != BEMPOL_REFINE_FINAL)
    bad("refine_scope must be BEMPOL_REFINE_EVERY or BEMPOL_REFINE_FINAL");
  if (p->thole_perm != 0 && p->thole_perm != 1) bad("thole_perm must be 0 or 1");
  if (p->near_rule != BEMPOL_NEAR_SEMI_ANALYTICAL && p->near_rule != BEMPOL_NEAR_GAUSS19)
    bad("near_rule must be BEMPOL_NEAR_SEMI_ANALYTICAL or BEMPOL_NEAR_GAUSS19");
}

bool op_fp32(int op) { return op == BEMPOL_OP_FP32_DIRECT || op == BEMPOL_OP_FP32_TREE; }
// Relative residual that GMRES with an FP32 operator form reliably reaches (FP32 pair
// terms with FP64 sums: the operator itself is accurate to ~1e-7).
constexpr double FP32_SOLVE_FLOOR = 1e-6;
bool op_tree(int op) { return op == BEMPOL_OP_FP32_TREE || op == BEMPOL_OP_FP64_TREE; }

template <typename T>
void to_device(DBuf<T>& dst, const T* src, size_t count, int where, cudaStream_t s) {
  dst.alloc(std::max<size_t>(1, count));
  if (count == 0) return;
  BP_CUDA(cudaMemcpyAsync(dst.p, src, count * sizeof(T),
                          where == BEMPOL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
}

template <typename T>
std::vector<T> to_host(const T* src, size_t count, int where, cudaStream_t s) {
  std::vector<T> h(count);
  if (count == 0) return h;
  if (where == BEMPOL_DEVICE) {
    BP_CUDA(cudaMemcpyAsync(h.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    BP_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(h.data(), src, count * sizeof(T));
  }
  return h;
}

// Pinned host and device scalar areas sized for per-system values.
void size_scalars(Ctx& c) {
  const size_t want = 4 * (size_t)c.nsys + 16;
  if (c.scal.n < want) {
    c.scal.alloc(want);
    if (c.h_pinned) cudaFreeHost(c.h_pinned);
    c.h_pinned = nullptr;
    BP_CUDA(cudaMallocHost(&c.h_pinned, want * sizeof(double)));
  }
}

// Groups (bodies of systems) from per-panel system and body ids (NULL = all 0):
// sorted (system, body) pairs; returns the group of every panel (caller order).
std::vector<int> make_groups(Ctx& c, int64_t nt, const std::vector<int32_t>& sy, const std::vector<int32_t>& bo) {
  std::vector<std::pair<int, int>> key, u;
  if (sy.empty() && bo.empty()) {
    u.assign(1, {0, 0});  // one system of one body
  } else {
    key.resize(nt);
    for (int64_t t = 0; t < nt; ++t) {
      const int a = sy.empty() ? 0 : sy[t], b = bo.empty() ? 0 : bo[t];
      if (a < 0 || b < 0) fail(BEMPOL_ERR_ARG, "system and body ids must be >= 0");
      key[t] = {a, b};
    }
    u = key;
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end()), u.end());
  }
  if (u.size() > 1023) fail(BEMPOL_ERR_ARG, "at most 1023 (system, body) groups");
  const int S = u.back().first + 1;
  c.ngroup = (int)u.size();
  c.nsys = S;
  c.h_grp_sys.resize(c.ngroup);
  c.h_grp_body.resize(c.ngroup);
  c.h_sys_grp.assign(S + 1, 0);
  for (int g = 0; g < c.ngroup; ++g) {
    c.h_grp_sys[g] = u[g].first;
    c.h_grp_body[g] = u[g].second;
    ++c.h_sys_grp[u[g].first + 1];
  }
  for (int q = 0; q < S; ++q) {
    if (c.h_sys_grp[q + 1] == 0)
      fail(BEMPOL_ERR_ARG, "system ids must be 0..S-1 with every system present (missing " + std::to_string(q) + ")");
    c.h_sys_grp[q + 1] += c.h_sys_grp[q];
  }
  std::vector<int> grp;
  if (c.ngroup > 1) {
    grp.resize(nt);
    for (int64_t t = 0; t < nt; ++t) grp[t] = (int)(std::lower_bound(u.begin(), u.end(), key[t]) - u.begin());
  }
  return grp;
}

void ensure_tree(Ctx& c, int op, cudaStream_t s) {
  if (op_tree(op) && c.stern) fail(BEMPOL_ERR_ARG, "a Stern-layer mesh takes the direct operator forms only");
  if (op_tree(op) && !c.tree_ready) build_tree(c, s);
}

__global__ void add_vec_scaled(const double* __restrict__ a, const double* __restrict__ b, double sb,
                               double* __restrict__ o, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = a[i] + sb * b[i];
}

__global__ void scale_kernel(double* __restrict__ a, double f, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] *= f;
}

__global__ void add_vec(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ o, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = a[i] + (b ? b[i] : 0.0);
}

// x[i] = a fixed pseudo-random value in [-1, 1) (integer hash of i and the seed)
__global__ void hash_vector_kernel(double* __restrict__ x, int len, unsigned seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  unsigned h = (unsigned)i * 2654435761u ^ seed;
  h ^= h >> 16;
  h *= 2246822519u;
  h ^= h >> 13;
  h *= 3266489917u;
  h ^= h >> 16;
  x[i] = (double)h * (2.0 / 4294967296.0) - 1.0;
}

__global__ void pack_sites(const double* __restrict__ pos, const double* __restrict__ alpha, int ns,
                           double4* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ns) out[i] = make_double4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], alpha[i]);
}

struct EventTimer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit EventTimer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  double ms() {
    float t = 0;
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&t, a, b);
    return t;
  }
  ~EventTimer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

void set_mesh_impl(Ctx* c, int64_t nv, const double* verts, int64_t nt, const int32_t* tris,
                   const int32_t* panel_system, const int32_t* panel_body, int where, cudaStream_t s,
                   bool stern = false) {
  if (nv < 4 || nt < 4 || !verts || !tris) fail(BEMPOL_ERR_ARG, "need nv >= 4, nt >= 4 and non-NULL arrays");
  if (nt >= (int64_t)1 << 24) fail(BEMPOL_ERR_ARG, "at most 16,777,215 triangles");
  if (nv >= (int64_t)1 << 31) fail(BEMPOL_ERR_ARG, "too many vertices");
  if (where != BEMPOL_HOST && where != BEMPOL_DEVICE) fail(BEMPOL_ERR_ARG, "bad `where`");
  c->have_mesh = false;
  c->have_sites = false;
  c->have_solution = false;
  c->tree_ready = false;
  c->stern = stern;
  c->n = (int)nt;
  c->nv = (int)nv;
  c->K = c->par.gauss_k;
  std::vector<int32_t> ht = to_host(tris, 3 * (size_t)nt, where, s);
  std::vector<int32_t> hs, hb;
  if (panel_system) hs = to_host(panel_system, (size_t)nt, where, s);
  if (panel_body) hb = to_host(panel_body, (size_t)nt, where, s);
  std::vector<int> grp = make_groups(*c, nt, hs, hb);
  size_scalars(*c);
  DBuf<double> dv;
  to_device(dv, verts, 3 * (size_t)nv, where, s);
  auto t = std::chrono::steady_clock::now();
  auto lap = [&](int k) {
    if (c->stats_on) BP_CUDA(cudaStreamSynchronize(s));
    const auto now = std::chrono::steady_clock::now();
    c->mesh_ms[k] = std::chrono::duration<double, std::milli>(now - t).count();
    t = now;
  };
  validate_closed(ht.data(), c->n, c->nv, grp);
  lap(0);
  build_geometry(*c, dv.p, ht.data(), grp, s);
  lap(1);
  build_blocks(*c, s);
  if (stern) {
    build_stern_blocks(*c, s);
    stern_check_nested(*c, s);
  }
  lap(2);
  build_tree(*c, s);  // the octree also narrows the near-pair search
  lap(3);
  build_near(*c, s);
  lap(4);
  size_t len = 2 * (size_t)c->n;
  c->vec_a.alloc(len);
  c->vec_b.alloc(len);
  c->vec_c.alloc(len);
  c->vec_d.alloc(len);
  c->gm_m = 0;  // GMRES workspace is sized per mesh
  c->have_mesh = true;
}

void set_sites_impl(Ctx* c, int64_t ns, const double* pos, const double* q, const double* d, const double* Q,
                    const double* alpha, const int32_t* group, const int32_t* site_system, const int32_t* site_body,
                    int where, cudaStream_t s) {
  if (!c->have_mesh) fail(BEMPOL_ERR_STATE, "set_mesh must come before set_sites");
  if (ns < 1 || ns > (1 << 24) || !pos || !q || !d || !Q || !alpha) fail(BEMPOL_ERR_ARG, "bad site arrays");
  if (where != BEMPOL_HOST && where != BEMPOL_DEVICE) fail(BEMPOL_ERR_ARG, "bad `where`");
  c->have_sites = false;
  c->have_solution = false;
  // group of every site; sites must come sorted by (system, body)
  std::vector<int32_t> hs, hb;
  if (site_system) hs = to_host(site_system, (size_t)ns, where, s);
  if (site_body) hb = to_host(site_body, (size_t)ns, where, s);
  std::vector<int> tag(ns);
  c->h_gsite.assign(c->ngroup + 1, 0);
  for (int64_t l = 0; l < ns; ++l) {
    const int a = hs.empty() ? 0 : hs[l], b = hb.empty() ? 0 : hb[l];
    int g = -1;
    for (int k = (a >= 0 && a < c->nsys) ? c->h_sys_grp[a] : 0; a >= 0 && a < c->nsys && k < c->h_sys_grp[a + 1]; ++k)
      if (c->h_grp_body[k] == b) g = k;
    if (g < 0)
      fail(BEMPOL_ERR_SITES, "site " + std::to_string(l) + ": its (system, body) has no surface");
    if (l > 0 && g < tag[l - 1])
      fail(BEMPOL_ERR_SITES, "sites must be ordered by system, then body (site " + std::to_string(l) + ")");
    if (c->stern && g != 0)
      fail(BEMPOL_ERR_SITES, "site " + std::to_string(l) + ": with a Stern layer every site lies inside body 0");
    tag[l] = g;
    ++c->h_gsite[g + 1];
  }
  for (int g = 0; g < c->ngroup; ++g) c->h_gsite[g + 1] += c->h_gsite[g];
  c->h_sys_site.assign(c->nsys + 1, 0);
  for (int k = 0; k <= c->nsys; ++k) c->h_sys_site[k] = c->h_gsite[c->h_sys_grp[k]];
  std::vector<int4> sblk;
  for (int g = 0; g < c->ngroup; ++g)
    for (int l = c->h_gsite[g]; l < c->h_gsite[g + 1]; l += 8)
      sblk.push_back(make_int4(l, std::min(8, c->h_gsite[g + 1] - l), g, 0));
  // host-side checks of the moments (small arrays)
  std::vector<double> hQ = to_host(Q, 9 * (size_t)ns, where, s);
  std::vector<double> ha = to_host(alpha, (size_t)ns, where, s);
  std::vector<double> Q6(6 * (size_t)ns);
  for (int64_t l = 0; l < ns; ++l) {
    const double* m = hQ.data() + 9 * l;
    double mx = 0;
    for (int k = 0; k < 9; ++k) mx = std::max(mx, std::fabs(m[k]));
    if (!std::isfinite(mx)) fail(BEMPOL_ERR_SITES, "site " + std::to_string(l) + " has a non-finite quadrupole");
    double asym = std::max(std::fabs(m[1] - m[3]), std::max(std::fabs(m[2] - m[6]), std::fabs(m[5] - m[7])));
    double tr = m[0] + m[4] + m[8];
    if (asym > 1e-9 * mx || std::fabs(tr) > 1e-9 * mx)
      fail(BEMPOL_ERR_SITES, "site " + std::to_string(l) + ": Q must be symmetric and traceless");
    double t3 = tr / 3.0;
    double* o = Q6.data() + 6 * l;
    o[0] = m[0] - t3;
    o[1] = m[1];
    o[2] = m[2];
    o[3] = m[4] - t3;
    o[4] = m[5];
    o[5] = m[8] - t3;
    if (!(ha[l] >= 0.0) || !std::isfinite(ha[l]))
      fail(BEMPOL_ERR_SITES, "site " + std::to_string(l) + ": alpha must be finite and >= 0");
  }
  c->ns = (int)ns;
  DBuf<double> dpos, dal;
  to_device(dpos, pos, 3 * (size_t)ns, where, s);
  to_device(dal, alpha, (size_t)ns, where, s);
  c->site_pos.alloc(ns);
  launch(pack_sites, cdiv(ns, 256), 256, 0, s, dpos.p, dal.p, (int)ns, c->site_pos.p);
  BP_CHECK_LAUNCH();
  to_device(c->site_q, q, (size_t)ns, where, s);
  to_device(c->site_d, d, 3 * (size_t)ns, where, s);
  to_device(c->site_Q, Q6.data(), 6 * (size_t)ns, BEMPOL_HOST, s);
  std::vector<int32_t> g(ns);
  if (group) {
    g = to_host(group, (size_t)ns, where, s);
  } else {
    for (int64_t l = 0; l < ns; ++l) g[l] = (int32_t)l;
  }
  to_device(c->site_group, g.data(), (size_t)ns, BEMPOL_HOST, s);
  to_device(c->stag, tag.data(), (size_t)ns, BEMPOL_HOST, s);
  to_device(c->gsite, c->h_gsite.data(), c->h_gsite.size(), BEMPOL_HOST, s);
  to_device(c->sys_site, c->h_sys_site.data(), c->h_sys_site.size(), BEMPOL_HOST, s);
  c->nsblk = (int)sblk.size();
  to_device(c->sblk, sblk.data(), sblk.size(), BEMPOL_HOST, s);
  c->stree.ready = false;
  site_validation(*c, s);
  BP_CUDA(cudaStreamSynchronize(s));
  c->have_sites = true;
}

}  // namespace
}  // namespace bp

using namespace bp;

extern "C" {

void bempol_default_params(bempol_params* p) {
  if (!p) return;
  p->eps_in = 1.0;
  p->eps_out = 80.0;
  p->kappa = 0.125;
  p->gauss_k = 4;
  p->near_factor = 2.0;
  p->theta = 0.5;
  p->order = 5;
  p->leaf = 256;
  p->gmres_tol = 1e-8;
  p->gmres_restart = 100;
  p->gmres_maxit = 500;
  p->scf_tol = 1e-8;
  p->sor_omega = 0.7;
  p->scf_maxit = 200;
  p->op = BEMPOL_OP_FP64_DIRECT;
  p->residual_op = BEMPOL_OP_FP64_DIRECT;
  p->inner_tol = 1e-3;
  p->refine_maxit = 20;
  p->thole_a = 0.39;
  p->refine_scope = BEMPOL_REFINE_EVERY;
  p->thole_perm = 0;
  p->near_rule = BEMPOL_NEAR_SEMI_ANALYTICAL;
}

bempol_status bempol_create(const bempol_params* p, int device, bempol_ctx** out) {
  if (!out) return BEMPOL_ERR_ARG;
  *out = nullptr;
  bempol_ctx* c = nullptr;
  try {
    check_params(p);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
      (void)cudaGetLastError();
      return BEMPOL_ERR_CUDA;
    }
    BP_CUDA(cudaSetDevice(device));
    c = new bempol_ctx();
    c->par = *p;
    c->device = device;
    init_near_rules();
    c->scal.alloc(16);
    c->dev_err.alloc(1);
    BP_CUDA(cudaMemset(c->dev_err.p, 0, sizeof(int)));
    BP_CUDA(cudaMallocHost(&c->h_pinned, 16 * sizeof(double)));
  } catch (const Error& e) {
    delete c;
    return e.st;
  }
  *out = c;
  return BEMPOL_OK;
}

bempol_status bempol_set_params(bempol_ctx* c, const bempol_params* p) {
  return guard(c, [&] {
    check_params(p);
    bool geo = p->gauss_k != c->par.gauss_k || p->near_factor != c->par.near_factor || p->kappa != c->par.kappa ||
               p->near_rule != c->par.near_rule;
    bool tree = p->leaf != c->par.leaf || p->theta != c->par.theta || geo;
    if (geo && c->have_mesh)
      fail(BEMPOL_ERR_STATE, "gauss_k, near_factor, near_rule and kappa are fixed once a mesh is set");
    c->par = *p;
    c->have_solution = false;
    if (tree) c->tree_ready = false;
  });
}

void bempol_destroy(bempol_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  delete c;
}

const char* bempol_last_error(const bempol_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

bempol_status bempol_set_mesh(bempol_ctx* c, int64_t nv, const double* verts, int64_t nt, const int32_t* tris,
                              int where, void* stream) {
  return guard(c, [&] { set_mesh_impl(c, nv, verts, nt, tris, nullptr, nullptr, where, (cudaStream_t)stream); });
}

bempol_status bempol_set_mesh_systems(bempol_ctx* c, int64_t nv, const double* verts, int64_t nt,
                                      const int32_t* tris, const int32_t* panel_system, const int32_t* panel_body,
                                      int where, void* stream) {
  return guard(c, [&] {
    set_mesh_impl(c, nv, verts, nt, tris, panel_system, panel_body, where, (cudaStream_t)stream);
  });
}

bempol_status bempol_set_mesh_stern(bempol_ctx* c, int64_t nv1, const double* verts1, int64_t nt1,
                                    const int32_t* tris1, int64_t nv2, const double* verts2, int64_t nt2,
                                    const int32_t* tris2, int where, void* stream) {
  return guard(c, [&] {
    if (where != BEMPOL_HOST) fail(BEMPOL_ERR_ARG, "the Stern-layer surfaces are read from host memory");
    if (nv1 < 4 || nt1 < 4 || nv2 < 4 || nt2 < 4 || !verts1 || !tris1 || !verts2 || !tris2)
      fail(BEMPOL_ERR_ARG, "need nv >= 4, nt >= 4 and non-NULL arrays for both surfaces");
    if (nv1 + nv2 >= (int64_t)1 << 31 || nt1 + nt2 >= (int64_t)1 << 24) fail(BEMPOL_ERR_ARG, "surfaces too large");
    // one mesh of two bodies: the dielectric boundary (body 0) and the ion-exclusion surface
    std::vector<double> v(3 * (size_t)(nv1 + nv2));
    std::copy(verts1, verts1 + 3 * nv1, v.begin());
    std::copy(verts2, verts2 + 3 * nv2, v.begin() + 3 * nv1);
    std::vector<int32_t> t(3 * (size_t)(nt1 + nt2)), body(nt1 + nt2, 0);
    std::copy(tris1, tris1 + 3 * nt1, t.begin());
    for (int64_t k = 0; k < 3 * nt2; ++k) {
      if (tris2[k] < 0 || tris2[k] >= nv2) fail(BEMPOL_ERR_MESH, "vertex index out of range in the second surface");
      t[3 * nt1 + k] = tris2[k] + (int32_t)nv1;
    }
    for (int64_t k = 0; k < 3 * nt1; ++k)
      if (tris1[k] < 0 || tris1[k] >= nv1) fail(BEMPOL_ERR_MESH, "vertex index out of range in the first surface");
    for (int64_t k = nt1; k < nt1 + nt2; ++k) body[k] = 1;
    set_mesh_impl(c, nv1 + nv2, v.data(), nt1 + nt2, t.data(), nullptr, body.data(), BEMPOL_HOST,
                  (cudaStream_t)stream, true);
  });
}

bempol_status bempol_set_sites(bempol_ctx* c, int64_t ns, const double* pos, const double* q, const double* d,
                               const double* Q, const double* alpha, const int32_t* group, int where,
                               void* stream) {
  return guard(c, [&] {
    if (c->ngroup != 1 && !c->stern)
      fail(BEMPOL_ERR_STATE, "the mesh has several bodies: use bempol_set_sites_systems");
    set_sites_impl(c, ns, pos, q, d, Q, alpha, group, nullptr, nullptr, where, (cudaStream_t)stream);
  });
}

bempol_status bempol_set_sites_systems(bempol_ctx* c, int64_t ns, const double* pos, const double* q,
                                       const double* d, const double* Q, const double* alpha, const int32_t* group,
                                       const int32_t* site_system, const int32_t* site_body, int where,
                                       void* stream) {
  return guard(c, [&] {
    set_sites_impl(c, ns, pos, q, d, Q, alpha, group, site_system, site_body, where, (cudaStream_t)stream);
  });
}

bempol_status bempol_systems(const bempol_ctx* cc, int64_t* n_systems, int64_t* n_bodies) {
  if (!cc) return BEMPOL_ERR_ARG;
  if (n_systems) *n_systems = cc->have_mesh ? cc->nsys : 0;
  if (n_bodies) *n_bodies = cc->have_mesh ? cc->ngroup : 0;
  return BEMPOL_OK;
}

bempol_status bempol_matvec(bempol_ctx* c, const double* x, double* y, int op, void* stream) {
  return guard(c, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->have_mesh) fail(BEMPOL_ERR_STATE, "no mesh");
    if (!x || !y || x == y) fail(BEMPOL_ERR_ARG, "x and y must be distinct device arrays");
    if (op < 0 || op > 3) fail(BEMPOL_ERR_ARG, "bad op");
    ensure_tree(*c, op, s);
    permute_to_internal(*c, x, c->vec_a.p, 2, s);
    matvec_internal(*c, c->vec_a.p, c->vec_b.p, op, s);
    permute_to_caller(*c, c->vec_b.p, y, 2, s);
  });
}

bempol_status bempol_matvec_transposed(bempol_ctx* c, const double* x, double* y, int op, void* stream) {
  return guard(c, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->have_mesh) fail(BEMPOL_ERR_STATE, "no mesh");
    if (!x || !y || x == y) fail(BEMPOL_ERR_ARG, "x and y must be distinct device arrays");
    if (op < 0 || op > 3) fail(BEMPOL_ERR_ARG, "bad op");
    ensure_tree(*c, op, s);
    permute_to_internal(*c, x, c->vec_a.p, 2, s);
    matvec_T_internal(*c, c->vec_a.p, c->vec_b.p, op, s);
    permute_to_caller(*c, c->vec_b.p, y, 2, s);
  });
}

bempol_status bempol_rhs(bempol_ctx* c, const double* p, double* b, int op, void* stream) {
  return guard(c, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->have_sites) fail(BEMPOL_ERR_STATE, "no sites");
    if (!b) fail(BEMPOL_ERR_ARG, "b is NULL");
    rhs_internal(*c, p, c->vec_a.p, op_fp32(op), s);
    permute_to_caller(*c, c->vec_a.p, b, 1, s);
  });
}

bempol_status bempol_site_reaction(bempol_ctx* c, const double* x, double* out, int op, void* stream) {
  return guard(c, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->have_sites) fail(BEMPOL_ERR_STATE, "no sites");
    if (!x || !out) fail(BEMPOL_ERR_ARG, "NULL array");
    permute_to_internal(*c, x, c->vec_a.p, 2, s);
    site_reaction_form(*c, c->vec_a.p, out, op, true, s);
  });
}

bempol_status bempol_multipole_field(bempol_ctx* c, const double* mu, int mode, double* out, void* stream) {
  return guard(c, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->have_sites) fail(BEMPOL_ERR_STATE, "no sites");
    if (!out || mode < 0 || mode > 3) fail(BEMPOL_ERR_ARG, "bad arguments");
    DBuf<double> zero;
    const double* m = mu;
    if (!m) {
      zero.alloc(3 * (size_t)c->ns);
      zero.zero(s);
      m = zero.p;
    }
    multipole_internal(*c, m, mode, out, s);
    if (!mu) BP_CUDA(cudaStreamSynchronize(s));
  });
}

bempol_status bempol_autotune(bempol_ctx* c, double target_err, bempol_tune_result* out, void* stream) {
  return guard(c, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->have_mesh) fail(BEMPOL_ERR_STATE, "no mesh");
    if (!(target_err > 0.0)) fail(BEMPOL_ERR_ARG, "target_err must be > 0");
    const int len = 2 * c->n;
    const bempol_params saved = c->par;
    DBuf<double> x, yref, y, d;
    x.alloc(len);
    yref.alloc(len);
    y.alloc(len);
    d.alloc(len);
    launch(hash_vector_kernel, cdiv(len, 256), 256, 0, s, x.p, len, 1810036980u);
    // reference: the FP32 direct product (every Gauss node, FP64 sums)
    matvec_internal(*c, x.p, yref.p, BEMPOL_OP_FP32_DIRECT, s);
    const double nref = std::sqrt(dot_dev(*c, yref.p, yref.p, len, s));
    const int leaves[] = {128, 192, 256, 384};
    const double thetas[] = {0.4, 0.5, 0.6};
    const int orders[] = {4, 5, 6};
    int best_leaf = saved.leaf, best_order = saved.order, tried = 0;
    double best_theta = saved.theta, best_ms = 1e300, best_err = -1.0;
    cudaEvent_t e0, e1;
    BP_CUDA(cudaEventCreate(&e0));
    BP_CUDA(cudaEventCreate(&e1));
    for (int lf : leaves)
      for (double th : thetas) {
        c->par.leaf = lf;
        c->par.theta = th;
        build_tree(*c, s);
        for (int P : orders) {
          c->par.order = P;
          matvec_internal(*c, x.p, y.p, BEMPOL_OP_FP32_TREE, s);  // warm (moment buffers)
          BP_CUDA(cudaEventRecord(e0, s));
          for (int r = 0; r < 3; ++r) matvec_internal(*c, x.p, y.p, BEMPOL_OP_FP32_TREE, s);
          BP_CUDA(cudaEventRecord(e1, s));
          BP_CUDA(cudaEventSynchronize(e1));
          float ms = 0;
          BP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          ms /= 3.0f;
          launch(add_vec_scaled, cdiv(len, 256), 256, 0, s, y.p, yref.p, -1.0, d.p, len);
          const double err = std::sqrt(dot_dev(*c, d.p, d.p, len, s)) / nref;
          ++tried;
          if (err <= target_err && ms < best_ms) {
            best_ms = ms;
            best_err = err;
            best_leaf = lf;
            best_theta = th;
            best_order = P;
          }
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->par = saved;
    if (best_err >= 0.0) {
      c->par.leaf = best_leaf;
      c->par.theta = best_theta;
      c->par.order = best_order;
    }
    build_tree(*c, s);
    c->have_solution = false;
    if (out) {
      out->leaf = c->par.leaf;
      out->theta = c->par.theta;
      out->order = c->par.order;
      out->matvec_ms = best_err >= 0.0 ? best_ms : -1.0;
      out->rel_err = best_err;
      out->candidates = tried;
    }
    if (best_err < 0.0) fail(BEMPOL_ERR_NOT_CONVERGED, "no candidate reached target_err; parameters unchanged");
  });
}

bempol_status bempol_sizes(const bempol_ctx* cc, int64_t* n_panels, int32_t* gauss_k, int64_t* n_sites,
                           int64_t* n_near, int64_t* n_cells, int64_t* n_leaves) {
  if (!cc) return BEMPOL_ERR_ARG;
  if (n_panels) *n_panels = cc->have_mesh ? cc->n : 0;
  if (gauss_k) *gauss_k = cc->K;
  if (n_sites) *n_sites = cc->have_sites ? cc->ns : 0;
  if (n_near) *n_near = cc->have_mesh ? cc->nnz : 0;
  if (n_cells) *n_cells = cc->tree_ready ? cc->tree.ncell : 0;
  if (n_leaves) *n_leaves = cc->tree_ready ? cc->tree.nleaf : 0;
  return BEMPOL_OK;
}

bempol_status bempol_shard_rows(int64_t n_units, const double* cost, int world, int64_t* bounds) {
  if (!bounds || n_units < 0 || world < 1) return BEMPOL_ERR_ARG;
  try {
    std::vector<double> v((size_t)n_units, 1.0);
    if (cost)
      for (int64_t i = 0; i < n_units; ++i) {
        if (!(cost[i] >= 0.0)) return BEMPOL_ERR_ARG;
        v[(size_t)i] = cost[i];
      }
    const std::vector<int64_t> b = shard_cuts(v, world);
    for (int r = 0; r <= world; ++r) bounds[r] = b[r];
    return BEMPOL_OK;
  } catch (...) {
    return BEMPOL_ERR_ARG;
  }
}

bempol_status bempol_set_shard(bempol_ctx* c, int rank, int world, double* exchange_buf, bempol_exchange_fn fn,
                               void* user) {
  return guard(c, [&] {
    if (!c->have_mesh) fail(BEMPOL_ERR_STATE, "bempol_set_shard needs a mesh");
    if (world < 1 || rank < 0 || rank >= world) fail(BEMPOL_ERR_ARG, "rank must be in [0, world)");
    if (world > 1 && (!fn || !exchange_buf)) fail(BEMPOL_ERR_ARG, "sharding needs an exchange buffer and callback");
    c->sh_rank = world > 1 ? rank : 0;
    c->sh_world = world;
    c->sh_buf = world > 1 ? exchange_buf : nullptr;
    c->sh_fn = world > 1 ? fn : nullptr;
    c->sh_user = world > 1 ? user : nullptr;
    c->sh_ready = false;
  });
}

bempol_status bempol_shard_bounds(bempol_ctx* c, int64_t* bounds) {
  return guard(c, [&] {
    if (!c->have_mesh) fail(BEMPOL_ERR_STATE, "no mesh");
    if (!bounds) fail(BEMPOL_ERR_ARG, "bounds is NULL");
    cudaStream_t s = 0;
    ensure_tree(*c, BEMPOL_OP_FP32_TREE, s);
    if (!c->sh_ready) build_shard(*c, s);
    for (int r = 0; r <= std::max(1, c->sh_world); ++r)
      bounds[r] = c->sh_world > 1 ? c->sh_bounds[r] : (r == 0 ? 0 : c->n);
  });
}

bempol_status bempol_stats_enable(bempol_ctx* c, int enable) {
  return guard(c, [&] { c->stats_on = enable != 0; });
}

bempol_status bempol_stats_read(bempol_ctx* c, bempol_stats* out, int reset) {
  return guard(c, [&] {
    if (!out) fail(BEMPOL_ERR_ARG, "out is NULL");
    BP_CUDA(cudaDeviceSynchronize());
    check_device_error(*c, 0);
    c->collect_timers();
    out->kernel_launches = g_launches.load() - c->launches_at_reset;
    out->pair_launches = c->stat_launches[0];
    out->pair_ms = c->stat_ms[0];
    out->far_launches = c->stat_launches[1];
    out->far_ms = c->stat_ms[1];
    out->pair_interactions = c->stat_pairs;
    out->far_evaluations = c->stat_far;
    out->tree_products = c->stat_launches[2];
    out->tree_ms = c->stat_ms[2];
    out->rhs_calls = c->stat_launches[3];
    out->rhs_ms = c->stat_ms[3];
    out->reaction_calls = c->stat_launches[4];
    out->reaction_ms = c->stat_ms[4];
    out->site_field_calls = c->stat_launches[5];
    out->site_field_ms = c->stat_ms[5];
    out->mesh_validate_ms = c->mesh_ms[0];
    out->mesh_geometry_ms = c->mesh_ms[1];
    out->mesh_blocks_ms = c->mesh_ms[2];
    out->mesh_tree_ms = c->mesh_ms[3];
    out->mesh_near_ms = c->mesh_ms[4];
    out->tree64_products = c->stat_launches[6];
    out->tree64_ms = c->stat_ms[6];
    if (reset) {
      c->launches_at_reset = g_launches.load();
      for (int k = 0; k < Ctx::NKIND; ++k) {
        c->stat_launches[k] = 0;
        c->stat_ms[k] = 0;
      }
      c->stat_pairs = c->stat_far = 0;
    }
  });
}

bempol_status bempol_get_geometry(bempol_ctx* c, double* centroid, double* normal, double* area,
                                  int64_t* near_ptr, int32_t* near_col, double* near_corr) {
  return guard(c, [&] {
    if (!c->have_mesh) fail(BEMPOL_ERR_STATE, "no mesh");
    const int n = c->n;
    cudaStream_t s = 0;
    std::vector<double4> t(n), nr(n);
    std::vector<int> perm(n), ptr(n + 1), col(c->nnz);
    std::vector<double4> corr(c->nnz);
    BP_CUDA(cudaMemcpy(t.data(), c->tgt64.p, sizeof(double4) * n, cudaMemcpyDeviceToHost));
    BP_CUDA(cudaMemcpy(nr.data(), c->nrm64.p, sizeof(double4) * n, cudaMemcpyDeviceToHost));
    BP_CUDA(cudaMemcpy(perm.data(), c->perm.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
    BP_CUDA(cudaMemcpy(ptr.data(), c->near_ptr.p, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
    if (c->nnz) {
      BP_CUDA(cudaMemcpy(col.data(), c->near_col.p, sizeof(int) * c->nnz, cudaMemcpyDeviceToHost));
      BP_CUDA(cudaMemcpy(corr.data(), c->near_corr.p, sizeof(double4) * c->nnz, cudaMemcpyDeviceToHost));
    }
    (void)s;
    for (int i = 0; i < n; ++i) {
      int p = perm[i];
      if (centroid) {
        centroid[3 * p] = t[i].x;
        centroid[3 * p + 1] = t[i].y;
        centroid[3 * p + 2] = t[i].z;
      }
      if (area) area[p] = t[i].w;
      if (normal) {
        normal[3 * p] = nr[i].x;
        normal[3 * p + 1] = nr[i].y;
        normal[3 * p + 2] = nr[i].z;
      }
    }
    if (near_ptr || near_col || near_corr) {
      // rows in caller order, columns as caller indices ascending
      std::vector<int64_t> cptr(n + 1, 0);
      for (int i = 0; i < n; ++i) cptr[perm[i] + 1] = ptr[i + 1] - ptr[i];
      for (int i = 0; i < n; ++i) cptr[i + 1] += cptr[i];
      if (near_ptr)
        for (int i = 0; i <= n; ++i) near_ptr[i] = cptr[i];
      std::vector<std::pair<int, int>> row;
      for (int i = 0; i < n; ++i) {
        int p = perm[i];
        row.clear();
        for (int e = ptr[i]; e < ptr[i + 1]; ++e) row.push_back({perm[col[e]], e});
        std::sort(row.begin(), row.end());
        int64_t o = cptr[p];
        for (auto& r : row) {
          if (near_col) near_col[o] = r.first;
          if (near_corr) {
            double4 v = corr[r.second];
            near_corr[4 * o] = v.x;
            near_corr[4 * o + 1] = v.y;
            near_corr[4 * o + 2] = v.z;
            near_corr[4 * o + 3] = v.w;
          }
          ++o;
        }
      }
    }
  });
}

bempol_status bempol_solve_systems(bempol_ctx* c, void* stream, bempol_result* out, bempol_system_result* per,
                                   int64_t n_per) {
  return guard(c, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->have_sites) fail(BEMPOL_ERR_STATE, "set_mesh and set_sites must come first");
    if (!out) fail(BEMPOL_ERR_ARG, "out is NULL");
    if (per && n_per < c->nsys) fail(BEMPOL_ERR_ARG, "per-system result array is shorter than the number of systems");
    auto wall0 = std::chrono::steady_clock::now();
    EventTimer tt(s);
    const bempol_params& P = c->par;
    const int n = c->n, ns = c->ns, len = 2 * n, S = c->nsys;
    ensure_tree(*c, P.op, s);
    ensure_tree(*c, P.residual_op, s);
    // Precision of the site-side sums (right-hand sides, reaction and multipole fields):
    // that of residual_op throughout, or, when only the final solve is refined, that of
    // op inside the induced-dipole iterations and of residual_op for the final solve and
    // the energy (f32_final).
    const bool refining = P.residual_op != P.op;
    const bool final_only = refining && P.refine_scope == BEMPOL_REFINE_FINAL;
    const bool f32_final = op_fp32(P.residual_op);
    const bool f32 = final_only ? op_fp32(P.op) : f32_final;
    // operator form of the reaction field inside the induced-dipole iterations (tree or
    // direct, FP32 or FP64): that of the solves' precision, as for the other site sums
    const int scf_form = final_only ? P.op : P.residual_op;
    DBuf<double>& mu = c->sol_mu;
    DBuf<double>& mu_v = c->sol_mu_v;
    DBuf<double>& x = c->sol_x;
    DBuf<double> emult, react, mult10, p, b;
    DBuf<int> d_act;
    c->have_solution = false;
    mu.alloc(3 * ns);
    mu_v.alloc(3 * ns);
    emult.alloc(3 * ns);
    react.alloc(10 * ns);
    mult10.alloc(10 * ns);
    p.alloc(3 * ns);
    b.alloc(len);
    x.alloc(len);
    d_act.alloc(S);
    mu.zero(s);
    mu_v.zero(s);
    x.zero(s);
    b.zero(s);
    double t_setup = tt.ms();
    EventTimer ts(s);
    int gm_iters = 0, matvecs = 0, res_matvecs = 0, solves = 0;
    std::vector<int> it_d(S, 0), it_v(S, 0), sys_gm(S, 0), sys_solves(S, 0);
    std::vector<double> sys_res(S, 0.0);
    std::vector<char> conv_v(S, 0), conv_d(S, 0), gm_ok(S, 1), diverged(S, 0);
    // Divergence guard (per system): the relaxed update converges only when every
    // eigenvalue of 4 pi alpha T (plus the reaction coupling) exceeds 1 - 2/omega.
    // A change that is not finite, or that has grown 8 times in a row to more than
    // 10x its smallest value, stops that system with an error (stagnation at the
    // operator's noise level instead runs to scf_maxit).
    struct Guard {
      double best = 1e300, prev = 1e300;
      int grow = 0;
      bool diverges(double rms) {
        if (!std::isfinite(rms)) return true;
        grow = (rms > prev) ? grow + 1 : 0;
        prev = rms;
        best = std::min(best, rms);
        return grow >= 8 && rms > 10.0 * best;
      }
    };
    auto upload_act = [&](const std::vector<int>& act) {
      int* hp = reinterpret_cast<int*>(c->h_pinned + 2 * S);
      std::copy(act.begin(), act.end(), hp);
      BP_CUDA(cudaMemcpyAsync(d_act.p, hp, sizeof(int) * S, cudaMemcpyHostToDevice, s));
      BP_CUDA(cudaStreamSynchronize(s));
    };
    // vacuum state: multipoles only, every site of a system interacting
    {
      std::vector<int> act(S, 1);
      std::vector<Guard> gv(S);
      for (int it = 1; it <= P.scf_maxit; ++it) {
        upload_act(act);
        Ctx::Timed tv;
        c->time_begin(5, s, tv);
        multipole_internal(*c, mu_v.p, 2, emult.p, s, f32);
        c->time_end(s, tv);
        std::vector<double> rms = sor_update(*c, mu_v.p, nullptr, emult.p, true, d_act.p, s);
        int left = 0;
        for (int q = 0; q < S; ++q) {
          if (!act[q]) continue;
          it_v[q] = it;
          if (rms[q] < P.scf_tol) {
            conv_v[q] = 1;
            act[q] = 0;
          } else if (gv[q].diverges(rms[q])) {
            diverged[q] = 1;
            act[q] = 0;
          } else {
            ++left;
          }
        }
        if (!left) break;
      }
    }
    std::vector<char> want(S, 1);
    auto bem = [&](const std::vector<char>& which, bool final) {
      launch(add_vec, cdiv(3 * ns, 256), 256, 0, s, c->site_d.p, mu.p, p.p, 3 * ns);
      Ctx::Timed tr;
      c->time_begin(3, s, tr);
      rhs_internal(*c, p.p, b.p, final ? f32_final : f32, s);
      c->time_end(s, tr);
      // under REFINE_FINAL the iteration's solves are plain GMRES with op, which for an
      // FP32 form cannot go below FP32_SOLVE_FLOOR; the final solve is refined to gmres_tol
      const double tol = (final_only && !final && op_fp32(P.op)) ? std::max(P.gmres_tol, FP32_SOLVE_FLOOR)
                                                                 : P.gmres_tol;
      GmresOut g = solve_bem(*c, b.p, x.p, which, s, refining && (final || !final_only), tol);
      gm_iters += g.iters;
      matvecs += g.matvecs;
      res_matvecs += g.residual_matvecs;
      ++solves;
      for (int q = 0; q < S; ++q) {
        if (!which[q]) continue;
        sys_gm[q] += g.sys_iters[q];
        ++sys_solves[q];
        sys_res[q] = g.sys_res[q];
        if (!g.sys_conv[q]) gm_ok[q] = 0;
      }
    };
    {
      std::vector<int> act(S, 1);
      std::vector<Guard> gd(S);
      for (int q = 0; q < S; ++q)
        if (diverged[q]) act[q] = 0;
      for (int it = 1; it <= P.scf_maxit; ++it) {
        for (int q = 0; q < S; ++q) want[q] = (char)act[q];
        bem(want, false);
        Ctx::Timed tx, tm;
        c->time_begin(4, s, tx);
        site_reaction_form(*c, x.p, react.p, scf_form, false, s);
        c->time_end(s, tx);
        c->time_begin(5, s, tm);
        multipole_internal(*c, mu.p, 0, emult.p, s, f32);
        c->time_end(s, tm);
        upload_act(act);
        std::vector<double> rms = sor_update(*c, mu.p, react.p, emult.p, false, d_act.p, s);
        int left = 0;
        for (int q = 0; q < S; ++q) {
          if (!act[q]) continue;
          it_d[q] = it;
          if (rms[q] < P.scf_tol) {
            conv_d[q] = 1;
            act[q] = 0;
          } else if (gd[q].diverges(rms[q])) {
            diverged[q] = 1;
            act[q] = 0;
          } else {
            ++left;
          }
        }
        if (!left) break;
      }
    }
    std::fill(want.begin(), want.end(), 1);
    bem(want, true);
    site_reaction_form(*c, x.p, react.p, P.residual_op, true, s);
    multipole_internal(*c, mu.p, 1, mult10.p, s, f32_final);
    std::vector<double> Gd = energy_internal(*c, react.p, mult10.p, s);
    multipole_internal(*c, mu_v.p, 3, mult10.p, s, f32_final);
    std::vector<double> Gv = energy_internal(*c, nullptr, mult10.p, s);
    double t_scf = ts.ms();
    bool ok = true;
    double Gd_sum = 0.0, Gv_sum = 0.0, res_max = 0.0;
    int itd_max = 0, itv_max = 0;
    for (int q = 0; q < S; ++q) {
      const bool sys_ok = conv_v[q] && conv_d[q] && gm_ok[q] && !diverged[q];
      ok = ok && sys_ok;
      Gd_sum += Gd[q];
      Gv_sum += Gv[q];
      res_max = std::max(res_max, sys_res[q]);
      itd_max = std::max(itd_max, it_d[q]);
      itv_max = std::max(itv_max, it_v[q]);
      if (per) {
        bempol_system_result& r = per[q];
        r.dG_solv_kcal = (Gd[q] - Gv[q]) * KCAL_PER_UNIT;
        r.G_diss = Gd[q];
        r.G_vac = Gv[q];
        r.scf_iters_diss = it_d[q];
        r.scf_iters_vac = it_v[q];
        r.gmres_iters = sys_gm[q];
        r.n_solves = sys_solves[q];
        r.last_rel_residual = sys_res[q];
        r.converged = sys_ok ? 1 : 0;
        r.n_panels = c->h_sys_pan[q + 1] - c->h_sys_pan[q];
        r.n_sites = c->h_sys_site[q + 1] - c->h_sys_site[q];
      }
    }
    out->G_diss = Gd_sum;
    out->G_vac = Gv_sum;
    out->dG_solv_kcal = (Gd_sum - Gv_sum) * KCAL_PER_UNIT;
    out->scf_iters_diss = itd_max;
    out->scf_iters_vac = itv_max;
    out->gmres_iters_total = gm_iters;
    out->matvecs_total = matvecs;
    out->residual_matvecs = res_matvecs;
    out->n_solves = solves;
    out->last_rel_residual = res_max;
    out->t_setup_ms = t_setup;
    out->t_scf_ms = t_scf;
    // optional arrays
    auto put = [&](double* dst, const double* src_dev, size_t count) {
      if (!dst) return;
      BP_CUDA(cudaMemcpyAsync(dst, src_dev, count * sizeof(double),
                              out->where == BEMPOL_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    };
    if (out->phi || out->dphidn) {
      permute_to_caller(*c, x.p, c->vec_d.p, 2, s);
      put(out->phi, c->vec_d.p, n);
      put(out->dphidn, c->vec_d.p + n, n);
    }
    put(out->site_reaction, react.p, 10 * (size_t)ns);
    put(out->mu_diss, mu.p, 3 * (size_t)ns);
    put(out->mu_vac, mu_v.p, 3 * (size_t)ns);
    BP_CUDA(cudaStreamSynchronize(s));
    check_device_error(*c, s);
    c->have_solution = true;
    out->t_total_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - wall0).count();
    for (int q = 0; q < S; ++q)
      if (diverged[q])
        fail(BEMPOL_ERR_NOT_CONVERGED,
             "induced-dipole iteration diverges in system " + std::to_string(q) +
                 " (RMS change grows); sor_omega is outside the convergence range of this polarizability coupling");
    if (!ok) fail(BEMPOL_ERR_NOT_CONVERGED, "GMRES or SCF reached its iteration limit");
  });
}

bempol_status bempol_solve(bempol_ctx* c, void* stream, bempol_result* out) {
  return bempol_solve_systems(c, stream, out, nullptr, 0);
}

bempol_status bempol_gradient(bempol_ctx* c, void* stream, double* grad_q, double* grad_d, double* grad_Q,
                              double* grad_pos, bempol_gradient_info* info, int units) {
  return guard(c, [&] {
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->have_sites || !c->have_solution) fail(BEMPOL_ERR_STATE, "bempol_gradient needs a completed solve");
    if (units != BEMPOL_UNITS_PAPER && units != BEMPOL_UNITS_KCAL) fail(BEMPOL_ERR_ARG, "bad units");
    if (c->par.thole_perm)
      fail(BEMPOL_ERR_ARG, "the adjoint gradient does not differentiate damped permanent fields (thole_perm = 1)");
    if (c->stern) fail(BEMPOL_ERR_ARG, "the adjoint gradient does not cover the Stern-layer system");
    EventTimer t(s);
    AdjointOut ao = gradient_internal(*c, grad_q, grad_d, grad_Q, grad_pos, s);
    if (units == BEMPOL_UNITS_KCAL) {
      const size_t ns = (size_t)c->ns;
      const std::pair<double*, size_t> outs[4] = {{grad_q, ns}, {grad_d, 3 * ns}, {grad_Q, 9 * ns}, {grad_pos, 3 * ns}};
      for (const auto& o : outs)
        if (o.first) launch(scale_kernel, cdiv((long long)o.second, 256), 256, 0, s, o.first, KCAL_PER_UNIT, (int)o.second);
      BP_CHECK_LAUNCH();
      BP_CUDA(cudaStreamSynchronize(s));
    }
    check_device_error(*c, s);
    const double ms = t.ms();
    if (info) {
      info->scf_iters_diss = ao.iters_diss;
      info->scf_iters_vac = ao.iters_vac;
      info->gmres_iters_total = ao.gmres_iters;
      info->n_solves = ao.solves;
      info->converged = ao.converged ? 1 : 0;
      info->t_ms = ms;
    }
    if (!ao.converged) fail(BEMPOL_ERR_NOT_CONVERGED, "the adjoint GMRES or SCF reached its iteration limit");
  });
}

}  // extern "C"
