// Internal declarations of the bempol library (not part of the ABI).
//
// Internal order: panels are sorted by group (a group is one body of one system,
// groups numbered in (system, body) order), then by the Morton code of their
// centroid within the group's bounding box (perm[i] = caller index of internal
// panel i).  So every group, and every system, owns a contiguous range of
// internal panels.  Gauss node g of internal panel j is source K*j + g.  Every
// device array below is in internal order.
//
// Coupling rules (Sec. "Calculation of the binding energy"): the Laplace layers
// and the multipole right-hand side of a body involve only that body's panels
// and sites; the Yukawa layers couple every panel of a system; different systems
// never interact.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <new>
#include <string>
#include <vector>

#include "../../include/bempol.h"

namespace bp {

// ---------------------------------------------------------------- errors
struct Error {
  bempol_status st;
  std::string msg;
};

#define BP_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::bp::Error{BEMPOL_ERR_CUDA, std::string(#call " failed: ") + cudaGetErrorString(e_)}; \
  } while (0)

#define BP_CHECK_LAUNCH() BP_CUDA(cudaGetLastError())

inline void fail(bempol_status st, const std::string& m) { throw Error{st, m}; }

// Every kernel of the library is launched through launch(): it counts launches
// (reported by bempol_stats_read) and checks the launch status.
void note_launch();
template <typename... KArgs, typename... Args>
inline void launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                   Args&&... args) {
  if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
  kernel<<<grid, block, smem, s>>>(static_cast<KArgs>(args)...);
  note_launch();
}

// ---------------------------------------------------------------- device buffer
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    if (count == n && p) return;
    release();
    if (count == 0) return;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      (void)cudaGetLastError();
      fail(e == cudaErrorMemoryAllocation ? BEMPOL_ERR_OOM : BEMPOL_ERR_CUDA,
           std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed: " +
               cudaGetErrorString(e));
    }
    n = count;
  }
  void zero(cudaStream_t s) {
    if (p) BP_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
};

// ---------------------------------------------------------------- tree
// Octree over the Morton-ordered panels.  Cells are stored in breadth-first
// order; cells of tree depth d are [h_depth_begin[d], h_depth_begin[d+1]).
// A cell owns the contiguous panel range [begin, end) and its Gauss nodes
// [K*begin, K*end).  Leaves are the target batches of the treecode.
struct Tree {
  int ncell = 0, nleaf = 0, ndepth = 0;
  std::vector<int> h_begin, h_end, h_child0, h_nchild;   // host topology
  std::vector<int> h_depth_begin;
  std::vector<int> h_leaf_cell;                          // leaf number -> cell
  std::vector<double4> h_center;                         // copy of `center`
  DBuf<int> begin, end, child0, nchild;
  DBuf<double4> center;                                  // x, y, z of the node bounding-box centre; w = radius
  DBuf<int> leaf_cell;                                   // leaf number -> cell
  DBuf<int> leaf_sys;                                    // leaf number -> system
  // group of each cell (-1 for the root when it holds several groups)
  std::vector<int> h_cell_grp;
  // interaction lists per leaf (CSR): accepted far cells (every body of the leaf's
  // system; far_lap flags those of the leaf's own body, the only ones with Laplace
  // terms) and near (direct) leaves; a near entry with bit 30 set is a leaf of another
  // body (Yukawa terms only)
  DBuf<int> far_ptr, far_list, near_ptr, near_list;
  bool farL_same = true;  // one group: every far cell carries Laplace terms
  // target blocks: (leaf number, first panel, count <= 128) for the far field,
  // (leaf number, first panel, count <= 32) for the FP64 near field and the transposed
  // kernels, and (leaf number, first panel, count <= 16) for the FP32 near field;
  // near_splits / near_splits16: pieces of each near list (grid y) of the 32- and
  // 16-target near kernels
  int nblk = 0, nblk32 = 0, nblk16 = 0, nblk16f = 0, near_splits = 1, near_splits16 = 1;
  DBuf<int4> blk, blk32, blk16;
  DBuf<int4> blk16f;  // the 16-target blocks in the order of the forward far field (most far work first)
  // interaction lists of the 16-target batches of the forward product (batch id = .w of
  // blk16 / blk16f; acceptance against each batch's own bounding sphere): far cells
  // (bfar_lap flags those with Laplace terms) and near leaves, CSR by batch id
  DBuf<int> bfar_ptr, bfar_list, bnear_ptr, bnear_list;
  DBuf<int> bfar_lap;  // per bfar_list entry: 1 if the cell is in the batch's own body (several bodies only)
  DBuf<int> far_lap;   // per far_list entry: 1 if the cell is in the leaf's own body (several bodies only)
  // host copies: the batches (leaf, first, count, id) in id order with their cost (near
  // pairs + far terms weighted by their flops), and the two launch orders
  std::vector<int4> h_batch, h_blk16, h_blk16f;
  std::vector<double> h_batch_cost;
  std::vector<long long> h_batch_pairs, h_batch_far;
  bool bfarL_same = true;
  int bm2m_min_depth = 0;
  long long bpairs_per_matvec = 0, bfar_per_matvec = 0;
  // multipole moments [ncell][2][NC]: single layer M_k, double layer D_k
  DBuf<float> mom32;
  DBuf<double> mom64;
  int mom_order = -1;
  // far-field coefficients of the cells, [ncell][NB][2] pairs (single, double layer),
  // formed from the moments in every product, and the table of their terms (entry ->
  // moment index and constant, CSR) for the product's order; the same for the
  // transposed product (pairs: Laplace, Yukawa charges)
  struct BTab {
    int order = -1;
    DBuf<int> ptr, k;
    DBuf<double> c;
  };
  DBuf<float> bco32, bcoT32;
  DBuf<double> bco64, bcoT64;
  BTab btab, btabT;
  // FP32 Gauss-node positions relative to the centre of their own leaf (x, y, z, 0),
  // and the same for the collocation points
  DBuf<float4> src_rel32, cen_rel32;
  // Gauss nodes of every leaf in pairs for the FP32 near field (a leaf with an odd count
  // ends with a padding node): leaf l owns pairs [pair_ptr[l], pair_ptr[l+1]); pair_src[p]
  // is the pair's first node (~node when the second is padding); positions relative to the
  // leaf centre PA = (x0, x1, y0, y1), PB = (z0, z1, 0, 0) and strengths SA = (m0, m1,
  // d0x, d1x), SB = (d0y, d1y, d0z, d1z) side by side
  int npair = 0;
  DBuf<int> pair_ptr, pair_src;
  DBuf<float4> pairPA, pairPB, pairSA, pairSB;
  // charge moments of the transposed product (Laplace, Yukawa)
  DBuf<float> momT32[2];
  DBuf<double> momT64[2];
  DBuf<float4> chgT32[2];   // charges (u, 0, 0, 0) at the collocation points, Laplace / Yukawa
  DBuf<double4> chgT64[2];
  int m2m_min_depth = 0;  // shallowest depth whose cells appear in a far list

  double theta_built = -1.0;
  long long pairs_per_matvec = 0, far_per_matvec = 0, farL_per_matvec = 0;
};

constexpr int NEAR_CROSS = 1 << 30;  // near-list flag: source leaf of another body

// Treecode evaluation of the reaction field at the sites: batches of <= 16 sites of one
// body in Morton order (bat: first position in perm, count, group, 0; bcen: centre and
// radius), their accepted cells and near leaves (CSR by batch), and the combined
// moments W = M - D of the cells.  Rebuilt after set_sites or a new tree.
struct SiteTree {
  bool ready = false;
  int nbat = 0, min_depth = 0;
  long long far_evals = 0, pairs = 0;  // (site, cell) terms and (site, node) pairs per evaluation
  DBuf<int4> bat;
  DBuf<double4> bcen;
  DBuf<int> perm, far_ptr, far_list, near_ptr, near_list;
  DBuf<float> w32;
  DBuf<double> w64;
};

// ---------------------------------------------------------------- context
struct Ctx {
  bempol_params par;
  int device = 0;
  std::string err;

  // geometry
  int n = 0;                 // panels
  int K = 0;                 // Gauss nodes per panel
  int nv = 0;
  bool have_mesh = false;
  DBuf<int> perm, iperm;     // internal -> caller, caller -> internal
  DBuf<double> vert9;        // [n][9] triangle vertices (internal order)
  DBuf<double4> tgt64;       // centroid x,y,z, area
  DBuf<float4> tgt32;        // centroid x,y,z, 0
  DBuf<double4> nrm64;       // unit normal, 0
  // target blocks of the direct kernels: (first target, count <= 128, group, 0), and
  // each block's source ranges (Yukawa begin, end, Laplace begin, end) in Gauss nodes
  int ndblk = 0;
  DBuf<int4> dblk, dblk_rng;
  DBuf<double4> blk_center;  // FP64 centre of each direct block's targets
  DBuf<double4> src64;       // Gauss node x,y,z, weight w_g*A_j   [n*K]
  DBuf<float4> src32;
  DBuf<double4> str64;       // per-matvec strengths m, d (x,y,z)  [n*K]
  DBuf<float4> str32;
  DBuf<int> near_ptr;        // [n+1]
  DBuf<int> near_col;        // [nnz]
  DBuf<double4> near_corr;   // [nnz] VL, KL, VY, KY corrections (Stern layer: a pair across the
                             // two surfaces holds VL, KL, 0, 0)
  int64_t nnz = 0;
  // the near table by columns: for panel j, entries [near_ptrT[j], near_ptrT[j+1])
  // hold (row i, index into near_corr) of every near pair (i, j)
  DBuf<int> near_ptrT, near_rowT, near_eT;
  bool nearT_ready = false;  // the three above match the current near table
  double bbox_lo[3], bbox_hi[3];
  double max_area = 0.0;     // largest panel area (near-field search radius)
  std::vector<unsigned> h_morton;  // 30-bit Morton code of each internal panel (sorted)
  Tree tree;
  bool tree_ready = false;
  SiteTree stree;

  // Stern (ion-exclusion) layer: group 0 is the dielectric boundary, group 1 the surface
  // where the ions begin; the direct blocks' source ranges over their own surface (A) and
  // over the other one (B), and the second pass's partial sums
  bool stern = false;
  DBuf<int4> stern_rngA, stern_rngB;
  DBuf<double> stern_part;
  int stern_splits = 0;

  // groups (bodies) and systems
  int ngroup = 1, nsys = 1;
  std::vector<int> h_grp_sys, h_grp_body;  // [G] system and caller body id of each group
  std::vector<int> h_gpan, h_sys_pan;      // [G+1], [S+1] internal panel ranges
  std::vector<int> h_sys_grp;              // [S+1] group ranges of the systems
  DBuf<int> ptag;                          // [n] group of each internal panel
  DBuf<int> psys;                          // [n] system of each internal panel
  DBuf<int> gpan, sys_pan, grp_sys;        // device copies
  std::vector<int> h_gsite, h_sys_site;    // [G+1], [S+1] site ranges (sites are sorted by group)
  DBuf<int> gsite, sys_site, stag;         // device copies; stag [ns] group of each site
  int nsblk = 0;
  DBuf<int4> sblk;                         // site blocks (first site, count <= 8, group, 0)
  // GMRES segmentation: chunks (system, begin, end, 0) of the [2n] vectors, each
  // inside one system and one half; chunks of system s are [chunk_ptr[s], chunk_ptr[s+1])
  int nchunk = 0;
  DBuf<int4> chunks;
  DBuf<int> chunk_ptr;

  // sites
  int ns = 0;
  bool have_sites = false;
  DBuf<double4> site_pos;    // x, y, z, alpha
  DBuf<double> site_q;       // [ns]
  DBuf<double> site_d;       // [ns*3]
  DBuf<double> site_Q;       // [ns*6] xx xy xz yy yz zz
  DBuf<int> site_group;      // [ns]

  // matvec / solver workspaces
  DBuf<double> part;         // P2P partial sums [S][4][n]
  int part_splits = 0;
  DBuf<double> site_part;    // site partial sums
  DBuf<double> gm_V, gm_H, gm_small, gm_dots;
  DBuf<int> gm_flags;        // [S] active flags and [S] Krylov sizes
  // Device flags [S] of the systems a matrix-vector product must compute (set by the
  // GMRES driver around its products; NULL = every system).  Rows of the other
  // systems are left unspecified.
  const int* mv_active = nullptr;
  // matrix-vector products apply A^T instead of A (set by the adjoint driver around
  // its solves)
  bool transposed = false;
  // state of the last solve, kept for the adjoint: surface solution (internal
  // order) and the dissolved and vacuum induced dipoles
  bool have_solution = false;
  DBuf<double> sol_x, sol_mu, sol_mu_v;
  DBuf<unsigned> gm_ticket;  // last-block ticket of the multi-dot kernel (kept at 0 between calls)
  DBuf<double> gm_tol;       // [S] absolute GMRES tolerances of the current solve (device copy)
  cudaEvent_t gm_ev[2] = {nullptr, nullptr};  // residual copies of alternate GMRES iterations
  DBuf<double> vec_a, vec_b, vec_c, vec_d;   // [2n] scratch vectors
  DBuf<double> scal;         // device scalars
  // set by a kernel whose bounded device-side wait ran out (read and cleared by the
  // synchronising entry points, which then return BEMPOL_ERR_TIMEOUT)
  DBuf<int> dev_err;
  double* h_pinned = nullptr;  // pinned host scalars
  int gm_m = 0;

  // target sharding: this rank computes the treecode rows [sh_bounds[rank],
  // sh_bounds[rank+1]) (internal order) with the block tables below, then sh_fn
  // exchanges the rest through the caller's buffer sh_buf [2n]
  int sh_rank = 0, sh_world = 1;
  std::vector<int64_t> sh_bounds;
  double* sh_buf = nullptr;
  bempol_exchange_fn sh_fn = nullptr;
  void* sh_user = nullptr;
  int sh_nblk16 = 0, sh_nblk16f = 0;
  DBuf<int4> sh_blk16, sh_blk16f;
  long long sh_pairs = 0, sh_far = 0;  // this rank's near pairs and far terms per product
  bool sh_ready = false;  // tables match the current tree
  // side stream (highest priority) of a treecode product: the moments, M2M shifts and
  // far-field kernels run on it while the near-field kernel runs on the caller's
  // stream; fork and join events order the two.  Created with the tree.
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  void ensure_aux();

  // optional CUDA-event timing of the pair (direct / near-field) and far-field kernels,
  // of whole treecode products (fork to join) and of the solve's other phases
  bool stats_on = false;
  struct Timed {
    cudaEvent_t a, b;
    int kind;  // 0 pair kernel, 1 far-field kernels, 2 FP32 treecode product, 3 right-hand side,
               // 4 reaction field at the sites, 5 multipole fields at the sites,
               // 6 FP64 treecode product
  };
  static constexpr int NKIND = 7;
  // host wall-clock of the phases of the last set_mesh (validation, geometry and Morton
  // order, block tables, tree, near table); the stream is synchronised at each phase
  // boundary only while stats are on
  double mesh_ms[5] = {};
  std::vector<Timed> timed;
  double stat_ms[NKIND] = {};
  long long stat_launches[NKIND] = {};
  long long stat_pairs = 0, stat_far = 0;
  long long stat_site_pairs = 0, stat_site_far = 0;  // treecode reaction-field terms at the sites
  long long launches_at_reset = 0;
  void time_begin(int kind, cudaStream_t s, Timed& t);
  void time_end(cudaStream_t s, Timed& t);
  void collect_timers();
  // accounting state, to drop the records of a product that turned out to have no
  // active system (its launches still count in kernel_launches)
  struct StatMark {
    size_t ntimed;
    long long launches[NKIND], pairs, far;
  };
  StatMark stat_mark() const {
    StatMark m{timed.size(), {}, stat_pairs, stat_far};
    for (int k = 0; k < NKIND; ++k) m.launches[k] = stat_launches[k];
    return m;
  }
  void stat_rewind(const StatMark& m);

  Ctx() = default;
  ~Ctx();
};

// Body of every C entry point taking a context: makes the context's device current,
// runs f, and turns exceptions into a status plus the context's message (nothing
// escapes an extern "C" function).
template <typename F>
bempol_status guard(Ctx* c, F&& f) {
  if (!c) return BEMPOL_ERR_ARG;
  try {
    if (cudaSetDevice(c->device) != cudaSuccess) fail(BEMPOL_ERR_CUDA, "cudaSetDevice failed");
    c->mv_active = nullptr;  // products outside a solve compute every system
    f();
    c->err.clear();
    return BEMPOL_OK;
  } catch (const Error& e) {
    c->err = e.msg;
    return e.st;
  } catch (const std::bad_alloc&) {
    c->err = "host allocation failed";
    return BEMPOL_ERR_OOM;
  } catch (const std::exception& e) {
    c->err = e.what();
    return BEMPOL_ERR_ARG;
  }
}

// BEMPOL_ERR_TIMEOUT if a kernel's bounded wait ran out since the last check (clears the
// flag; synchronises s)
void check_device_error(Ctx& c, cudaStream_t s);

// ---------------------------------------------------------------- launch helpers
inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }
int num_sms(int device);

// geometry.cu
// closed, consistently oriented surfaces, no edge shared by two bodies (fails with BEMPOL_ERR_MESH)
void validate_closed(const int* tris, int n, int nv, const std::vector<int>& grp);
void build_geometry(Ctx& c, const double* d_verts, const int* h_tris, const std::vector<int>& h_group,
                    cudaStream_t s);
void build_blocks(Ctx& c, cudaStream_t s);
// near.cu
void build_near(Ctx& c, cudaStream_t s);
void init_near_rules();  // Gauss-Legendre nodes and the 19-node triangle rule (constant memory)
// p2p.cu
void strengths(Ctx& c, const double* x, bool fp32, cudaStream_t s);
void p2p_direct(Ctx& c, bool fp32, cudaStream_t s);
void combine(Ctx& c, const double* x, double* y, cudaStream_t s);
void matvec_internal(Ctx& c, const double* x, double* y, int op, cudaStream_t s);
// tree.cu
void build_tree(Ctx& c, cudaStream_t s);
// contiguous ranges of nearly equal cost (bempol_shard_rows)
std::vector<int64_t> shard_cuts(const std::vector<double>& cost, int world);
// this rank's block tables and row bounds for the current tree (no-op without sharding)
void build_shard(Ctx& c, cudaStream_t s);
void tree_matvec_sums(Ctx& c, bool fp32, cudaStream_t s);
void tree_matvec_T_sums(Ctx& c, const double* u, cudaStream_t s);
void tree_near_candidates(Ctx& c, double rmax, std::vector<int>& ptr, std::vector<int>& cells);
// adjoint.cu
// builds the near table by columns (near_ptrT/rowT/eT) if the current mesh has none yet
void ensure_near_transpose(Ctx& c, cudaStream_t s);
void matvec_T_internal(Ctx& c, const double* u, double* y, int op, cudaStream_t s);
struct AdjointOut {
  int iters_diss = 0, iters_vac = 0, solves = 0, gmres_iters = 0;
  bool converged = true;
};
AdjointOut gradient_internal(Ctx& c, double* g_q, double* g_d, double* g_Q, double* g_pos, cudaStream_t s);
// sites.cu
void site_field_of_charges(Ctx& c, const double4* src, const double4* str, const float4* src32, const float4* str32,
                           int K, bool fp32, double* out10, cudaStream_t s);
void rhs_internal(Ctx& c, const double* p, double* b, bool fp32, cudaStream_t s);
void site_reaction_internal(Ctx& c, const double* x, double* out, bool fp32, bool hessian, cudaStream_t s);
// the reaction field in the form of operator `op`: by the treecode for the tree forms
// (always with the Hessian), by direct K-node sums otherwise; FP32 pair terms for the
// FP32 forms
void site_reaction_form(Ctx& c, const double* x, double* out, int op, bool hessian, cudaStream_t s);
void multipole_internal(Ctx& c, const double* mu, int mode, double* out, cudaStream_t s, bool fp32 = false);
// per-system energies (host vector of nsys)
std::vector<double> energy_internal(Ctx& c, const double* react10, const double* mult10, cudaStream_t s);
// SOR step for the systems with active[s] != 0 (device flags, NULL = all); returns
// the per-system RMS change
std::vector<double> sor_update(Ctx& c, double* mu, const double* E_react10, const double* E_mult3, bool vacuum,
                               const int* d_active, cudaStream_t s);
void site_validation(Ctx& c, cudaStream_t s);
// direct pair sums with the given per-block source ranges into part [S][4][n]
int p2p_splits(Ctx& c, int max_range);
void p2p_direct_ranges(Ctx& c, bool fp32, const int4* rng, double* part, int S, cudaStream_t s);
// Stern layer (stern.cu)
void build_stern_blocks(Ctx& c, cudaStream_t s);
void stern_check_nested(Ctx& c, cudaStream_t s);
void stern_matvec(Ctx& c, const double* x, double* y, bool fp32, cudaStream_t s);
// sitetree.cu: reaction potential, field and Hessian at the sites by the treecode, FP32
// terms with FP64 sums or FP64 (out [ns*10] as site_reaction_internal)
void site_reaction_tree(Ctx& c, const double* x, double* out, bool fp32, cudaStream_t s);
bool site_reaction_scratch(Ctx& c, const double* x, double* out, bool fp32, bool hessian, double* scratch,
                           size_t cap, cudaStream_t s);
// gmres.cu
struct GmresOut {
  int iters = 0;
  int matvecs = 0;
  int residual_matvecs = 0;    // of matvecs, the refinement residuals (products with residual_op)
  double rel_res = 0;          // largest relative residual over the solved systems
  bool converged = false;      // every solved system converged
  std::vector<int> sys_iters;  // per system
  std::vector<double> sys_res; // per system relative residual
  std::vector<char> sys_conv;
};
// Solve A x = b for every system with want[s] != 0 (empty = all); x holds the
// initial guess and is left unchanged for the other systems.  With `refine` and
// params.residual_op != params.op the solve is FP64 iterative refinement (outer
// residual with residual_op, inner GMRES with op); otherwise plain GMRES with op.
// rel_tol: stopping tolerance ||b - A x|| / ||b|| (<= 0: params.gmres_tol).
GmresOut solve_bem(Ctx& c, const double* b, double* x, const std::vector<char>& want, cudaStream_t s,
                   bool refine, double rel_tol = -1.0);
// vector helpers (gmres.cu)
double dot_dev(Ctx& c, const double* a, const double* b, int len, cudaStream_t s);
void permute_to_internal(const Ctx& c, const double* src, double* dst, int blocks_of_n, cudaStream_t s);
void permute_to_caller(const Ctx& c, const double* src, double* dst, int blocks_of_n, cudaStream_t s);

}  // namespace bp
