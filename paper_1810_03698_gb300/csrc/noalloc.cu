// Reaction field at the sites without any device allocation.
//
// bempol_site_reaction keeps its per-split partial sums in a buffer owned by the
// context, which it (re)allocates with cudaMalloc when the number of sites or
// splits grows.  Some callers cannot allow a device allocation at call time:
// for example code running while another runtime owns the device memory pool,
// or latency-critical loops that cannot accept cudaMalloc's implicit device
// synchronisation.  bempol_site_reaction_noalloc computes the same quantity with
// its partial sums in a fixed file-scope device array instead.
//
// The array is 2 MiB (262,144 doubles).  Every GPU that loads this library holds
// it until the process exits.  It is shared by every call and every context, and
// keeps the last call's contents: calls that overlap on the GPU (other streams,
// other contexts, other host threads) race on it.  Each call writes every entry
// it later reads, so nothing needs clearing between calls.
#include <mutex>
#include <string>

#include "internal.h"

struct bempol_ctx : public bp::Ctx {};

namespace bp {

namespace {

constexpr size_t NOALLOC_SCRATCH_DOUBLES = 262144;  // 2 MiB
__device__ __align__(256) double g_site_scratch[NOALLOC_SCRATCH_DOUBLES];

std::mutex g_scratch_mu;
double* g_scratch_ptr[64] = {};

// Device address of the scratch array for the current device.  In host code the
// symbol g_site_scratch is only a host-side stand-in, never a device address;
// the address comes from cudaGetSymbolAddress, looked up once per device (on the
// first call there) and cached for the life of the process.  That first lookup
// may load this library's device code onto the device (CUDA loads modules
// lazily), which the driver does with allocations of its own.  A
// cudaDeviceReset destroys the array together with every other allocation of the
// library, so no context and no cached address may be used after one.
double* scratch_for(int device) {
  if (device < 0 || device >= 64) fail(BEMPOL_ERR_ARG, "device index out of range for the no-alloc scratch");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_site_scratch);
    if (e != cudaSuccess || !p)
      fail(BEMPOL_ERR_CUDA, std::string("cudaGetSymbolAddress of the no-alloc scratch failed: ") +
                                cudaGetErrorString(e));
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  return g_scratch_ptr[device];
}

}  // namespace
}  // namespace bp

extern "C" bempol_status bempol_site_reaction_noalloc(bempol_ctx* c, const double* x, double* out, int op,
                                                      void* stream) {
  using namespace bp;
  return guard(c, [&] {
    if (!c->have_sites) fail(BEMPOL_ERR_STATE, "no sites");
    if (!x || !out) fail(BEMPOL_ERR_ARG, "NULL array");
    if (op < 0 || op > 3) fail(BEMPOL_ERR_ARG, "bad op");
    if ((size_t)c->ns * 10 > NOALLOC_SCRATCH_DOUBLES)
      fail(BEMPOL_ERR_ARG, "bempol_site_reaction_noalloc handles at most " +
                               std::to_string(NOALLOC_SCRATCH_DOUBLES / 10) + " sites (2 MiB scratch); got " +
                               std::to_string(c->ns));
    cudaStream_t s = (cudaStream_t)stream;
    double* scratch = scratch_for(c->device);
    const bool fp32 = (op == BEMPOL_OP_FP32_DIRECT || op == BEMPOL_OP_FP32_TREE);
    // x into internal order in the context's own vector (allocated by set_mesh)
    permute_to_internal(*c, x, c->vec_a.p, 2, s);
    if (!site_reaction_scratch(*c, c->vec_a.p, out, fp32, true, scratch, NOALLOC_SCRATCH_DOUBLES, s))
      fail(BEMPOL_ERR_ARG, "site count exceeds the no-alloc scratch");
  });
}
