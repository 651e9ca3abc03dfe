// Treecode matvec (Sec. "The treecode algorithm").  Placeholder until the
// Morton-octree far field lands: the tree operators report an argument error.
#include "internal.h"

namespace bp {

void build_tree(Ctx& c, cudaStream_t s) {
  (void)s;
  c.tree_ready = false;
}

void tree_matvec_sums(Ctx& c, bool fp32, cudaStream_t s) {
  (void)c;
  (void)fp32;
  (void)s;
  fail(BEMPOL_ERR_ARG, "treecode operators are not available in this build");
}

}  // namespace bp
