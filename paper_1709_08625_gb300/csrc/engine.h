// engine.h -- host tree, layout and planner interfaces.
#pragma once

#include "hlc_internal.h"

namespace hlc {

struct HTree {
  int64_t n = 0;
  int leaf = 64;
  double eta = 2.0;
  double eps = 1e-6;
  int kmax = 64;
  int kfix = 0;  // fixed-rank mode: at most kfix columns per low-rank block
  int depth = 0;
  std::vector<double> px, py;   // points in tree order
  std::vector<int32_t> perm;    // tree position -> caller index
  std::vector<Cluster> cl;      // breadth-first, root = 0
  std::vector<Block> blk;       // block-cluster tree, root = 0 (diagonal)
  std::vector<int32_t> leaves;  // leaf blocks, depth-first
  int64_t arena_doubles = 0;
  int32_t nslots = 0;
  int64_t max_dense_dim = 0;
  std::vector<DenseAsm> dense_asm;
  std::vector<LrAsm> lr_asm;
};

// Leaf list (depth-first) of the block tree built on the device.
void collect_leaf_list(HTree& T);
// Arena offsets, rank capacities and rank slots of the leaves.
void layout(HTree& T, int kmax);

// accumulate: updates of a low-rank block are truncated together right before
// the block is next used (accumulated updates) instead of one at a time.
// flow: also build the plan's dataflow form (op-level dependencies) for the
// dependency-driven factorisation kernel
void plan_cholesky(HTree& T, Plan& P, bool accumulate = false, bool flow = false);
// chains: the solve of every subdivided diagonal block of at most 1024 rows
// becomes one op (a chain run by one CTA)
void plan_solve(HTree& T, Plan& P, int trans, int64_t voff, int64_t ncols, bool chains = false);
void plan_matvec(HTree& T, Plan& P, int64_t xoff, int64_t yoff, int64_t ncols);
// X := L X (trans 0) or L^T X (trans 1), in place, L the lower factor
void plan_trmv(HTree& T, Plan& P, int trans, int64_t voff, int64_t ncols, bool chains = false);
void plan_recompress(HTree& T, Plan& P);
// Bounds check of every view against the buffer sizes (in doubles) and of
// every rank slot against the rank array's length.
std::string validate_plan(const Plan& P, const int64_t* bufsize, int64_t nslots);

}  // namespace hlc
