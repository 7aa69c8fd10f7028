// hlc_internal.h -- structures shared by the host planner and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/hlc.h"

namespace hlc {

// ---------------------------------------------------------------------------
// Device-visible descriptors.
// ---------------------------------------------------------------------------

// Buffers an op view can point into.
enum Buf : int32_t {
  BUF_L = 0,     // arena of the matrix being factored / solved with
  BUF_TMP = 1,   // zero-initialised temporaries of a plan
  BUF_VEC = 2,   // vectors of the solves (n x c, tree order)
  BUF_C = 3,     // arena of C~ (matvec, assembly)
  NBUF = 4
};

// A strided matrix view: element (i, j) at base[buf] + off + i*rs + j*cs.
struct Mv {
  int64_t off;
  int64_t rs, cs;
  int32_t buf;
  int32_t pad;
};

// A dimension that is either static or the runtime rank of a block
// (ranks[slot]); the static value is the capacity.
struct Dim {
  int32_t n;
  int32_t slot;
};

// Y (m x c) = beta * Y + alpha * A (m x k) * B (k x c), beta in {0, 1};
// B.buf == MV_IDENTITY marks B as the identity (Y = beta Y + alpha A, k = c),
// B.buf == MV_ONES as the k x 1 vector of ones (a fixed-order row sum of A).
constexpr int32_t MV_IDENTITY = -1;
constexpr int32_t MV_ONES = -2;
struct OpGemm {
  Mv Y, A, B;
  Dim m, k, c;
  int32_t beta;
  int32_t pad;
  double alpha;
};

// X (n x c) := L^-1 X (trans = 0), L^-T X (trans = 1), L X (trans = 2) or
// L^T X (trans = 3); L dense lower n x n (its upper triangle is not read).
struct OpTrsm {
  Mv L, X;
  int32_t n, trans;
  Dim c;
};

// In-place lower Cholesky of a dense n x n block.
struct OpPotrf {
  Mv A;
  int32_t n;
  int32_t row0;  // global row of the block (for the error report)
};

// One low-rank term of a truncated sum: alpha * U V^T placed at row offset
// roff / column offset coff of the target.  flags bit 0: U is the identity of
// size urows (k = urows); bit 1: V is the identity of size vrows.
struct TermD {
  Mv U, V;
  int32_t urows, vrows;
  int32_t roff, coff;
  Dim k;
  int32_t flags;
  int32_t pad;
  double alpha;
};

// Target := trunc(target + sum of terms[term0 .. term0 + nterms)) at block
// accuracy eps (and at most kfix columns when kfix > 0); target U (m x kcap),
// V (n x kcap), rank in ranks[slot].
// keep = 0 ignores the target's current content (assembly).
struct OpTrunc {
  Mv U, V;
  int32_t m, n;
  int32_t kcap, slot;
  int32_t nterms, keep;
  int64_t term0;
  double eps;
  int32_t kfix;  // fixed-rank mode: keep at most kfix columns (0: adaptive)
  int32_t pad;
};

// Base pointers handed to every op kernel.
struct Bases {
  double* buf[NBUF];
  int* ranks;      // rank slots of the matrix in BUF_L
  int* status;     // [0] error code, [1] detail (first error wins)
  double* scratch; // per-CTA scratch of the truncation kernel
  int mixed;       // 1: FP32 arithmetic for panels, products and QR (mixed modes)
  int core64;      // 1: FP64 truncation core in a mixed mode (HLC_MIXED_SVD64)
  double* flops;   // per op type algorithmic flop counters, or null
  unsigned long long* phase;  // truncation phase cycle counters, or null
};

enum OpType : int32_t {
  OP_POTRF = 0,
  OP_TRSM = 1,
  OP_GEMM = 2,
  OP_TRUNC = 3,
  OP_TRUNC_BIG = 4,
  OP_CHAIN = 5,
  NOPTYPES = 6
};

// A chain: the TRSM and GEMM ops of one small diagonal block's triangular
// solve (or product with the factor), run in order by one CTA with a block
// barrier between consecutive ops, instead of one wave each.  Items index
// the plan's chain arrays (ctrsm for OP_TRSM, cgemm for OP_GEMM).
struct ChainItem {
  int32_t type;
  int32_t pad;
  int64_t idx;
};
struct OpChain {
  int64_t item0;
  int32_t nitems;
  int32_t pad;
};
// Device tables of a plan's chains.
struct ChainTab {
  const ChainItem* items;
  const OpTrsm* trsm;
  const OpGemm* gemm;
};

// Device error codes recorded in status[0].
enum DevErr : int32_t { DEV_OK = 0, DEV_NOT_SPD = 1, DEV_RANK = 2, DEV_BAD = 3, DEV_TIMEOUT = 4 };

// ---------------------------------------------------------------------------
// Host-side tree.
// ---------------------------------------------------------------------------
enum BlkType : int32_t { BT_DENSE = 0, BT_LR = 1, BT_SUB = 2 };

struct Cluster {
  int64_t lo, hi;
  double bmin[2], bmax[2];
  int32_t child[2];
  int32_t level;
  bool leaf() const { return child[0] < 0; }
  int64_t size() const { return hi - lo; }
};

struct Block {
  int32_t r, s;
  int32_t type;
  int32_t diag;
  int32_t ch[4];     // off-diagonal: ch[2i+j] = (r_i, s_j); diagonal: 0,2,3
  int64_t m, n;
  int64_t offD;      // dense: m x n column-major (ld = m)
  int64_t offU, offV;// low-rank: U m x kcap (ld m), V n x kcap (ld n)
  int32_t kcap;
  int32_t slot;      // rank slot (low-rank) or -1
  int32_t leaf_index;// position in the leaf list, -1 for SUB
};

// Assembly descriptors (device).
struct DenseAsm {
  int64_t off;   // arena offset
  int64_t r0, c0;
  int32_t m, n;
};
struct LrAsm {
  int64_t offU, offV;
  int64_t r0, c0;
  int32_t m, n;
  int32_t kcap, slot;
};

// A dependency-ordered op program ("plan"): ops grouped into waves; within a
// wave ops are independent and run as one launch per op type.
struct Launch {
  int32_t type;
  int32_t wave;
  int64_t first, count;  // range in the per-type device arrays
};

// State of the persistent kernel's grid barrier (zeroed before each launch).
struct GridBar {
  unsigned int count, gen, abort, pad;
  unsigned long long ticket;  // next op number (solves) or ready-queue slot (factorisation) to take
  unsigned long long tail;    // ready-queue slots filled beyond the initially ready ops
};

// TRSM, GEMM and chain op ranges of one wave (persistent execution of a
// plan).
struct WaveRange {
  int64_t trsm0, ntrsm;
  int64_t gemm0, ngemm;
  int64_t chain0, nchain;
};

// An op of a dataflow plan: its type and index in that type's array.  A
// truncation run by a group of CTAs (OP_TRUNC_BIG) has one entry per part
// (part 0..parts-1, consecutive), sharing the group record `group`.  For a
// TRSM of a dataflow solve, `group` is the GEMM (a one-column product into
// the TRSM's rows) that the same CTA runs first, or -1.
struct FlowOp {
  int32_t type;
  int32_t part;
  int64_t idx;
  int64_t group;
};

// Rendezvous of the CTAs that run the parts of one group truncation in the
// dataflow factorisation (zeroed before each run): a bounded barrier and the
// CTA of every part (whose scratch slice the others read).
struct TrGroup {
  unsigned int count, gen;
  int32_t cta[8];
};

// Timeline record of one op of the dataflow factorisation (optional): global
// timer nanoseconds when a CTA took the op's ticket, when its producers were
// done and when it finished; the CTA; the producer whose signal released it
// (-1: none, the op had no producers).
struct FactorTrace {
  unsigned long long t_take, t_ready, t_done;
  uint32_t cta;
  int32_t releaser;
};

struct Plan {
  std::vector<OpGemm> gemm;
  std::vector<OpTrsm> trsm;
  std::vector<OpPotrf> potrf;
  std::vector<OpTrunc> trunc;
  std::vector<TermD> terms;
  std::vector<OpChain> chain;
  std::vector<ChainItem> citems;
  std::vector<OpTrsm> ctrsm;
  std::vector<OpGemm> cgemm;
  std::vector<Launch> launches;
  // dataflow form of a TRSM/GEMM plan (ops in wave order; predecessors
  // counted, successors as CSR), for the dependency-driven persistent kernel
  std::vector<FlowOp> flow;
  std::vector<int32_t> npred;
  std::vector<int64_t> succ_off;
  std::vector<int32_t> succ;
  // the ops without producers, in flow order (a group with all its parts):
  // the first entries of the factorisation's ready queue
  std::vector<int32_t> ready0;
  FlowOp* d_flow = nullptr;
  int32_t* d_npred = nullptr;
  int64_t* d_succ_off = nullptr;
  int32_t* d_succ = nullptr;
  int32_t* d_count = nullptr;  // arrivals per op (zeroed before each run)
  int32_t* d_ready0 = nullptr; // device copy of ready0
  int32_t* d_ready = nullptr;  // ready queue of the factorisation (one slot per op)
  int64_t ngroups = 0;         // group truncations (OP_TRUNC_BIG) of a dataflow factorisation
  TrGroup* d_groups = nullptr;
  int64_t tmp_doubles = 0;
  int32_t tmp_slots = 0;  // rank slots of temporary partial sums (after the matrix's)
  int32_t nwaves = 0;
  int64_t max_trunc_per_wave = 0;
  bool checked = false;
  // the plan captured as a CUDA graph for one set of base pointers
  mutable cudaGraphExec_t graph = nullptr;
  mutable Bases graph_key{};
  mutable int64_t graph_kernels = 0;
  // waves of a TRSM/GEMM-only plan, for the persistent kernel
  std::vector<WaveRange> waves;
  WaveRange* d_waves = nullptr;
  // online tuning of the persistent kernel's CTAs per SM: candidate i is
  // launched tune_tries[i] times and its best event time is tune_ms[i];
  // tuned_per_sm is set once every candidate has two timed runs
  mutable int tuned_per_sm = 0;
  mutable int tune_tries[3] = {0, 0, 0};
  mutable int tune_done[3] = {0, 0, 0};
  mutable float tune_ms[3] = {0.f, 0.f, 0.f};
  // device copies
  OpGemm* d_gemm = nullptr;
  OpTrsm* d_trsm = nullptr;
  OpPotrf* d_potrf = nullptr;
  OpTrunc* d_trunc = nullptr;
  TermD* d_terms = nullptr;
  OpChain* d_chain = nullptr;
  ChainItem* d_citems = nullptr;
  OpTrsm* d_ctrsm = nullptr;
  OpGemm* d_cgemm = nullptr;
  ChainTab chains() const { return ChainTab{d_citems, d_ctrsm, d_cgemm}; }
  int64_t nops() const {
    return (int64_t)gemm.size() + trsm.size() + potrf.size() + trunc.size() + ctrsm.size() + cgemm.size();
  }
};

}  // namespace hlc
