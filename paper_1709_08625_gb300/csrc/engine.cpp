// engine.cpp -- host side of the library: tree structures, storage layout and
// the planner that turns the recursive H-arithmetic into a wave-ordered op
// program executed by the batched kernels.
//
// The planner walks the recursion of the H-Cholesky factorisation (Table 1:
// truncated addition and multiply-add, the Cholesky of eq. 2) symbolically:
// it touches no numbers, only block structure, and emits primitive ops
// (dense POTRF, dense TRSM, strided GEMM, low-rank truncation) with the
// ranks of low-rank blocks left as runtime values read by the kernels.
// Every op is placed in the earliest wave after the ops it depends on
// (read-after-write, write-after-read and write-after-write on 2-D regions of
// the block storage), so each wave is a set of independent ops that run as
// one launch per op type.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <queue>
#include <stdexcept>

#include "engine.h"

namespace hlc {

// ---------------------------------------------------------------------------
// Leaf list of the block-cluster tree (built on the device, tree.cu).
// ---------------------------------------------------------------------------
static void collect_leaves(HTree& T, int32_t b) {
  Block& B = T.blk[b];
  if (B.type != BT_SUB) {
    B.leaf_index = (int32_t)T.leaves.size();
    T.leaves.push_back(b);
    return;
  }
  for (int q = 0; q < 4; ++q)
    if (T.blk[b].ch[q] >= 0) collect_leaves(T, T.blk[b].ch[q]);
}

void collect_leaf_list(HTree& T) {
  T.leaves.clear();
  collect_leaves(T, 0);
}

void layout(HTree& T, int kmax) {
  T.kmax = kmax;
  int64_t off = 0;
  int32_t slots = 0;
  T.dense_asm.clear();
  T.lr_asm.clear();
  T.max_dense_dim = 0;
  for (int32_t b : T.leaves) {
    Block& B = T.blk[b];
    const Cluster& cr = T.cl[B.r];
    const Cluster& cs = T.cl[B.s];
    if (B.type == BT_DENSE) {
      B.offD = off;
      off += B.m * B.n;
      off = (off + 3) & ~int64_t(3);  // 32-byte alignment of every block
      T.dense_asm.push_back(DenseAsm{B.offD, cr.lo, cs.lo, (int32_t)B.m, (int32_t)B.n});
      T.max_dense_dim = std::max<int64_t>(T.max_dense_dim, std::max(B.m, B.n));
    } else {
      B.kcap = (int32_t)std::min<int64_t>(kmax, std::min(B.m, B.n));
      B.slot = slots++;
      B.offU = off;
      off += B.m * B.kcap;
      off = (off + 3) & ~int64_t(3);
      B.offV = off;
      off += B.n * B.kcap;
      off = (off + 3) & ~int64_t(3);
      T.lr_asm.push_back(LrAsm{B.offU, B.offV, cr.lo, cs.lo, (int32_t)B.m, (int32_t)B.n, B.kcap, B.slot});
    }
  }
  T.arena_doubles = off;
  T.nslots = slots;
}

// ---------------------------------------------------------------------------
// Planner
// ---------------------------------------------------------------------------
namespace {

struct Rect {
  int64_t r0, r1, c0, c1;
  bool overlaps(const Rect& o) const { return r0 < o.r1 && o.r0 < r1 && c0 < o.c1 && o.c0 < c1; }
  bool operator==(const Rect& o) const { return r0 == o.r0 && r1 == o.r1 && c0 == o.c0 && c1 == o.c1; }
};

struct Acc {
  Rect rc;
  int32_t lw, lr;  // wave of the last write / latest read
  // op-level dependencies (tracked for the dataflow plans): the op that
  // last wrote the region and the ops that read it since
  int64_t wop = -1;
  std::vector<int64_t> rops;
};

struct Obj {
  int32_t buf;
  int64_t off, ld;
  std::vector<Acc> acc;
  // temporaries: size, lifetime in waves, rows already written (union)
  int64_t size = 0;
  int32_t birth = INT32_MAX, death = -1;
  std::vector<std::pair<int64_t, int64_t>> written;
  // dataflow plans: the ops that touch this temporary, and those that write it
  std::vector<int64_t> touch, wr;
};

// A view in storage coordinates of an object: element (i, j) of the view is
// storage element (sr + i, sc + j), or (sr + j, sc + i) when transposed.
struct PV {
  int32_t obj;
  int64_t sr, sc;
  int64_t rows, cols;  // static extents (capacities)
  bool tr;
  int32_t drow, dcol;  // rank slot of a dynamic extent, -1 if static
};

const int32_t NOSLOT = -1;

struct TermP {
  PV U, V;
  int64_t urows, vrows;
  int64_t roff, coff;
  Dim k;
  int32_t flags;
  double alpha;
};
const int64_t kTruncBigRows = 4096;   // m + n above which a truncation uses a cluster
const int64_t kTruncManyCols = 128;   // term columns (at capacity) beyond which ...
const int64_t kTruncManyRows = 512;   // ... a target with m + n above this uses a cluster too
const int64_t kGemmSplitRows = 4096;  // row block of a split product
const int64_t kGemmSplitK = 2048;     // inner block of a split matrix-vector product
const int64_t kPendingCols = INT64_MAX;  // no size-forced truncation: flush only on use
const size_t kTreeMinTerms = 9;          // a truncated sum of this many terms or more ...
const size_t kTreeLeafTerms = 4;         // ... is summed as a tree over groups of this many
const int64_t kTempKcap = 128;           // rank capacity of a partial sum
const int64_t kChainRows = 1024;         // largest diagonal block whose solve is one chain

struct Planner {
  HTree& T;
  Plan& P;
  int32_t mat_buf;
  std::vector<Obj> objs;
  std::vector<int32_t> objD, objU, objV;  // per block id
  int64_t tmp_top = 0;
  struct Ref {
    int32_t type;
    int64_t idx;
    int32_t wave;
  };
  std::vector<Ref> seq;
  int32_t maxwave = -1;

  // Accumulated updates: terms added to a low-rank block wait here and are
  // truncated together (in batches of 64 columns) right before the block is
  // read or written otherwise, or when too many columns have piled up.
  bool defer = false;
  std::vector<std::vector<struct TermP>> pending;
  std::vector<int64_t> pending_cols;

  Planner(HTree& t, Plan& p, int32_t mbuf) : T(t), P(p), mat_buf(mbuf) {
    objD.assign(T.blk.size(), -1);
    objU.assign(T.blk.size(), -1);
    objV.assign(T.blk.size(), -1);
    pending.assign(T.blk.size(), {});
    pending_cols.assign(T.blk.size(), 0);
    for (int32_t b : T.leaves) {
      const Block& B = T.blk[b];
      if (B.type == BT_DENSE) {
        objD[b] = add_obj(mat_buf, B.offD, B.m);
      } else {
        objU[b] = add_obj(mat_buf, B.offU, B.m);
        objV[b] = add_obj(mat_buf, B.offV, B.n);
      }
    }
  }

  int32_t add_obj(int32_t buf, int64_t off, int64_t ld) {
    Obj o;
    o.buf = buf;
    o.off = off;
    o.ld = ld;
    objs.push_back(std::move(o));
    return (int32_t)objs.size() - 1;
  }

  // Temporaries get a virtual offset here; finish() maps them onto reused
  // physical storage according to their lifetimes.
  std::vector<int32_t> tmp_objs;
  int32_t new_tmp(int64_t rows, int64_t cols) {
    const int64_t off = tmp_top;
    const int64_t sz = ((std::max<int64_t>(rows * cols, 1)) + 3) & ~int64_t(3);
    tmp_top += sz;
    const int32_t o = add_obj(BUF_TMP, off, std::max<int64_t>(rows, 1));
    objs[o].size = sz;
    tmp_objs.push_back(o);
    return o;
  }

  // beta for a write of rows [a, b) into a temporary: 0 when nothing of it
  // was written before, 1 when all of it was; a partial overlap cannot
  // arise for cluster-aligned row ranges and is rejected.
  int32_t first_write_beta(const PV& v) {
    Obj& o = objs[v.obj];
    if (o.buf != BUF_TMP) return 1;
    const Rect rc = rect(v);
    const int64_t a = rc.r0, b = rc.r1;
    int64_t cov = 0;
    for (auto& iv : o.written) cov += std::max<int64_t>(0, std::min(b, iv.second) - std::max(a, iv.first));
    if (cov != 0 && cov != b - a) throw std::runtime_error("planner: partial first write of a temporary");
    if (cov == 0) {
      // merge [a, b) into the union
      o.written.push_back({a, b});
      std::sort(o.written.begin(), o.written.end());
      std::vector<std::pair<int64_t, int64_t>> mg;
      for (auto& iv : o.written) {
        if (!mg.empty() && iv.first <= mg.back().second)
          mg.back().second = std::max(mg.back().second, iv.second);
        else
          mg.push_back(iv);
      }
      o.written.swap(mg);
      return 0;
    }
    return 1;
  }

  // ---- views ----
  PV whole(int32_t obj, int64_t rows, int64_t cols, int32_t drow = NOSLOT, int32_t dcol = NOSLOT) {
    return PV{obj, 0, 0, rows, cols, false, drow, dcol};
  }
  static PV T_(const PV& v) {
    PV t = v;
    t.tr = !v.tr;
    t.rows = v.cols;
    t.cols = v.rows;
    t.drow = v.dcol;
    t.dcol = v.drow;
    return t;
  }
  static PV rows(const PV& v, int64_t a, int64_t b) {
    PV t = v;
    if (!v.tr)
      t.sr += a;
    else
      t.sc += a;
    t.rows = b - a;
    t.drow = NOSLOT;
    return t;
  }
  static PV cols(const PV& v, int64_t a, int64_t b) {
    PV t = v;
    if (!v.tr)
      t.sc += a;
    else
      t.sr += a;
    t.cols = b - a;
    t.dcol = NOSLOT;
    return t;
  }
  Rect rect(const PV& v) const {
    if (!v.tr) return Rect{v.sr, v.sr + v.rows, v.sc, v.sc + v.cols};
    return Rect{v.sr, v.sr + v.cols, v.sc, v.sc + v.rows};
  }
  Mv mv(const PV& v) const {
    const Obj& o = objs[v.obj];
    Mv m;
    m.buf = o.buf;
    m.pad = 0;
    m.off = o.off + v.sr + v.sc * o.ld;
    m.rs = v.tr ? o.ld : 1;
    m.cs = v.tr ? 1 : o.ld;
    return m;
  }
  static Dim dim(int64_t n, int32_t slot) { return Dim{(int32_t)n, slot}; }

  // ---- dependency analysis ----
  // Op-level dependency lists (track = true): preds[i] holds the ops that op
  // i (its index in seq) must wait for -- the last writer of every region it
  // reads or writes (read/write after write) and, for the regions it
  // writes, the readers since that write (write after read).
  bool track = false;
  std::vector<std::vector<int64_t>> preds;

  int32_t place(const std::vector<PV>& reads, const std::vector<PV>& writes) {
    const int64_t me = (int64_t)seq.size();  // the op being placed
    std::vector<int64_t> dep;
    int32_t w = 0;
    for (const PV& v : reads) {
      if (v.rows <= 0 || v.cols <= 0) continue;
      const Rect rc = rect(v);
      for (const Acc& a : objs[v.obj].acc)
        if (a.rc.overlaps(rc)) {
          w = std::max(w, a.lw + 1);
          if (track && a.wop >= 0) dep.push_back(a.wop);
        }
    }
    for (const PV& v : writes) {
      if (v.rows <= 0 || v.cols <= 0) continue;
      const Rect rc = rect(v);
      for (const Acc& a : objs[v.obj].acc)
        if (a.rc.overlaps(rc)) {
          w = std::max(w, std::max(a.lw, a.lr) + 1);
          if (track) {
            if (a.wop >= 0) dep.push_back(a.wop);
            dep.insert(dep.end(), a.rops.begin(), a.rops.end());
          }
        }
    }
    if (track) {
      std::sort(dep.begin(), dep.end());
      dep.erase(std::unique(dep.begin(), dep.end()), dep.end());
      dep.erase(std::remove(dep.begin(), dep.end(), me), dep.end());
      if ((int64_t)preds.size() <= me) preds.resize(me + 1);
      preds[me] = std::move(dep);
    }
    for (const PV& v : reads) {
      if (v.rows <= 0 || v.cols <= 0) continue;
      Obj& ob = objs[v.obj];
      if (ob.buf == BUF_TMP) {
        ob.birth = std::min(ob.birth, w);
        ob.death = std::max(ob.death, w);
        if (track) ob.touch.push_back(me);
      }
      const Rect rc = rect(v);
      bool found = false;
      for (Acc& a : objs[v.obj].acc)
        if (a.rc == rc) {
          a.lr = std::max(a.lr, w);
          if (track) a.rops.push_back(me);
          found = true;
          break;
        }
      if (!found) {
        Acc a{rc, -1, w};
        if (track) a.rops.push_back(me);
        objs[v.obj].acc.push_back(std::move(a));
      }
    }
    for (const PV& v : writes) {
      if (v.rows <= 0 || v.cols <= 0) continue;
      Obj& ob = objs[v.obj];
      if (ob.buf == BUF_TMP) {
        ob.birth = std::min(ob.birth, w);
        ob.death = std::max(ob.death, w);
        if (track) {
          ob.touch.push_back(me);
          ob.wr.push_back(me);
        }
      }
      const Rect rc = rect(v);
      std::vector<Acc>& L = objs[v.obj].acc;
      // accesses covered by this write are superseded by it
      L.erase(std::remove_if(L.begin(), L.end(),
                             [&](const Acc& a) {
                               return a.rc.r0 >= rc.r0 && a.rc.r1 <= rc.r1 && a.rc.c0 >= rc.c0 &&
                                      a.rc.c1 <= rc.c1;
                             }),
              L.end());
      Acc a{rc, w, -1};
      a.wop = track ? me : -1;
      L.push_back(std::move(a));
    }
    maxwave = std::max(maxwave, w);
    return w;
  }

  // ---- op emission ----
  void gemm(const PV& Y, const PV& A, const PV& B, Dim m, Dim k, Dim c, double alpha) {
    if (m.n <= 0 || c.n <= 0 || k.n <= 0) return;
    // matrix-vector products with a long inner dimension: partial products
    // of inner blocks into disjoint slices of a temporary (one CTA each),
    // then their sum in a fixed order
    if (c.slot < 0 && c.n == 1 && k.slot < 0 && k.n > kGemmSplitK) {
      const int64_t nq = (k.n + kGemmSplitK - 1) / kGemmSplitK, mc = m.n;
      const int32_t t = new_tmp(mc * nq, 1);
      const PV Pt = whole(t, mc * nq, 1);
      for (int64_t q = 0; q < nq; ++q) {
        const int64_t k0 = q * kGemmSplitK, k1 = std::min<int64_t>(k.n, k0 + kGemmSplitK);
        gemm(rows(Pt, q * mc, (q + 1) * mc), cols(A, k0, k1), rows(B, k0, k1), m, dim(k1 - k0, NOSLOT), c, 1.0);
      }
      OpGemm op;
      op.Y = mv(Y);
      op.A = mv(Pt);
      op.A.cs = mc;  // the slices side by side: element (i, q) at i + q mc
      op.B = Mv{0, 0, 0, MV_ONES, 0};
      op.m = m;
      op.k = dim(nq, NOSLOT);
      op.c = c;
      op.alpha = alpha;
      op.beta = first_write_beta(Y);
      op.pad = 0;
      emit_gemm(op, {Pt}, {Y});
      return;
    }
    // tall products split into independent row blocks (one CTA each)
    if (m.slot < 0 && m.n > kGemmSplitRows) {
      for (int64_t r0 = 0; r0 < m.n; r0 += kGemmSplitRows) {
        const int64_t r1 = std::min<int64_t>(m.n, r0 + kGemmSplitRows);
        gemm(rows(Y, r0, r1), rows(A, r0, r1), B, dim(r1 - r0, NOSLOT), k, c, alpha);
      }
      return;
    }
    OpGemm op;
    op.Y = mv(Y);
    op.A = mv(A);
    op.B = mv(B);
    op.m = m;
    op.k = k;
    op.c = c;
    op.alpha = alpha;
    op.beta = first_write_beta(Y);
    op.pad = 0;
    emit_gemm(op, {A, B}, {Y});
  }
  // Y += alpha * X (B marked as the identity)
  void axpy(const PV& Y, const PV& X, Dim m, Dim c, double alpha) {
    if (m.n <= 0 || c.n <= 0) return;
    OpGemm op;
    op.Y = mv(Y);
    op.A = mv(X);
    op.B = Mv{0, 0, 0, MV_IDENTITY, 0};
    op.m = m;
    op.k = c;
    op.c = c;
    op.alpha = alpha;
    op.beta = first_write_beta(Y);
    op.pad = 0;
    emit_gemm(op, {X}, {Y});
  }
  void trsm(const PV& L, const PV& X, int64_t n, int trans, Dim c) {
    if (n <= 0 || c.n <= 0) return;
    OpTrsm op;
    op.L = mv(L);
    op.X = mv(X);
    op.n = (int32_t)n;
    op.trans = trans;
    op.c = c;
    if (in_chain) {
      P.ctrsm.push_back(op);
      P.citems.push_back(ChainItem{OP_TRSM, 0, (int64_t)P.ctrsm.size() - 1});
      chain_access({L}, {X});
      return;
    }
    const int32_t w = place({L}, {X});
    P.trsm.push_back(op);
    seq.push_back(Ref{OP_TRSM, (int64_t)P.trsm.size() - 1, w});
  }

  // ---- chains: the ops of a small diagonal block's solve run by one CTA ----
  bool chains = false;    // emit chains (solve plans)
  bool in_chain = false;  // collecting the ops of a chain
  int64_t chain_item0 = 0;
  std::vector<PV> chain_reads, chain_writes;

  void emit_gemm(const OpGemm& op, const std::vector<PV>& reads, const std::vector<PV>& writes) {
    if (in_chain) {
      P.cgemm.push_back(op);
      P.citems.push_back(ChainItem{OP_GEMM, 0, (int64_t)P.cgemm.size() - 1});
      chain_access(reads, writes);
      return;
    }
    const int32_t w = place(reads, writes);
    P.gemm.push_back(op);
    seq.push_back(Ref{OP_GEMM, (int64_t)P.gemm.size() - 1, w});
  }
  void chain_access(const std::vector<PV>& reads, const std::vector<PV>& writes) {
    chain_reads.insert(chain_reads.end(), reads.begin(), reads.end());
    chain_writes.insert(chain_writes.end(), writes.begin(), writes.end());
  }
  void begin_chain() {
    in_chain = true;
    chain_item0 = (int64_t)P.citems.size();
    chain_reads.clear();
    chain_writes.clear();
  }
  // The chain is one op: it waits for every producer of what any of its ops
  // reads or writes, and everything after it waits for it.  Temporaries
  // written inside the chain are among its writes, so they live for its
  // wave.
  void end_chain() {
    in_chain = false;
    const int64_t nit = (int64_t)P.citems.size() - chain_item0;
    if (nit == 0) return;
    // reads that the chain itself wrote first are internal: only the writes
    // need to be placed for those regions, and a region both read and
    // written orders the same way as written
    const int32_t w = place(chain_reads, chain_writes);
    P.chain.push_back(OpChain{chain_item0, (int32_t)nit, 0});
    seq.push_back(Ref{OP_CHAIN, (int64_t)P.chain.size() - 1, w});
  }
  void potrf(int32_t b) {
    const Block& B = T.blk[b];
    OpPotrf op;
    PV A = whole(objD[b], B.m, B.n);
    op.A = mv(A);
    op.n = (int32_t)B.m;
    op.row0 = (int32_t)T.cl[B.r].lo;
    const int32_t w = place({}, {A});
    P.potrf.push_back(op);
    seq.push_back(Ref{OP_POTRF, (int64_t)P.potrf.size() - 1, w});
  }

  // The low-rank target of a truncation: a leaf block of the matrix or a
  // temporary partial sum (views in BUF_TMP, a rank slot after the
  // matrix's own).
  struct Target {
    PV U, V;
    int64_t m, n;
    int32_t kcap, slot;
  };
  Target block_target(int32_t b) {
    const Block& B = T.blk[b];
    return Target{whole(objU[b], B.m, B.kcap), whole(objV[b], B.n, B.kcap), B.m, B.n, B.kcap, B.slot};
  }
  // Rank slots of temporary partial sums, numbered after the matrix's
  // nslots (the rank array of a matrix holds nslots + P.tmp_slots words).
  Target temp_target(int64_t m, int64_t n) {
    const int32_t kc = (int32_t)std::min<int64_t>(kTempKcap, std::min(m, n));
    const int32_t ou = new_tmp(m, kc), ov = new_tmp(n, kc);
    const int32_t slot = T.nslots + P.tmp_slots++;
    return Target{whole(ou, m, kc), whole(ov, n, kc), m, n, kc, slot};
  }
  TermP as_term(const Target& t) {
    return TermP{PV{t.U.obj, 0, 0, t.m, t.kcap, false, NOSLOT, t.slot},
                 PV{t.V.obj, 0, 0, t.n, t.kcap, false, NOSLOT, t.slot}, t.m, t.n, 0, 0, dim(t.kcap, t.slot), 0,
                 1.0};
  }

  // One truncation op: target := trunc(target (keep) + sum of the terms),
  // the terms taken in batches of at most 64 new columns by the kernel.
  void trunc_op(const Target& tg, const std::vector<TermP>& terms, int keep) {
    OpTrunc op;
    PV U = tg.U, V = tg.V;
    op.U = mv(U);
    op.V = mv(V);
    op.m = (int32_t)tg.m;
    op.n = (int32_t)tg.n;
    op.kcap = tg.kcap;
    op.slot = tg.slot;
    op.nterms = (int32_t)terms.size();
    op.keep = keep;
    op.term0 = (int64_t)P.terms.size();
    op.eps = T.eps;
    op.kfix = T.kfix;
    op.pad = 0;
    std::vector<PV> reads;
    for (const TermP& t : terms) {
      TermD d;
      d.U = (t.flags & 1) ? Mv{0, 0, 0, -1, 0} : mv(t.U);
      d.V = (t.flags & 2) ? Mv{0, 0, 0, -1, 0} : mv(t.V);
      d.urows = (int32_t)t.urows;
      d.vrows = (int32_t)t.vrows;
      d.roff = (int32_t)t.roff;
      d.coff = (int32_t)t.coff;
      d.k = t.k;
      d.flags = t.flags;
      d.pad = 0;
      d.alpha = t.alpha;
      P.terms.push_back(d);
      if (!(t.flags & 1)) reads.push_back(t.U);
      if (!(t.flags & 2)) reads.push_back(t.V);
    }
    const int32_t w = place(reads, {U, V});
    P.trunc.push_back(op);
    // a cluster of CTAs streams the rows of large targets, and of mid-size
    // targets that take many terms (several sequential batches of columns)
    int64_t tcols = 0;
    for (const TermP& t : terms) tcols += (t.flags & 1) ? t.urows : (t.flags & 2) ? t.vrows : t.k.n;
    const bool many = tcols > kTruncManyCols && tg.m + tg.n > kTruncManyRows;
    const int32_t ty = (tg.m + tg.n > kTruncBigRows || many) ? OP_TRUNC_BIG : OP_TRUNC;
    seq.push_back(Ref{ty, (int64_t)P.trunc.size() - 1, w});
  }

  // Truncated sum of many terms (Table 1's truncated addition over a sum
  // whose order the paper leaves open): fewer than kTreeMinTerms terms go
  // into one op in order; more are summed as a balanced tree -- groups of
  // kTreeLeafTerms terms truncated on their own into temporaries, adjacent
  // partial sums combined pairwise (an odd last one moves up) until two
  // remain, then target := trunc(target + S_1 + S_2).  The ops of a tree
  // level are independent, so the depth is logarithmic in the number of
  // terms instead of linear in their columns.
  void trunc(int32_t b, const std::vector<TermP>& terms, int keep) {
    const Target tg = block_target(b);
    if (terms.size() < kTreeMinTerms) {
      trunc_op(tg, terms, keep);
      return;
    }
    std::vector<Target> level;
    for (size_t g = 0; g < terms.size(); g += kTreeLeafTerms) {
      const size_t e = std::min(terms.size(), g + kTreeLeafTerms);
      const std::vector<TermP> grp(terms.begin() + g, terms.begin() + e);
      const Target s = temp_target(tg.m, tg.n);
      trunc_op(s, grp, 0);
      level.push_back(s);
    }
    while (level.size() > 2) {
      std::vector<Target> next;
      for (size_t i = 0; i < level.size(); i += 2) {
        if (i + 1 == level.size()) {
          next.push_back(level[i]);
          break;
        }
        const Target s = temp_target(tg.m, tg.n);
        trunc_op(s, {as_term(level[i]), as_term(level[i + 1])}, 0);
        next.push_back(s);
      }
      level.swap(next);
    }
    std::vector<TermP> last;
    for (const Target& s : level) last.push_back(as_term(s));
    trunc_op(tg, last, keep);
  }

  static int64_t term_cap(const TermP& t) {
    return (t.flags & 1) ? t.urows : (t.flags & 2) ? t.vrows : t.k.n;
  }
  void add_terms(int32_t c, const std::vector<TermP>& terms) {
    if (!defer) {
      trunc(c, terms, 1);
      return;
    }
    for (const TermP& t : terms) {
      pending[c].push_back(t);
      pending_cols[c] += term_cap(t);
    }
    if (pending_cols[c] > kPendingCols) flush(c);
  }
  void flush(int32_t b) {
    if (b < 0 || pending[b].empty()) return;
    std::vector<TermP> terms;
    terms.swap(pending[b]);
    pending_cols[b] = 0;
    trunc(b, terms, 1);
  }
  void flush_all() {
    for (size_t b = 0; b < pending.size(); ++b) flush((int32_t)b);
  }
  // a leaf block is about to be read (or rewritten): its pending updates first
  void use(int32_t b) {
    if (T.blk[b].type == BT_LR) flush(b);
  }

  // ---- block views ----
  const Block& blk(int32_t b) const { return T.blk[b]; }
  int64_t rlo(int32_t b) const { return T.cl[T.blk[b].r].lo; }
  int64_t slo(int32_t b) const { return T.cl[T.blk[b].s].lo; }
  PV D(int32_t b) { return whole(objD[b], blk(b).m, blk(b).n); }
  PV U(int32_t b) { return whole(objU[b], blk(b).m, blk(b).kcap, NOSLOT, blk(b).slot); }
  PV V(int32_t b) { return whole(objV[b], blk(b).n, blk(b).kcap, NOSLOT, blk(b).slot); }
  Dim rk(int32_t b) { return dim(blk(b).kcap, blk(b).slot); }

  // ---- H-arithmetic (mirrors the recursion of the H-Cholesky) ----

  // Y += alpha * A X  (A off-diagonal)
  void hmul(int32_t a, const PV& X, const PV& Y, double alpha) {
    use(a);
    const Block& A = blk(a);
    const Dim c = dim(X.cols, X.dcol);
    if (A.type == BT_DENSE) {
      gemm(Y, D(a), X, dim(A.m, NOSLOT), dim(A.n, NOSLOT), c, alpha);
    } else if (A.type == BT_LR) {
      const int32_t t = new_tmp(A.kcap, X.cols);
      PV Tv = whole(t, A.kcap, X.cols, A.slot, X.dcol);
      gemm(Tv, T_(V(a)), X, rk(a), dim(A.n, NOSLOT), c, 1.0);
      gemm(Y, U(a), Tv, dim(A.m, NOSLOT), rk(a), c, alpha);
    } else {
      const int64_t r0 = rlo(a), s0 = slo(a);
      for (int q = 0; q < 4; ++q) {
        const int32_t cb = A.ch[q];
        if (cb < 0) continue;
        const Cluster& cr = T.cl[blk(cb).r];
        const Cluster& cs = T.cl[blk(cb).s];
        hmul(cb, rows(X, cs.lo - s0, cs.hi - s0), rows(Y, cr.lo - r0, cr.hi - r0), alpha);
      }
    }
  }

  // Y += alpha * A^T X  (A off-diagonal)
  void hmul_t(int32_t a, const PV& X, const PV& Y, double alpha) {
    use(a);
    const Block& A = blk(a);
    const Dim c = dim(X.cols, X.dcol);
    if (A.type == BT_DENSE) {
      gemm(Y, T_(D(a)), X, dim(A.n, NOSLOT), dim(A.m, NOSLOT), c, alpha);
    } else if (A.type == BT_LR) {
      const int32_t t = new_tmp(A.kcap, X.cols);
      PV Tv = whole(t, A.kcap, X.cols, A.slot, X.dcol);
      gemm(Tv, T_(U(a)), X, rk(a), dim(A.m, NOSLOT), c, 1.0);
      gemm(Y, V(a), Tv, dim(A.n, NOSLOT), rk(a), c, alpha);
    } else {
      // children from the bottom row of blocks up: in the backward solve the
      // bottom rows of X are final first, and the products accumulate into
      // Y in this order, so no contribution waits behind a later one
      const int64_t r0 = rlo(a), s0 = slo(a);
      for (int q = 3; q >= 0; --q) {
        const int32_t cb = A.ch[q];
        if (cb < 0) continue;
        const Cluster& cr = T.cl[blk(cb).r];
        const Cluster& cs = T.cl[blk(cb).s];
        hmul_t(cb, rows(X, cr.lo - r0, cr.hi - r0), rows(Y, cs.lo - s0, cs.hi - s0), alpha);
      }
    }
  }

  int64_t cut(int32_t l) const {
    const Cluster& t = T.cl[blk(l).r];
    return T.cl[t.child[0]].hi - t.lo;
  }

  // A subdivided diagonal block of at most kChainRows rows starts a chain
  // (when chains are on and none is open): its whole solve or product
  // becomes one op.
  bool chain_here(int32_t l) const {
    const Block& L = blk(l);
    return chains && !in_chain && L.type == BT_SUB && L.m <= kChainRows;
  }

  // X := L^-1 X
  void trsv(int32_t l, const PV& X) {
    const Block& L = blk(l);
    if (chain_here(l)) {
      begin_chain();
      trsv(l, X);
      end_chain();
      return;
    }
    if (L.type == BT_DENSE) {
      trsm(D(l), X, L.m, 0, dim(X.cols, X.dcol));
      return;
    }
    const int64_t c = cut(l);
    const PV X0 = rows(X, 0, c), X1 = rows(X, c, X.rows);
    trsv(L.ch[0], X0);
    hmul(L.ch[2], X0, X1, -1.0);
    trsv(L.ch[3], X1);
  }

  // X := L^-T X
  void trsv_t(int32_t l, const PV& X) {
    const Block& L = blk(l);
    if (chain_here(l)) {
      begin_chain();
      trsv_t(l, X);
      end_chain();
      return;
    }
    if (L.type == BT_DENSE) {
      trsm(D(l), X, L.m, 1, dim(X.cols, X.dcol));
      return;
    }
    const int64_t c = cut(l);
    const PV X0 = rows(X, 0, c), X1 = rows(X, c, X.rows);
    trsv_t(L.ch[3], X1);
    hmul_t(L.ch[2], X1, X0, -1.0);
    trsv_t(L.ch[0], X0);
  }

  // X := L X (L the lower factor): with L = [L11 0; L21 L22],
  // X1 := L22 X1 + L21 X0 (X0 still unchanged), then X0 := L11 X0
  void trmv(int32_t l, const PV& X) {
    const Block& L = blk(l);
    if (chain_here(l)) {
      begin_chain();
      trmv(l, X);
      end_chain();
      return;
    }
    if (L.type == BT_DENSE) {
      trsm(D(l), X, L.m, 2, dim(X.cols, X.dcol));
      return;
    }
    const int64_t c = cut(l);
    const PV X0 = rows(X, 0, c), X1 = rows(X, c, X.rows);
    trmv(L.ch[3], X1);
    hmul(L.ch[2], X0, X1, 1.0);
    trmv(L.ch[0], X0);
  }

  // X := L^T X: X0 := L11^T X0 + L21^T X1 (X1 still unchanged), then
  // X1 := L22^T X1
  void trmv_t(int32_t l, const PV& X) {
    const Block& L = blk(l);
    if (chain_here(l)) {
      begin_chain();
      trmv_t(l, X);
      end_chain();
      return;
    }
    if (L.type == BT_DENSE) {
      trsm(D(l), X, L.m, 3, dim(X.cols, X.dcol));
      return;
    }
    const int64_t c = cut(l);
    const PV X0 = rows(X, 0, c), X1 = rows(X, c, X.rows);
    trmv_t(L.ch[0], X0);
    hmul_t(L.ch[2], X1, X0, 1.0);
    trmv_t(L.ch[3], X1);
  }

  // C += alpha U V^T
  void add_lr(int32_t c, const PV& Uv, const PV& Vv, Dim k, double alpha) {
    const Block& C = blk(c);
    if (k.n <= 0) return;
    if (C.type == BT_DENSE) {
      gemm(D(c), Uv, T_(Vv), dim(C.m, NOSLOT), k, dim(C.n, NOSLOT), alpha);
    } else if (C.type == BT_LR) {
      TermP t{Uv, Vv, C.m, C.n, 0, 0, k, 0, alpha};
      add_terms(c, {t});
    } else {
      const int64_t r0 = rlo(c), s0 = slo(c);
      for (int q = 0; q < 4; ++q) {
        const int32_t cb = C.ch[q];
        if (cb < 0) continue;
        const Cluster& cr = T.cl[blk(cb).r];
        const Cluster& cs = T.cl[blk(cb).s];
        add_lr(cb, rows(Uv, cr.lo - r0, cr.hi - r0), rows(Vv, cs.lo - s0, cs.hi - s0), k, alpha);
      }
    }
  }

  // C += P (P a dense |r| x |s| view, already scaled)
  void add_dense(int32_t c, const PV& Pv) {
    const Block& C = blk(c);
    if (C.type == BT_DENSE) {
      axpy(D(c), Pv, dim(C.m, NOSLOT), dim(C.n, NOSLOT), 1.0);
    } else if (C.type == BT_LR) {
      TermP t;
      t.roff = t.coff = 0;
      t.alpha = 1.0;
      t.urows = C.m;
      t.vrows = C.n;
      if (C.m <= C.n) {  // P = I (P^T)^T
        t.U = Pv;
        t.V = T_(Pv);
        t.flags = 1;
        t.k = dim(C.m, NOSLOT);
      } else {  // P = P I^T
        t.U = Pv;
        t.V = Pv;
        t.flags = 2;
        t.k = dim(C.n, NOSLOT);
      }
      add_terms(c, {t});
    } else {
      const int64_t r0 = rlo(c), s0 = slo(c);
      for (int q = 0; q < 4; ++q) {
        const int32_t cb = C.ch[q];
        if (cb < 0) continue;
        const Cluster& cr = T.cl[blk(cb).r];
        const Cluster& cs = T.cl[blk(cb).s];
        add_dense(cb, cols(rows(Pv, cr.lo - r0, cr.hi - r0), cs.lo - s0, cs.hi - s0));
      }
    }
  }

  // exact product A B^T as low-rank terms inside the |r| x |r'| target
  void prod_terms(int32_t a, int32_t b, int64_t roff, int64_t coff, double alpha, std::vector<TermP>& out) {
    use(a);
    use(b);
    const Block& A = blk(a);
    const Block& B = blk(b);
    if (A.type == BT_LR) {
      const int32_t w = new_tmp(B.m, A.kcap);
      PV W = whole(w, B.m, A.kcap, NOSLOT, A.slot);
      hmul(b, V(a), W, 1.0);
      out.push_back(TermP{U(a), W, A.m, B.m, roff, coff, rk(a), 0, alpha});
    } else if (B.type == BT_LR) {
      const int32_t w = new_tmp(A.m, B.kcap);
      PV W = whole(w, A.m, B.kcap, NOSLOT, B.slot);
      hmul(a, V(b), W, 1.0);
      out.push_back(TermP{W, U(b), A.m, B.m, roff, coff, rk(b), 0, alpha});
    } else if (A.type == BT_DENSE && B.type == BT_DENSE) {
      out.push_back(TermP{D(a), D(b), A.m, B.m, roff, coff, dim(A.n, NOSLOT), 0, alpha});
    } else if (A.type == BT_DENSE) {
      const int32_t w = new_tmp(B.m, A.m);
      PV W = whole(w, B.m, A.m);
      hmul(b, T_(D(a)), W, 1.0);
      out.push_back(TermP{W, W, A.m, B.m, roff, coff, dim(A.m, NOSLOT), 1, alpha});
    } else if (B.type == BT_DENSE) {
      const int32_t w = new_tmp(A.m, B.m);
      PV W = whole(w, A.m, B.m);
      hmul(a, T_(D(b)), W, 1.0);
      out.push_back(TermP{W, W, A.m, B.m, roff, coff, dim(B.m, NOSLOT), 2, alpha});
    } else {
      const int64_t ar0 = rlo(a), br0 = rlo(b);
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
          for (int l = 0; l < 2; ++l) {
            const int32_t ai = A.ch[2 * i + l], bj = B.ch[2 * j + l];
            prod_terms(ai, bj, roff + rlo(ai) - ar0, coff + rlo(bj) - br0, alpha, out);
          }
    }
  }

  // C += alpha A B^T with truncation; A = (r, s), B = (r', s), C = (r, r')
  void mul_add(int32_t c, int32_t a, int32_t b, double alpha) {
    use(a);
    use(b);
    const Block& A = blk(a);
    const Block& B = blk(b);
    const Block& C = blk(c);
    if (A.type == BT_LR) {
      const int32_t w = new_tmp(B.m, A.kcap);
      PV W = whole(w, B.m, A.kcap, NOSLOT, A.slot);
      hmul(b, V(a), W, 1.0);
      add_lr(c, U(a), W, rk(a), alpha);
    } else if (B.type == BT_LR) {
      const int32_t w = new_tmp(A.m, B.kcap);
      PV W = whole(w, A.m, B.kcap, NOSLOT, B.slot);
      hmul(a, V(b), W, alpha);
      add_lr(c, W, U(b), rk(b), 1.0);
    } else if (A.type == BT_DENSE && B.type == BT_DENSE) {
      if (C.type == BT_DENSE) {
        gemm(D(c), D(a), T_(D(b)), dim(C.m, NOSLOT), dim(A.n, NOSLOT), dim(C.n, NOSLOT), alpha);
      } else {
        const int32_t p = new_tmp(A.m, B.m);
        PV Pv = whole(p, A.m, B.m);
        gemm(Pv, D(a), T_(D(b)), dim(A.m, NOSLOT), dim(A.n, NOSLOT), dim(B.m, NOSLOT), alpha);
        add_dense(c, Pv);
      }
    } else if (A.type == BT_DENSE) {
      const int32_t w = new_tmp(B.m, A.m);
      PV W = whole(w, B.m, A.m);
      hmul(b, T_(D(a)), W, alpha);
      add_dense(c, T_(W));
    } else if (B.type == BT_DENSE) {
      const int32_t w = new_tmp(A.m, B.m);
      PV W = whole(w, A.m, B.m);
      hmul(a, T_(D(b)), W, alpha);
      add_dense(c, W);
    } else if (C.type == BT_SUB) {
      const bool dg = C.diag;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          if (dg && j > i) continue;
          const int32_t cc = C.ch[2 * i + j];
          for (int l = 0; l < 2; ++l) mul_add(cc, A.ch[2 * i + l], B.ch[2 * j + l], alpha);
        }
    } else {
      std::vector<TermP> terms;
      prod_terms(a, b, 0, 0, alpha, terms);
      if (C.type == BT_LR) {
        add_terms(c, terms);
      } else {
        // not reachable for geometric trees (a dense target has a leaf
        // cluster); expand the terms into a temporary and add it
        const int32_t p = new_tmp(C.m, C.n);
        PV Pv = whole(p, C.m, C.n);
        for (const TermP& t : terms) {
          PV Y = cols(rows(Pv, t.roff, t.roff + t.urows), t.coff, t.coff + t.vrows);
          if (t.flags == 1)
            axpy(Y, T_(t.V), dim(t.urows, NOSLOT), dim(t.vrows, NOSLOT), t.alpha);
          else if (t.flags == 2)
            axpy(Y, t.U, dim(t.urows, NOSLOT), dim(t.vrows, NOSLOT), t.alpha);
          else
            gemm(Y, t.U, T_(t.V), dim(t.urows, NOSLOT), t.k, dim(t.vrows, NOSLOT), t.alpha);
        }
        add_dense(c, Pv);
      }
    }
  }

  // B := B L^-T
  void trsm_blk(int32_t l, int32_t b) {
    use(b);
    const Block& B = blk(b);
    if (B.type == BT_DENSE) {
      trsv(l, T_(D(b)));
    } else if (B.type == BT_LR) {
      trsv(l, V(b));
    } else {
      const Block& L = blk(l);
      for (int i = 0; i < 2; ++i) {
        const int32_t b0 = B.ch[2 * i], b1 = B.ch[2 * i + 1];
        trsm_blk(L.ch[0], b0);
        mul_add(b1, b0, L.ch[2], -1.0);
        trsm_blk(L.ch[3], b1);
      }
    }
  }

  void chol(int32_t m) {
    const Block& M = blk(m);
    if (M.type == BT_DENSE) {
      potrf(m);
      return;
    }
    chol(M.ch[0]);
    trsm_blk(M.ch[0], M.ch[2]);
    mul_add(M.ch[3], M.ch[2], M.ch[2], -1.0);
    chol(M.ch[3]);
  }

  // y += C x for the symmetric matrix stored as lower block triangle
  void symv(int32_t b, const PV& x, const PV& y) {
    const Block& B = blk(b);
    const Cluster& cr = T.cl[B.r];
    const Cluster& cs = T.cl[B.s];
    if (B.diag) {
      if (B.type == BT_DENSE) {
        gemm(rows(y, cr.lo, cr.hi), D(b), rows(x, cs.lo, cs.hi), dim(B.m, NOSLOT), dim(B.n, NOSLOT),
             dim(x.cols, NOSLOT), 1.0);
      } else {
        symv(B.ch[0], x, y);
        symv(B.ch[2], x, y);
        symv(B.ch[3], x, y);
      }
      return;
    }
    hmul(b, rows(x, cs.lo, cs.hi), rows(y, cr.lo, cr.hi), 1.0);
    hmul_t(b, rows(x, cr.lo, cr.hi), rows(y, cs.lo, cs.hi), 1.0);
  }

  // ---- finish: group ops into launches ----
  // Map the temporaries onto physical storage: a temporary lives from the
  // first wave that writes it to the last wave that reads it; storage is
  // reused first-fit once a temporary is dead.
  void allocate_temps() {
    std::vector<int32_t> order = tmp_objs;
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
      if (objs[a].birth != objs[b].birth) return objs[a].birth < objs[b].birth;
      return a < b;
    });
    std::map<int64_t, int64_t> freel;  // offset -> size
    // dataflow plans: the last temporary that occupied each stretch of the
    // buffer (start -> (end, temporary))
    std::map<int64_t, std::pair<int64_t, int32_t>> occupant;
    int64_t top = 0;
    using Live = std::pair<int32_t, int32_t>;  // (death, obj)
    std::priority_queue<Live, std::vector<Live>, std::greater<Live>> live;
    std::vector<int64_t> phys(objs.size(), -1);
    auto release = [&](int64_t off, int64_t sz) {
      auto it = freel.emplace(off, sz).first;
      auto nx = std::next(it);
      if (nx != freel.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        freel.erase(nx);
      }
      if (it != freel.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
          pv->second += it->second;
          freel.erase(it);
        }
      }
    };
    for (int32_t o : order) {
      Obj& ob = objs[o];
      if (ob.death < 0) {  // never used
        ob.birth = ob.death = 0;
      }
      while (!live.empty() && live.top().first < ob.birth) {
        const int32_t d = live.top().second;
        live.pop();
        release(phys[d], objs[d].size);
      }
      int64_t at = -1;
      for (auto it = freel.begin(); it != freel.end(); ++it)
        if (it->second >= ob.size) {
          at = it->first;
          const int64_t rest = it->second - ob.size;
          freel.erase(it);
          if (rest > 0) freel.emplace(at + ob.size, rest);
          break;
        }
      if (at < 0) {
        at = top;
        top += ob.size;
      }
      phys[o] = at;
      live.push(Live{ob.death, o});
      if (track) reuse_edges(occupant, at, at + ob.size, o);
    }
    P.tmp_doubles = top;
    // virtual -> physical: temporaries are contiguous in virtual space in
    // creation order
    std::vector<int64_t> vbase(tmp_objs.size());
    for (size_t i = 0; i < tmp_objs.size(); ++i) vbase[i] = objs[tmp_objs[i]].off;
    auto patch = [&](Mv& m) {
      if (m.buf != BUF_TMP) return;
      const size_t i = std::upper_bound(vbase.begin(), vbase.end(), m.off) - vbase.begin() - 1;
      const int32_t o = tmp_objs[i];
      m.off += phys[o] - objs[o].off;
    };
    for (OpGemm& g : P.gemm) {
      patch(g.Y);
      patch(g.A);
      if (g.B.buf >= 0) patch(g.B);
    }
    for (OpTrsm& t : P.trsm) {
      patch(t.L);
      patch(t.X);
    }
    for (TermD& t : P.terms) {
      if (!(t.flags & 1)) patch(t.U);
      if (!(t.flags & 2)) patch(t.V);
    }
    for (OpTrunc& t : P.trunc) {  // targets that are temporary partial sums
      patch(t.U);
      patch(t.V);
    }
    for (OpGemm& g : P.cgemm) {
      patch(g.Y);
      patch(g.A);
      if (g.B.buf >= 0) patch(g.B);
    }
    for (OpTrsm& t : P.ctrsm) {
      patch(t.L);
      patch(t.X);
    }
  }

  // Storage reuse in a dataflow plan: a temporary placed where earlier
  // (dead) temporaries lived must not be written before every op that
  // touched them is done -- in waves their lifetimes order them, without
  // barriers an edge must.  Edges go from the previous occupants' ops to the
  // new temporary's writers; the occupant map is updated to the new one.
  void reuse_edges(std::map<int64_t, std::pair<int64_t, int32_t>>& occ, int64_t a, int64_t b, int32_t o) {
    std::vector<int32_t> prev;
    auto it = occ.lower_bound(a);
    if (it != occ.begin()) {
      auto pv = std::prev(it);
      if (pv->second.first > a) it = pv;
    }
    std::vector<std::pair<int64_t, std::pair<int64_t, int32_t>>> keep;
    while (it != occ.end() && it->first < b) {
      const int64_t s0 = it->first, s1 = it->second.first;
      const int32_t t = it->second.second;
      prev.push_back(t);
      if (s0 < a) keep.push_back({s0, {a, t}});  // the part before [a, b) stays
      if (s1 > b) keep.push_back({b, {s1, t}});  // the part after [a, b) stays
      it = occ.erase(it);
    }
    for (auto& k : keep) occ[k.first] = k.second;
    occ[a] = {b, o};
    std::sort(prev.begin(), prev.end());
    prev.erase(std::unique(prev.begin(), prev.end()), prev.end());
    for (int32_t t : prev) {
      // the readers of the previous occupant: its writers precede them
      // already (read after write); a temporary never read: its writers
      std::vector<int64_t> last;
      for (int64_t q : objs[t].touch)
        if (!std::binary_search(objs[t].wr.begin(), objs[t].wr.end(), q)) last.push_back(q);
      if (last.empty()) last = objs[t].wr;
      for (int64_t w : objs[o].wr) {
        if ((int64_t)preds.size() <= w) preds.resize(w + 1);
        preds[w].insert(preds[w].end(), last.begin(), last.end());
      }
    }
  }

  void finish() {
    allocate_temps();
    if (track)  // the reuse edges may repeat producers
      for (auto& d : preds) {
        std::sort(d.begin(), d.end());
        d.erase(std::unique(d.begin(), d.end()), d.end());
      }
    P.nwaves = maxwave + 1;
    // stable order by (wave, type)
    std::vector<int64_t> order(seq.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
      if (seq[a].wave != seq[b].wave) return seq[a].wave < seq[b].wave;
      return seq[a].type < seq[b].type;
    });
    std::vector<OpGemm> g;
    std::vector<OpTrsm> t;
    std::vector<OpPotrf> p;
    std::vector<OpTrunc> u;
    std::vector<OpChain> ch;
    P.launches.clear();
    P.max_trunc_per_wave = 0;
    for (size_t i = 0; i < order.size(); ++i) {
      const Ref& r = seq[order[i]];
      int64_t pos = 0;
      switch (r.type) {
        case OP_GEMM: pos = (int64_t)g.size(); g.push_back(P.gemm[r.idx]); break;
        case OP_TRSM: pos = (int64_t)t.size(); t.push_back(P.trsm[r.idx]); break;
        case OP_POTRF: pos = (int64_t)p.size(); p.push_back(P.potrf[r.idx]); break;
        case OP_CHAIN: pos = (int64_t)ch.size(); ch.push_back(P.chain[r.idx]); break;
        default: pos = (int64_t)u.size(); u.push_back(P.trunc[r.idx]); break;  // OP_TRUNC, OP_TRUNC_BIG
      }
      if (!P.launches.empty() && P.launches.back().wave == r.wave && P.launches.back().type == r.type) {
        P.launches.back().count++;
      } else {
        P.launches.push_back(Launch{r.type, r.wave, pos, 1});
      }
      if (r.type == OP_TRUNC || r.type == OP_TRUNC_BIG) P.max_trunc_per_wave = std::max(P.max_trunc_per_wave, P.launches.back().count);
    }
    P.gemm.swap(g);
    P.trsm.swap(t);
    P.potrf.swap(p);
    P.trunc.swap(u);
    P.chain.swap(ch);
    if (track) build_flow(order);
  }

  // Dataflow form of a plan: the ops in wave order (flow), the number of
  // predecessors of each and its successors (CSR).  A group truncation
  // (OP_TRUNC_BIG) becomes kGroupParts consecutive entries: the op's
  // producers count towards part 0 only, all parts become ready together,
  // and part 0 alone signals the op's consumers (after the group's last
  // barrier, when every part is done).
  //
  // In a solve, a one-column product whose only consumer is the TRSM of the
  // same rows (the update of a diagonal block's right-hand side by its
  // neighbour, then its substitution) joins that TRSM: the TRSM's flow entry
  // names the product (FlowOp::group), which the same CTA runs first, and the
  // product's producers become the TRSM's.  One dependency hop less per
  // diagonal block; each op computes what it computes alone.
  static constexpr int kGroupParts = 8;
  void build_flow(const std::vector<int64_t>& order) {
    P.flow.clear();
    P.npred.clear();
    P.succ_off.clear();
    P.succ.clear();
    P.ngroups = 0;
    const int64_t N = (int64_t)order.size();
    // final array index of every op (the arrays are in wave order)
    std::vector<int64_t> aidx(N);
    {
      std::vector<int64_t> cnt_t(NOPTYPES, 0);
      for (int64_t i = 0; i < N; ++i) {
        const Ref& r = seq[order[i]];
        const int32_t arr = r.type == OP_TRUNC_BIG ? OP_TRUNC : r.type;  // both truncation kinds share one array
        aidx[order[i]] = cnt_t[arr]++;
      }
    }
    std::vector<int64_t> joined_into(N, -1);  // product -> the TRSM it joins
    std::vector<int64_t> pre_of(N, -1);       // TRSM -> the product it runs first
    if (P.trunc.empty()) {
      std::vector<int32_t> nsucc_op(N, 0);
      for (int64_t q = 0; q < (int64_t)preds.size(); ++q)
        for (int64_t d : preds[q]) nsucc_op[d] += 1;
      for (int64_t q = 0; q < (int64_t)preds.size(); ++q) {
        if (seq[q].type != OP_TRSM) continue;
        const OpTrsm& t = P.trsm[aidx[q]];
        for (int64_t d : preds[q]) {
          if (seq[d].type != OP_GEMM || nsucc_op[d] != 1 || joined_into[d] >= 0) continue;
          const OpGemm& g = P.gemm[aidx[d]];
          const bool one_col = g.c.slot < 0 && g.c.n == 1 && t.c.slot < 0 && t.c.n == 1;
          const bool same_rows = g.Y.buf == t.X.buf && g.Y.off == t.X.off && g.Y.rs == t.X.rs && g.m.slot < 0 &&
                                 g.m.n == t.n;
          const bool matrix_a = (g.A.buf == BUF_L || g.A.buf == BUF_C) && g.B.buf >= 0;
          if (one_col && same_rows && matrix_a) {
            joined_into[d] = q;
            pre_of[q] = d;
            break;
          }
        }
      }
    }
    std::vector<int64_t> pos_of(N, -1), parts_of(N, 0);  // seq index -> first flow index, parts
    for (int64_t i = 0; i < N; ++i) {
      const int64_t q = order[i];
      if (joined_into[q] >= 0) continue;
      const Ref& r = seq[q];
      pos_of[q] = (int64_t)P.flow.size();
      const int np = r.type == OP_TRUNC_BIG ? kGroupParts : 1;
      parts_of[q] = np;
      const int64_t grp = np > 1 ? P.ngroups++ : (pre_of[q] >= 0 ? aidx[pre_of[q]] : -1);
      for (int p = 0; p < np; ++p) P.flow.push_back(FlowOp{r.type, p, aidx[q], grp});
    }
    // the producers of a joined product become its TRSM's
    for (int64_t q = 0; q < N; ++q) {
      if (pre_of[q] < 0 || pre_of[q] >= (int64_t)preds.size()) continue;
      std::vector<int64_t>& d = preds[q];
      d.erase(std::remove(d.begin(), d.end(), pre_of[q]), d.end());
      d.insert(d.end(), preds[pre_of[q]].begin(), preds[pre_of[q]].end());
      std::sort(d.begin(), d.end());
      d.erase(std::unique(d.begin(), d.end()), d.end());
      preds[pre_of[q]].clear();
    }
    // a group's producers signal its first part only; the parts become ready
    // together (the kernel queues all of them when the first is released)
    const int64_t F = (int64_t)P.flow.size();
    std::vector<int64_t> nsucc(F, 0);
    P.npred.assign(F, 0);
    for (int64_t q = 0; q < N; ++q) {
      if (q >= (int64_t)preds.size() || pos_of[q] < 0) continue;
      for (int64_t d : preds[q]) {
        P.npred[pos_of[q]] += 1;
        nsucc[pos_of[d]] += 1;
      }
    }
    P.succ_off.assign(F + 1, 0);
    for (int64_t i = 0; i < F; ++i) P.succ_off[i + 1] = P.succ_off[i] + nsucc[i];
    P.succ.assign(P.succ_off[F], 0);
    std::vector<int64_t> fill(P.succ_off.begin(), P.succ_off.end() - 1);
    for (int64_t q = 0; q < N; ++q) {
      if (q >= (int64_t)preds.size() || pos_of[q] < 0) continue;
      for (int64_t d : preds[q]) P.succ[fill[pos_of[d]]++] = (int32_t)pos_of[q];
    }
    // the ops ready at the start, in flow order (a group with all its parts)
    P.ready0.clear();
    for (int64_t q = 0; q < N; ++q) {
      const int64_t f = pos_of[order[q]];
      if (f < 0 || P.npred[f] != 0) continue;
      for (int64_t p = 0; p < parts_of[order[q]]; ++p) P.ready0.push_back((int32_t)(f + p));
    }
  }
};

}  // namespace

void plan_cholesky(HTree& T, Plan& P, bool accumulate, bool flow) {
  P = Plan();
  Planner pl(T, P, BUF_L);
  pl.defer = accumulate;
  pl.track = flow;
  pl.chol(0);
  pl.flush_all();
  pl.finish();
}

// Forward (trans = 0) or backward (trans = 1) solve of the factor against
// the vector(s) in BUF_VEC at offset voff (n x ncols, ld n).
void plan_solve(HTree& T, Plan& P, int trans, int64_t voff, int64_t ncols, bool chains) {
  P = Plan();
  Planner pl(T, P, BUF_L);
  pl.chains = chains;
  pl.track = !chains;
  const int32_t v = pl.add_obj(BUF_VEC, voff, T.n);
  PV X = pl.whole(v, T.n, ncols);
  if (trans)
    pl.trsv_t(0, X);
  else
    pl.trsv(0, X);
  pl.finish();
}

// In-place product of the lower factor (trans = 0: X := L X) or of its
// transpose (trans = 1: X := L^T X) with the vector(s) in BUF_VEC at voff.
void plan_trmv(HTree& T, Plan& P, int trans, int64_t voff, int64_t ncols, bool chains) {
  P = Plan();
  Planner pl(T, P, BUF_L);
  pl.chains = chains;
  pl.track = !chains;
  const int32_t v = pl.add_obj(BUF_VEC, voff, T.n);
  PV X = pl.whole(v, T.n, ncols);
  if (trans)
    pl.trmv_t(0, X);
  else
    pl.trmv(0, X);
  pl.finish();
}

// y (BUF_VEC at yoff) += C x (BUF_VEC at xoff); C in BUF_C.
void plan_matvec(HTree& T, Plan& P, int64_t xoff, int64_t yoff, int64_t ncols) {
  P = Plan();
  Planner pl(T, P, BUF_C);
  pl.track = true;
  const int32_t xo = pl.add_obj(BUF_VEC, xoff, T.n);
  const int32_t yo = pl.add_obj(BUF_VEC, yoff, T.n);
  pl.symv(0, pl.whole(xo, T.n, ncols), pl.whole(yo, T.n, ncols));
  pl.finish();
}

// Recompression of every assembled low-rank block (in place, BUF_C).
void plan_recompress(HTree& T, Plan& P) {
  P = Plan();
  Planner pl(T, P, BUF_C);
  for (int32_t b : T.leaves)
    if (T.blk[b].type == BT_LR) pl.trunc(b, {}, 1);
  pl.finish();
}

// Every view of every op must stay inside its buffer at full capacity
// (static extents, ranks at their caps).  Returns an empty string or the
// first violation.
std::string validate_plan(const Plan& P, const int64_t* bufsize, int64_t nslots) {
  char msg[256];
  auto slot_ok = [&](const Dim& d) { return d.slot < (int32_t)nslots; };
  auto check = [&](const Mv& v, int64_t rows, int64_t cols, const char* what, int64_t i) -> bool {
    if (rows <= 0 || cols <= 0) return true;
    if (v.buf < 0 || v.buf >= NBUF || v.off < 0 || v.rs < 0 || v.cs < 0) {
      snprintf(msg, sizeof msg, "%s op %lld: bad view (buf %d off %lld)", what, (long long)i, v.buf,
               (long long)v.off);
      return false;
    }
    const int64_t last = v.off + (rows - 1) * v.rs + (cols - 1) * v.cs;
    if (last >= bufsize[v.buf]) {
      snprintf(msg, sizeof msg, "%s op %lld: view ends at %lld beyond buffer %d of %lld", what, (long long)i,
               (long long)last, v.buf, (long long)bufsize[v.buf]);
      return false;
    }
    return true;
  };
  for (size_t i = 0; i < P.gemm.size(); ++i) {
    const OpGemm& g = P.gemm[i];
    if (!slot_ok(g.m) || !slot_ok(g.k) || !slot_ok(g.c)) return "gemm: rank slot out of range";
    if (!check(g.Y, g.m.n, g.c.n, "gemm.Y", i)) return msg;
    if (g.B.buf == MV_IDENTITY) {
      if (!check(g.A, g.m.n, g.c.n, "axpy.X", i)) return msg;
    } else if (g.B.buf == MV_ONES) {
      if (!check(g.A, g.m.n, g.k.n, "gemm.A", i)) return msg;
    } else {
      if (!check(g.A, g.m.n, g.k.n, "gemm.A", i) || !check(g.B, g.k.n, g.c.n, "gemm.B", i)) return msg;
    }
  }
  for (size_t i = 0; i < P.trsm.size(); ++i) {
    const OpTrsm& t = P.trsm[i];
    if (t.n > 128) return "trsm: block larger than 128";
    if (!slot_ok(t.c)) return "trsm: rank slot out of range";
    if (!check(t.L, t.n, t.n, "trsm.L", i) || !check(t.X, t.n, t.c.n, "trsm.X", i)) return msg;
  }
  for (size_t i = 0; i < P.cgemm.size(); ++i) {
    const OpGemm& g = P.cgemm[i];
    if (!slot_ok(g.m) || !slot_ok(g.k) || !slot_ok(g.c)) return "chain gemm: rank slot out of range";
    if (!check(g.Y, g.m.n, g.c.n, "chain gemm.Y", i)) return msg;
    if (g.B.buf == MV_IDENTITY) {
      if (!check(g.A, g.m.n, g.c.n, "chain axpy.X", i)) return msg;
    } else if (g.B.buf == MV_ONES) {
      if (!check(g.A, g.m.n, g.k.n, "chain gemm.A", i)) return msg;
    } else {
      if (!check(g.A, g.m.n, g.k.n, "chain gemm.A", i) || !check(g.B, g.k.n, g.c.n, "chain gemm.B", i)) return msg;
    }
  }
  for (size_t i = 0; i < P.ctrsm.size(); ++i) {
    const OpTrsm& t = P.ctrsm[i];
    if (t.n > 128) return "chain trsm: block larger than 128";
    if (!slot_ok(t.c)) return "chain trsm: rank slot out of range";
    if (!check(t.L, t.n, t.n, "chain trsm.L", i) || !check(t.X, t.n, t.c.n, "chain trsm.X", i)) return msg;
  }
  for (const OpChain& c : P.chain) {
    if (c.item0 < 0 || c.nitems <= 0 || c.item0 + c.nitems > (int64_t)P.citems.size()) return "chain: item range";
    for (int64_t q = c.item0; q < c.item0 + c.nitems; ++q) {
      const ChainItem& it = P.citems[q];
      if (it.type == OP_TRSM) {
        if (it.idx < 0 || it.idx >= (int64_t)P.ctrsm.size()) return "chain: trsm index";
      } else if (it.type == OP_GEMM) {
        if (it.idx < 0 || it.idx >= (int64_t)P.cgemm.size()) return "chain: gemm index";
      } else {
        return "chain: item type";
      }
    }
  }
  for (size_t i = 0; i < P.potrf.size(); ++i) {
    const OpPotrf& t = P.potrf[i];
    if (t.n > 128) return "potrf: block larger than 128";
    if (!check(t.A, t.n, t.n, "potrf.A", i)) return msg;
  }
  for (size_t i = 0; i < P.trunc.size(); ++i) {
    const OpTrunc& t = P.trunc[i];
    if (t.kcap > 128) return "trunc: rank capacity above 128";
    if (t.slot < 0 || t.slot >= nslots) return "trunc: rank slot out of range";
    if (!check(t.U, t.m, t.kcap, "trunc.U", i) || !check(t.V, t.n, t.kcap, "trunc.V", i)) return msg;
    if (t.term0 < 0 || t.term0 + t.nterms > (int64_t)P.terms.size()) return "trunc: term range";
    for (int q = 0; q < t.nterms; ++q) {
      const TermD& d = P.terms[t.term0 + q];
      if (d.roff < 0 || d.coff < 0 || d.roff + d.urows > t.m || d.coff + d.vrows > t.n) return "term: placement";
      const int64_t k = (d.flags & 1) ? d.urows : (d.flags & 2) ? d.vrows : d.k.n;
      if (k > 128) return "term: more than 128 columns";
      if (!slot_ok(d.k)) return "term: rank slot out of range";
      if (!(d.flags & 1) && !check(d.U, d.urows, k, "term.U", t.term0 + q)) return msg;
      if (!(d.flags & 2) && !check(d.V, d.vrows, k, "term.V", t.term0 + q)) return msg;
    }
  }
  return std::string();
}

}  // namespace hlc
