// selftest.cpp -- host-only check of the planner's dataflow programs (no
// device involved).  A synthetic cluster tree and block-cluster tree take
// the place of the device-built trees: midpoint bisection of the index
// interval [0, n), with the clusters' boxes either the intervals themselves
// (1-D) or the tight boxes of the points of a square grid numbered in Morton
// order (2-D: the structure of uniformly spread points), and admissibility
// min(diam) <= eta * dist between the boxes.  The factorisation (also with
// accumulated updates), solve, matvec and factor-product plans are built
// from them exactly as for a real tree, and the checks are the invariants
// the dependency-driven kernels rely on:
//   * every plan passes validate_plan (views inside their buffers, rank
//     slots inside the rank array);
//   * every dependency edge points forward in flow order (the solve kernel
//     takes ops in that order and needs every producer to come first), and
//     the predecessor counts equal the edges into each op;
//   * a group truncation is TR_CL consecutive parts of one op, its producers
//     and consumers attached to part 0 only;
//   * the ready list is exactly the ops without producers in flow order,
//     each group with all its parts;
//   * in a solve, a product joined into a TRSM is a one-column product into
//     the TRSM's own rows, and every product of the plan runs exactly once
//     (as a flow entry or inside its TRSM);
//   * a discrete-event model of the factorisation kernel's ready-queue
//     protocol (G CTAs, seeded op durations, a group's parts waiting for
//     each other) runs every op after all of its producers and finishes.

#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <queue>
#include <random>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/hlc.h"
#include "engine.h"

namespace hlc {
namespace {

constexpr int kParts = 8;  // parts of a group truncation (the kernel's cluster size)

// Clusters: midpoint bisection of index intervals, breadth-first like the
// device build (children of a cluster are consecutive).
// grid point of Morton index i: x from the even bits, y from the odd ones
inline int64_t morton_compact(uint64_t v) {
  uint64_t x = v & 0x5555555555555555ull;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
  x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
  x = (x | (x >> 16)) & 0x00000000ffffffffull;
  return (int64_t)x;
}

void synth_clusters(HTree& T, int64_t n, int leaf, int geometry) {
  T.cl.clear();
  Cluster root{};
  root.lo = 0;
  root.hi = n;
  root.child[0] = root.child[1] = -1;
  root.level = 0;
  T.cl.push_back(root);
  for (size_t c = 0; c < T.cl.size(); ++c) {
    if (T.cl[c].size() <= leaf) continue;
    const int64_t mid = T.cl[c].lo + T.cl[c].size() / 2;
    Cluster a{}, b{};
    a.lo = T.cl[c].lo;
    a.hi = mid;
    b.lo = mid;
    b.hi = T.cl[c].hi;
    a.child[0] = a.child[1] = b.child[0] = b.child[1] = -1;
    a.level = b.level = T.cl[c].level + 1;
    const int32_t first = (int32_t)T.cl.size();
    T.cl[c].child[0] = first;
    T.cl[c].child[1] = first + 1;
    T.cl.push_back(a);
    T.cl.push_back(b);
  }
  T.depth = 0;
  for (int64_t i = 0; i < (int64_t)T.cl.size(); ++i) {
    Cluster& C = T.cl[i];
    if (geometry == 0) {
      C.bmin[0] = (double)C.lo;
      C.bmax[0] = (double)C.hi - 1.0;
      C.bmin[1] = C.bmax[1] = 0.0;
    } else {
      C.bmin[0] = C.bmin[1] = 1e300;
      C.bmax[0] = C.bmax[1] = -1e300;
      for (int64_t p = C.lo; p < C.hi; ++p) {
        const double x = (double)morton_compact((uint64_t)p), y = (double)morton_compact((uint64_t)p >> 1);
        C.bmin[0] = std::min(C.bmin[0], x);
        C.bmax[0] = std::max(C.bmax[0], x);
        C.bmin[1] = std::min(C.bmin[1], y);
        C.bmax[1] = std::max(C.bmax[1], y);
      }
    }
    T.depth = std::max(T.depth, C.level);
  }
}

double box_diam(const Cluster& c) {
  const double a = c.bmax[0] - c.bmin[0], b = c.bmax[1] - c.bmin[1];
  return std::sqrt(a * a + b * b);
}

double box_dist(const Cluster& r, const Cluster& s) {
  double d2 = 0.0;
  for (int k = 0; k < 2; ++k) {
    const double g = std::max(0.0, std::max(r.bmin[k] - s.bmax[k], s.bmin[k] - r.bmax[k]));
    d2 += g * g;
  }
  return std::sqrt(d2);
}

// Block-cluster tree on the lower triangle, breadth-first: a diagonal block
// has children (0: r0 x r0, 2: r1 x r0, 3: r1 x r1), an off-diagonal one the
// four pairs of children.
void synth_blocks(HTree& T, double eta) {
  T.blk.clear();
  auto make = [&](int32_t r, int32_t s) {
    Block B{};
    B.r = r;
    B.s = s;
    for (int q = 0; q < 4; ++q) B.ch[q] = -1;
    B.m = T.cl[r].size();
    B.n = T.cl[s].size();
    B.slot = -1;
    B.leaf_index = -1;
    return B;
  };
  T.blk.push_back(make(0, 0));
  for (size_t b = 0; b < T.blk.size(); ++b) {
    const int32_t r = T.blk[b].r, s = T.blk[b].s;
    const Cluster R = T.cl[r], S = T.cl[s];
    const bool lr = R.child[0] < 0, ls = S.child[0] < 0;
    if (r == s) {
      T.blk[b].diag = 1;
      if (lr) {
        T.blk[b].type = BT_DENSE;
        continue;
      }
      T.blk[b].type = BT_SUB;
      const int32_t f = (int32_t)T.blk.size();
      T.blk[b].ch[0] = f;
      T.blk[b].ch[2] = f + 1;
      T.blk[b].ch[3] = f + 2;
      T.blk.push_back(make(R.child[0], R.child[0]));
      T.blk.push_back(make(R.child[1], R.child[0]));
      T.blk.push_back(make(R.child[1], R.child[1]));
      continue;
    }
    T.blk[b].diag = 0;
    const double d = box_dist(R, S);
    const bool adm = d > 0.0 && std::min(box_diam(R), box_diam(S)) <= eta * d;
    if (adm) {
      T.blk[b].type = BT_LR;
    } else if (lr || ls) {
      T.blk[b].type = BT_DENSE;
    } else {
      T.blk[b].type = BT_SUB;
      const int32_t f = (int32_t)T.blk.size();
      for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q) {
          T.blk[b].ch[2 * p + q] = f + 2 * p + q;
          T.blk.push_back(make(R.child[p], S.child[q]));
        }
    }
  }
}

struct Check {
  std::string err;
  void fail(const std::string& what) {
    if (err.empty()) err = what;
  }
};

bool same_view(const Mv& a, const Mv& b) { return a.buf == b.buf && a.off == b.off && a.rs == b.rs; }

// FNV-1a over the bytes of a plan's op program (op descriptors, terms,
// launches and the dataflow arrays): equal hashes mean the same program
template <class V>
void hash_vec(uint64_t& h, const V& v) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(v.data());
  const size_t nb = v.size() * sizeof(typename V::value_type);
  for (size_t i = 0; i < nb; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  h ^= (uint64_t)v.size();
  h *= 1099511628211ull;
}

uint64_t plan_hash(const Plan& P) {
  uint64_t h = 1469598103934665603ull;
  hash_vec(h, P.gemm);
  hash_vec(h, P.trsm);
  hash_vec(h, P.potrf);
  hash_vec(h, P.trunc);
  hash_vec(h, P.terms);
  hash_vec(h, P.launches);
  hash_vec(h, P.flow);
  hash_vec(h, P.npred);
  hash_vec(h, P.succ_off);
  hash_vec(h, P.succ);
  hash_vec(h, P.ready0);
  h ^= (uint64_t)P.tmp_doubles * 31 + (uint64_t)P.tmp_slots;
  return h;
}

// The flow invariants of one plan; returns its number of edges.
int64_t check_flow(const Plan& P, const char* name, bool solve, Check& ck, int64_t* joins) {
  const int64_t F = (int64_t)P.flow.size();
  char buf[256];
  if ((int64_t)P.npred.size() != F || (int64_t)P.succ_off.size() != F + 1) {
    ck.fail(std::string(name) + ": flow arrays of inconsistent length");
    return 0;
  }
  std::vector<int32_t> indeg(F, 0);
  for (int64_t i = 0; i < F; ++i)
    for (int64_t e = P.succ_off[i]; e < P.succ_off[i + 1]; ++e) {
      const int64_t j = P.succ[e];
      if (j <= i || j >= F) {
        snprintf(buf, sizeof(buf), "%s: edge %lld -> %lld does not point forward", name, (long long)i, (long long)j);
        ck.fail(buf);
        return 0;
      }
      indeg[j] += 1;
    }
  for (int64_t i = 0; i < F; ++i)
    if (indeg[i] != P.npred[i]) {
      snprintf(buf, sizeof(buf), "%s: op %lld counts %d producers, has %d edges in", name, (long long)i, P.npred[i],
               indeg[i]);
      ck.fail(buf);
      return 0;
    }
  // group truncations: consecutive parts, edges on part 0 only
  for (int64_t i = 0; i < F; ++i) {
    const FlowOp& f = P.flow[i];
    if (f.type != OP_TRUNC_BIG) continue;
    if (f.part == 0) {
      for (int p = 1; p < kParts; ++p) {
        if (i + p >= F || P.flow[i + p].type != OP_TRUNC_BIG || P.flow[i + p].part != p ||
            P.flow[i + p].idx != f.idx || P.flow[i + p].group != f.group) {
          ck.fail(std::string(name) + ": a group's parts are not consecutive");
          return 0;
        }
      }
    } else if (P.npred[i] != 0 || P.succ_off[i + 1] != P.succ_off[i]) {
      ck.fail(std::string(name) + ": a group part other than the first has edges");
      return 0;
    }
  }
  // the ready list
  std::vector<int32_t> r0;
  for (int64_t i = 0; i < F; ++i) {
    const FlowOp& f = P.flow[i];
    if (f.type == OP_TRUNC_BIG && f.part != 0) continue;
    if (P.npred[i] != 0) continue;
    const int np = f.type == OP_TRUNC_BIG ? kParts : 1;
    for (int p = 0; p < np; ++p) r0.push_back((int32_t)(i + p));
  }
  if (r0 != P.ready0) ck.fail(std::string(name) + ": the ready list is not the ops without producers");
  // joined products
  *joins = 0;
  std::vector<int32_t> runs(P.gemm.size(), 0);
  for (int64_t i = 0; i < F; ++i) {
    const FlowOp& f = P.flow[i];
    if (f.type == OP_GEMM) runs[f.idx] += 1;
    if (f.type != OP_TRSM || f.group < 0) continue;
    if (!solve) {
      ck.fail(std::string(name) + ": a TRSM of the factorisation names a product");
      return 0;
    }
    const OpTrsm& t = P.trsm[f.idx];
    const OpGemm& g = P.gemm[f.group];
    if (!(g.c.slot < 0 && g.c.n == 1 && g.m.slot < 0 && g.m.n == t.n && same_view(g.Y, t.X))) {
      ck.fail(std::string(name) + ": a joined product does not write its TRSM's rows");
      return 0;
    }
    runs[f.group] += 1;
    *joins += 1;
  }
  for (size_t g = 0; g < runs.size(); ++g)
    if (runs[g] != 1) {
      snprintf(buf, sizeof(buf), "%s: product %lld runs %d times", name, (long long)g, runs[g]);
      ck.fail(buf);
      return 0;
    }
  return P.succ_off[F];
}

// Discrete-event model of the factorisation kernel's scheduling: ctas CTAs;
// a free CTA claims the next queue slot and waits for it to be filled; a
// single-CTA op runs for its duration; the parts of a group wait until all of
// them have started and finish together; the CTA completing a consumer's
// count appends it (a group with all its parts).  Returns the makespan in
// model units, or -1 after recording a violation.
double simulate_queue(const Plan& P, int ctas, uint64_t seed, Check& ck) {
  const int64_t F = (int64_t)P.flow.size();
  std::vector<int32_t> slot(F, -1);
  int64_t filled = 0;
  for (int32_t v : P.ready0) slot[filled++] = v;
  std::vector<int32_t> count(F, 0), started(F, 0), done(F, 0);
  std::vector<int32_t> group_arrived(P.ngroups > 0 ? P.ngroups : 1, 0);
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> dur(1.0, 10.0);
  int64_t head = 0, finished = 0;
  // events: (time, kind, cta, op); kind 0 = op finished
  using Ev = std::tuple<double, int, int, int64_t>;
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> ev;
  std::vector<int32_t> waiter(F, -1);  // the CTA that claimed a slot not filled yet
  std::vector<std::vector<std::pair<int, int64_t>>> group_wait(group_arrived.size());
  double now = 0.0;
  std::function<void(int)> claim;
  auto start = [&](int c, int64_t op) {
    const FlowOp& f = P.flow[op];
    const int64_t head_op = f.type == OP_TRUNC_BIG ? op - f.part : op;
    if (count[head_op] != P.npred[head_op]) {
      ck.fail("queue model: an op started before its producers finished");
      return;
    }
    started[op] = 1;
    if (f.type == OP_TRUNC_BIG) {
      group_wait[f.group].push_back({c, op});
      if (++group_arrived[f.group] == kParts) {
        const double d = dur(rng) * 4.0;
        for (auto& w : group_wait[f.group]) ev.push(Ev{now + d, 0, w.first, w.second});
      }
      return;
    }
    ev.push(Ev{now + dur(rng), 0, c, op});
  };
  claim = [&](int c) {
    if (head >= F) return;
    const int64_t s = head++;
    if (s < filled) {
      start(c, slot[s]);
    } else {
      waiter[s] = c;
    }
  };
  auto push = [&](int32_t v) {
    const int np = P.flow[v].type == OP_TRUNC_BIG ? kParts : 1;
    for (int p = 0; p < np; ++p) {
      const int64_t s = filled++;
      slot[s] = v + p;
      if (waiter[s] >= 0) start(waiter[s], slot[s]);
    }
  };
  for (int c = 0; c < ctas; ++c) claim(c);
  while (!ev.empty() && ck.err.empty()) {
    const Ev e = ev.top();
    ev.pop();
    now = std::get<0>(e);
    const int c = std::get<2>(e);
    const int64_t op = std::get<3>(e);
    done[op] = 1;
    finished += 1;
    const FlowOp& f = P.flow[op];
    if (!(f.type == OP_TRUNC_BIG && f.part != 0))
      for (int64_t q = P.succ_off[op]; q < P.succ_off[op + 1]; ++q) {
        const int32_t v = P.succ[q];
        if (++count[v] == P.npred[v]) push(v);
      }
    claim(c);
  }
  if (!ck.err.empty()) return -1.0;
  if (finished != F) {
    char buf[160];
    snprintf(buf, sizeof(buf), "queue model: stopped with %lld of %lld ops done", (long long)finished, (long long)F);
    ck.fail(buf);
    return -1.0;
  }
  return now;
}

}  // namespace
}  // namespace hlc

extern "C" int hlc_selftest_plans(int64_t n, int leaf, double eta, int geometry, int kmax, int ctas, uint64_t seed,
                                  int64_t* stats, int nstats, char* msg, int msglen) {
  using namespace hlc;
  if (n < 2 || n > ((int64_t)1 << 26) || leaf < 1 || leaf > 128 || !(eta > 0.0) || (geometry != 0 && geometry != 1) ||
      kmax < 1 || kmax > 128 || ctas <= kParts || (nstats > 0 && !stats) || (msglen > 0 && !msg))
    return HLC_ERR_ARG;
  Check ck;
  int64_t st[15] = {0};
  try {
    HTree T;
    T.n = n;
    T.leaf = leaf;
    T.eta = eta;
    T.eps = 1e-6;
    synth_clusters(T, n, leaf, geometry);
    synth_blocks(T, eta);
    collect_leaf_list(T);
    layout(T, kmax);
    Plan chol, fwd, bwd, mv;
    const auto t0 = std::chrono::steady_clock::now();
    plan_cholesky(T, chol, false, true);
    st[12] = (int64_t)std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    plan_solve(T, fwd, 0, 0, 1, false);
    plan_solve(T, bwd, 1, 0, 1, false);
    plan_matvec(T, mv, n, 2 * n, 1);
    // also checked, not counted in the stats: the factorisation with
    // accumulated updates and the products with the factor and its transpose
    Plan chol_acc, lmv, lmvt;
    plan_cholesky(T, chol_acc, true, true);
    plan_trmv(T, lmv, 0, 0, 1, false);
    plan_trmv(T, lmvt, 1, 0, 1, false);
    const struct {
      const Plan* P;
      const char* name;
      bool solve;
    } plans[7] = {{&chol, "factorisation", false},        {&fwd, "forward solve", true},
                  {&bwd, "backward solve", true},         {&mv, "matvec", true},
                  {&chol_acc, "accumulated factorisation", false}, {&lmv, "product with L", true},
                  {&lmvt, "product with L^T", true}};
    for (int k = 0; k < 7 && ck.err.empty(); ++k) {
      const Plan& P = *plans[k].P;
      int64_t bufsize[NBUF] = {0, 0, 0, 0};
      bufsize[BUF_L] = T.arena_doubles;
      bufsize[BUF_C] = T.arena_doubles;
      bufsize[BUF_TMP] = P.tmp_doubles;
      bufsize[BUF_VEC] = 6 * n;
      const std::string v = validate_plan(P, bufsize, (int64_t)T.nslots + P.tmp_slots);
      if (!v.empty()) ck.fail(std::string(plans[k].name) + ": " + v);
      int64_t joins = 0;
      const int64_t edges = check_flow(P, plans[k].name, plans[k].solve, ck, &joins);
      if (k == 0) {
        st[0] = (int64_t)P.flow.size();
        st[1] = edges;
        st[2] = P.ngroups;
        st[3] = (int64_t)P.ready0.size();
        st[13] = (int64_t)plan_hash(P);
      } else if (k == 1) {
        st[4] = (int64_t)P.flow.size();
        st[5] = joins;
      } else if (k == 2) {
        st[6] = (int64_t)P.flow.size();
        st[7] = joins;
      } else if (k == 3) {
        st[8] = (int64_t)P.flow.size();
      }
      if (k > 0 && k < 4) st[14] = (int64_t)(((uint64_t)st[14] * 1099511628211ull) ^ plan_hash(P));
    }
    if (ck.err.empty()) simulate_queue(chol_acc, ctas, seed + 1, ck);
    if (ck.err.empty()) {
      const double span = simulate_queue(chol, ctas, seed, ck);
      st[9] = (int64_t)span;
      st[10] = (int64_t)T.leaves.size();
      st[11] = (int64_t)T.nslots;
    }
  } catch (const std::bad_alloc&) {
    return HLC_ERR_OOM;
  }
  for (int i = 0; i < nstats && i < 15; ++i) stats[i] = st[i];
  if (msglen > 0) {
    strncpy(msg, ck.err.c_str(), (size_t)msglen - 1);
    msg[msglen - 1] = '\0';
  }
  return ck.err.empty() ? HLC_OK : HLC_ERR_STATE;
}
