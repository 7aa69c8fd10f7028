// api.cu -- the C ABI (include/hlc.h): contexts, trees, H-matrices and the
// likelihood evaluation, executing the planner's op programs on one stream.

#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <stdexcept>
#include <vector>

#include "engine.h"
#include "kernels.h"
#include "matern.cuh"
#include "serve.h"

using namespace hlc;

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct hlc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  double* d_part = nullptr;   // reduction partials
  double* d_scalar = nullptr; // 8 scalars
  int* d_status = nullptr;    // [0] code, [1] detail
  double* d_scratch = nullptr;
  cudaEvent_t ev[4];
  hlc::Serve* serve = nullptr;
  // measurement
  double* d_flops = nullptr;  // NOPTYPES algorithmic flop counters
  unsigned long long* d_phase = nullptr;  // truncation phase cycles (HLC_PHASES=1)
  GridBar* d_gridbar = nullptr;           // barrier state of the persistent solve kernel
  bool persistent = true;                 // off in serve slots (several contexts share the SMs)
  bool profiling = false;
  double launches = 0;
  double op_launches[NOPTYPES] = {};
  double persistent_launches = 0;
  // timed runs of the persistent kernel still to be read (grid tuning)
  struct TuneRec {
    const Plan* P;
    int cand;
    cudaEvent_t e0, e1;
  };
  std::vector<TuneRec> tune_pending;
  std::vector<cudaEvent_t> tune_free;
  // side streams for the independent launches of one wave (POTRF, TRSM,
  // GEMM), forked from and joined back into the context's stream
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join[3] = {nullptr, nullptr, nullptr};
  bool side_ok = false;
  double op_ms[NOPTYPES] = {};
  std::vector<cudaEvent_t> evpool;
  struct Pending {
    int type;
    int ev;
  };
  std::vector<Pending> pending;
};

struct hlc_hmat {
  hlc_tree* t = nullptr;
  int which = 0;  // 0: C~, 1: L~
  double* arena = nullptr;
  int* ranks = nullptr;
  bool valid = false;
};

struct hlc_tree {
  hlc_ctx* ctx = nullptr;
  hlc_params p{};
  HTree T;
  int32_t* d_perm = nullptr;
  double* d_px = nullptr;
  double* d_py = nullptr;
  DenseAsm* d_dense = nullptr;
  LrAsm* d_lr = nullptr;
  int64_t* d_diag_off = nullptr;
  int32_t* d_diag_dim = nullptr;
  int64_t ndiag = 0;
  double* d_knu = nullptr;  // 2 * KNU_NODES node table
  std::vector<double> h_knu;
  Plan chol, fwd, bwd, mv, recomp;
  Plan lmv, lmvt;  // products with the lower factor and its transpose
  bool chol_ready = false, solve_ready = false, lmv_ready = false;
  double* d_tmp = nullptr;
  int64_t tmp_cap = 0;
  double* d_vec = nullptr;  // 6 n: W0 | X | Y | Z | XS | R
  hlc_hmat* wsC = nullptr;
  hlc_hmat* wsL = nullptr;
};

namespace {

// largest n for the diagnostics that evaluate the exact covariance (O(n^2)
// kernel evaluations per product)
constexpr int64_t kDiagExactMax = 131072;

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HLC_OK;
  if (e == cudaErrorMemoryAllocation) return HLC_ERR_OOM;
  return HLC_ERR_CUDA;
}

#define CK(x)                             \
  do {                                    \
    cudaError_t e_ = (x);                 \
    if (e_ != cudaSuccess) {              \
      return cuda_status(e_);             \
    }                                     \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
int upload(T** d, const std::vector<T>& h) {
  *d = nullptr;
  if (h.empty()) return HLC_OK;
  CK(cudaMalloc(d, h.size() * sizeof(T)));
  CK(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return HLC_OK;
}

// Wave table of a plan made of TRSM, GEMM and chain ops only (solves,
// products with the factor, matvec).
void build_waves(Plan& P) {
  P.waves.clear();
  for (const Launch& L : P.launches)
    if (L.type != OP_TRSM && L.type != OP_GEMM && L.type != OP_CHAIN) return;
  int32_t cur = -1;
  for (const Launch& L : P.launches) {
    if (L.wave != cur) {
      P.waves.push_back(WaveRange{0, 0, 0, 0, 0, 0});
      cur = L.wave;
    }
    WaveRange& w = P.waves.back();
    if (L.type == OP_TRSM) {
      w.trsm0 = L.first;
      w.ntrsm = L.count;
    } else if (L.type == OP_GEMM) {
      w.gemm0 = L.first;
      w.ngemm = L.count;
    } else {
      w.chain0 = L.first;
      w.nchain = L.count;
    }
  }
}

int upload_plan(Plan& P) {
  int st;
  P.checked = true;
  build_waves(P);
  if ((st = upload(&P.d_waves, P.waves))) return st;
  if ((st = upload(&P.d_gemm, P.gemm))) return st;
  if ((st = upload(&P.d_trsm, P.trsm))) return st;
  if ((st = upload(&P.d_potrf, P.potrf))) return st;
  if ((st = upload(&P.d_trunc, P.trunc))) return st;
  if ((st = upload(&P.d_terms, P.terms))) return st;
  if ((st = upload(&P.d_flow, P.flow))) return st;
  if ((st = upload(&P.d_npred, P.npred))) return st;
  if ((st = upload(&P.d_succ_off, P.succ_off))) return st;
  if ((st = upload(&P.d_succ, P.succ))) return st;
  if (!P.flow.empty()) CK(cudaMalloc(&P.d_count, P.flow.size() * sizeof(int32_t)));
  if (P.ngroups > 0) CK(cudaMalloc(&P.d_groups, P.ngroups * sizeof(TrGroup)));
  // the ready queue serves the factorisation (the plan with truncations)
  if (!P.flow.empty() && !P.trunc.empty()) {
    if ((st = upload(&P.d_ready0, P.ready0))) return st;
    CK(cudaMalloc(&P.d_ready, P.flow.size() * sizeof(int32_t)));
  }
  if ((st = upload(&P.d_chain, P.chain))) return st;
  if ((st = upload(&P.d_citems, P.citems))) return st;
  if ((st = upload(&P.d_ctrsm, P.ctrsm))) return st;
  if ((st = upload(&P.d_cgemm, P.cgemm))) return st;
  return HLC_OK;
}

void free_plan(Plan& P) {
  if (P.graph) cudaGraphExecDestroy(P.graph);
  P.graph = nullptr;
  cudaFree(P.d_waves);
  P.d_waves = nullptr;
  cudaFree(P.d_gemm);
  cudaFree(P.d_trsm);
  cudaFree(P.d_potrf);
  cudaFree(P.d_trunc);
  cudaFree(P.d_terms);
  cudaFree(P.d_flow);
  cudaFree(P.d_npred);
  cudaFree(P.d_succ_off);
  cudaFree(P.d_succ);
  cudaFree(P.d_count);
  cudaFree(P.d_groups);
  cudaFree(P.d_ready0);
  cudaFree(P.d_ready);
  P.d_ready0 = nullptr;
  P.d_ready = nullptr;
  P.d_groups = nullptr;
  P.d_flow = nullptr;
  P.d_npred = nullptr;
  P.d_succ_off = nullptr;
  P.d_succ = nullptr;
  P.d_count = nullptr;
  cudaFree(P.d_chain);
  cudaFree(P.d_citems);
  cudaFree(P.d_ctrsm);
  cudaFree(P.d_cgemm);
  P.d_chain = nullptr;
  P.d_citems = nullptr;
  P.d_ctrsm = nullptr;
  P.d_cgemm = nullptr;
  P.d_gemm = nullptr;
  P.d_trsm = nullptr;
  P.d_potrf = nullptr;
  P.d_trunc = nullptr;
  P.d_terms = nullptr;
}

int ensure_tmp(hlc_tree* t, int64_t doubles) {
  if (doubles <= t->tmp_cap) return HLC_OK;
  cudaFree(t->d_tmp);
  t->d_tmp = nullptr;
  t->tmp_cap = 0;
  CK(cudaMalloc(&t->d_tmp, std::max<int64_t>(doubles, 4) * sizeof(double)));
  t->tmp_cap = doubles;
  return HLC_OK;
}

// Optional per-launch timing (environment HLC_PROFILE=1): every launch is
// synchronised and timed on the host; totals per op type and the slowest
// launches are printed when the process exits.
struct Prof {
  bool on = false;
  double ms[NOPTYPES] = {};
  int64_t launches[NOPTYPES] = {}, ops[NOPTYPES] = {};
  struct Slow {
    double ms;
    int type, wave;
    int64_t count;
  };
  std::vector<Slow> slow;
  Prof() { on = getenv("HLC_PROFILE") && getenv("HLC_PROFILE")[0] == '1'; }
  ~Prof() {
    if (!on) return;
    static const char* nm[NOPTYPES] = {"potrf", "trsm", "gemm", "trunc", "truncC", "chain"};
    for (int i = 0; i < NOPTYPES; ++i)
      fprintf(stderr, "hlc-profile %-6s launches %9lld ops %11lld  %10.2f ms\n", nm[i], (long long)launches[i],
              (long long)ops[i], ms[i]);
    std::sort(slow.begin(), slow.end(), [](const Slow& a, const Slow& b) { return a.ms > b.ms; });
    for (size_t i = 0; i < slow.size() && i < 12; ++i)
      fprintf(stderr, "hlc-profile slow %-6s wave %6d ops %7lld %8.3f ms\n", nm[slow[i].type], slow[i].wave,
              (long long)slow[i].count, slow[i].ms);
  }
} g_prof;

bool same_bases(const Bases& a, const Bases& b) { return std::memcmp(&a, &b, sizeof(Bases)) == 0; }

bool graphs_enabled() {
  static const bool on = !(getenv("HLC_GRAPHS") && getenv("HLC_GRAPHS")[0] == '0');
  return on;
}

void run_plan_launches(hlc_tree* t, const Plan& P, const Bases& B, cudaStream_t st, bool count);
void run_launch(hlc_tree* t, const Plan& P, const Bases& B, const Launch& L, int md, cudaStream_t st, bool count);

// CTAs per SM tried by the grid tuning of the persistent kernel (capped at
// what fits on an SM when launched)
constexpr int kTuneCandidates[3] = {1, 2, 4};

// solves and products with the factor as chains of small diagonal blocks
// (HLC_CHAINS=1); off by default: one CTA running a chain's ops one after
// another waits out each op's memory latency in turn, which measured slower
// than the waves of independent ops (17.2 s against 11.2 s of solves per
// evaluation at n = 524,288)
bool chains_enabled() {
  static const bool on = getenv("HLC_CHAINS") && getenv("HLC_CHAINS")[0] == '1';
  return on;
}

// The factorisation runs as one dependency-driven launch (k_factor) unless
// HLC_FACTOR_FLOW=0, which replays its waves from a CUDA graph
bool factor_flow_enabled() {
  static const bool on = !(getenv("HLC_FACTOR_FLOW") && getenv("HLC_FACTOR_FLOW")[0] == '0');
  return on;
}

// TRSM/GEMM plans run dependency-driven (k_flow) unless HLC_FLOW=0, which
// keeps the wave-by-wave persistent kernel (k_waves)
bool flow_enabled() {
  static const bool on = !(getenv("HLC_FLOW") && getenv("HLC_FLOW")[0] == '0');
  return on;
}

// One persistent launch of a TRSM/GEMM plan: dependency-driven when the plan
// has its dataflow form, else wave by wave.  0 or -1 (launch unavailable).
// HLC_FACTOR_TRACE=<path> (HLC_SOLVE_TRACE=<path>): the dataflow
// factorisation (each dataflow solve or matvec) records a timeline
// (FactorTrace per op) and writes it to <path> (<path>.<plan>, the plan's
// last run) after the launch.  File: the 8 bytes "HLCFTR01", int64 nops,
// then nops records of six int32 (type, part and four sizes: POTRF n; TRSM n,
// c, trans; GEMM m, k, c; truncations m, n, term columns, rank after), then
// the nops FactorTrace records.  Sizes that are ranks are read after the run
// (a temporary's slot holds its last value).
const char* factor_trace_path() {
  static const char* p = getenv("HLC_FACTOR_TRACE");
  return p && p[0] ? p : nullptr;
}

const char* solve_trace_path() {
  static const char* p = getenv("HLC_SOLVE_TRACE");
  return p && p[0] ? p : nullptr;
}

int write_trace(hlc_tree* t, const Plan& P, const int* d_ranks, int64_t nsl, const FactorTrace* d_trace,
                const std::string& path) {
  hlc_ctx* c = t->ctx;
  const int64_t nops = (int64_t)P.flow.size();
  std::vector<FactorTrace> tr(nops);
  std::vector<int> rk(std::max<int64_t>(nsl, 1));
  CK(cudaMemcpyAsync(tr.data(), d_trace, nops * sizeof(FactorTrace), cudaMemcpyDeviceToHost, c->stream));
  if (nsl) CK(cudaMemcpyAsync(rk.data(), d_ranks, nsl * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  auto dim = [&](const Dim& d) { return d.slot >= 0 && d.slot < nsl ? rk[d.slot] : d.n; };
  std::vector<int32_t> meta(6 * nops, 0);
  for (int64_t i = 0; i < nops; ++i) {
    const FlowOp& f = P.flow[i];
    int32_t* m = &meta[6 * i];
    m[0] = f.type;
    m[1] = f.part;
    if (f.type == OP_POTRF) {
      m[2] = P.potrf[f.idx].n;
    } else if (f.type == OP_TRSM) {
      const OpTrsm& o = P.trsm[f.idx];
      m[2] = o.n;
      m[3] = dim(o.c);
      m[4] = o.trans;
    } else if (f.type == OP_GEMM) {
      const OpGemm& o = P.gemm[f.idx];
      m[2] = dim(o.m);
      m[3] = dim(o.k);
      m[4] = dim(o.c);
    } else {
      const OpTrunc& o = P.trunc[f.idx];
      m[2] = o.m;
      m[3] = o.n;
      int64_t cols = 0;
      for (int64_t e = o.term0; e < o.term0 + o.nterms; ++e) {
        const TermD& d = P.terms[e];
        cols += (d.flags & 1) ? d.urows : (d.flags & 2) ? d.vrows : dim(d.k);
      }
      m[4] = (int32_t)cols;
      m[5] = o.slot >= 0 && o.slot < nsl ? rk[o.slot] : -1;
    }
  }
  FILE* fp = fopen(path.c_str(), "wb");
  if (!fp) return HLC_ERR_ARG;
  bool ok = fwrite("HLCFTR01", 1, 8, fp) == 8 && fwrite(&nops, sizeof(nops), 1, fp) == 1 &&
            fwrite(meta.data(), sizeof(int32_t), meta.size(), fp) == meta.size() &&
            fwrite(tr.data(), sizeof(FactorTrace), tr.size(), fp) == tr.size();
  ok = (fclose(fp) == 0) && ok;
  return ok ? HLC_OK : HLC_ERR_ARG;
}

int launch_persistent(const Plan& P, const Bases& B, GridBar* gb, int md, int per, cudaStream_t st,
                      FactorTrace* trace = nullptr) {
  if (flow_enabled() && P.d_flow && P.d_count)
    return launch_flow(P.d_flow, (int64_t)P.flow.size(), P.d_npred, P.d_succ_off, P.d_succ, P.d_count, P.d_trsm,
                       P.d_gemm, B, gb, md, per, trace, st);
  return launch_waves(P.d_waves, (int)P.waves.size(), P.d_trsm, P.d_gemm, P.d_chain, P.chains(), B, gb, md, per, st);
}

bool persistent_enabled() {
  static const bool on = !(getenv("HLC_PERSISTENT") && getenv("HLC_PERSISTENT")[0] == '0');
  return on;
}

// Run a plan: replayed from a CUDA graph when possible (the op program is the
// same for every evaluation on a tree; only the ranks in device memory vary),
// captured on first use for a given set of base pointers.
void run_plan(hlc_tree* t, const Plan& P, const Bases& B, cudaStream_t st) {
  hlc_ctx* c = t->ctx;
  // TRSM/GEMM plans (solves, matvec): one persistent cooperative launch
  if (P.d_waves && !P.waves.empty() && c->persistent && !c->profiling && !g_prof.on && persistent_enabled()) {
    const int md = (int)std::max<int64_t>(t->T.max_dense_dim, t->T.leaf);
    // autotuning of the grid: until the plan is tuned, every run takes the
    // candidate with the fewest runs so far and is timed with events; the
    // grid does not change the result (each op of a wave writes its own
    // region), only the time
    int per = P.tuned_per_sm, cand = -1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (per == 0) {
      cand = 0;
      for (int i = 1; i < 3; ++i)
        if (P.tune_tries[i] < P.tune_tries[cand]) cand = i;
      per = kTuneCandidates[cand];
      for (cudaEvent_t* e : {&e0, &e1}) {
        if (!c->tune_free.empty()) {
          *e = c->tune_free.back();
          c->tune_free.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
          *e = nullptr;
        }
      }
      if (e0 && e1) cudaEventRecord(e0, st);
    }
    FactorTrace* d_trace = nullptr;
    const char* tpath = P.d_flow && flow_enabled() ? solve_trace_path() : nullptr;
    if (tpath && cudaMalloc(&d_trace, P.flow.size() * sizeof(FactorTrace)) == cudaSuccess)
      cudaMemsetAsync(d_trace, 0xff, P.flow.size() * sizeof(FactorTrace), st);
    const int lst = launch_persistent(P, B, c->d_gridbar, md, per, st, d_trace);
    if (d_trace) {
      const char* name = &P == &t->fwd ? "fwd" : &P == &t->bwd ? "bwd" : &P == &t->mv ? "mv" : "other";
      if (lst == 0) write_trace(t, P, B.ranks, t->T.nslots, d_trace, std::string(tpath) + "." + name);
      cudaFree(d_trace);
    }
    if (lst == 0) {
      c->launches += 1;
      c->persistent_launches += 1;
      if (cand >= 0) {
        P.tune_tries[cand] += 1;
        if (e0 && e1) {
          cudaEventRecord(e1, st);
          c->tune_pending.push_back(hlc_ctx::TuneRec{&P, cand, e0, e1});
          e0 = e1 = nullptr;
        }
      }
      for (cudaEvent_t e : {e0, e1})
        if (e) c->tune_free.push_back(e);
      return;
    }
    for (cudaEvent_t e : {e0, e1})
      if (e) c->tune_free.push_back(e);
    cudaGetLastError();
  }
  if (c->profiling || g_prof.on || !graphs_enabled() || P.launches.empty()) {
    run_plan_launches(t, P, B, st, true);
    return;
  }
  if (!P.graph || !same_bases(P.graph_key, B)) {
    if (P.graph) {
      cudaGraphExecDestroy(P.graph);
      P.graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      run_plan_launches(t, P, B, st, false);
      if (cudaStreamEndCapture(st, &g) == cudaSuccess && g) {
        if (cudaGraphInstantiate(&P.graph, g, 0) != cudaSuccess) P.graph = nullptr;
        cudaGraphDestroy(g);
      }
    }
    cudaGetLastError();
    if (!P.graph) {  // capture unavailable: plain launches
      run_plan_launches(t, P, B, st, true);
      return;
    }
    P.graph_key = B;
  }
  cudaGraphLaunch(P.graph, st);
  c->launches += (double)P.launches.size();
  for (const Launch& L : P.launches) c->op_launches[L.type] += 1;
}

// The ops of one wave are independent (the planner puts an op in the first
// wave after all of its producers and earlier readers), so the POTRF, TRSM
// and GEMM launches of a wave run on side streams beside the truncations,
// forked from the context's stream at the start of the wave and joined back
// before the next one (in a captured graph: parallel branches).  The two
// truncation kernels stay on the context's stream: they share the per-CTA
// scratch.  Timed (profiling) runs keep one stream.
void run_plan_launches(hlc_tree* t, const Plan& P, const Bases& B, cudaStream_t st, bool count) {
  const int md = (int)std::max<int64_t>(t->T.max_dense_dim, t->T.leaf);
  hlc_ctx* cx = t->ctx;
  const bool conc = cx->side_ok && !cx->profiling && !g_prof.on;
  size_t wave_end = 0;
  bool forked = false, used[3] = {false, false, false};
  for (size_t li = 0; li < P.launches.size(); ++li) {
    const Launch& L = P.launches[li];
    if (li == wave_end) {  // a new wave starts: its launches are [li, wave_end)
      wave_end = li;
      while (wave_end < P.launches.size() && P.launches[wave_end].wave == L.wave) ++wave_end;
      forked = conc && wave_end - li > 1;
      used[0] = used[1] = used[2] = false;
      if (forked) cudaEventRecord(cx->ev_fork, st);
    }
    cudaStream_t ls = st;
    if (forked && L.type <= OP_GEMM) {
      ls = cx->side[L.type];
      if (!used[L.type]) {
        cudaStreamWaitEvent(ls, cx->ev_fork, 0);
        used[L.type] = true;
      }
    }
    run_launch(t, P, B, L, md, ls, count);
    if (forked && li + 1 == wave_end) {
      for (int k = 0; k < 3; ++k)
        if (used[k]) {
          cudaEventRecord(cx->ev_join[k], cx->side[k]);
          cudaStreamWaitEvent(st, cx->ev_join[k], 0);
        }
    }
  }
}

void run_launch(hlc_tree* t, const Plan& P, const Bases& B, const Launch& L, int md, cudaStream_t st, bool count) {
  {
    const void* ops = nullptr;
    switch (L.type) {
      case OP_GEMM: ops = P.d_gemm + L.first; break;
      case OP_TRSM: ops = P.d_trsm + L.first; break;
      case OP_POTRF: ops = P.d_potrf + L.first; break;
      case OP_CHAIN: ops = P.d_chain + L.first; break;
      default: ops = P.d_trunc + L.first; break;  // OP_TRUNC, OP_TRUNC_BIG
    }
    hlc_ctx* c = t->ctx;
    if (count) {
      c->launches += 1;
      c->op_launches[L.type] += 1;
    }
    if (c->profiling) {
      const int ev = (int)c->pending.size() * 2;
      while ((int)c->evpool.size() < ev + 2) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        c->evpool.push_back(e);
      }
      cudaEventRecord(c->evpool[ev], st);
      launch_ops(L.type, ops, L.count, P.d_terms, P.chains(), B, md, st);
      cudaEventRecord(c->evpool[ev + 1], st);
      c->pending.push_back(hlc_ctx::Pending{L.type, ev});
      return;
    }
    if (!g_prof.on) {
      launch_ops(L.type, ops, L.count, P.d_terms, P.chains(), B, md, st);
      return;
    }
    cudaStreamSynchronize(st);
    const auto t0 = std::chrono::steady_clock::now();
    launch_ops(L.type, ops, L.count, P.d_terms, P.chains(), B, md, st);
    cudaStreamSynchronize(st);
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    g_prof.ms[L.type] += ms;
    g_prof.launches[L.type] += 1;
    g_prof.ops[L.type] += L.count;
    if (g_prof.slow.size() < 4096 || ms > 1.0) g_prof.slow.push_back(Prof::Slow{ms, L.type, L.wave, L.count});
  }
}

Bases make_bases(hlc_tree* t, double* mat_L, double* mat_C, int* ranks, bool mixed) {
  Bases B;
  B.mixed = mixed ? 1 : 0;
  B.core64 = (mixed && t->p.precision == HLC_MIXED_SVD64) ? 1 : 0;
  B.buf[BUF_L] = mat_L;
  B.buf[BUF_TMP] = t->d_tmp;
  B.buf[BUF_VEC] = t->d_vec;
  B.buf[BUF_C] = mat_C;
  B.ranks = ranks;
  B.status = t->ctx->d_status;
  B.scratch = t->ctx->d_scratch;
  B.flops = t->ctx->d_flops;
  B.phase = t->ctx->d_phase;
  return B;
}

// Timed runs of the persistent kernel (the stream has been synchronised):
// record each candidate's best time; once every candidate has two runs the
// plan keeps the fastest.
void read_tuning(hlc_ctx* c) {
  for (const hlc_ctx::TuneRec& r : c->tune_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) {
      float& best = r.P->tune_ms[r.cand];
      if (r.P->tune_done[r.cand] == 0 || ms < best) best = ms;
      r.P->tune_done[r.cand] += 1;
      bool all = true;
      int arg = 0;
      for (int i = 0; i < 3; ++i) {
        all = all && r.P->tune_done[i] >= 2;
        if (r.P->tune_done[i] > 0 && r.P->tune_ms[i] < r.P->tune_ms[arg]) arg = i;
      }
      if (all && r.P->tuned_per_sm == 0) r.P->tuned_per_sm = kTuneCandidates[arg];
    }
    c->tune_free.push_back(r.e0);
    c->tune_free.push_back(r.e1);
  }
  c->tune_pending.clear();
  cudaGetLastError();
}

// device status -> ABI status (also resets it)
int take_status(hlc_ctx* c) {
  int h[2] = {0, 0};
  cudaError_t e = cudaMemcpyAsync(h, c->d_status, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_status(e);
  read_tuning(c);
  cudaMemsetAsync(c->d_status, 0, 2 * sizeof(int), c->stream);
  switch (h[0]) {
    case DEV_OK: return HLC_OK;
    case DEV_NOT_SPD: return HLC_ERR_NOT_SPD;
    case DEV_RANK: return HLC_ERR_RANK;
    case DEV_TIMEOUT: return HLC_ERR_TIMEOUT;
    default: return HLC_ERR_NUMERIC;
  }
}

bool valid_theta(const hlc_theta* th) {
  return th && th->sigma2 > 0.0 && th->ell > 0.0 && th->nu > 0.0 && th->nugget >= 0.0 && th->nu < 20.0;
}

MaternDev matern_params(hlc_tree* t, const hlc_theta* th) {
  MaternDev mp;
  mp.sigma2 = th->sigma2;
  mp.ell = th->ell;
  mp.nu = th->nu;
  mp.nugget = th->nugget;
  mp.coef = th->sigma2 / (pow(2.0, th->nu - 1.0) * tgamma(th->nu));
  mp.kind = th->nu == 0.5 ? 0 : th->nu == 1.5 ? 1 : th->nu == 2.5 ? 2 : 3;
  mp.nnodes = KNU_NODES;
  t->h_knu.resize(2 * KNU_NODES);
  for (int j = 0; j < KNU_NODES; ++j) {
    const double tj = j * KNU_STEP;
    const double sh = sinh(0.5 * tj);
    t->h_knu[j] = 2.0 * sh * sh;  // cosh t - 1 without cancellation
    t->h_knu[KNU_NODES + j] = cosh(th->nu * tj);
  }
  mp.cm1 = t->d_knu;
  mp.wnu = t->d_knu + KNU_NODES;
  return mp;
}

int hmat_alloc(hlc_tree* t, int which, hlc_hmat** out) {
  hlc_hmat* M = new (std::nothrow) hlc_hmat();
  if (!M) return HLC_ERR_OOM;
  M->t = t;
  M->which = which;
  cudaError_t e = cudaMalloc(&M->arena, std::max<int64_t>(t->T.arena_doubles, 4) * sizeof(double));
  // a factor's rank array also holds the slots of the factorisation plan's
  // temporary partial sums (the plan is built before a factor is allocated)
  const int64_t slots = (int64_t)t->T.nslots + (which == 1 ? t->chol.tmp_slots : 0);
  if (e == cudaSuccess) e = cudaMalloc(&M->ranks, std::max<int64_t>(slots, 1) * sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(M->arena);
    cudaFree(M->ranks);
    delete M;
    return cuda_status(e);
  }
  *out = M;
  return HLC_OK;
}

// Refuse to run a plan whose views leave their buffers.
int check_plan(hlc_tree* t, const Plan& P) {
  int64_t sz[NBUF];
  sz[BUF_L] = t->T.arena_doubles;
  sz[BUF_C] = t->T.arena_doubles;
  sz[BUF_TMP] = P.tmp_doubles;
  sz[BUF_VEC] = 6 * t->T.n;
  const std::string err = validate_plan(P, sz, (int64_t)t->T.nslots + P.tmp_slots);
  if (!err.empty()) {
    fprintf(stderr, "hlc: plan rejected: %s\n", err.c_str());
    return HLC_ERR_STATE;
  }
  return HLC_OK;
}

int build_plans(hlc_tree* t, bool chol, bool solve) {
  try {
    if (chol && !t->chol_ready) {
      const bool acc = getenv("HLC_ACCUMULATE") && getenv("HLC_ACCUMULATE")[0] == '1';
      plan_cholesky(t->T, t->chol, acc, factor_flow_enabled());
      int st = check_plan(t, t->chol);
      if (st) return st;
      st = upload_plan(t->chol);
      if (st) return st;
      t->chol_ready = true;
    }
    if (solve && !t->solve_ready) {
      const int64_t n = t->T.n;
      plan_solve(t->T, t->fwd, 0, 0, 1, chains_enabled());
      plan_solve(t->T, t->bwd, 1, 0, 1, chains_enabled());
      plan_matvec(t->T, t->mv, n, 2 * n, 1);
      int st;
      if ((st = check_plan(t, t->fwd)) || (st = check_plan(t, t->bwd)) || (st = check_plan(t, t->mv))) return st;
      if ((st = upload_plan(t->fwd)) || (st = upload_plan(t->bwd)) || (st = upload_plan(t->mv))) return st;
      t->solve_ready = true;
    }
  } catch (const std::bad_alloc&) {
    return HLC_ERR_OOM;
  } catch (const std::exception&) {
    return HLC_ERR_CUDA;
  }
  int64_t need = std::max(t->recomp.tmp_doubles, t->chol.tmp_doubles);
  need = std::max(need, std::max(t->fwd.tmp_doubles, std::max(t->bwd.tmp_doubles, t->mv.tmp_doubles)));
  need = std::max(need, std::max(t->lmv.tmp_doubles, t->lmvt.tmp_doubles));
  return ensure_tmp(t, need);
}

// Plans of the products with the lower factor (in place on the vector at
// offset 0 of the tree's vector workspace).
int build_lmv_plans(hlc_tree* t) {
  if (t->lmv_ready) return HLC_OK;
  try {
    plan_trmv(t->T, t->lmv, 0, 0, 1, chains_enabled());
    plan_trmv(t->T, t->lmvt, 1, 0, 1, chains_enabled());
    int st;
    if ((st = check_plan(t, t->lmv)) || (st = check_plan(t, t->lmvt))) return st;
    if ((st = upload_plan(t->lmv)) || (st = upload_plan(t->lmvt))) return st;
  } catch (const std::bad_alloc&) {
    return HLC_ERR_OOM;
  } catch (const std::exception&) {
    return HLC_ERR_CUDA;
  }
  t->lmv_ready = true;
  return ensure_tmp(t, std::max(t->lmv.tmp_doubles, t->lmvt.tmp_doubles));
}

// y = L~ x (trans 0) or L~^T x (trans 1) in caller order, FP64 arithmetic;
// x, y host or device.
int factor_apply(hlc_tree* t, const hlc_hmat* L, int trans, const double* x, double* y) {
  hlc_ctx* c = t->ctx;
  int st = build_lmv_plans(t);
  if (st) return st;
  const int64_t n = t->T.n;
  double* W0 = t->d_vec;
  double* S = t->d_vec + 3 * n;  // staging
  cudaStream_t s = c->stream;
  if (is_device_ptr(x)) {
    launch_gather(x, t->d_perm, W0, n, s);
  } else {
    CK(cudaMemcpyAsync(S, x, n * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gather(S, t->d_perm, W0, n, s);
  }
  c->launches += 1;
  Bases B = make_bases(t, L->arena, nullptr, L->ranks, false);
  run_plan(t, trans ? t->lmvt : t->lmv, B, s);
  if (is_device_ptr(y)) {
    launch_scatter(W0, t->d_perm, y, n, s);
  } else {
    launch_scatter(W0, t->d_perm, S, n, s);
    CK(cudaMemcpyAsync(y, S, n * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  c->launches += 1;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return take_status(c);
}

int do_assemble(hlc_tree* t, const hlc_theta* th, hlc_hmat* C) {
  hlc_ctx* c = t->ctx;
  MaternDev mp = matern_params(t, th);
  CK(cudaMemcpyAsync(t->d_knu, t->h_knu.data(), t->h_knu.size() * sizeof(double), cudaMemcpyHostToDevice,
                     c->stream));
  launch_dense_asm(t->d_dense, (int64_t)t->T.dense_asm.size(), C->arena, t->d_px, t->d_py, mp, c->stream);
  c->launches += 2;  // dense assembly + ACA
  // C~ is assembled and recompressed in FP64 in every precision mode: it is
  // the matrix the FP64 residual of the refinement is taken against, and the
  // quadratic form z^T C~^-1 z inherits every perturbation of C~ amplified by
  // its condition number (FP32 ACA panels moved |dL|/n by ~5e-4 at
  // n = 524,288, ell = 0.0864, nugget 1e-4).
  launch_aca(t->d_lr, (int64_t)t->T.lr_asm.size(), C->arena, t->d_px, t->d_py, mp, t->p.eps, t->p.fixed_rank,
             C->ranks, c->d_status, c->stream);
  Bases B = make_bases(t, nullptr, C->arena, C->ranks, false);
  run_plan(t, t->recomp, B, c->stream);
  CK(cudaGetLastError());
  C->valid = false;
  const int st = take_status(c);
  if (st == HLC_OK) C->valid = true;
  return st;
}

int do_cholesky(hlc_tree* t, const hlc_hmat* C, hlc_hmat* L) {
  hlc_ctx* c = t->ctx;
  int st = build_plans(t, true, false);
  if (st) return st;
  CK(cudaMemcpyAsync(L->arena, C->arena, t->T.arena_doubles * sizeof(double), cudaMemcpyDeviceToDevice,
                     c->stream));
  if (t->T.nslots)
    CK(cudaMemcpyAsync(L->ranks, C->ranks, t->T.nslots * sizeof(int), cudaMemcpyDeviceToDevice, c->stream));
  Bases B = make_bases(t, L->arena, nullptr, L->ranks, t->p.precision != HLC_FP64);
  // one dependency-driven launch (serve slots share the SMs and take the
  // waves; so do the timed profiling passes, which time launches by type)
  bool flowed = false;
  if (factor_flow_enabled() && c->persistent && !c->profiling && !g_prof.on && t->chol.d_flow) {
    const int md = (int)std::max<int64_t>(t->T.max_dense_dim, t->T.leaf);
    const char* tpath = factor_trace_path();
    FactorTrace* d_trace = nullptr;
    if (tpath) {
      const size_t bytes = t->chol.flow.size() * sizeof(FactorTrace);
      CK(cudaMalloc(&d_trace, bytes));
      // releaser -1 where no producer signals
      CK(cudaMemsetAsync(d_trace, 0xff, bytes, c->stream));
    }
    if (launch_factor(t->chol, B, c->d_gridbar, md, d_trace, c->stream) == 0) {
      flowed = true;
      c->launches += 1;
      c->persistent_launches += 1;
      if (d_trace) st = write_trace(t, t->chol, L->ranks, (int64_t)t->T.nslots + t->chol.tmp_slots, d_trace, tpath);
    } else {
      cudaGetLastError();
    }
    if (d_trace) CK(cudaFree(d_trace));
    if (st) return st;
  }
  if (!flowed) run_plan(t, t->chol, B, c->stream);
  CK(cudaGetLastError());
  L->valid = false;
  st = take_status(c);
  if (st == HLC_OK) L->valid = true;
  return st;
}

// Extreme eigenvalues of the symmetric tridiagonal matrix with diagonal d
// and off-diagonal e (e[i] couples i and i+1) by bisection on the Sturm
// sequence count (the number of eigenvalues below x is the number of
// negative pivots of T - x I).
int tridiag_count_below(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int cnt = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    const double off = i ? e[i - 1] * e[i - 1] : 0.0;
    q = d[i] - x - (i ? off / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

void tridiag_extremes(const std::vector<double>& d, const std::vector<double>& e, double* lo, double* hi) {
  double a = INFINITY, b = -INFINITY;
  for (size_t i = 0; i < d.size(); ++i) {
    const double r = (i ? fabs(e[i - 1]) : 0.0) + (i + 1 < d.size() ? fabs(e[i]) : 0.0);
    a = std::min(a, d[i] - r);
    b = std::max(b, d[i] + r);
  }
  const int k = (int)d.size();
  for (int which = 0; which < 2; ++which) {
    // which 0: smallest (count below x >= 1), 1: largest (count below x >= k)
    double l = a, h = b;
    for (int it = 0; it < 200 && h - l > 1e-15 * std::max(fabs(l), fabs(h)); ++it) {
      const double m = 0.5 * (l + h);
      if (tridiag_count_below(d, e, m) >= (which ? k : 1))
        h = m;
      else
        l = m;
    }
    (which ? *hi : *lo) = 0.5 * (l + h);
  }
}

// Estimate of |I - (L~ L~^T)^-1 C~|_2 from the preconditioned CG run (the
// quantity of Table 5's last column).  CG with step lengths a_j and update
// coefficients b_j is the Lanczos process of the preconditioned operator,
// with tridiagonal T: T_00 = 1/a_0, T_jj = 1/a_j + b_{j-1}/a_{j-1},
// T_{j-1,j} = sqrt(b_{j-1})/a_{j-1}.  The extreme eigenvalues of T (Ritz
// values) approach those of the operator from inside, so the estimate is a
// lower bound that tightens with the number of iterations.  -1 when no
// iteration ran.
double lanczos_rel_err(const std::vector<double>& al, const std::vector<double>& be) {
  const size_t k = al.size();
  if (k == 0) return -1.0;
  std::vector<double> d(k), e(k > 1 ? k - 1 : 0);
  for (size_t j = 0; j < k; ++j) {
    if (!(al[j] > 0.0)) return -1.0;
    d[j] = 1.0 / al[j] + (j ? be[j - 1] / al[j - 1] : 0.0);
    if (j) e[j - 1] = sqrt(std::max(be[j - 1], 0.0)) / al[j - 1];
  }
  double lo = d[0], hi = d[0];
  if (k > 1) tridiag_extremes(d, e, &lo, &hi);
  return std::max(fabs(1.0 - lo), fabs(hi - 1.0));
}

double read_scalar(hlc_ctx* c, int idx) {
  double v = 0.0;
  cudaMemcpyAsync(&v, c->d_scalar + idx, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  return v;
}

void hmat_stats(hlc_tree* t, const hlc_hmat* M, size_t* bytes, int* maxr) {
  std::vector<int> r(t->T.nslots);
  if (!r.empty()) cudaMemcpy(r.data(), M->ranks, r.size() * sizeof(int), cudaMemcpyDeviceToHost);
  size_t b = 0;
  int mx = 0;
  for (int32_t bl : t->T.leaves) {
    const Block& B = t->T.blk[bl];
    if (B.type == BT_DENSE) {
      b += (size_t)B.m * B.n * 8;
    } else {
      const int k = r[B.slot];
      b += (size_t)(B.m + B.n) * k * 8;
      mx = std::max(mx, k);
    }
  }
  *bytes = b;
  *maxr = mx;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
namespace hlc {
Serve*& serve_of(hlc_ctx* c) { return c->serve; }
void set_persistent(hlc_ctx* c, bool on) { c->persistent = on; }
int device_of(hlc_ctx* c) { return c->device; }
}  // namespace hlc

extern "C" {

int hlc_ctx_stream(hlc_ctx* c, void** stream) {
  if (!c || !stream) return HLC_ERR_ARG;
  *stream = (void*)c->stream;
  return HLC_OK;
}

int hlc_ctx_set_profiling(hlc_ctx* c, int on) {
  if (!c) return HLC_ERR_ARG;
  c->profiling = on != 0;
  return HLC_OK;
}

int hlc_ctx_counters(hlc_ctx* c, int reset, double* out) {
  if (!c || !out) return HLC_ERR_ARG;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->stream));
  for (const hlc_ctx::Pending& p : c->pending) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->evpool[p.ev], c->evpool[p.ev + 1]) == cudaSuccess) c->op_ms[p.type] += ms;
  }
  c->pending.clear();
  double fl[NOPTYPES];
  CK(cudaMemcpy(fl, c->d_flops, sizeof(fl), cudaMemcpyDeviceToHost));
  out[0] = c->launches;
  for (int t = 0; t < NOPTYPES; ++t) {
    out[1 + 3 * t] = c->op_launches[t];
    out[2 + 3 * t] = c->op_ms[t];
    out[3 + 3 * t] = fl[t];
  }
  out[1 + 3 * NOPTYPES] = c->persistent_launches;
  if (reset) {
    c->launches = 0;
    c->persistent_launches = 0;
    for (int t = 0; t < NOPTYPES; ++t) c->op_launches[t] = c->op_ms[t] = 0;
    CK(cudaMemset(c->d_flops, 0, NOPTYPES * sizeof(double)));
  }
  return HLC_OK;
}

void hlc_default_params(hlc_params* p) {
  if (!p) return;
  p->leaf = 64;
  p->eta = 2.0;
  p->eps = 1e-6;
  p->precision = HLC_FP64;
  p->refine_tol = 1e-12;
  p->refine_maxit = 100;
  p->kmax = 64;
  p->admissibility = HLC_ADM_STANDARD;
  p->split = HLC_SPLIT_GEOMETRIC;
  p->fixed_rank = 0;
}

const char* hlc_strerror(int s) {
  switch (s) {
    case HLC_OK: return "ok";
    case HLC_PENDING: return "request pending";
    case HLC_ERR_ARG: return "invalid argument";
    case HLC_ERR_OOM: return "out of memory";
    case HLC_ERR_NOT_SPD: return "matrix not positive definite (non-positive pivot)";
    case HLC_ERR_TIMEOUT: return "bounded device wait expired";
    case HLC_ERR_CUDA: return "CUDA runtime error";
    case HLC_ERR_RANK: return "low-rank block exceeded the rank capacity kmax";
    case HLC_ERR_STATE: return "call out of order";
    case HLC_ERR_UNSUPPORTED: return "unsupported";
    case HLC_ERR_NUMERIC: return "numerical breakdown (NaN)";
    case HLC_ERR_SCRATCH: return "problem larger than the fixed buffer of the no-alloc call";
    default: return "unknown status";
  }
}

int hlc_create(hlc_ctx** out, int device) {
  if (!out) return HLC_ERR_ARG;
  *out = nullptr;
  int nd = 0;
  if (cudaGetDeviceCount(&nd) != cudaSuccess || device < 0 || device >= nd) {
    cudaGetLastError();
    return HLC_ERR_CUDA;
  }
  CK(cudaSetDevice(device));
  hlc_ctx* c = new (std::nothrow) hlc_ctx();
  if (!c) return HLC_ERR_OOM;
  c->device = device;
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  {
    bool ok = e == cudaSuccess;
    for (int k = 0; k < 3 && ok; ++k) {
      ok = cudaStreamCreateWithFlags(&c->side[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    }
    ok = ok && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    c->side_ok = ok;  // without side streams every launch stays on the context's stream
    cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->d_part, 1 << 20);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_scalar, 64);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, 16);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_flops, NOPTYPES * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->d_flops, 0, NOPTYPES * sizeof(double));
  if (e == cudaSuccess && getenv("HLC_PHASES") && getenv("HLC_PHASES")[0] == '1') {
    e = cudaMalloc(&c->d_phase, 32 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->d_phase, 0, 32 * sizeof(unsigned long long));
  }
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, 16);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_gridbar, sizeof(GridBar));
  if (e == cudaSuccess)
    e = cudaMalloc(&c->d_scratch, (size_t)max_trunc_ctas() * trunc_scratch_doubles() * sizeof(double));
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
  if (e == cudaSuccess && configure_kernels(128) != 0) e = cudaErrorInvalidValue;
  if (e != cudaSuccess) {
    hlc_destroy(c);
    return cuda_status(e);
  }
  *out = c;
  return HLC_OK;
}

// After the CUDA runtime has begun unloading (process exit), device
// resources are gone with the context: release host memory only.
static bool runtime_alive(int device) {
  const cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) return true;
  cudaGetLastError();
  return false;
}

void hlc_destroy(hlc_ctx* c) {
  if (!c) return;
  if (!runtime_alive(c->device)) {
    delete c;
    return;
  }
  if (c->serve) hlc_serve_stop(c);
  cudaFree(c->d_part);
  cudaFree(c->d_scalar);
  cudaFree(c->d_status);
  cudaFree(c->d_gridbar);
  cudaFree(c->d_scratch);
  cudaFree(c->d_flops);
  if (c->d_phase) {
    // two sets of counters: batches of K <= 32 columns, and wider ones
    unsigned long long all[32];
    if (cudaMemcpy(all, c->d_phase, sizeof(all), cudaMemcpyDeviceToHost) == cudaSuccess) {
      for (int set = 0; set < 2; ++set) {
        const unsigned long long* ph = all + 16 * set;
        if (!ph[11]) continue;
        static const char* nm[8] = {"", "qr U", "qr V", "core M", "core QRCP", "core QR+Jacobi", "core vectors",
                                    "apply"};
        double tot = 0;
        for (int i = 1; i < 8; ++i) tot += (double)ph[i];
        fprintf(stderr, "hlc-phases %s batches %llu  mean K %.1f  mean rank %.1f\n", set ? "K > 32" : "K <= 32",
                ph[11], (double)ph[12] / ph[11], (double)ph[10] / ph[11]);
        for (int i = 1; i < 8; ++i)
          fprintf(stderr, "hlc-phases %-16s %14.0f cycles (%5.1f %%) %10.1f per batch\n", nm[i], (double)ph[i],
                  100.0 * ph[i] / tot, (double)ph[i] / ph[11]);
      }
    }
    cudaFree(c->d_phase);
  }
  for (cudaEvent_t e : c->evpool) cudaEventDestroy(e);
  for (const hlc_ctx::TuneRec& r : c->tune_pending) {
    cudaEventDestroy(r.e0);
    cudaEventDestroy(r.e1);
  }
  for (cudaEvent_t e : c->tune_free) cudaEventDestroy(e);
  for (int i = 0; i < 4; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  if (c->stream) cudaStreamDestroy(c->stream);
  for (int k = 0; k < 3; ++k) {
    if (c->side[k]) cudaStreamDestroy(c->side[k]);
    if (c->ev_join[k]) cudaEventDestroy(c->ev_join[k]);
  }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  delete c;
}

int hlc_build_tree(hlc_ctx* c, const double* xy, int64_t n, const hlc_params* p, hlc_tree** out) {
  if (!c || !xy || !out || n <= 0 || n > (int64_t)1 << 30) return HLC_ERR_ARG;
  hlc_params q;
  if (p)
    q = *p;
  else
    hlc_default_params(&q);
  if (q.leaf < 1 || q.leaf > 128 || !(q.eta > 0.0) || !(q.eps > 0.0) || q.kmax < 1 || q.kmax > 128 ||
      (q.precision != HLC_FP64 && q.precision != HLC_MIXED && q.precision != HLC_MIXED_SVD64) ||
      q.refine_maxit < 0 || q.admissibility < HLC_ADM_STANDARD || q.admissibility > HLC_ADM_WEAK ||
      (q.split != HLC_SPLIT_GEOMETRIC && q.split != HLC_SPLIT_CARDINALITY) || q.fixed_rank < 0 ||
      q.fixed_rank > q.kmax)
    return HLC_ERR_ARG;
  *out = nullptr;
  CK(cudaSetDevice(c->device));
  std::unique_ptr<hlc_tree> t(new (std::nothrow) hlc_tree());
  if (!t) return HLC_ERR_OOM;
  t->ctx = c;
  t->p = q;
  // points on the device; the trees are built there (Morton sort, bisection,
  // block-cluster tree) and their structure copied to the host planner
  double* d_xy = nullptr;
  CK(cudaMalloc(&d_xy, 2 * n * sizeof(double)));
  CK(cudaMemcpy(d_xy, xy, 2 * n * sizeof(double), is_device_ptr(xy) ? cudaMemcpyDeviceToDevice
                                                                    : cudaMemcpyHostToDevice));
  try {
    t->T.n = n;
    t->T.leaf = q.leaf;
    t->T.eta = q.eta;
    t->T.eps = q.eps;
    int depth = 0;
    if (device_tree_build(d_xy, n, q.leaf, q.eta, q.admissibility, q.split, c->stream, t->T.perm, t->T.cl, t->T.blk,
                          &depth) != 0) {
      cudaFree(d_xy);
      return HLC_ERR_CUDA;
    }
    t->T.depth = depth;
    collect_leaf_list(t->T);
    t->T.eps = q.eps;
    t->T.kfix = q.fixed_rank;
    layout(t->T, q.kmax);
    plan_recompress(t->T, t->recomp);
  } catch (const std::bad_alloc&) {
    cudaFree(d_xy);
    return HLC_ERR_OOM;
  }
  int st;
  if ((st = upload(&t->d_perm, t->T.perm))) return st;
  CK(cudaMalloc(&t->d_px, n * sizeof(double)));
  CK(cudaMalloc(&t->d_py, n * sizeof(double)));
  launch_points(d_xy, t->d_perm, t->d_px, t->d_py, n, c->stream);
  CK(cudaStreamSynchronize(c->stream));
  cudaFree(d_xy);
  if ((st = upload(&t->d_dense, t->T.dense_asm))) return st;
  if ((st = upload(&t->d_lr, t->T.lr_asm))) return st;
  std::vector<int64_t> doff;
  std::vector<int32_t> ddim;
  for (int32_t b : t->T.leaves) {
    const Block& B = t->T.blk[b];
    if (B.diag) {
      doff.push_back(B.offD);
      ddim.push_back((int32_t)B.m);
    }
  }
  t->ndiag = (int64_t)doff.size();
  if ((st = upload(&t->d_diag_off, doff))) return st;
  if ((st = upload(&t->d_diag_dim, ddim))) return st;
  CK(cudaMalloc(&t->d_knu, 2 * KNU_NODES * sizeof(double)));
  CK(cudaMalloc(&t->d_vec, 6 * n * sizeof(double)));
  if ((st = check_plan(t.get(), t->recomp))) return st;
  if ((st = upload_plan(t->recomp))) return st;
  if ((st = ensure_tmp(t.get(), t->recomp.tmp_doubles))) return st;
  *out = t.release();
  return HLC_OK;
}

void hlc_tree_free(hlc_tree* t) {
  if (!t) return;
  if (!runtime_alive(t->ctx->device)) {
    delete t;
    return;
  }
  cudaStreamSynchronize(t->ctx->stream);
  read_tuning(t->ctx);  // no timing record may outlive the tree's plans
  hlc_hmat_free(t->wsC);
  hlc_hmat_free(t->wsL);
  cudaFree(t->d_perm);
  cudaFree(t->d_px);
  cudaFree(t->d_py);
  cudaFree(t->d_dense);
  cudaFree(t->d_lr);
  cudaFree(t->d_diag_off);
  cudaFree(t->d_diag_dim);
  cudaFree(t->d_knu);
  cudaFree(t->d_tmp);
  cudaFree(t->d_vec);
  free_plan(t->chol);
  free_plan(t->fwd);
  free_plan(t->bwd);
  free_plan(t->mv);
  free_plan(t->recomp);
  free_plan(t->lmv);
  free_plan(t->lmvt);
  delete t;
}

int hlc_tree_info(const hlc_tree* t, int64_t* info) {
  if (!t || !info) return HLC_ERR_ARG;
  int64_t leaves = 0, nd = 0, nl = 0;
  for (const Cluster& c : t->T.cl) leaves += c.leaf() ? 1 : 0;
  for (int32_t b : t->T.leaves) (t->T.blk[b].type == BT_DENSE ? nd : nl)++;
  info[0] = t->T.n;
  info[1] = (int64_t)t->T.cl.size();
  info[2] = leaves;
  info[3] = nd;
  info[4] = nl;
  info[5] = t->T.depth;
  info[6] = t->chol_ready ? t->chol.nops() : -1;
  info[7] = t->chol_ready ? t->chol.nwaves : -1;
  return HLC_OK;
}

int hlc_tree_memory(const hlc_tree* t, int64_t* out) {
  if (!t || !out) return HLC_ERR_ARG;
  const HTree& T = t->T;
  const int64_t arena = T.arena_doubles * 8 + (int64_t)T.nslots * 4;
  const int64_t held = (t->wsC ? 1 : 0) + (t->wsL ? 1 : 0);
  const int64_t tmp = t->tmp_cap * 8;
  const int64_t vec = 6 * T.n * 8 + T.n * (4 + 16) + (int64_t)T.dense_asm.size() * sizeof(DenseAsm) +
                      (int64_t)T.lr_asm.size() * sizeof(LrAsm) + t->ndiag * 12 + 2 * KNU_NODES * 8;
  auto plan_bytes = [](const Plan& P) -> int64_t {
    if (!P.checked) return 0;
    return (int64_t)(P.gemm.size() * sizeof(OpGemm) + P.trsm.size() * sizeof(OpTrsm) +
                     P.potrf.size() * sizeof(OpPotrf) + P.trunc.size() * sizeof(OpTrunc) +
                     P.terms.size() * sizeof(TermD) + P.waves.size() * sizeof(WaveRange));
  };
  const int64_t plans = plan_bytes(t->chol) + plan_bytes(t->fwd) + plan_bytes(t->bwd) + plan_bytes(t->mv) +
                        plan_bytes(t->recomp) + plan_bytes(t->lmv) + plan_bytes(t->lmvt);
  out[0] = arena;
  out[1] = held;
  out[2] = tmp;
  out[3] = vec;
  out[4] = plans;
  out[5] = arena * held + tmp + vec + plans;
  return HLC_OK;
}

int hlc_tree_perm(const hlc_tree* t, int32_t* perm) {
  if (!t || !perm) return HLC_ERR_ARG;
  std::copy(t->T.perm.begin(), t->T.perm.end(), perm);
  return HLC_OK;
}

int hlc_tree_leaf_blocks(const hlc_tree* t, int64_t* out) {
  if (!t || !out) return HLC_ERR_ARG;
  size_t q = 0;
  for (int32_t b : t->T.leaves) {
    const Block& B = t->T.blk[b];
    out[5 * q + 0] = t->T.cl[B.r].lo;
    out[5 * q + 1] = t->T.cl[B.r].hi;
    out[5 * q + 2] = t->T.cl[B.s].lo;
    out[5 * q + 3] = t->T.cl[B.s].hi;
    out[5 * q + 4] = B.type;
    ++q;
  }
  return HLC_OK;
}

int hlc_assemble(hlc_ctx* c, hlc_tree* t, const hlc_theta* th, hlc_hmat** C) {
  if (!c || !t || !C || t->ctx != c || !valid_theta(th)) return HLC_ERR_ARG;
  CK(cudaSetDevice(c->device));
  *C = nullptr;
  hlc_hmat* M = nullptr;
  int st = hmat_alloc(t, 0, &M);
  if (st) return st;
  st = do_assemble(t, th, M);
  if (st) {
    hlc_hmat_free(M);
    return st;
  }
  *C = M;
  return HLC_OK;
}

int hlc_cholesky(hlc_ctx* c, const hlc_hmat* C, hlc_hmat** L) {
  if (!c || !C || !L || C->which != 0 || C->t->ctx != c) return HLC_ERR_ARG;
  if (!C->valid) return HLC_ERR_STATE;
  CK(cudaSetDevice(c->device));
  *L = nullptr;
  hlc_hmat* M = nullptr;
  int st = build_plans(C->t, true, false);  // sizes the factor's rank array
  if (st) return st;
  st = hmat_alloc(C->t, 1, &M);
  if (st) return st;
  st = do_cholesky(C->t, C, M);
  if (st) {
    hlc_hmat_free(M);
    return st;
  }
  *L = M;
  return HLC_OK;
}

int hlc_matvec(hlc_ctx* c, const hlc_hmat* C, const double* x, double* y) {
  if (!c || !C || !x || !y || C->which != 0 || C->t->ctx != c) return HLC_ERR_ARG;
  if (!C->valid) return HLC_ERR_STATE;
  hlc_tree* t = C->t;
  CK(cudaSetDevice(c->device));
  int st = build_plans(t, false, true);
  if (st) return st;
  const int64_t n = t->T.n;
  double* X = t->d_vec + n;
  double* Y = t->d_vec + 2 * n;
  double* S = t->d_vec + 3 * n;  // staging
  const bool dx = is_device_ptr(x), dy = is_device_ptr(y);
  if (dx) {
    launch_gather(x, t->d_perm, X, n, c->stream);
  } else {
    CK(cudaMemcpyAsync(S, x, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    launch_gather(S, t->d_perm, X, n, c->stream);
  }
  CK(cudaMemsetAsync(Y, 0, n * sizeof(double), c->stream));
  Bases B = make_bases(t, nullptr, C->arena, C->ranks, false);
  run_plan(t, t->mv, B, c->stream);
  if (dy) {
    launch_scatter(Y, t->d_perm, y, n, c->stream);
  } else {
    launch_scatter(Y, t->d_perm, S, n, c->stream);
    CK(cudaMemcpyAsync(y, S, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return take_status(c);
}

int hlc_factor_apply(hlc_ctx* c, const hlc_hmat* L, int trans, const double* x, double* y) {
  if (!c || !L || !x || !y || L->which != 1 || L->t->ctx != c || (trans != 0 && trans != 1)) return HLC_ERR_ARG;
  if (!L->valid) return HLC_ERR_STATE;
  CK(cudaSetDevice(c->device));
  return factor_apply(L->t, L, trans, x, y);
}

int hlc_sample(hlc_ctx* c, hlc_tree* t, const hlc_theta* th, const double* xi, double* z) {
  if (!c || !t || !xi || !z || t->ctx != c || !valid_theta(th)) return HLC_ERR_ARG;
  CK(cudaSetDevice(c->device));
  int st = build_plans(t, true, false);
  if (st) return st;
  if (!t->wsC && (st = hmat_alloc(t, 0, &t->wsC))) return st;
  if (!t->wsL && (st = hmat_alloc(t, 1, &t->wsL))) return st;
  if ((st = do_assemble(t, th, t->wsC))) return st;
  if ((st = do_cholesky(t, t->wsC, t->wsL))) return st;
  return factor_apply(t, t->wsL, 0, xi, z);
}

// ---------------------------------------------------------------------------
// Accuracy diagnostics (Sec. 3, Tables 2, 3 and 5)
// ---------------------------------------------------------------------------
namespace {

// deterministic N(0, 1) draws on the host: SplitMix64 (Steele, Lea, Flood,
// OOPSLA 2014) for uniforms, Box-Muller for the normals
struct Probe {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  void normals(std::vector<double>& v) {
    for (size_t i = 0; i < v.size(); i += 2) {
      const double r = sqrt(-2.0 * log(uniform())), a = 6.283185307179586 * uniform();
      v[i] = r * cos(a);
      if (i + 1 < v.size()) v[i + 1] = r * sin(a);
    }
  }
};

struct Diag {
  hlc_tree* t;
  hlc_ctx* c;
  cudaStream_t s;
  int64_t n;
  MaternDev mp;
  Bases BL, BC;
  double *W0, *X, *Y;  // the tree's solve / matvec vectors (tree order)
  double dot(const double* a, const double* b) {
    launch_dot(a, b, n, c->d_part, c->d_scalar + 7, s);
    c->launches += 2;
    return read_scalar(c, 7);
  }
  void copy(double* d, const double* a) { cudaMemcpyAsync(d, a, n * sizeof(double), cudaMemcpyDeviceToDevice, s); }
  void scale(double* v, double a) { launch_axpby(0.0, v, a, v, n, s); }
  // out = C~ in
  void hmv(double* out, const double* in) {
    copy(X, in);
    cudaMemsetAsync(Y, 0, n * sizeof(double), s);
    run_plan(t, t->mv, BC, s);
    copy(out, Y);
  }
  // out = C in (exact)
  void xmv(double* out, const double* in) {
    launch_exact_matvec(t->d_px, t->d_py, in, out, n, mp, s);
    c->launches += 1;
  }
  // out = L~^-1 in (trans 0) or L~^-T in (trans 1)
  void solve(double* out, const double* in, int trans) {
    copy(W0, in);
    run_plan(t, trans ? t->bwd : t->fwd, BL, s);
    copy(out, W0);
  }
  // out = L~ in (trans 0) or L~^T in (trans 1)
  void lmul(double* out, const double* in, int trans) {
    copy(W0, in);
    run_plan(t, trans ? t->lmvt : t->lmv, BL, s);
    copy(out, W0);
  }
};

}  // namespace

int hlc_diagnostics(hlc_ctx* c, hlc_tree* t, const hlc_theta* th, int iters, int probes, uint64_t seed,
                    double* out) {
  if (!c || !t || !out || t->ctx != c || !valid_theta(th) || iters < 1 || iters > 1000 || probes < 0 ||
      probes > 10000)
    return HLC_ERR_ARG;
  CK(cudaSetDevice(c->device));
  for (int i = 0; i < 6; ++i) out[i] = -1.0;
  int st = build_plans(t, true, true);
  if (st) return st;
  if ((st = build_lmv_plans(t))) return st;
  if (!t->wsC && (st = hmat_alloc(t, 0, &t->wsC))) return st;
  if (!t->wsL && (st = hmat_alloc(t, 1, &t->wsL))) return st;
  if ((st = do_assemble(t, th, t->wsC))) return st;
  if ((st = do_cholesky(t, t->wsC, t->wsL))) return st;
  const int64_t n = t->T.n;
  const bool exact = n <= kDiagExactMax;
  Diag D;
  D.t = t;
  D.c = c;
  D.s = c->stream;
  D.n = n;
  D.mp = matern_params(t, th);  // the node table is on the device since the assembly
  // FP64 arithmetic throughout (the factor is stored in FP64 in every mode)
  D.BL = make_bases(t, t->wsL->arena, nullptr, t->wsL->ranks, false);
  D.BC = make_bases(t, nullptr, t->wsC->arena, t->wsC->ranks, false);
  D.W0 = t->d_vec;
  D.X = t->d_vec + n;
  D.Y = t->d_vec + 2 * n;
  double* buf = nullptr;
  CK(cudaMalloc(&buf, 5 * n * sizeof(double)));
  double *v = buf, *w = buf + n, *a = buf + 2 * n, *b = buf + 3 * n, *g = buf + 4 * n;
  Probe rng{seed};
  std::vector<double> h(n);
  auto start = [&](double* dst) {
    rng.normals(h);
    cudaMemcpyAsync(dst, h.data(), n * sizeof(double), cudaMemcpyHostToDevice, D.s);
    D.scale(dst, 1.0 / sqrt(D.dot(dst, dst)));
  };
  // power iteration on a symmetric operator: |A v_k| with v_k normalised
  auto power = [&](auto&& apply) {
    start(v);
    double est = 0.0;
    for (int k = 0; k < iters; ++k) {
      apply(w, v);
      est = sqrt(D.dot(w, w));
      if (!(est > 0.0)) break;
      D.copy(v, w);
      D.scale(v, 1.0 / est);
    }
    return est;
  };
  // |C~ - L~ L~^T|_2 and |C~|_2
  out[2] = power([&](double* o, const double* in) {
    D.hmv(a, in);
    D.lmul(b, in, 1);
    D.lmul(o, b, 0);
    launch_axpby(1.0, a, -1.0, o, n, D.s);  // o = C~ in - L L^T in
  });
  out[5] = power([&](double* o, const double* in) { D.hmv(o, in); });
  // |I - (L~ L~^T)^-1 C~|_2: power iteration on A^T A with
  // A = I - P^-1 C~, A^T = I - C~ P^-1, P = L~ L~^T
  {
    auto pinv = [&](double* o, const double* in) {
      D.solve(b, in, 0);
      D.solve(o, b, 1);
    };
    auto A = [&](double* o, const double* in) {
      D.hmv(a, in);
      pinv(o, a);
      launch_axpby(1.0, in, -1.0, o, n, D.s);  // o = in - P^-1 C~ in
    };
    auto At = [&](double* o, const double* in) {
      pinv(a, in);
      D.hmv(o, a);
      launch_axpby(1.0, in, -1.0, o, n, D.s);  // o = in - C~ P^-1 in
    };
    start(v);
    double est = 0.0;
    for (int k = 0; k < iters; ++k) {
      A(g, v);
      est = sqrt(D.dot(g, g));  // |A v|, v the current right singular vector estimate
      At(w, g);
      const double nw = sqrt(D.dot(w, w));
      if (!(nw > 0.0)) break;
      D.copy(v, w);
      D.scale(v, 1.0 / nw);
    }
    out[3] = est;
  }
  if (exact) {
    // |C - C~|_2 and |C|_2 with the exact covariance
    out[0] = power([&](double* o, const double* in) {
      D.xmv(o, in);
      D.hmv(a, in);
      launch_axpby(-1.0, a, 1.0, o, n, D.s);
    });
    out[1] = power([&](double* o, const double* in) { D.xmv(o, in); });
    // KLD(C, C~) = 1/2 (tr(C~^-1 C) - n - log det(C~^-1 C)) = 1/2 sum (d_i - log(1 + d_i)) with d_i the
    // eigenvalues of B = L~^-1 (C - C~) L~^-T; to second order 1/4 |B|_F^2, estimated with Gaussian probes
    // (E |B g|^2 = |B|_F^2)
    if (probes > 0) {
      double acc = 0.0;
      for (int p = 0; p < probes; ++p) {
        rng.normals(h);
        cudaMemcpyAsync(g, h.data(), n * sizeof(double), cudaMemcpyHostToDevice, D.s);
        D.solve(v, g, 1);  // v = L^-T g
        D.xmv(w, v);
        D.hmv(a, v);
        launch_axpby(-1.0, a, 1.0, w, n, D.s);  // w = (C - C~) v
        D.solve(b, w, 0);
        acc += D.dot(b, b);
      }
      out[4] = 0.25 * acc / probes;
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(D.s);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_status(e);
  return take_status(c);
}

int hlc_hmat_expand(hlc_ctx* c, const hlc_hmat* M, double* out) {
  if (!c || !M || !out) return HLC_ERR_ARG;
  hlc_tree* t = M->t;
  const int64_t n = t->T.n;
  if (n > 16384) return HLC_ERR_ARG;
  if (!M->valid) return HLC_ERR_STATE;
  CK(cudaSetDevice(c->device));
  std::vector<double> ar(t->T.arena_doubles);
  std::vector<int> rk(t->T.nslots);
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(ar.data(), M->arena, ar.size() * sizeof(double), cudaMemcpyDeviceToHost));
  if (!rk.empty()) CK(cudaMemcpy(rk.data(), M->ranks, rk.size() * sizeof(int), cudaMemcpyDeviceToHost));
  std::fill(out, out + n * n, 0.0);
  for (int32_t b : t->T.leaves) {
    const Block& B = t->T.blk[b];
    const int64_t r0 = t->T.cl[B.r].lo, c0 = t->T.cl[B.s].lo;
    for (int64_t j = 0; j < B.n; ++j)
      for (int64_t i = 0; i < B.m; ++i) {
        double v = 0.0;
        if (B.type == BT_DENSE) {
          v = ar[B.offD + i + j * B.m];
        } else {
          const int k = rk[B.slot];
          for (int l = 0; l < k; ++l) v += ar[B.offU + i + (int64_t)l * B.m] * ar[B.offV + j + (int64_t)l * B.n];
        }
        if (M->which == 1 && B.diag && j > i) v = 0.0;
        const int64_t ui = t->T.perm[r0 + i], uj = t->T.perm[c0 + j];
        out[ui + uj * n] = v;
        if (M->which == 0 && (r0 + i) != (c0 + j)) out[uj + ui * n] = v;
      }
  }
  return HLC_OK;
}

int hlc_hmat_ranks(hlc_ctx* c, const hlc_hmat* M, int32_t* out) {
  if (!c || !M || !out) return HLC_ERR_ARG;
  hlc_tree* t = M->t;
  CK(cudaSetDevice(c->device));
  std::vector<int> rk(t->T.nslots);
  CK(cudaStreamSynchronize(c->stream));
  if (!rk.empty()) CK(cudaMemcpy(rk.data(), M->ranks, rk.size() * sizeof(int), cudaMemcpyDeviceToHost));
  size_t q = 0;
  for (int32_t b : t->T.leaves) {
    const Block& B = t->T.blk[b];
    out[q++] = B.type == BT_DENSE ? -1 : rk[B.slot];
  }
  return HLC_OK;
}

void hlc_hmat_free(hlc_hmat* M) {
  if (!M) return;
  if (!runtime_alive(M->t->ctx->device)) {
    delete M;
    return;
  }
  cudaFree(M->arena);
  cudaFree(M->ranks);
  delete M;
}

int hlc_loglik(hlc_ctx* c, hlc_tree* t, const hlc_theta* th, const double* z, hlc_result* out) {
  if (!c || !t || !z || !out || t->ctx != c || !valid_theta(th)) return HLC_ERR_ARG;
  CK(cudaSetDevice(c->device));
  std::memset(out, 0, sizeof(*out));
  int st = build_plans(t, true, true);
  if (st) return st;
  if (!t->wsC && (st = hmat_alloc(t, 0, &t->wsC))) return st;
  if (!t->wsL && (st = hmat_alloc(t, 1, &t->wsL))) return st;
  const int64_t n = t->T.n;
  cudaStream_t s = c->stream;
  double* W0 = t->d_vec;
  double* X = t->d_vec + n;
  double* Y = t->d_vec + 2 * n;
  double* Z = t->d_vec + 3 * n;
  double* XS = t->d_vec + 4 * n;
  // data vector to tree order
  if (is_device_ptr(z)) {
    launch_gather(z, t->d_perm, Z, n, s);
    c->launches += 1;
  } else {
    CK(cudaMemcpyAsync(Y, z, n * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_gather(Y, t->d_perm, Z, n, s);
    c->launches += 1;
  }
  CK(cudaEventRecord(c->ev[0], s));
  if ((st = do_assemble(t, th, t->wsC))) return st;
  CK(cudaEventRecord(c->ev[1], s));
  if ((st = do_cholesky(t, t->wsC, t->wsL))) return st;
  CK(cudaEventRecord(c->ev[2], s));
  // the preconditioner solves follow the factor's precision; the residual
  // matvec against C~ is always FP64
  Bases BL = make_bases(t, t->wsL->arena, nullptr, t->wsL->ranks, t->p.precision != HLC_FP64);
  Bases BC = make_bases(t, nullptr, t->wsC->arena, t->wsC->ranks, false);
  // log det = 2 sum log L_ii  (2 launches), and the vector kernels below
  c->launches += 2;
  launch_logdet(t->d_diag_off, t->d_diag_dim, t->ndiag, t->wsL->arena, c->d_part, c->d_scalar + 0, s);
  // v = L^-1 z, quad_factor = v^T v, x = L^-T v
  CK(cudaMemcpyAsync(W0, Z, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  run_plan(t, t->fwd, BL, s);
  launch_dot(W0, W0, n, c->d_part, c->d_scalar + 1, s);
  c->launches += 2;
  run_plan(t, t->bwd, BL, s);
  CK(cudaMemcpyAsync(XS, W0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  launch_dot(Z, Z, n, c->d_part, c->d_scalar + 2, s);
  c->launches += 2;
  const double logdet_half = read_scalar(c, 0);
  const double qf = read_scalar(c, 1);
  const double zn = sqrt(read_scalar(c, 2));
  // Quadratic form: conjugate gradients on C~ preconditioned with
  // (L~ L~^T)^-1, started from x0 = (L~ L~^T)^-1 z (App. B listing).
  // vectors: XS = x, X = p (matvec input), Y = C~ p, W0 = preconditioned r,
  // R = residual (tree workspace slot 5).
  double* R = t->d_vec + 5 * n;
  auto matvec = [&](double* in) {
    if (in != X) cudaMemcpyAsync(X, in, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(Y, 0, n * sizeof(double), s);
    run_plan(t, t->mv, BC, s);
  };
  matvec(XS);
  launch_sub(Z, Y, R, n, s);
  c->launches += 1;
  launch_dot(R, R, n, c->d_part, c->d_scalar + 3, s);
  c->launches += 2;
  int it = 0;
  std::vector<double> cg_alpha, cg_beta;  // CG step and update coefficients
  double rel = zn > 0.0 ? sqrt(read_scalar(c, 3)) / zn : 0.0;
  if (rel > t->p.refine_tol && t->p.refine_maxit > 0) {
    CK(cudaMemcpyAsync(W0, R, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    run_plan(t, t->fwd, BL, s);
    run_plan(t, t->bwd, BL, s);
    CK(cudaMemcpyAsync(X, W0, n * sizeof(double), cudaMemcpyDeviceToDevice, s));  // p = w
    launch_dot(R, W0, n, c->d_part, c->d_scalar + 5, s);
    c->launches += 2;
    double rw = read_scalar(c, 5);
    while (it < t->p.refine_maxit) {
      matvec(X);  // Y = C p
      launch_dot(X, Y, n, c->d_part, c->d_scalar + 6, s);
      c->launches += 2;
      const double alpha = rw / read_scalar(c, 6);
      cg_alpha.push_back(alpha);
      launch_axpby(alpha, X, 1.0, XS, n, s);
      c->launches += 1;
      launch_axpby(-alpha, Y, 1.0, R, n, s);
      c->launches += 1;
      ++it;
      launch_dot(R, R, n, c->d_part, c->d_scalar + 3, s);
      c->launches += 2;
      rel = zn > 0.0 ? sqrt(read_scalar(c, 3)) / zn : 0.0;
      if (!(rel > t->p.refine_tol)) break;
      CK(cudaMemcpyAsync(W0, R, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      run_plan(t, t->fwd, BL, s);
      run_plan(t, t->bwd, BL, s);
      launch_dot(R, W0, n, c->d_part, c->d_scalar + 5, s);
      c->launches += 2;
      const double rw1 = read_scalar(c, 5);
      const double beta = rw1 / rw;
      cg_beta.push_back(beta);
      rw = rw1;
      launch_axpby(1.0, W0, beta, X, n, s);
      c->launches += 1;  // p = w + beta p
    }
    // true residual at exit
    matvec(XS);
    launch_sub(Z, Y, R, n, s);
    c->launches += 1;
    launch_dot(R, R, n, c->d_part, c->d_scalar + 3, s);
    c->launches += 2;
    rel = zn > 0.0 ? sqrt(read_scalar(c, 3)) / zn : 0.0;
  }
  launch_dot(Z, XS, n, c->d_part, c->d_scalar + 4, s);
  c->launches += 2;
  const double quad = read_scalar(c, 4);
  CK(cudaEventRecord(c->ev[3], s));
  CK(cudaEventSynchronize(c->ev[3]));
  if ((st = take_status(c))) return st;
  float ms[3];
  cudaEventElapsedTime(&ms[0], c->ev[0], c->ev[1]);
  cudaEventElapsedTime(&ms[1], c->ev[1], c->ev[2]);
  cudaEventElapsedTime(&ms[2], c->ev[2], c->ev[3]);
  const double logdet = 2.0 * logdet_half;
  if (!(logdet == logdet) || !(quad == quad)) return HLC_ERR_NUMERIC;
  out->logdet = logdet;
  out->quad = quad;
  out->quad_factor = qf;
  out->loglik = -0.5 * (double)n * log(2.0 * M_PI) - 0.5 * logdet - 0.5 * quad;
  out->refine_iters = it;
  out->rel_residual = rel;
  out->est_rel_err = lanczos_rel_err(cg_alpha, cg_beta);
  out->ms_assemble = ms[0];
  out->ms_factor = ms[1];
  out->ms_solve = ms[2];
  hmat_stats(t, t->wsC, &out->bytes_C, &out->max_rank_C);
  hmat_stats(t, t->wsL, &out->bytes_L, &out->max_rank_L);
  return HLC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The matvec without allocation.  The paper has no counterpart: it concerns
// how the library meets callers that may not allocate device memory during a
// call.  Such callers exist.  A host framework may hold all free device memory
// in its own caching pool, so a cudaMalloc of ours would fail or force the
// pool to release memory.  A latency-bound loop may not afford the
// device-wide synchronisation that cudaMalloc and cudaFree can cause.  An
// out-of-memory handler must not allocate at all.  hlc_matvec can allocate (it
// builds and uploads plans and sizes the tree's workspaces on demand); this
// variant keeps its vectors and the plan's temporaries in one fixed buffer
// that belongs to the loaded module and allocates nothing per call.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocDoubles = int64_t(8) << 20;  // 64 MiB
__device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kNoAllocMaxDevices = 256;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the buffer on `device`, which the caller has made
// current; looked up once per device.  The first lookup may load the module
// on that device (lazy loading), which is where the buffer's memory comes
// from.
int noalloc_scratch(int device, double** out) {
  if (device < 0 || device >= kNoAllocMaxDevices) return HLC_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return HLC_ERR_CUDA;
    }
    g_noalloc_addr[device] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[device];
  return HLC_OK;
}

}  // namespace

extern "C" {

int64_t hlc_matvec_noalloc_capacity(void) { return kNoAllocDoubles; }

int hlc_selftest_barrier_timeout(hlc_ctx* c) {
  if (!c) return HLC_ERR_ARG;
  CK(cudaSetDevice(c->device));
  if (launch_barrier_probe(c->d_gridbar, c->d_status, c->stream) != 0) {
    cudaGetLastError();
    return HLC_ERR_CUDA;
  }
  return take_status(c);
}

int hlc_matvec_noalloc(hlc_ctx* c, const hlc_hmat* C, const double* x, double* y) {
  if (!c || !C || !x || !y || C->which != 0 || C->t->ctx != c) return HLC_ERR_ARG;
  if (!C->valid) return HLC_ERR_STATE;
  hlc_tree* t = C->t;
  // the matvec plan must exist already (built by hlc_matvec or hlc_loglik)
  if (!t->solve_ready || !t->mv.d_waves || t->mv.waves.empty()) return HLC_ERR_STATE;
  CK(cudaSetDevice(c->device));
  if (!is_device_ptr(x) || !is_device_ptr(y)) return HLC_ERR_ARG;
  const int64_t n = t->T.n;
  // buffer layout (doubles): [0, n) unused, x in tree order at [n, 2n), y at
  // [2n, 3n) (the offsets the matvec plan was built with), temporaries after
  if (3 * n + t->mv.tmp_doubles > kNoAllocDoubles) return HLC_ERR_SCRATCH;
  double* S = nullptr;
  int st = noalloc_scratch(c->device, &S);
  if (st) return st;
  launch_gather(x, t->d_perm, S + n, n, c->stream);
  // y accumulates, so it starts at zero; the temporaries are written before
  // they are read and the grid barrier's state is zeroed by its launch
  CK(cudaMemsetAsync(S + 2 * n, 0, n * sizeof(double), c->stream));
  Bases B = make_bases(t, nullptr, C->arena, C->ranks, false);
  B.buf[BUF_VEC] = S;
  B.buf[BUF_TMP] = S + 3 * n;
  // the same choice as for every other plan run: one persistent launch when
  // the context and the environment allow it and the cooperative launch is
  // available, else the waves one launch at a time (neither allocates)
  const int md = (int)std::max<int64_t>(t->T.max_dense_dim, t->T.leaf);
  bool done = false;
  if (c->persistent && !c->profiling && !g_prof.on && persistent_enabled()) {
    if (launch_persistent(t->mv, B, c->d_gridbar, md, t->mv.tuned_per_sm, c->stream) == 0) {
      done = true;
      c->launches += 1;
      c->persistent_launches += 1;
    } else {
      cudaGetLastError();
    }
  }
  if (!done) run_plan_launches(t, t->mv, B, c->stream, true);
  launch_scatter(S + 2 * n, t->d_perm, y, n, c->stream);
  c->launches += 2;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return take_status(c);
}

}  // extern "C"
