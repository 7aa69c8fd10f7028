// kernels.cu -- sm_103a kernels of the H-matrix likelihood.
//
//   k_dense_asm   dense inadmissible leaves of C~ (eq. 3 + nugget, Sec. 4.1)
//   k_aca         ACA with partial pivoting for admissible leaves (App. B)
//   k_potrf       Cholesky of dense diagonal leaves (eq. 2), FP64
//   k_trsm        triangular solves with dense diagonal leaves (FP64, or
//                 FP32 in the mixed modes)
//   k_gemm        strided multiply-add of dense views (H-arithmetic, Table 1),
//                 with a matrix-vector path for one column
//   k_chain       chains: the ops of a small diagonal block's solve in order,
//                 by one CTA
//   k_flow        a whole triangular solve or matvec as one cooperative launch,
//                 every op started when its own producers are done (bounded
//                 waits on per-op arrival counters)
//   k_waves       the same, wave by wave with a bounded grid barrier between
//                 waves
//   reductions    log det = 2 sum log L_ii, dot products (fixed order)
//
// The truncated low-rank sums (Remark A.1) are in trunc.cu.  Op kernels take
// a list of descriptors produced by the planner and loop over it
// grid-stride, one op per CTA at a time.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hlc_internal.h"
#include "kernels.h"
#include "matern.cuh"
#include "devutil.cuh"
#include "ops.cuh"

namespace hlc {

// ---------------------------------------------------------------------------
// Assembly
// ---------------------------------------------------------------------------
__global__ void k_dense_asm(const DenseAsm* blks, int64_t count, double* arena, const double* px,
                            const double* py, MaternDev mp) {
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) {
    const DenseAsm b = blks[o];
    double* D = arena + b.off;
    const int64_t tot = (int64_t)b.m * b.n;
    for (int64_t e = threadIdx.x; e < tot; e += blockDim.x) {
      const int64_t i = e % b.m, j = e / b.m;
      const int64_t gi = b.r0 + i, gj = b.c0 + j;
      double v = matern_f64(dist_f64(px[gi], py[gi], px[gj], py[gj]), mp);
      if (gi == gj) v += mp.nugget;
      D[e] = v;
    }
  }
}

constexpr int ACA_THREADS = 256;

// ACA with partial pivoting.  U (m x kcap) gets the residual columns, V
// (n x kcap) the residual rows divided by the pivot.  Stops when
// |u_k| |v_k| <= eps |S_k|_F (running Frobenius norm of the approximant).
// A vanishing pivot row moves to the first unused row, at most three times
// in a row.  Used rows and columns are excluded from the pivot searches.
// The assembled C~ is the matrix the FP64 refinement residual is taken
// against in every precision mode, so the ACA runs in FP64 (T = double).
template <class T>
__device__ __forceinline__ T aca_entry(double x0, double y0, double x1, double y1, const MaternDev& mp);
template <>
__device__ __forceinline__ double aca_entry<double>(double x0, double y0, double x1, double y1, const MaternDev& mp) {
  return matern_f64(dist_f64(x0, y0, x1, y1), mp);
}

// Capacities of the per-block pivot bookkeeping: ranks up to ACA_KCAP
// (the largest kmax a tree accepts), and every used row, including the
// rows that were skipped as zero (at most 3 in a row per accepted pivot).
constexpr int ACA_KCAP = 128;
constexpr int ACA_ROWS = 4 * ACA_KCAP;

template <class T>
__global__ void __launch_bounds__(ACA_THREADS) k_aca(const LrAsm* blks, int64_t count, double* arena,
                                                      const double* px, const double* py, MaternDev mp,
                                                      double eps, int kfix, int* ranks, int* status) {
  __shared__ double s_ui[ACA_KCAP], s_vj[ACA_KCAP];
  __shared__ double s_cu[ACA_THREADS / 32][8], s_cv[ACA_THREADS / 32][8];
  __shared__ int used_r[ACA_ROWS], used_c[ACA_KCAP];
  __shared__ double redv[33];
  __shared__ int redi[33];
  const int tid = threadIdx.x;
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) {
    const LrAsm b = blks[o];
    const int m = b.m, n = b.n;
    // kcap > ACA_KCAP is refused when the tree is laid out; clamp anyway so
    // that no index below can leave the shared arrays
    int kcap = b.kcap < ACA_KCAP ? b.kcap : ACA_KCAP;
    // fixed-rank mode: at most kfix crosses, reaching them is not an error
    const bool fixed_stop = kfix > 0 && kfix < kcap;
    if (fixed_stop) kcap = kfix;
    double* U = arena + b.offU;
    double* V = arena + b.offV;
    int k = 0, next = 0, zero_tries = 0, nur = 0, nuc = 0;
    double s2 = 0.0;
    bool converged = false;
    while (k < kcap && nur < ACA_ROWS) {
      const int i = next;
      __syncthreads();
      if (tid == 0) used_r[nur] = i;
      if (tid < k) s_ui[tid] = U[i + (int64_t)tid * m];
      __syncthreads();
      ++nur;
      // residual row i into V[:, k]; pivot search over unused columns
      double best = -1.0;
      int bj = -1;
      const double xi = px[b.r0 + i], yi = py[b.r0 + i];
      for (int j = tid; j < n; j += blockDim.x) {
        T v = aca_entry<T>(xi, yi, px[b.c0 + j], py[b.c0 + j], mp);
        for (int l = 0; l < k; ++l) v -= (T)s_ui[l] * (T)V[j + (int64_t)l * n];
        V[j + (int64_t)k * n] = (double)v;
        bool used = false;
        for (int q = 0; q < nuc; ++q) used |= (used_c[q] == j);
        const double a = fabs((double)v);
        if (!used && (a > best || (a == best && (bj < 0 || j < bj)))) {
          best = a;
          bj = j;
        }
      }
      double bval;
      const int jp = block_argmax(best, bj, redv, redi, &bval);
      if (jp < 0) {  // every column used: the approximant is exact
        converged = true;
        break;
      }
      if (bval == 0.0) {
        // the residual vanishes on this row; after three such rows in a
        // row the residual is taken to be zero (the stopping rule of ACA)
        if (++zero_tries > 3) {
          converged = true;
          break;
        }
        // first unused row
        int nx = -1;
        for (int t = 0; t < m && nx < 0; ++t) {
          bool u = false;
          for (int q = 0; q < nur; ++q) u |= (used_r[q] == t);
          if (!u) nx = t;
        }
        if (nx < 0) {  // every row used: exact
          converged = true;
          break;
        }
        next = nx;
        continue;
      }
      zero_tries = 0;
      __syncthreads();
      const double piv = V[jp + (int64_t)k * n];
      __syncthreads();
      for (int j = tid; j < n; j += blockDim.x) V[j + (int64_t)k * n] = (double)((T)V[j + (int64_t)k * n] / (T)piv);
      if (tid < k) s_vj[tid] = V[jp + (int64_t)tid * n];
      if (tid == 0) used_c[nuc] = jp;
      __syncthreads();
      ++nuc;
      // residual column jp into U[:, k]
      const double xj = px[b.c0 + jp], yj = py[b.c0 + jp];
      for (int t = tid; t < m; t += blockDim.x) {
        T u = aca_entry<T>(px[b.r0 + t], py[b.r0 + t], xj, yj, mp);
        for (int l = 0; l < k; ++l) u -= (T)U[t + (int64_t)l * m] * (T)s_vj[l];
        U[t + (int64_t)k * m] = (double)u;
      }
      __syncthreads();
      // norms: |u|^2, |v|^2 and the cross terms (U_l . u)(V_l . v)
      double uu = 0.0, vv = 0.0;
      for (int t = tid; t < m; t += blockDim.x) uu += U[t + (int64_t)k * m] * U[t + (int64_t)k * m];
      for (int t = tid; t < n; t += blockDim.x) vv += V[t + (int64_t)k * n] * V[t + (int64_t)k * n];
      uu = block_sum(uu, redv);
      vv = block_sum(vv, redv);
      double cross = 0.0;
      for (int l0 = 0; l0 < k; l0 += 8) {
        const int nl = min(8, k - l0);
        double au[8], av[8];
        for (int q = 0; q < 8; ++q) au[q] = av[q] = 0.0;
        for (int t = tid; t < m; t += blockDim.x) {
          const double ut = U[t + (int64_t)k * m];
          for (int q = 0; q < nl; ++q) au[q] += U[t + (int64_t)(l0 + q) * m] * ut;
        }
        for (int t = tid; t < n; t += blockDim.x) {
          const double vt = V[t + (int64_t)k * n];
          for (int q = 0; q < nl; ++q) av[q] += V[t + (int64_t)(l0 + q) * n] * vt;
        }
        const int lane = tid & 31, w = tid >> 5;
        for (int q = 0; q < 8; ++q) {
          au[q] = warp_sum(au[q]);
          av[q] = warp_sum(av[q]);
        }
        __syncthreads();
        if (lane == 0)
          for (int q = 0; q < 8; ++q) {
            s_cu[w][q] = au[q];
            s_cv[w][q] = av[q];
          }
        __syncthreads();
        double c = 0.0;
        for (int q = 0; q < nl; ++q) {
          double a = 0.0, bb = 0.0;
          for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) {
            a += s_cu[ww][q];
            bb += s_cv[ww][q];
          }
          c += a * bb;
        }
        cross += c;
      }
      s2 += 2.0 * cross + uu * vv;
      ++k;
      if (sqrt(uu) * sqrt(vv) <= eps * sqrt(fmax(s2, 0.0))) {
        converged = true;
        break;
      }
      // next pivot row: largest |u| among unused rows
      best = -1.0;
      int bi = -1;
      for (int t = tid; t < m; t += blockDim.x) {
        bool used = false;
        for (int q = 0; q < nur; ++q) used |= (used_r[q] == t);
        const double a = fabs(U[t + (int64_t)(k - 1) * m]);
        if (!used && (a > best || (a == best && (bi < 0 || t < bi)))) {
          best = a;
          bi = t;
        }
      }
      const int ip = block_argmax(best, bi, redv, redi, &bval);
      if (ip < 0) {
        converged = true;
        break;
      }
      next = ip;
    }
    __syncthreads();
    // A block that reached its rank capacity before the stopping test held
    // is not accurate to eps: reported as a rank overflow, unless the
    // capacity is the full rank min(m, n), where the approximant is exact.
    if (tid == 0) {
      ranks[b.slot] = k;
      if (!converged && !fixed_stop && k < (m < n ? m : n)) record_error(status, DEV_RANK, k);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// POTRF: dense lower Cholesky of a diagonal leaf (n <= 128), right-looking,
// one op per CTA (do_potrf in ops.cuh).
// ---------------------------------------------------------------------------
__global__ void k_potrf(const OpPotrf* ops, int64_t count, Bases B) {
  extern __shared__ double sm[];
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) do_potrf(ops[o], B, sm);
}

template <class T>
__global__ void k_trsm(const OpTrsm* ops, int64_t count, Bases B) {
  extern __shared__ double smd[];
  T* sL = reinterpret_cast<T*>(smd);
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) do_trsm<T>(ops[o], B, sL);
}

template <class T>
__global__ void __launch_bounds__(256) k_gemm(const OpGemm* ops, int64_t count, Bases B) {
  __shared__ GemmSmem<T> sm;
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) do_gemm<T>(ops[o], B, sm);
}

// A chain: its TRSM and GEMM ops in order, by the whole CTA, a block barrier
// after each (the next op may read what this one wrote).
template <class T>
__device__ void do_chain(const OpChain& c, const ChainTab& ct, const Bases& B, T* sL, GemmSmem<T>& gs) {
  for (int32_t q = 0; q < c.nitems; ++q) {
    const ChainItem it = ct.items[c.item0 + q];
    if (it.type == OP_TRSM)
      do_trsm<T>(ct.trsm[it.idx], B, sL);
    else
      do_gemm<T>(ct.gemm[it.idx], B, gs);
    __syncthreads();
  }
}

template <class T>
__global__ void __launch_bounds__(256) k_chain(const OpChain* ops, int64_t count, ChainTab ct, Bases B) {
  extern __shared__ double smd[];
  __shared__ GemmSmem<T> gs;
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) do_chain<T>(ops[o], ct, B, reinterpret_cast<T*>(smd), gs);
}

// Grid-wide barrier of the persistent kernel: bounded_barrier (devutil.cuh)
// over all CTAs of the grid, on the grid's barrier record.
// `expected`: arrivals that release the barrier (the grid size; the
// self-test asks for one more than the grid has, so only the time limit can
// end the wait).
__device__ bool grid_barrier(GridBar* gb, int* status, unsigned int expected) {
  return bounded_barrier(&gb->count, &gb->gen, expected, &gb->abort, status);
}

// Persistent execution of a plan made of TRSM and GEMM ops (the solves and
// the matvec): one cooperative launch (all CTAs co-resident) walks the waves;
// within a wave the CTAs take the ops round-robin, and a grid barrier
// separates consecutive waves.
__global__ void __launch_bounds__(256) k_waves(const WaveRange* waves, int nwaves, const OpTrsm* trsm,
                                               const OpGemm* gemm, const OpChain* chain, ChainTab ct, Bases B,
                                               GridBar* gb) {
  extern __shared__ double sL[];
  __shared__ GemmSmem<double> gd;
  __shared__ GemmSmem<float> gf;
  for (int w = 0; w < nwaves; ++w) {
    const WaveRange wr = waves[w];
    const int64_t tot = wr.ntrsm + wr.ngemm + wr.nchain;
    for (int64_t o = blockIdx.x; o < tot; o += gridDim.x) {
      if (o < wr.ntrsm) {
        if (B.mixed)
          do_trsm<float>(trsm[wr.trsm0 + o], B, reinterpret_cast<float*>(sL));
        else
          do_trsm<double>(trsm[wr.trsm0 + o], B, sL);
      } else if (o < wr.ntrsm + wr.ngemm) {
        if (B.mixed)
          do_gemm<float>(gemm[wr.gemm0 + (o - wr.ntrsm)], B, gf);
        else
          do_gemm<double>(gemm[wr.gemm0 + (o - wr.ntrsm)], B, gd);
      } else {
        const OpChain& c = chain[wr.chain0 + (o - wr.ntrsm - wr.ngemm)];
        if (B.mixed)
          do_chain<float>(c, ct, B, reinterpret_cast<float*>(sL), gf);
        else
          do_chain<double>(c, ct, B, sL, gd);
      }
      __syncthreads();
    }
    if (w + 1 < nwaves && !grid_barrier(gb, B.status, gridDim.x)) return;
  }
}

// Dependency-driven execution of a TRSM/GEMM plan (one cooperative launch,
// all CTAs resident).  The ops are numbered in wave order; each CTA takes
// the next number from a ticket counter, waits until every producer of that
// op has signalled (count[i] == npred[i]), runs it, and signals its
// successors.  Because tickets go out in wave order and every producer has a
// smaller number, the unfinished op with the smallest number always has all
// of its producers done, so the launch always progresses.  The wait is
// bounded like the grid barrier's: after kBarrierNs, or once another CTA has
// given up, the CTA records DEV_TIMEOUT, raises the abort flag and leaves.
// Every op computes exactly what it computes in a wave, in the same order
// relative to the ops it depends on: the results are those of the waves.
__global__ void __launch_bounds__(256) k_flow(const FlowOp* flow, int64_t nops, const int32_t* npred,
                                              const int64_t* succ_off, const int32_t* succ, int32_t* count,
                                              const OpTrsm* trsm, const OpGemm* gemm, Bases B, GridBar* gb,
                                              FactorTrace* trace, int64_t smem_entries) {
  extern __shared__ double sL[];
  __shared__ GemmSmem<double> gd;
  __shared__ GemmSmem<float> gf;
  __shared__ long long s_op;
  __shared__ int s_ok, s_go;
  unsigned long long* ticket = &gb->ticket;
  for (;;) {
    if (threadIdx.x == 0) {
      volatile unsigned int* abort = &gb->abort;
      long long i = -1;
      if (!*abort) i = (long long)atomicAdd(ticket, 1ull);
      s_op = i;
      s_ok = i >= 0 && i < nops;
      if (s_ok && trace) {
        trace[i].t_take = global_ns();
        trace[i].cta = (uint32_t)blockIdx.x;
      }
    }
    __syncthreads();
    if (!s_ok) return;
    const FlowOp f = flow[s_op];
    // a solve's factor block (a matvec's block of C~) is final: load it while
    // the producers finish
    bool pre = false;
    const OpGemm* g = f.type == OP_GEMM ? gemm + f.idx : f.group >= 0 ? gemm + f.group : nullptr;
    if (f.type == OP_TRSM) {
      // the block, then (when it fits beside it) the joined product's operand
      const int64_t used = (int64_t)trsm[f.idx].n * trsm[f.idx].n + trsm[f.idx].n;
      if (B.mixed) {
        trsm_load<float>(trsm[f.idx], B, reinterpret_cast<float*>(sL));
        if (g) pre = gemv_prefetch<float>(*g, B, reinterpret_cast<float*>(sL) + used, 2 * smem_entries - used);
      } else {
        trsm_load<double>(trsm[f.idx], B, sL);
        if (g) pre = gemv_prefetch<double>(*g, B, sL + used, smem_entries - used);
      }
    } else if (B.mixed) {
      pre = gemv_prefetch<float>(gemm[f.idx], B, reinterpret_cast<float*>(sL), 2 * smem_entries);
    } else {
      pre = gemv_prefetch<double>(gemm[f.idx], B, sL, smem_entries);
    }
    if (threadIdx.x == 0) {
      // wait for the producers of the op
      volatile unsigned int* abort = &gb->abort;
      const volatile int32_t* cnt = count + s_op;
      const int32_t need = npred[s_op];
      const unsigned long long t0 = global_ns();
      int ok = 1;
      while (*cnt < need) {
        if (*abort || global_ns() - t0 > kBarrierNs) {
          atomicExch(&gb->abort, 1u);
          record_error(B.status, DEV_TIMEOUT, 1);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
      __threadfence();
      if (trace) trace[s_op].t_ready = global_ns();
      s_go = ok;  // not s_ok: another thread may still be reading it
    }
    __syncthreads();
    if (!s_go) return;
    if (f.type == OP_TRSM) {
      const int64_t used = (int64_t)trsm[f.idx].n * trsm[f.idx].n + trsm[f.idx].n;
      if (g) {  // the joined product first: it writes the rows the TRSM reads
        if (pre && B.mixed)
          do_gemv_pre<float>(*g, B, reinterpret_cast<const float*>(sL) + used);
        else if (pre)
          do_gemv_pre<double>(*g, B, sL + used);
        else if (B.mixed)
          do_gemm<float>(*g, B, gf);
        else
          do_gemm<double>(*g, B, gd);
        __syncthreads();
      }
      if (B.mixed)
        trsm_apply<float>(trsm[f.idx], B, reinterpret_cast<const float*>(sL));
      else
        trsm_apply<double>(trsm[f.idx], B, sL);
    } else if (pre) {
      if (B.mixed)
        do_gemv_pre<float>(gemm[f.idx], B, reinterpret_cast<const float*>(sL));
      else
        do_gemv_pre<double>(gemm[f.idx], B, sL);
    } else if (B.mixed) {
      do_gemm<float>(gemm[f.idx], B, gf);
    } else {
      do_gemm<double>(gemm[f.idx], B, gd);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // the op's writes before its signals
      if (trace) {
        trace[s_op].t_done = global_ns();
        for (int64_t e = succ_off[s_op]; e < succ_off[s_op + 1]; ++e) {
          const int32_t v = succ[e];
          if (atomicAdd(count + v, 1) + 1 == npred[v]) trace[v].releaser = (int32_t)s_op;
        }
      } else {
        for (int64_t e = succ_off[s_op]; e < succ_off[s_op + 1]; ++e) atomicAdd(count + succ[e], 1);
      }
    }
  }
}

int launch_flow(const FlowOp* flow, int64_t nops, const int32_t* npred, const int64_t* succ_off, const int32_t* succ,
                int32_t* count, const OpTrsm* trsm, const OpGemm* gemm, const Bases& B, GridBar* gb, int max_dense,
                int per_sm, FactorTrace* trace, cudaStream_t st) {
  int maxper = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&maxper, k_flow, 256, trsm_smem(max_dense)) != cudaSuccess)
    return -1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per = (per_sm <= 0 || per_sm > maxper) ? maxper : per_sm;
  const int grid = per * sms;
  if (grid <= 0 || nops <= 0 || !gb || !count) return -1;
  if (cudaMemsetAsync(gb, 0, sizeof(GridBar), st) != cudaSuccess) return -1;
  if (cudaMemsetAsync(count, 0, nops * sizeof(int32_t), st) != cudaSuccess) return -1;
  int64_t sent = (int64_t)(trsm_smem(max_dense) / sizeof(double));  // dynamic shared memory in doubles
  void* args[] = {(void*)&flow, (void*)&nops, (void*)&npred, (void*)&succ_off, (void*)&succ, (void*)&count,
                  (void*)&trsm, (void*)&gemm, (void*)&B, (void*)&gb, (void*)&trace, (void*)&sent};
  return cudaLaunchCooperativeKernel((void*)k_flow, grid, 256, args, trsm_smem(max_dense), st) == cudaSuccess ? 0
                                                                                                               : -1;
}

// Self-test of the bounded wait: every CTA arrives, one arrival more is
// expected, so the barrier ends only by its time limit (DEV_TIMEOUT).
__global__ void k_barrier_probe(GridBar* gb, int* status) {
  grid_barrier(gb, status, gridDim.x + 1);
}

int launch_barrier_probe(GridBar* gb, int* status, cudaStream_t st) {
  if (!gb || !status) return -1;
  if (cudaMemsetAsync(gb, 0, sizeof(GridBar), st) != cudaSuccess) return -1;
  k_barrier_probe<<<2, 32, 0, st>>>(gb, status);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// CTAs of the persistent kernel that fit on one SM (all must be resident)
int waves_max_per_sm(int max_dense) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_waves, 256, trsm_smem(max_dense)) != cudaSuccess)
    return 0;
  return per;
}

int launch_waves(const WaveRange* waves, int nwaves, const OpTrsm* trsm, const OpGemm* gemm, const OpChain* chain,
                 const ChainTab& ct, const Bases& B, GridBar* gb, int max_dense, int per_sm, cudaStream_t st) {
  const int maxper = waves_max_per_sm(max_dense);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per = (per_sm <= 0 || per_sm > maxper) ? maxper : per_sm;
  const int grid = per * sms;
  if (grid <= 0 || nwaves <= 0 || !gb) return -1;
  if (cudaMemsetAsync(gb, 0, sizeof(GridBar), st) != cudaSuccess) return -1;
  void* args[] = {(void*)&waves, (void*)&nwaves, (void*)&trsm, (void*)&gemm, (void*)&chain, (void*)&ct, (void*)&B,
                  (void*)&gb};
  return cudaLaunchCooperativeKernel((void*)k_waves, grid, 256, args, trsm_smem(max_dense),
                                     st) == cudaSuccess
             ? 0
             : -1;
}

// ---------------------------------------------------------------------------
// Exact covariance matvec (accuracy diagnostics): y = C x with C_ij the
// Matern function of eq. (3) plus the nugget on the diagonal, every entry
// evaluated on the fly in FP64; one thread per row, the columns in tiles
// staged in shared memory and summed in increasing order (deterministic).
// ---------------------------------------------------------------------------
constexpr int XMV_TILE = 256;

__global__ void __launch_bounds__(XMV_TILE) k_exact_matvec(const double* px, const double* py, const double* x,
                                                           double* y, int64_t n, MaternDev mp) {
  __shared__ double sx[XMV_TILE], sy[XMV_TILE], sv[XMV_TILE];
  for (int64_t r0 = (int64_t)blockIdx.x * XMV_TILE; r0 < n; r0 += (int64_t)gridDim.x * XMV_TILE) {
    const int64_t i = r0 + threadIdx.x;
    const double xi = i < n ? px[i] : 0.0, yi = i < n ? py[i] : 0.0;
    double acc = 0.0;
    for (int64_t c0 = 0; c0 < n; c0 += XMV_TILE) {
      const int64_t j = c0 + threadIdx.x;
      __syncthreads();
      sx[threadIdx.x] = j < n ? px[j] : 0.0;
      sy[threadIdx.x] = j < n ? py[j] : 0.0;
      sv[threadIdx.x] = j < n ? x[j] : 0.0;
      __syncthreads();
      const int cnt = (int)(n - c0 < XMV_TILE ? n - c0 : XMV_TILE);
      if (i < n)
        for (int q = 0; q < cnt; ++q) {
          double c = matern_f64(dist_f64(xi, yi, sx[q], sy[q]), mp);
          if (c0 + q == i) c += mp.nugget;
          acc += c * sv[q];
        }
    }
    if (i < n) y[i] = acc;
  }
}

void launch_exact_matvec(const double* px, const double* py, const double* x, double* y, int64_t n,
                         const MaternDev& mp, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t blocks = (n + XMV_TILE - 1) / XMV_TILE;
  k_exact_matvec<<<(int)(blocks < 152 * 8 ? blocks : 152 * 8), XMV_TILE, 0, st>>>(px, py, x, y, n, mp);
}

// ---------------------------------------------------------------------------
// small utilities
// ---------------------------------------------------------------------------
__global__ void k_gather(const double* src, const int32_t* perm, double* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[perm[i]];
}
__global__ void k_scatter(const double* src, const int32_t* perm, double* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[perm[i]] = src[i];
}
__global__ void k_points(const double* xy, const int32_t* perm, double* px, double* py, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p = perm[i];
    px[i] = xy[2 * (int64_t)p];
    py[i] = xy[2 * (int64_t)p + 1];
  }
}
// y = a*x + b*y
__global__ void k_axpby(double a, const double* x, double b, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}
// z = x - y
__global__ void k_sub(const double* x, const double* y, double* z, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = x[i] - y[i];
}

// Deterministic dot product: fixed grid of RED_BLOCKS partial sums, then a
// single-CTA pairwise sum.
constexpr int RED_BLOCKS = 304;
__global__ void k_dot_part(const double* x, const double* y, int64_t n, double* part) {
  __shared__ double red[33];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += x[i] * y[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}
__global__ void k_sum_final(const double* part, int64_t count, double* out) {
  __shared__ double red[33];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// log det contribution of the dense diagonal leaves: part[b] = sum log L_ii
__global__ void k_logdet_part(const int64_t* offs, const int32_t* dims, int64_t count, const double* arena,
                              double* part) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < count; b += (int64_t)gridDim.x * blockDim.x) {
    const double* D = arena + offs[b];
    const int n = dims[b];
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += log(D[i + (int64_t)i * n]);
    part[b] = s;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_for(int64_t count, int cap) { return (int)(count < cap ? count : cap); }

void launch_dense_asm(const DenseAsm* d, int64_t count, double* arena, const double* px, const double* py,
                      const MaternDev& mp, cudaStream_t st) {
  if (count <= 0) return;
  k_dense_asm<<<grid_for(count, 152 * 16), 256, 0, st>>>(d, count, arena, px, py, mp);
}
void launch_aca(const LrAsm* d, int64_t count, double* arena, const double* px, const double* py,
                const MaternDev& mp, double eps, int kfix, int* ranks, int* status, cudaStream_t st) {
  if (count <= 0) return;
  k_aca<double><<<grid_for(count, 152 * 8), ACA_THREADS, 0, st>>>(d, count, arena, px, py, mp, eps, kfix, ranks,
                                                                   status);
}


void launch_ops(int type, const void* ops, int64_t count, const TermD* terms, const ChainTab& ct, const Bases& B,
                int max_dense, cudaStream_t st) {
  if (count <= 0) return;
  switch (type) {
    case OP_CHAIN:
      if (B.mixed)
        k_chain<float><<<grid_for(count, 152 * 8), 256, trsm_smem(max_dense), st>>>((const OpChain*)ops, count, ct, B);
      else
        k_chain<double><<<grid_for(count, 152 * 8), 256, trsm_smem(max_dense), st>>>((const OpChain*)ops, count, ct,
                                                                                      B);
      break;
    case OP_POTRF:
      k_potrf<<<grid_for(count, 152 * 8), 128, (size_t)max_dense * max_dense * sizeof(double), st>>>(
          (const OpPotrf*)ops, count, B);
      break;
    case OP_TRSM:
      if (B.mixed)
        k_trsm<float><<<grid_for(count, 152 * 8), 256, trsm_smem(max_dense), st>>>((const OpTrsm*)ops, count, B);
      else
        k_trsm<double><<<grid_for(count, 152 * 8), 256, trsm_smem(max_dense), st>>>((const OpTrsm*)ops, count, B);
      break;
    case OP_GEMM:
      if (B.mixed)
        k_gemm<float><<<grid_for(count, 152 * 16), 256, 0, st>>>((const OpGemm*)ops, count, B);
      else
        k_gemm<double><<<grid_for(count, 152 * 16), 256, 0, st>>>((const OpGemm*)ops, count, B);
      break;
    case OP_TRUNC:
      launch_trunc((const OpTrunc*)ops, count, terms, B, false, st);
      break;
    case OP_TRUNC_BIG:
      launch_trunc((const OpTrunc*)ops, count, terms, B, true, st);
      break;
  }
}

void launch_gather(const double* src, const int32_t* perm, double* dst, int64_t n, cudaStream_t st) {
  k_gather<<<grid_for((n + 255) / 256, 152 * 8), 256, 0, st>>>(src, perm, dst, n);
}
void launch_scatter(const double* src, const int32_t* perm, double* dst, int64_t n, cudaStream_t st) {
  k_scatter<<<grid_for((n + 255) / 256, 152 * 8), 256, 0, st>>>(src, perm, dst, n);
}
void launch_points(const double* xy, const int32_t* perm, double* px, double* py, int64_t n, cudaStream_t st) {
  k_points<<<grid_for((n + 255) / 256, 152 * 8), 256, 0, st>>>(xy, perm, px, py, n);
}
void launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st) {
  k_axpby<<<grid_for((n + 255) / 256, 152 * 8), 256, 0, st>>>(a, x, b, y, n);
}
void launch_sub(const double* x, const double* y, double* z, int64_t n, cudaStream_t st) {
  k_sub<<<grid_for((n + 255) / 256, 152 * 8), 256, 0, st>>>(x, y, z, n);
}
void launch_dot(const double* x, const double* y, int64_t n, double* part, double* out, cudaStream_t st) {
  k_dot_part<<<RED_BLOCKS, 256, 0, st>>>(x, y, n, part);
  k_sum_final<<<1, 256, 0, st>>>(part, RED_BLOCKS, out);
}
void launch_logdet(const int64_t* offs, const int32_t* dims, int64_t count, const double* arena, double* part,
                   double* out, cudaStream_t st) {
  k_logdet_part<<<grid_for((count + 127) / 128, 152 * 4), 128, 0, st>>>(offs, dims, count, arena, part);
  k_sum_final<<<1, 256, 0, st>>>(part, count, out);
}

int configure_kernels(int max_dense) {
  const size_t need = (size_t)max_dense * max_dense * sizeof(double);
  cudaError_t e1 = cudaFuncSetAttribute(k_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
  const int tneed = (int)trsm_smem(max_dense);
  cudaError_t e2 = cudaFuncSetAttribute(k_trsm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, tneed);
  if (e2 == cudaSuccess) e2 = cudaFuncSetAttribute(k_trsm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, tneed);
  cudaError_t e4 = cudaFuncSetAttribute(k_waves, cudaFuncAttributeMaxDynamicSharedMemorySize, tneed);
  if (e4 == cudaSuccess) e4 = cudaFuncSetAttribute(k_flow, cudaFuncAttributeMaxDynamicSharedMemorySize, tneed);
  if (e4 == cudaSuccess) e4 = cudaFuncSetAttribute(k_chain<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, tneed);
  if (e4 == cudaSuccess) e4 = cudaFuncSetAttribute(k_chain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, tneed);
  const int e3 = configure_trunc();
  return (e1 == cudaSuccess && e2 == cudaSuccess && e3 == 0 && e4 == cudaSuccess) ? 0 : -1;
}

}  // namespace hlc
