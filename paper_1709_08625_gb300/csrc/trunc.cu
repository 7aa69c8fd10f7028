// trunc.cu -- truncated low-rank sums (the recompression of Remark A.1 and
// the truncated addition of Table 1):
//
//   target := trunc(target + sum_t alpha_t U_t V_t^T),  keep sigma_i > eps sigma_1,
//
// taken in batches of at most TR_KB new columns, acc := trunc(acc + batch).
// For one batch with K = rank(acc) + batch columns and the concatenated
// factors Ucat (m x K), Vcat (n x K):
//
//   1. R_u, R_v: R factors of Ucat and Vcat by Householder QR streamed over
//      row chunks ([R; chunk] -> R); Q is never formed.  For K <= 32 a
//      warp-level tall-skinny QR (both sides at once, qr_tsqr_pair), else
//      block-wide (qr_stream);
//   2. M = R_u R_v^T (K x K);
//   3. the SVD of M: QR with column pivoting reduces M to its numerical rank
//      r (the trailing part dropped is below max(1e-3 eps, 8 u) |M|), then
//      one-sided Jacobi on the transpose of the R factor of (R P^T)^T:
//      M = X S Y^T;
//   4. keep the k values sigma_i > eps sigma_1 and write
//        U_new = Ucat R_v^T Y_k S_k^-1/2 = Q_u X_k S_k^1/2,
//        V_new = Vcat R_u^T X_k G^-1 S_k^-1/2,  G = X_k^T X_k (~ I),
//      row by row, in place (G^-1 makes U_new V_new^T the orthogonal
//      projection of the block onto span(Q_u X_k) even where the computed
//      X_k is not exactly orthonormal).
//
// Steps 1 and 4 run in the panel type: FP64 (HLC_FP64) or FP32 (mixed
// modes).  Steps 2-3 (the core) run in the core type: FP32 in HLC_MIXED,
// whose R factors carry FP32 rounding already, FP64 in HLC_FP64 and
// HLC_MIXED_SVD64; the core's stopping rules scale with its unit roundoff.
//
// Large targets (m + n above 4096 rows, or above 512 rows with many term
// columns; the planner decides) run on a cluster of TR_CL CTAs: each CTA
// streams its share of the rows, CTAs 0 and 1 combine the partial R factors,
// CTA 0 computes the core, all CTAs apply; the phases are separated by
// cluster barriers.

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "devutil.cuh"
#include "hlc_internal.h"
#include "kernels.h"
#include "ops.cuh"

namespace cg = cooperative_groups;

namespace hlc {

constexpr int TR_KB = 64;      // new columns per batch
constexpr int TR_KT = 256;     // columns of one truncation: rank (<= 128) + batch (<= 128)
constexpr int TR_KCAP = 128;   // rank capacity of a block
// the streamed chunk buffer: 64 KB of shared memory either way (3 CTAs per
// SM); a chunk has as many rows as fit for the batch's K (at least 32)
template <class T>
struct TrCh {
  static constexpr int value = sizeof(T) == 8 ? 32 : 64;  // rows at K = TR_KT
  static constexpr int elems = value * TR_KT;
};
// the core's work arrays reuse the chunk buffer (free between the QR and
// the apply): its size in entries of the core type
template <class T, class C>
__host__ __device__ constexpr int64_t core_smem_elems() {
  return (int64_t)TrCh<T>::elems * (int64_t)sizeof(T) / (int64_t)sizeof(C);
}
constexpr int TR_THREADS = 256;
constexpr int TR_CL = 8;       // CTAs per cluster for large targets
constexpr int64_t TR_REG = (int64_t)TR_KT * TR_KT;
// per-CTA scratch: Pu, Pv, M, W, J, X (K x K each), Cu, Cv (K x 128 each)
// and a few words for cluster broadcasts
constexpr int64_t TR_PANEL = (int64_t)TR_KT * TR_KCAP;
constexpr int64_t TR_OFF_X = 5 * TR_REG;
constexpr int64_t TR_OFF_CU = TR_OFF_X + TR_REG;  // X holds the rank x rank Jacobi matrix
constexpr int64_t TR_OFF_CV = TR_OFF_CU + TR_PANEL;
constexpr int64_t TR_OFF_FLAG = TR_OFF_CV + TR_PANEL;
constexpr int64_t TR_SCRATCH = TR_OFF_FLAG + 8;

int64_t trunc_scratch_doubles() { return TR_SCRATCH; }
int max_trunc_ctas() { return 152 * 3; }

struct TrCat {
  int kacc;                   // leading columns from the target itself
  int nt;                     // terms in the batch
  const TermD* terms;         // batch terms
  int col0[65];               // first concatenated column of each term; col0[nt] = K
  unsigned char tcol[TR_KT];  // term of every concatenated column beyond kacc
};

__device__ __forceinline__ int term_cols(const TermD& d, const int* ranks) {
  return (d.flags & 1) ? d.urows : (d.flags & 2) ? d.vrows : dimv(d.k, ranks);
}

// value of column `col` of Ucat (side 0) or Vcat (side 1) at row `row`
__device__ __forceinline__ double cat_value(const Bases& B, const OpTrunc& op, const TrCat& cat, int side,
                                            int row, int col) {
  if (col < cat.kacc) {
    return side == 0 ? B.buf[op.U.buf][op.U.off + row + (int64_t)col * op.m]
                     : B.buf[op.V.buf][op.V.off + row + (int64_t)col * op.n];
  }
  const int t = cat.tcol[col];
  const TermD& d = cat.terms[t];
  const int lc = col - cat.col0[t];
  if (side == 0) {
    const int ii = row - d.roff;
    if (ii < 0 || ii >= d.urows) return 0.0;
    if (d.flags & 1) return ii == lc ? d.alpha : 0.0;
    return d.alpha * B.buf[d.U.buf][d.U.off + (int64_t)ii * d.U.rs + (int64_t)lc * d.U.cs];
  } else {
    const int jj = row - d.coff;
    if (jj < 0 || jj >= d.vrows) return 0.0;
    if (d.flags & 2) return jj == lc ? 1.0 : 0.0;
    return B.buf[d.V.buf][d.V.off + (int64_t)jj * d.V.rs + (int64_t)lc * d.V.cs];
  }
}

// Streaming Householder QR: R (K x K, ld TR_KT, type T) of the nrows x K
// matrix whose entries rowval(i, c) returns; buf: the TrCh<T> chunk buffer.
// Row chunks are folded into R one at a time ([R; chunk] -> R).  Step j
// reflects column j of [R; chunk]: the reflector is (1 at row j of R;
// sc x_j on the chunk), and since Q is never formed the chunk column x_j is
// left unscaled (sc is folded into the updates).  Every warp computes the
// step's scalars itself from R(j, j) and the squared norm of x_j, which the
// warp that updated column j in the previous step left in shared memory
// (look-ahead), so a step takes one block barrier.  R stays in shared memory
// while it leaves room for a 32-row chunk, and is copied out at the end.
template <class T, class F>
__device__ void qr_stream(F rowval, int nrows, int K, T* Rout, T* buf, double* sh) {
  (void)sh;
  __shared__ T s_xn[2];
  constexpr int64_t E = TrCh<T>::elems;
  const bool rsm = (int64_t)K * K + 32LL * K <= E;
  T* R = rsm ? buf : Rout;
  const int ldr = rsm ? K : TR_KT;
  T* sC = rsm ? buf + (int64_t)K * K : buf;
  const int64_t cap = rsm ? E - (int64_t)K * K : E;
  const int TR_CH = max(32, (int)((cap / max(K, 1)) & ~31));
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < K * K; e += blockDim.x) R[(e % K) + (int64_t)(e / K) * ldr] = T(0);
  __syncthreads();
  for (int r0 = 0; r0 < nrows; r0 += TR_CH) {
    const int rows = min(TR_CH, nrows - r0);
    for (int e = tid; e < rows * K; e += blockDim.x) {
      const int i = e % rows, c = e / rows;
      sC[i + c * TR_CH] = (T)rowval(r0 + i, c);
    }
    __syncthreads();
    if (w == 0) {
      T xn = T(0);
      for (int i = lane; i < rows; i += 32) xn += sC[i] * sC[i];
      xn = warp_sum(xn);
      if (lane == 0) s_xn[0] = xn;
    }
    __syncthreads();
    for (int j = 0; j < K; ++j) {
      const T xn = s_xn[j & 1];
      const T alpha = R[j + (int64_t)j * ldr];
      T tau = T(0), sc = T(0), beta = alpha;
      if (xn > T(0)) {
        beta = -copysign(sqrt(alpha * alpha + xn), alpha);
        tau = (beta - alpha) / beta;
        sc = T(1) / (alpha - beta);
      }
      const T* xj = sC + j * TR_CH;
      for (int l = j + 1 + w; l < K; l += nw) {
        T* xl = sC + l * TR_CH;
        if (tau != T(0)) {
          T p = T(0);
          for (int i = lane; i < rows; i += 32) p += xj[i] * xl[i];
          p = warp_sum(p);
          const T rjl = R[j + (int64_t)l * ldr];
          const T wv = tau * (rjl + sc * p), ws = wv * sc;
          T q = T(0);
          for (int i = lane; i < rows; i += 32) {
            const T v = xl[i] - ws * xj[i];
            xl[i] = v;
            q += v * v;
          }
          if (l == j + 1) {
            q = warp_sum(q);
            if (lane == 0) s_xn[(j + 1) & 1] = q;
          }
          __syncwarp();
          if (lane == 0) R[j + (int64_t)l * ldr] = rjl - wv;
        } else if (l == j + 1) {
          T q = T(0);
          for (int i = lane; i < rows; i += 32) q += xl[i] * xl[i];
          q = warp_sum(q);
          if (lane == 0) s_xn[(j + 1) & 1] = q;
        }
      }
      __syncthreads();
      if (tid == 0) R[j + (int64_t)j * ldr] = beta;
    }
    __syncthreads();
  }
  if (rsm) {
    for (int e = tid; e < K * K; e += blockDim.x) {
      const int i = e % K, c = e / K;
      Rout[i + (int64_t)c * TR_KT] = R[i + (int64_t)c * K];
    }
    __syncthreads();
  }
}

// Tall-skinny QR for K <= 32 columns, warp-level: every warp streams its own
// 32-row chunks, one row per lane held in registers, and folds them into its
// own R (K x K, shared memory) by Householder steps on [R; chunk]; the
// per-warp factors are then combined pairwise (R_a := qr([R_a; R_b])) in a
// binary tree.  Within a step the pivot column is always v[0]: after the
// step the row shifts left, so every register index is static.  The column
// dot products of a step are summed by a reduce-scatter butterfly (31
// shuffles; lane l ends with the sum for column l), and the resulting
// updates reach every lane through a 32-entry shared array.
constexpr int TSQR_LD = 32;

template <class T>
__device__ __forceinline__ void tsqr_absorb(T (&v)[32], int K, T* R, T* wsh) {
  constexpr int RL = TSQR_LD;
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  for (int j = 0; j < K; ++j) {
    const T x0 = v[0];
    const T xn = warp_sum(x0 * x0);
    const T alpha = R[j + j * RL];
    T tau = T(0), sc = T(0), beta = alpha;
    if (xn > T(0)) {
      beta = -copysign(sqrt(alpha * alpha + xn), alpha);
      tau = (beta - alpha) / beta;
      sc = T(1) / (alpha - beta);
    }
    if (tau != T(0)) {
      const T u0 = x0 * sc;  // the reflector's chunk part (its R part is 1 at row j)
      const int nl = K - j;
      T d[32];
#pragma unroll
      for (int l = 0; l < 32; ++l) d[l] = u0 * v[l];
#pragma unroll
      for (int h = 16; h > 0; h >>= 1) {
        const bool hi = (lane & h) != 0;
#pragma unroll
        for (int t = 0; t < h; ++t) {
          const T send = hi ? d[t] : d[t + h];
          const T keep = hi ? d[t + h] : d[t];
          d[t] = keep + __shfl_xor_sync(FULL, send, h);
        }
      }
      T wv = T(0);
      if (lane >= 1 && lane < nl) {
        const T rjl = R[j + (j + lane) * RL];
        wv = tau * (rjl + d[0]);
        R[j + (j + lane) * RL] = rjl - wv;
      }
      if (lane == 0) R[j + j * RL] = beta;
      wsh[lane] = wv;
      __syncwarp();
#pragma unroll
      for (int l = 1; l < 32; ++l) v[l] -= wsh[l] * u0;
    }
#pragma unroll
    for (int l = 0; l < 31; ++l) v[l] = v[l + 1];
    v[31] = T(0);
    __syncwarp();
  }
}

// R (K x K upper, ld TR_KT) of the nrows x K matrix rowval(i, c), K <= 32;
// sW: per warp a 32 x 32 factor, then per warp 32 entries and a flag.
template <class T, class F>
__device__ void qr_tsqr(F rowval, int nrows, int K, T* R, T* sW) {
  constexpr int RL = TSQR_LD;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T* Rw = sW + w * 32 * RL;
  T* wsh = sW + nw * 32 * RL + w * 32;
  for (int e = lane; e < 32 * RL; e += 32) Rw[e] = T(0);
  __syncwarp();
  T v[32];
  for (int r0 = w * 32; r0 < nrows; r0 += nw * 32) {
    const int row = r0 + lane;
#pragma unroll
    for (int l = 0; l < 32; ++l) v[l] = (l < K && row < nrows) ? (T)rowval(row, l) : T(0);
    tsqr_absorb<T>(v, K, Rw, wsh);
  }
  __syncthreads();
  // warp w holds rows iff w * 32 < nrows; a factor without rows is zero
  for (int st = 1; st < nw; st <<= 1) {
    if ((w % (2 * st)) == 0 && w + st < nw && (w + st) * 32 < nrows) {
      const T* Rb = sW + (w + st) * 32 * RL;
#pragma unroll
      for (int l = 0; l < 32; ++l) v[l] = (l < K && lane < K && lane <= l) ? Rb[lane + l * RL] : T(0);
      tsqr_absorb<T>(v, K, Rw, wsh);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int i = e % K, j = e / K;
    R[i + (int64_t)j * TR_KT] = sW[i + j * RL];
  }
  __syncthreads();
}

// Both R factors of a batch at once, for K <= 32: the first half of the
// warps runs the tall-skinny QR of U's rows, the second half V's, each with
// its own binary tree; the block barriers between tree levels are shared.
template <class T, class FU, class FV>
__device__ void qr_tsqr_pair(FU rowu, int mrows, FV rowv, int nrows, int K, T* Ru, T* Rv, T* sW) {
  constexpr int RL = TSQR_LD;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int half = nw >> 1, side = w >= half, wl = w - side * half;
  const int rows = side ? nrows : mrows;
  T* Rw = sW + w * 32 * RL;
  T* wsh = sW + nw * 32 * RL + w * 32;
  for (int e = lane; e < 32 * RL; e += 32) Rw[e] = T(0);
  __syncwarp();
  T v[32];
  for (int r0 = wl * 32; r0 < rows; r0 += half * 32) {
    const int row = r0 + lane;
    if (side) {
#pragma unroll
      for (int l = 0; l < 32; ++l) v[l] = (l < K && row < rows) ? (T)rowv(row, l) : T(0);
    } else {
#pragma unroll
      for (int l = 0; l < 32; ++l) v[l] = (l < K && row < rows) ? (T)rowu(row, l) : T(0);
    }
    tsqr_absorb<T>(v, K, Rw, wsh);
  }
  __syncthreads();
  for (int st = 1; st < half; st <<= 1) {
    if ((wl % (2 * st)) == 0 && wl + st < half && (wl + st) * 32 < rows) {
      const T* Rb = sW + (w + st) * 32 * RL;
#pragma unroll
      for (int l = 0; l < 32; ++l) v[l] = (l < K && lane < K && lane <= l) ? Rb[lane + l * RL] : T(0);
      tsqr_absorb<T>(v, K, Rw, wsh);
    }
    __syncthreads();
  }
  const T* R0 = sW;
  const T* R1 = sW + half * 32 * RL;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int i = e % K, j = e / K;
    Ru[i + (int64_t)j * TR_KT] = R0[i + j * RL];
    Rv[i + (int64_t)j * TR_KT] = R1[i + j * RL];
  }
  __syncthreads();
}

template <class T>
struct CoreShared {
  T cn[TR_KT];
  T cn2[TR_KT];
  T scl[TR_KT];
  T tauq[TR_KT];
  T sv[TR_KT];
  int piv[TR_KT];
  int order[TR_KT];
  T red[40];
  int stop, jmax, rank, k, rot;
};

// FP64 core: SVD of M = R_u R_v^T reduced by column-pivoted QR, truncation
// rank, and the coefficient matrices Cu, Cv (K x k, ld TR_KT).
__device__ __forceinline__ void phase_mark(unsigned long long* ph, int slot, long long& t) {
  if (ph && threadIdx.x == 0) {
    const long long now = clock64();
    atomicAdd(ph + slot, (unsigned long long)(now - t));
    t = now;
  }
}

// Work arrays, all with leading dimension K: M (K x K), and once the
// numerical rank r of M is known W (K x r), J and X (r x r, in K x r
// regions).  They live in the shared buffer sm (sm_elems entries of the core
// type) as far as they fit -- M when K^2 <= sm_elems, the others when
// K^2 + 3 K r <= sm_elems as well -- and otherwise in the CTA's scratch scr.
// Cu, Cv: K x k outputs in the scratch (leading dimension TR_KT); Ru, Rv:
// the R factors (TR_KT).
template <class T, class C>
__device__ void tr_core(const T* Ru, const T* Rv, int K, double eps, int kcap, int kfix, C* sm, int64_t sm_elems,
                        double* scr, C* Cu, C* Cv, CoreShared<C>& cs, int* status,
                        unsigned long long* ph = nullptr) {
  constexpr int ldc = TR_KT;
  const int ld = K;
  C* M = (int64_t)K * K <= sm_elems ? sm : reinterpret_cast<C*>(scr + 2 * TR_REG);
  C *W, *J, *X;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  long long t0 = clock64();
  // M = Ru Rv^T (both upper triangular)
  for (int e = tid; e < K * K; e += blockDim.x) {
    const int i = e % K, j = e / K;
    C s = C(0);
    for (int c = max(i, j); c < K; ++c) s += (C)Ru[i + (int64_t)c * TR_KT] * (C)Rv[j + (int64_t)c * TR_KT];
    M[i + (int64_t)j * ld] = s;
  }
  for (int j = tid; j < K; j += blockDim.x) cs.piv[j] = j;
  __syncthreads();
  phase_mark(ph, 3, t0);
  // Householder QR with column pivoting, stopped at the numerical rank: the
  // remaining columns are dropped once their norm is below 1e-3 eps |M|
  // (or 8 unit roundoffs of the core type, when that is larger)
  const C stop_rel = (C)fmax(1e-3 * eps, sizeof(C) == 8 ? 8.0 * 2.220446049250313e-16 : 8.0 * 1.1920929e-7);
    int r = 0;
  // Column norms once; afterwards every warp recomputes the norm (below the
  // current row) of each column it updates, into the other of two buffers,
  // so that the pivot choice of a step reads a buffer nobody writes.  Every
  // warp picks the pivot itself (same data, same result), computes the
  // reflector of the pivot column itself, and applies it with its scale
  // folded in; the diagonal of R and the scaled reflectors are written after
  // the loop.  Two block barriers per pivot.
  C* cn0 = cs.cn;
  C* cn1 = cs.cn2;
  for (int j = w; j < K; j += nw) {
    C p = C(0);
    for (int i = lane; i < K; i += 32) p += M[i + (int64_t)j * ld] * M[i + (int64_t)j * ld];
    p = warp_sum(p);
    if (lane == 0) cn0[j] = p;
  }
  __syncthreads();
  C ref = C(0);
  for (; r < K; ++r) {
    const C* cur = (r & 1) ? cn1 : cn0;
    C* nxt = (r & 1) ? cn0 : cn1;
    int jm = -1;
    C best = C(-1), rem = C(0);
    for (int j = r + lane; j < K; j += 32) {
      rem += cur[j];
      if (cur[j] > best) {
        best = cur[j];
        jm = j;
      }
    }
    rem = warp_sum(rem);
    for (int o = 16; o > 0; o >>= 1) {  // max, ties to the smaller index
      const C ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oj = __shfl_xor_sync(0xffffffffu, jm, o);
      if (ob > best || (ob == best && oj >= 0 && (jm < 0 || oj < jm))) {
        best = ob;
        jm = oj;
      }
    }
    if (r == 0) ref = sqrt(best);
    if (ref == C(0) || !(sqrt(rem) > stop_rel * ref)) break;
    if (jm != r) {
      for (int i = tid; i < K; i += blockDim.x) {
        const C a = M[i + (int64_t)r * ld];
        M[i + (int64_t)r * ld] = M[i + (int64_t)jm * ld];
        M[i + (int64_t)jm * ld] = a;
      }
      if (tid == 0) {
        const int t = cs.piv[r];
        cs.piv[r] = cs.piv[jm];
        cs.piv[jm] = t;
      }
    }
    __syncthreads();
    C xn = C(0);
    for (int i = r + 1 + lane; i < K; i += 32) xn += M[i + (int64_t)r * ld] * M[i + (int64_t)r * ld];
    xn = warp_sum(xn);
    const C alpha = M[r + (int64_t)r * ld];
    C tau = C(0), sc = C(1), beta = alpha;
    if (xn > C(0)) {
      beta = -copysign(sqrt(alpha * alpha + xn), alpha);
      tau = (beta - alpha) / beta;
      sc = C(1) / (alpha - beta);
    }
    if (tid == 0) {
      cs.tauq[r] = tau;
      cs.sv[r] = beta;  // the diagonal of R, written after the loop
      cs.scl[r] = sc;
    }
    for (int l = r + 1 + w; l < K; l += nw) {
      C p = C(0);
      for (int i = r + 1 + lane; i < K; i += 32) p += M[i + (int64_t)r * ld] * M[i + (int64_t)l * ld];
      p = warp_sum(p);
      const C wv = tau * (M[r + (int64_t)l * ld] + sc * p), ws = wv * sc;
      C q = C(0);
      for (int i = r + 1 + lane; i < K; i += 32) {
        const C v = M[i + (int64_t)l * ld] - ws * M[i + (int64_t)r * ld];
        M[i + (int64_t)l * ld] = v;
        q += v * v;
      }
      q = warp_sum(q);
      if (lane == 0) {
        M[r + (int64_t)l * ld] -= wv;
        nxt[l] = q;
      }
    }
    __syncthreads();
  }
  // the diagonal of R and the reflectors scaled to a unit leading entry
  for (int e = tid; e < r * K; e += blockDim.x) {
    const int q = e / K, i = e % K;
    if (i == q)
      M[q + (int64_t)q * ld] = cs.sv[q];
    else if (i > q && cs.tauq[q] != C(0))
      M[i + (int64_t)q * ld] *= cs.scl[q];
  }
  __syncthreads();
  const int rank = r;
  if (M == sm && (int64_t)K * K + 3 * (int64_t)K * rank <= sm_elems) {
    W = M + (int64_t)K * K;
    J = W + (int64_t)K * rank;
    X = J + (int64_t)K * rank;
  } else {
    W = reinterpret_cast<C*>(scr + 3 * TR_REG);
    J = reinterpret_cast<C*>(scr + 4 * TR_REG);
    X = reinterpret_cast<C*>(scr + TR_OFF_X);
  }
  phase_mark(ph, 4, t0);
  if (ph && tid == 0) atomicAdd(ph + 10, (unsigned long long)rank);
  if (rank == 0) {
    if (tid == 0) cs.k = 0;
    __syncthreads();
    return;
  }
  // B = (R P^T)^T (K x rank) into W
  for (int e = tid; e < K * rank; e += blockDim.x) {
    const int j = e % K, i = e / K;  // R(i, j) -> B(piv[j], i)
    W[cs.piv[j] + (int64_t)i * ld] = (i <= j) ? M[i + (int64_t)j * ld] : C(0);
  }
  __syncthreads();
  // Householder QR of B (K x rank): B = Q_B R_B; the one-sided Jacobi then
  // works on the rank x rank triangle R_B (QR preconditioning of the Jacobi
  // SVD), and the left vectors of B are Q_B times those of R_B.
  for (int q = 0; q < rank; ++q) {
    if (w == 0) {
      C xn = C(0);
      for (int i = q + 1 + lane; i < K; i += 32) xn += W[i + (int64_t)q * ld] * W[i + (int64_t)q * ld];
      xn = warp_sum(xn);
      const C alpha = W[q + (int64_t)q * ld];
      C tau = C(0), sc = C(0), beta = alpha;
      if (xn > C(0)) {
        beta = -copysign(sqrt(alpha * alpha + xn), alpha);
        tau = (beta - alpha) / beta;
        sc = C(1) / (alpha - beta);
      }
      if (tau != C(0))
        for (int i = q + 1 + lane; i < K; i += 32) W[i + (int64_t)q * ld] *= sc;
      if (lane == 0) {
        W[q + (int64_t)q * ld] = beta;
        cs.cn[q] = tau;  // tau of the B reflectors
      }
    }
    __syncthreads();
    const C tau = cs.cn[q];
    if (tau != C(0)) {
      for (int l = q + 1 + w; l < rank; l += nw) {
        C p = C(0);
        for (int i = q + 1 + lane; i < K; i += 32) p += W[i + (int64_t)q * ld] * W[i + (int64_t)l * ld];
        p = warp_sum(p);
        const C wv = tau * (p + W[q + (int64_t)l * ld]);
        for (int i = q + 1 + lane; i < K; i += 32) W[i + (int64_t)l * ld] -= wv * W[i + (int64_t)q * ld];
        if (lane == 0) W[q + (int64_t)l * ld] -= wv;
      }
    }
    __syncthreads();
  }
  // The one-sided Jacobi works on A = R_B^T (lower triangular; the
  // transpose of the triangular factor is what the QR preconditioning makes
  // nearly orthogonal), in the X region; J accumulates its rotations.
  C* A = X;
  for (int e = tid; e < rank * rank; e += blockDim.x) {
    const int i = e % rank, j = e / rank;
    A[i + (int64_t)j * ld] = (i >= j) ? W[j + (int64_t)i * ld] : C(0);
    J[i + (int64_t)j * ld] = (i == j) ? C(1) : C(0);
  }
  __syncthreads();
  // one-sided Jacobi on the rank columns of A, round-robin pairs
  C fro2 = C(0);
  for (int e = tid; e < rank * rank; e += blockDim.x) {
    const C v = A[(e % rank) + (int64_t)(e / rank) * ld];
    fro2 += v * v;
  }
  fro2 = block_sum(fro2, cs.red + 1);
  // pairs of columns both at rounding level (below 1e-13 |A|_F in FP64,
  // 1e-6 |A|_F in FP32) cannot affect any truncation decision and are left
  // alone; a pair is rotated while |gamma| > max(rank, 16) c sqrt(alpha beta)
  // with c = 1e-14 (FP64) or 1e-6 (FP32), i.e. some tens of unit roundoffs
  // per column: the columns end up orthogonal far below any truncation
  // threshold, without chasing the rounding noise of the dot products
  const C tiny = (sizeof(C) == 8 ? C(1e-26) : C(1e-12)) * fro2;
  const C rtol = (C)max(rank, 16) * (sizeof(C) == 8 ? C(1e-14) : C(1e-6));
  const int Kp = rank + (rank & 1);
  for (int sweep = 0; sweep < 80 && Kp > 1; ++sweep) {
    if (tid == 0) cs.rot = 0;
    __syncthreads();
    for (int step = 0; step < Kp - 1; ++step) {
      for (int q = w; q < Kp / 2; q += nw) {
        const int pa = q, pb = Kp - 1 - q;
        int a = pa == 0 ? 0 : 1 + (pa - 1 + step) % (Kp - 1);
        int b = pb == 0 ? 0 : 1 + (pb - 1 + step) % (Kp - 1);
        if (a > b) {
          const int t = a;
          a = b;
          b = t;
        }
        if (b >= rank) continue;
        C al = C(0), be = C(0), ga = C(0);
        for (int i = lane; i < rank; i += 32) {
          const C x = A[i + (int64_t)a * ld], y = A[i + (int64_t)b * ld];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al <= tiny && be <= tiny) continue;
        if (ga == C(0) || fabs(ga) <= rtol * sqrt(al * be)) continue;
        const C zeta = (be - al) / (C(2) * ga);
        const C t = (zeta >= C(0) ? C(1) : C(-1)) / (fabs(zeta) + sqrt(C(1) + zeta * zeta));
        const C c = C(1) / sqrt(C(1) + t * t), sn = c * t;
        for (int i = lane; i < rank; i += 32) {
          const C x = A[i + (int64_t)a * ld], y = A[i + (int64_t)b * ld];
          A[i + (int64_t)a * ld] = c * x - sn * y;
          A[i + (int64_t)b * ld] = sn * x + c * y;
          const C jx = J[i + (int64_t)a * ld], jy = J[i + (int64_t)b * ld];
          J[i + (int64_t)a * ld] = c * jx - sn * jy;
          J[i + (int64_t)b * ld] = sn * jx + c * jy;
        }
        if (lane == 0) cs.rot = 1;
      }
      __syncthreads();
    }
    if (!cs.rot) break;
    __syncthreads();
  }
  phase_mark(ph, 5, t0);
  // singular values, order (ties: smaller index first), truncation rank
  for (int j = w; j < rank; j += nw) {
    C s = C(0);
    for (int i = lane; i < rank; i += 32) s += A[i + (int64_t)j * ld] * A[i + (int64_t)j * ld];
    s = warp_sum(s);
    if (lane == 0) cs.sv[j] = sqrt(s);
  }
  __syncthreads();
  for (int j = tid; j < rank; j += blockDim.x) {
    int pos = 0;
    for (int i = 0; i < rank; ++i) pos += (cs.sv[i] > cs.sv[j]) || (cs.sv[i] == cs.sv[j] && i < j);
    cs.order[pos] = j;
  }
  __syncthreads();
  if (tid == 0) {
    const C smax = cs.sv[cs.order[0]];
    const C thr = (C)eps * smax;
    int k = 0;
    if (smax > C(0))
      while (k < rank && cs.sv[cs.order[k]] > thr) ++k;
    if (!(smax == smax)) {
      record_error(status, DEV_BAD, 1);
      k = 0;
    }
    if (kfix > 0 && k > kfix) k = kfix;  // fixed-rank mode
    if (k > kcap) {
      record_error(status, DEV_RANK, k);
      k = kcap;
    }
    cs.k = k;
  }
  __syncthreads();
  const int k = cs.k;
  // The Jacobi gives R_B^T J = Wa (orthogonal columns, Wa = Wa_n S), so
  // R_B = J S Wa_n^T, B = Q_B R_B = (Q_B J) S Wa_n^T, and with M = Q R P^T =
  // Q B^T = (Q Wa_n) S (Q_B J)^T:
  //   left vectors of M:  x_c = Q [Wa_n(:, j_c); 0]  (reflectors of the pivoted QR, in M)
  //   right vectors of M: y_c = Q_B [J(:, j_c); 0]   (reflectors of the QR of B, in W)
  // Both are built in the Cu/Cv regions' columns (K x k each) before the
  // coefficients overwrite them: x_c in Cv, y_c in Cu.
  for (int c = w; c < k; c += nw) {
    const int j = cs.order[c];
    const C sv = cs.sv[j];
    C* x = Cv + (int64_t)c * ldc;
    C* y = Cu + (int64_t)c * ldc;
    for (int i = lane; i < K; i += 32) {
      x[i] = i < rank ? A[i + (int64_t)j * ld] / sv : C(0);
      y[i] = i < rank ? J[i + (int64_t)j * ld] : C(0);
    }
    __syncwarp();
    for (int q = rank - 1; q >= 0; --q) {
      const C tq = cs.tauq[q], tb = cs.cn[q];
      C p = C(0), pb = C(0);
      for (int i = q + lane; i < K; i += 32) {
        p += (i == q ? C(1) : M[i + (int64_t)q * ld]) * x[i];
        pb += (i == q ? C(1) : W[i + (int64_t)q * ld]) * y[i];
      }
      p = warp_sum(p);
      pb = warp_sum(pb);
      for (int i = q + lane; i < K; i += 32) {
        if (tq != C(0)) x[i] -= tq * p * (i == q ? C(1) : M[i + (int64_t)q * ld]);
        if (tb != C(0)) y[i] -= tb * pb * (i == q ? C(1) : W[i + (int64_t)q * ld]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // G = X_k^T X_k, the Gram matrix of the kept left vectors (the identity up
  // to the orthogonality the Jacobi reached), lower triangle in the X region
  // (A is no longer needed).  V_new carries G^-1: then U_new V_new^T =
  // Q_u P M Q_v^T with P the orthogonal projector onto span(X_k), whose
  // distance from M is bounded by the dropped columns whether or not X_k is
  // exactly orthogonal (in FP32 it is only to ~1e-6, which is not below eps).
  C* G = X;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    if (i < j) continue;
    const C* xi = Cv + (int64_t)i * ldc;
    const C* xj = Cv + (int64_t)j * ldc;
    C g = C(0);
    for (int q = 0; q < K; ++q) g += xi[q] * xj[q];
    G[i + (int64_t)j * ld] = g;
  }
  __syncthreads();
  // G = L L^T in place (warp 0, left-looking); G is near the identity, so a
  // pivot below 1/4 means the vectors are unusable and the correction is
  // skipped
  if (w == 0) {
    int ok = 1;
    for (int j = 0; j < k; ++j) {
      C part = C(0);
      for (int q = lane; q < j; q += 32) part += G[j + (int64_t)q * ld] * G[j + (int64_t)q * ld];
      part = warp_sum(part);
      const C d = G[j + (int64_t)j * ld] - part;
      if (!(d > C(0.25))) ok = 0;
      const C ljj = sqrt(d > C(0.25) ? d : C(1));
      for (int i = j + 1 + lane; i < k; i += 32) {
        C g = G[i + (int64_t)j * ld];
        for (int q = 0; q < j; ++q) g -= G[i + (int64_t)q * ld] * G[j + (int64_t)q * ld];
        G[i + (int64_t)j * ld] = g / ljj;
      }
      __syncwarp();
      if (lane == 0) G[j + (int64_t)j * ld] = ljj;
      __syncwarp();
    }
    if (lane == 0) cs.rot = ok;
  }
  // Cu = R_v^T y_c / s^0.5 and Cv = R_u^T x_c, one entry per thread; y_c,
  // x_c sit in Cu, Cv, the results go to W, M (free now)
  for (int e = tid; e < K * k; e += blockDim.x) {
    const int col = e % K, c = e / K;
    const C isq = C(1) / sqrt(cs.sv[cs.order[c]]);
    const C* y = Cu + (int64_t)c * ldc;
    const C* x = Cv + (int64_t)c * ldc;
    C a = C(0), b = C(0);
    for (int q = 0; q <= col; ++q) {
      a += (C)Rv[q + (int64_t)col * TR_KT] * y[q];
      b += (C)Ru[q + (int64_t)col * TR_KT] * x[q];
    }
    W[col + (int64_t)c * ld] = a * isq;
    M[col + (int64_t)c * ld] = b;
  }
  __syncthreads();
  // each row of R_u^T X_k times G^-1 (one thread per row), then S^-1/2
  if (cs.rot) {
    for (int col = tid; col < K; col += blockDim.x) {
      C* row = M + col;
      for (int c = 0; c < k; ++c) {
        C v = row[(int64_t)c * ld];
        for (int q = 0; q < c; ++q) v -= G[c + (int64_t)q * ld] * row[(int64_t)q * ld];
        row[(int64_t)c * ld] = v / G[c + (int64_t)c * ld];
      }
      for (int c = k - 1; c >= 0; --c) {
        C v = row[(int64_t)c * ld];
        for (int q = c + 1; q < k; ++q) v -= G[q + (int64_t)c * ld] * row[(int64_t)q * ld];
        row[(int64_t)c * ld] = v / G[c + (int64_t)c * ld];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < K * k; e += blockDim.x) {
    const int col = e % K, c = e / K;
    const C isq = C(1) / sqrt(cs.sv[cs.order[c]]);
    Cu[col + (int64_t)c * ldc] = W[col + (int64_t)c * ld];
    Cv[col + (int64_t)c * ldc] = M[col + (int64_t)c * ld] * isq;
  }
  __syncthreads();
  phase_mark(ph, 6, t0);
}

// Rows [r0, r1) of one side: out(row, c) = sum_col cat(row, col) C(col, c),
// tile by tile: a tile of the concatenation is staged in shared memory, so the
// rows of the tile can be overwritten in place once it is loaded.
template <class T, class C>
__device__ void tr_apply(const Bases& B, const OpTrunc& op, const TrCat& cat, int side, int r0, int r1, int K,
                         int k, const C* Co, T* sC) {
  const int tid = threadIdx.x;
  const int ld = side == 0 ? op.m : op.n;
  double* out = side == 0 ? B.buf[op.U.buf] + op.U.off : B.buf[op.V.buf] + op.V.off;
  const int TR = max(32, (TrCh<T>::elems / max(K, 1)) & ~31);
  for (int t0 = r0; t0 < r1; t0 += TR) {
    const int rows = min(TR, r1 - t0);
    for (int e = tid; e < rows * K; e += blockDim.x) {
      const int i = e % rows, c = e / rows;
      sC[i + c * TR] = (T)cat_value(B, op, cat, side, t0 + i, c);
    }
    __syncthreads();
    for (int e = tid; e < rows * k; e += blockDim.x) {
      const int i = e % rows, c = e / rows;
      const C* Cc = Co + (int64_t)c * TR_KT;
      T acc = T(0);
      for (int col = 0; col < K; ++col) acc += sC[i + col * TR] * (T)Cc[col];
      out[(t0 + i) + (int64_t)c * ld] = (double)acc;
    }
    __syncthreads();
  }
}

// batch [t0, t1) of the op's terms: sets cat and returns K
__device__ int tr_batch(const OpTrunc& op, const TermD* tl, const int* ranks, int kacc, int t0, int* t1out,
                        TrCat& cat) {
  int t1 = t0, kb = 0;
  while (t1 < op.nterms) {
    const int kt = term_cols(tl[t1], ranks);
    if (kb != 0 && kb + kt > TR_KB) break;
    if (t1 - t0 >= 64) break;
    kb += kt;
    ++t1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cat.kacc = kacc;
    cat.nt = t1 - t0;
    cat.terms = tl + t0;
    int c = kacc;
    for (int t = t0; t < t1; ++t) {
      cat.col0[t - t0] = c;
      const int kt = term_cols(tl[t], ranks);
      for (int q = 0; q < kt && c + q < TR_KT; ++q) cat.tcol[c + q] = (unsigned char)(t - t0);
      c += kt;
    }
    cat.col0[t1 - t0] = c;
  }
  __syncthreads();
  *t1out = t1;
  return kacc + kb;
}

// Shared-memory state of one CTA running truncation ops.
template <class C>
struct TrShared {
  TrCat cat;
  CoreShared<C> cs;
  double sh[2];
};

// One truncation op by one CTA (scr: the CTA's scratch slice).
template <class T, class C>
__device__ void trunc_one(const OpTrunc& op, const TermD* terms, const Bases& B, double* scr, T* sC,
                          TrShared<C>& ts) {
  TrCat& cat = ts.cat;
  CoreShared<C>& cs = ts.cs;
  double* sh = ts.sh;
  T* Pu = reinterpret_cast<T*>(scr);
  T* Pv = reinterpret_cast<T*>(scr + TR_REG);
  C* Cu = reinterpret_cast<C*>(scr + TR_OFF_CU);
  C* Cv = reinterpret_cast<C*>(scr + TR_OFF_CV);
  const TermD* tl = terms + op.term0;
  int kacc = op.keep ? B.ranks[op.slot] : 0;
  int t0 = 0;
  bool first = true;
  while (first || t0 < op.nterms) {
    first = false;
    int t1;
    const int K = tr_batch(op, tl, B.ranks, kacc, t0, &t1, cat);
    t0 = t1;
    if (K == 0) {
      kacc = 0;
      continue;
    }
    if (K > TR_KT) {
      if (threadIdx.x == 0) record_error(B.status, DEV_RANK, K);
      kacc = 0;
      break;
    }
    long long tp = clock64();
    // phase counters (HLC_PHASES): one set for K <= 32, one for wider batches
    unsigned long long* ph = B.phase ? B.phase + (K > 32 ? 16 : 0) : nullptr;
    if (ph && threadIdx.x == 0) {
      atomicAdd(ph + 11, 1ull);
      atomicAdd(ph + 12, (unsigned long long)K);
    }
    if (K <= 32) {
      qr_tsqr_pair<T>([&](int r, int c) { return cat_value(B, op, cat, 0, r, c); }, op.m,
                      [&](int r, int c) { return cat_value(B, op, cat, 1, r, c); }, op.n, K, Pu, Pv, sC);
      phase_mark(ph, 1, tp);
    } else {
      qr_stream<T>([&](int r, int c) { return cat_value(B, op, cat, 0, r, c); }, op.m, K, Pu, sC, sh);
      phase_mark(ph, 1, tp);
      qr_stream<T>([&](int r, int c) { return cat_value(B, op, cat, 1, r, c); }, op.n, K, Pv, sC, sh);
    }
    phase_mark(ph, 2, tp);
    tr_core<T, C>(Pu, Pv, K, op.eps, op.kcap, op.kfix, reinterpret_cast<C*>(sC), core_smem_elems<T, C>(), scr, Cu,
                  Cv, cs, B.status, ph);
    tp = clock64();
    const int k = cs.k;
    // algorithmic flops of the batch: two streamed R factors and the apply
    if (B.flops && threadIdx.x == 0)
      atomicAdd(B.flops + OP_TRUNC, 2.0 * K * K * (double)(op.m + op.n) + 2.0 * K * (double)k * (op.m + op.n));
    tr_apply<T, C>(B, op, cat, 0, 0, op.m, K, k, Cu, sC);
    tr_apply<T, C>(B, op, cat, 1, 0, op.n, K, k, Cv, sC);
    phase_mark(ph, 7, tp);
    kacc = k;
    __syncthreads();
  }
  if (threadIdx.x == 0) B.ranks[op.slot] = kacc;
  __syncthreads();
}

template <class T, class C>
__global__ void __launch_bounds__(TR_THREADS, sizeof(T) == 4 ? 2 : 1) k_trunc(const OpTrunc* ops, int64_t count, const TermD* terms,
                                                       Bases B) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ TrShared<C> ts;
  double* scr = B.scratch + (int64_t)blockIdx.x * TR_SCRATCH;
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x)
    trunc_one<T, C>(ops[o], terms, B, scr, reinterpret_cast<T*>(smraw), ts);
}

// One part (rk of TR_CL) of a truncation op shared by TR_CL CTAs: each
// streams its share of the rows, parts 0 and 1 combine the partial R
// factors, part 0 computes the core, all apply.  scr_of(r) is part r's
// scratch slice; sync() separates the phases (a cluster barrier, or a
// bounded barrier in global memory: false when it gave up, and then the part
// stops).
template <class T, class C, class ScrOf, class Sync>
__device__ void trunc_part(const OpTrunc& op, const TermD* terms, const Bases& B, int rk, ScrOf scr_of, Sync sync,
                           T* sC, TrShared<C>& ts) {
  TrCat& cat = ts.cat;
  CoreShared<C>& cs = ts.cs;
  double* sh = ts.sh;
  double* scr = scr_of(rk);
  T* Pu = reinterpret_cast<T*>(scr);
  T* Pv = reinterpret_cast<T*>(scr + TR_REG);
  C* J = reinterpret_cast<C*>(scr + 4 * TR_REG);  // the combined R factor of this part's side
  C* Cu0 = reinterpret_cast<C*>(scr_of(0) + TR_OFF_CU);  // coefficients live with part 0
  C* Cv0 = reinterpret_cast<C*>(scr_of(0) + TR_OFF_CV);
  int* flag0 = reinterpret_cast<int*>(scr_of(0) + TR_OFF_FLAG);
  const TermD* tl = terms + op.term0;
  int kacc = op.keep ? B.ranks[op.slot] : 0;
  int t0 = 0;
  bool first = true;
  while (first || t0 < op.nterms) {
    first = false;
    int t1;
    const int K = tr_batch(op, tl, B.ranks, kacc, t0, &t1, cat);
    t0 = t1;
    if (K == 0) {
      kacc = 0;
      continue;
    }
    if (K > TR_KT) {
      if (threadIdx.x == 0 && rk == 0) record_error(B.status, DEV_RANK, K);
      kacc = 0;
      break;
    }
    const int mu0 = (int)((int64_t)op.m * rk / TR_CL), mu1 = (int)((int64_t)op.m * (rk + 1) / TR_CL);
    const int nv0 = (int)((int64_t)op.n * rk / TR_CL), nv1 = (int)((int64_t)op.n * (rk + 1) / TR_CL);
    // 1. partial R factors of this part's rows
    if (K <= 32) {
      qr_tsqr<T>([&](int r, int c) { return cat_value(B, op, cat, 0, mu0 + r, c); }, mu1 - mu0, K, Pu, sC);
      qr_tsqr<T>([&](int r, int c) { return cat_value(B, op, cat, 1, nv0 + r, c); }, nv1 - nv0, K, Pv, sC);
    } else {
      qr_stream<T>([&](int r, int c) { return cat_value(B, op, cat, 0, mu0 + r, c); }, mu1 - mu0, K, Pu, sC, sh);
      qr_stream<T>([&](int r, int c) { return cat_value(B, op, cat, 1, nv0 + r, c); }, nv1 - nv0, K, Pv, sC, sh);
    }
    if (!sync()) return;
    // 2. part 0 combines the U partials into its J region, part 1 the V partials
    if (rk < 2) {
      const int64_t poff = rk == 0 ? 0 : TR_REG;
      T* fin = reinterpret_cast<T*>(J);
      auto part = [&](int r, int c) {
        const T* P = reinterpret_cast<const T*>(scr_of(r / K) + poff);
        const int i = r % K;
        return i <= c ? (double)P[i + (int64_t)c * TR_KT] : 0.0;
      };
      if (K <= 32)
        qr_tsqr<T>(part, TR_CL * K, K, fin, sC);
      else
        qr_stream<T>(part, TR_CL * K, K, fin, sC, sh);
    }
    if (!sync()) return;
    // 3. part 0: core from R_u (own J) and R_v (part 1's J)
    if (rk == 0) {
      T* Ru = Pu;
      T* Rv = Pv;
      const T* fu = reinterpret_cast<const T*>(J);
      const T* fv = reinterpret_cast<const T*>(scr_of(1) + 4 * TR_REG);
      for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e % K, j = e / K;
        Ru[i + (int64_t)j * TR_KT] = fu[i + (int64_t)j * TR_KT];
        Rv[i + (int64_t)j * TR_KT] = fv[i + (int64_t)j * TR_KT];
      }
      __syncthreads();
      tr_core<T, C>(Ru, Rv, K, op.eps, op.kcap, op.kfix, reinterpret_cast<C*>(sC), core_smem_elems<T, C>(), scr,
                    Cu0, Cv0, cs, B.status);
      if (threadIdx.x == 0) flag0[0] = cs.k;
    }
    if (!sync()) return;
    const int k = reinterpret_cast<const volatile int*>(flag0)[0];
    if (B.flops && threadIdx.x == 0 && rk == 0)
      atomicAdd(B.flops + OP_TRUNC_BIG,
                2.0 * K * K * (double)(op.m + op.n) + 2.0 * K * (double)k * (op.m + op.n));
    // 4. all parts apply to their rows
    tr_apply<T, C>(B, op, cat, 0, mu0, mu1, K, k, Cu0, sC);
    tr_apply<T, C>(B, op, cat, 1, nv0, nv1, K, k, Cv0, sC);
    kacc = k;
    if (!sync()) return;
  }
  if (threadIdx.x == 0 && rk == 0) B.ranks[op.slot] = kacc;
}

// Cluster variant for large targets: the TR_CL CTAs of a cluster share one op.
template <class T, class C>
__global__ void __cluster_dims__(TR_CL, 1, 1) __launch_bounds__(TR_THREADS, sizeof(T) == 4 ? 2 : 1)
    k_trunc_cl(const OpTrunc* ops, int64_t count, const TermD* terms, Bases B) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ TrShared<C> ts;
  cg::cluster_group cluster = cg::this_cluster();
  const int rk = (int)cluster.block_rank();
  const int64_t cid = blockIdx.x / TR_CL, ncl = gridDim.x / TR_CL;
  const int64_t base_cta = cid * TR_CL;  // first CTA of this cluster
  auto scr_of = [&](int r) { return B.scratch + (base_cta + r) * TR_SCRATCH; };
  auto sync = [&]() {
    __threadfence();
    cluster.sync();
    return true;
  };
  for (int64_t o = cid; o < count; o += ncl) {
    trunc_part<T, C>(ops[o], terms, B, rk, scr_of, sync, reinterpret_cast<T*>(smraw), ts);
    sync();
  }
}

// ---------------------------------------------------------------------------
// The whole H-Cholesky as one dependency-driven cooperative launch.  The ops
// of the plan (POTRF, TRSM, GEMM, truncations) run in the order they become
// ready: a ready queue holds one slot per op, its first n0 slots the ops
// without producers; a free CTA takes the next slot number from a counter,
// waits until that slot is filled, runs the op and signals its consumers; the
// CTA whose signal completes a consumer's count appends the consumer to the
// queue.  A group truncation is TR_CL consecutive ops, one per part, queued
// together in TR_CL consecutive slots when its first part is released: its
// CTAs meet at the start (each publishes its scratch slice) and at every
// phase of the op through bounded barriers in global memory, and part 0
// signals the consumers when all parts are done.  Progress: every queued op
// can run (its producers are done), a group's parts are taken by the next
// TR_CL free CTAs (the grid has more than TR_CL CTAs), and every op is
// queued once its producers finish, so every slot is filled.  Every wait is
// bounded (kBarrierNs): a CTA that gives up records DEV_TIMEOUT and raises
// the abort flag, and every CTA leaves.  Each op computes what it computes in
// the wave launches, after the same producers: the results are the waves'.
// With a trace buffer (FactorTrace per op) the kernel records when a CTA
// took the op's slot, when the slot was filled and when the op finished, its
// CTA, and the producer whose signal released it.
// ---------------------------------------------------------------------------
template <class T, class C>
__global__ void __launch_bounds__(TR_THREADS, sizeof(T) == 4 ? 2 : 1)
    k_factor(const FlowOp* flow, int64_t nops, const int32_t* npred, const int64_t* succ_off, const int32_t* succ,
             int32_t* count, int32_t* ready, int64_t n0, const OpPotrf* potrf, const OpTrsm* trsm,
             const OpGemm* gemm, const OpTrunc* trunc, const TermD* terms, TrGroup* groups, Bases B, GridBar* gb,
             FactorTrace* trace) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ TrShared<C> ts;
  __shared__ GemmSmem<T> gs;
  __shared__ long long s_op;
  __shared__ int s_ok;
  double* my_scr = B.scratch + (int64_t)blockIdx.x * TR_SCRATCH;
  for (;;) {
    if (threadIdx.x == 0) {
      volatile unsigned int* abort = &gb->abort;
      long long slot = -1, i = -1;
      if (!*abort) slot = (long long)atomicAdd(&gb->ticket, 1ull);
      int ok = slot >= 0 && slot < nops;
      if (ok) {
        const unsigned long long t0 = global_ns();
        const volatile int32_t* q = ready + slot;
        while ((i = *q) < 0) {
          if (*abort || global_ns() - t0 > kBarrierNs) {
            atomicExch(&gb->abort, 1u);
            record_error(B.status, DEV_TIMEOUT, 2);
            ok = 0;
            break;
          }
          __nanosleep(20);
        }
        __threadfence();
        if (ok && trace) {
          trace[i].t_take = t0;
          trace[i].t_ready = global_ns();
          trace[i].cta = (uint32_t)blockIdx.x;
        }
      }
      s_op = i;
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    const FlowOp f = flow[s_op];
    bool done = true;
    switch (f.type) {
      case OP_POTRF:
        do_potrf(potrf[f.idx], B, reinterpret_cast<double*>(smraw));
        break;
      case OP_TRSM:
        do_trsm<T>(trsm[f.idx], B, reinterpret_cast<T*>(smraw));
        break;
      case OP_GEMM:
        do_gemm<T>(gemm[f.idx], B, gs);
        break;
      case OP_TRUNC:
        trunc_one<T, C>(trunc[f.idx], terms, B, my_scr, reinterpret_cast<T*>(smraw), ts);
        break;
      default: {  // OP_TRUNC_BIG: part f.part of a group
        TrGroup* g = groups + f.group;
        if (threadIdx.x == 0) g->cta[f.part] = (int32_t)blockIdx.x;
        auto sync = [&]() { return bounded_barrier(&g->count, &g->gen, TR_CL, &gb->abort, B.status); };
        if (!sync()) return;  // every part has published its scratch slice
        auto scr_of = [&](int r) {
          return B.scratch + (int64_t)reinterpret_cast<volatile int32_t*>(g->cta)[r] * TR_SCRATCH;
        };
        trunc_part<T, C>(trunc[f.idx], terms, B, f.part, scr_of, sync, reinterpret_cast<T*>(smraw), ts);
        done = sync();  // all parts finished, the rank is written
        if (!done) return;
        if (f.part != 0) {  // part 0 signals for the group
          if (trace && threadIdx.x == 0) trace[s_op].t_done = global_ns();
          continue;
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // the op's writes before its signals
      if (trace) trace[s_op].t_done = global_ns();
      for (int64_t e = succ_off[s_op]; e < succ_off[s_op + 1]; ++e) {
        const int32_t v = succ[e];
        if (atomicAdd(count + v, 1) + 1 != npred[v]) continue;
        // the last producer of v: queue it (a group with all its parts)
        const int np = flow[v].type == OP_TRUNC_BIG ? TR_CL : 1;
        const long long pos = n0 + (long long)atomicAdd(&gb->tail, (unsigned long long)np);
        if (trace) trace[v].releaser = (int32_t)s_op;
        for (int p = 0; p < np; ++p) atomicExch(ready + pos + p, v + p);
      }
    }
  }
}

// dynamic shared memory of the factorisation kernel: the truncation chunk
// or TRSM / POTRF block, whichever is larger
template <class T, class C>
static size_t factor_smem(int max_dense);

// dynamic shared memory: the streamed chunk, or the per-warp R factors and
// update arrays of the warp-level QR, whichever is larger
template <class T, class C>
static size_t smem_bytes() {
  const size_t chunk = (size_t)TrCh<T>::elems * sizeof(T);
  const size_t tsqr = (size_t)(TR_THREADS / 32) * 32 * (TSQR_LD + 1) * sizeof(T);
  return chunk > tsqr ? chunk : tsqr;
}

template <class T, class C>
static int configure_pair() {
  int bad = 0;
  const int sm = (int)smem_bytes<T, C>();
  bad |= cudaFuncSetAttribute(k_trunc<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess;
  bad |= cudaFuncSetAttribute(k_trunc_cl<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess;
  return bad;
}

int configure_trunc() {
  const int bad = configure_pair<double, double>() | configure_pair<float, float>() | configure_pair<float, double>();
  return bad ? -1 : 0;
}

template <class T, class C>
static void launch_pair(const OpTrunc* ops, int64_t count, const TermD* terms, const Bases& B, bool big,
                        cudaStream_t st) {
  const int cap = max_trunc_ctas();
  const size_t sm = smem_bytes<T, C>();
  if (!big) {
    const int grid = (int)(count < cap ? count : cap);
    k_trunc<T, C><<<grid, TR_THREADS, sm, st>>>(ops, count, terms, B);
  } else {
    const int64_t ncl = count < cap / TR_CL ? count : cap / TR_CL;
    k_trunc_cl<T, C><<<(int)(ncl * TR_CL), TR_THREADS, sm, st>>>(ops, count, terms, B);
  }
}

template <class T, class C>
static size_t factor_smem(int max_dense) {
  const size_t tr = smem_bytes<T, C>(), blk = trsm_smem(max_dense);
  return tr > blk ? tr : blk;
}

template <class T, class C>
static int launch_factor_t(const Plan& P, const Bases& B, GridBar* gb, int max_dense, FactorTrace* trace,
                           cudaStream_t st) {
  const size_t sm = factor_smem<T, C>(max_dense);
  if (cudaFuncSetAttribute(k_factor<T, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
    return -1;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_factor<T, C>, TR_THREADS, sm) != cudaSuccess) return -1;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int grid = per * sms;
  if (grid > max_trunc_ctas()) grid = max_trunc_ctas();  // one truncation scratch slice per CTA
  const int64_t nops = (int64_t)P.flow.size();
  if (grid <= TR_CL || nops <= 0 || !gb || !P.d_count) return -1;
  if (cudaMemsetAsync(gb, 0, sizeof(GridBar), st) != cudaSuccess) return -1;
  if (cudaMemsetAsync(P.d_count, 0, nops * sizeof(int32_t), st) != cudaSuccess) return -1;
  if (P.ngroups && cudaMemsetAsync(P.d_groups, 0, P.ngroups * sizeof(TrGroup), st) != cudaSuccess) return -1;
  // the ready queue: the ops without producers, then empty slots (-1)
  const int64_t n0 = (int64_t)P.ready0.size();
  if (!P.d_ready || !P.d_ready0 || n0 <= 0) return -1;
  if (cudaMemsetAsync(P.d_ready, 0xff, nops * sizeof(int32_t), st) != cudaSuccess) return -1;
  if (cudaMemcpyAsync(P.d_ready, P.d_ready0, n0 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return -1;
  const FlowOp* flow = P.d_flow;
  const int32_t* npred = P.d_npred;
  const int64_t* so = P.d_succ_off;
  const int32_t* sc = P.d_succ;
  int32_t* cnt = P.d_count;
  int32_t* rq = P.d_ready;
  const OpPotrf* po = P.d_potrf;
  const OpTrsm* tr = P.d_trsm;
  const OpGemm* ge = P.d_gemm;
  const OpTrunc* tu = P.d_trunc;
  const TermD* te = P.d_terms;
  TrGroup* gr = P.d_groups;
  Bases b = B;
  void* args[] = {(void*)&flow, (void*)&nops, (void*)&npred, (void*)&so,  (void*)&sc, (void*)&cnt,
                  (void*)&rq,   (void*)&n0,   (void*)&po,    (void*)&tr,  (void*)&ge, (void*)&tu,
                  (void*)&te,   (void*)&gr,   (void*)&b,     (void*)&gb,  (void*)&trace};
  return cudaLaunchCooperativeKernel((void*)k_factor<T, C>, grid, TR_THREADS, args, sm, st) == cudaSuccess ? 0 : -1;
}

int launch_factor(const Plan& P, const Bases& B, GridBar* gb, int max_dense, FactorTrace* trace, cudaStream_t st) {
  if (!B.mixed) return launch_factor_t<double, double>(P, B, gb, max_dense, trace, st);
  if (B.core64) return launch_factor_t<float, double>(P, B, gb, max_dense, trace, st);
  return launch_factor_t<float, float>(P, B, gb, max_dense, trace, st);
}

// FP64: FP64 throughout; mixed: FP32 panels with an FP32 core, or with an
// FP64 core (B.core64)
void launch_trunc(const OpTrunc* ops, int64_t count, const TermD* terms, const Bases& B, bool big,
                  cudaStream_t st) {
  if (count <= 0) return;
  if (!B.mixed)
    launch_pair<double, double>(ops, count, terms, B, big, st);
  else if (B.core64)
    launch_pair<float, double>(ops, count, terms, B, big, st);
  else
    launch_pair<float, float>(ops, count, terms, B, big, st);
}

}  // namespace hlc
