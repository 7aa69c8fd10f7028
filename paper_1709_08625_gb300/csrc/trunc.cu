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
//      row chunks ([R; chunk] -> R); Q is never formed;
//   2. M = R_u R_v^T (K x K, FP64);
//   3. the SVD of M in FP64: QR with column pivoting reduces M to its
//      numerical rank r (the trailing part dropped is below 1e-3 eps |M|),
//      then one-sided Jacobi on the r columns of (R P^T)^T: M = X S Y^T;
//   4. keep the k values sigma_i > eps sigma_1 and write
//        U_new = Ucat R_v^T Y_k S_k^-1/2 = Q_u X_k S_k^1/2,
//        V_new = Vcat R_u^T X_k S_k^-1/2 = Q_v Y_k S_k^1/2,
//      row by row, in place.
//
// Steps 1 and 4 run in FP64 (HLC_FP64) or FP32 (HLC_MIXED); step 3 is FP64
// in both.  Targets with m + n above TR_BIG_ROWS run on a cluster of TR_CL
// CTAs: each CTA streams its share of the rows, CTAs 0 and 1 combine the
// partial R factors, CTA 0 computes the core, all CTAs apply; the phases are
// separated by cluster barriers.

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "devutil.cuh"
#include "hlc_internal.h"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace hlc {

constexpr int TR_KB = 64;      // new columns per batch
constexpr int TR_KT = 256;     // columns of one truncation: rank (<= 128) + batch (<= 128)
constexpr int TR_KCAP = 128;   // rank capacity of a block
// rows per streamed chunk: 64 KB of shared memory either way (3 CTAs per SM)
template <class T>
struct TrCh {
  static constexpr int value = sizeof(T) == 8 ? 32 : 64;
};
constexpr int TR_THREADS = 256;
constexpr int TR_OUT_LD = TR_KCAP + 1;
constexpr int TR_CL = 8;       // CTAs per cluster for large targets
constexpr int64_t TR_REG = (int64_t)TR_KT * TR_KT;
// per-CTA scratch: Pu, Pv, M, W, J, X (K x K each), Cu, Cv (K x 128 each),
// the apply stage, and a few words for cluster broadcasts
constexpr int64_t TR_PANEL = (int64_t)TR_KT * TR_KCAP;
constexpr int64_t TR_OFF_X = 5 * TR_REG;
constexpr int64_t TR_OFF_CU = TR_OFF_X + TR_REG;  // X holds the rank x rank Jacobi matrix
constexpr int64_t TR_OFF_CV = TR_OFF_CU + TR_PANEL;
constexpr int64_t TR_OFF_STAGE = TR_OFF_CV + TR_PANEL;
constexpr int64_t TR_OFF_FLAG = TR_OFF_STAGE + (int64_t)TR_THREADS * TR_OUT_LD;
constexpr int64_t TR_SCRATCH = TR_OFF_FLAG + 8;

int64_t trunc_scratch_doubles() { return TR_SCRATCH; }
int max_trunc_ctas() { return 152 * 3; }

struct TrCat {
  int kacc;            // leading columns from the target itself
  int nt;              // terms in the batch
  const TermD* terms;  // batch terms
  int col0[65];        // first concatenated column of each term; col0[nt] = K
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
  int t = 0;
  while (col >= cat.col0[t + 1]) ++t;
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
// matrix whose entries rowval(i, c) returns.  sC: TrCh<T> x K chunk buffer.
template <class T, class F>
__device__ void qr_stream(F rowval, int nrows, int K, T* R, T* sC, double* sh) {
  constexpr int TR_CH = TrCh<T>::value;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  for (int e = tid; e < K * K; e += blockDim.x) R[(e % K) + (int64_t)(e / K) * TR_KT] = T(0);
  __syncthreads();
  for (int r0 = 0; r0 < nrows; r0 += TR_CH) {
    const int rows = min(TR_CH, nrows - r0);
    for (int e = tid; e < rows * K; e += blockDim.x) {
      const int i = e % rows, c = e / rows;
      sC[i + c * TR_CH] = (T)rowval(r0 + i, c);
    }
    __syncthreads();
    for (int j = 0; j < K; ++j) {
      if (w == 0) {
        T xn = T(0);
        for (int i = lane; i < rows; i += 32) xn += sC[i + j * TR_CH] * sC[i + j * TR_CH];
        for (int o = 16; o > 0; o >>= 1) xn += __shfl_xor_sync(0xffffffffu, xn, o);
        const T alpha = R[j + (int64_t)j * TR_KT];
        T tau = T(0), sc = T(0), beta = alpha;
        if (xn > T(0)) {
          beta = -copysign(sqrt(alpha * alpha + xn), alpha);
          tau = (beta - alpha) / beta;
          sc = T(1) / (alpha - beta);
        }
        if (tau != T(0))
          for (int i = lane; i < rows; i += 32) sC[i + j * TR_CH] *= sc;
        if (lane == 0) {
          R[j + (int64_t)j * TR_KT] = beta;
          sh[0] = (double)tau;
        }
      }
      __syncthreads();
      const T tau = (T)sh[0];
      if (tau != T(0)) {
        for (int l = j + 1 + w; l < K; l += nw) {
          T p = T(0);
          for (int i = lane; i < rows; i += 32) p += sC[i + j * TR_CH] * sC[i + l * TR_CH];
          for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
          const T wv = tau * (p + R[j + (int64_t)l * TR_KT]);
          for (int i = lane; i < rows; i += 32) sC[i + l * TR_CH] -= wv * sC[i + j * TR_CH];
          if (lane == 0) R[j + (int64_t)l * TR_KT] -= wv;
        }
      }
      __syncthreads();
    }
  }
}

struct CoreShared {
  double cn[TR_KT];
  double tauq[TR_KT];
  double sv[TR_KT];
  int piv[TR_KT];
  int order[TR_KT];
  double red[40];
  int stop, jmax, rank, k, rot;
};

// FP64 core: SVD of M = R_u R_v^T reduced by column-pivoted QR, truncation
// rank, and the coefficient matrices Cu, Cv (K x k, ld TR_KT).
template <class T>
__device__ void tr_core(const T* Ru, const T* Rv, int K, double eps, int kcap, double* M, double* W, double* J,
                        double* X, double* Cu, double* Cv, CoreShared& cs, int* status) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  // M = Ru Rv^T (both upper triangular)
  for (int e = tid; e < K * K; e += blockDim.x) {
    const int i = e % K, j = e / K;
    double s = 0.0;
    for (int c = max(i, j); c < K; ++c) s += (double)Ru[i + (int64_t)c * TR_KT] * (double)Rv[j + (int64_t)c * TR_KT];
    M[i + (int64_t)j * TR_KT] = s;
  }
  for (int j = tid; j < K; j += blockDim.x) cs.piv[j] = j;
  __syncthreads();
  // Householder QR with column pivoting, stopped at the numerical rank
  double ref = 0.0;
  int r = 0;
  for (; r < K; ++r) {
    for (int j = r + w; j < K; j += nw) {
      double p = 0.0;
      for (int i = r + lane; i < K; i += 32) p += M[i + (int64_t)j * TR_KT] * M[i + (int64_t)j * TR_KT];
      p = warp_sum(p);
      if (lane == 0) cs.cn[j] = p;
    }
    __syncthreads();
    if (tid == 0) {
      int jm = r;
      double rem = 0.0;
      for (int j = r; j < K; ++j) {
        rem += cs.cn[j];
        if (cs.cn[j] > cs.cn[jm]) jm = j;
      }
      cs.jmax = jm;
      if (r == 0) cs.red[0] = sqrt(cs.cn[jm]);
      cs.stop = (cs.red[0] == 0.0) || !(sqrt(rem) > 1e-3 * eps * cs.red[0]);
    }
    __syncthreads();
    ref = cs.red[0];
    if (cs.stop) break;
    const int jm = cs.jmax;
    if (jm != r) {
      for (int i = tid; i < K; i += blockDim.x) {
        const double a = M[i + (int64_t)r * TR_KT];
        M[i + (int64_t)r * TR_KT] = M[i + (int64_t)jm * TR_KT];
        M[i + (int64_t)jm * TR_KT] = a;
      }
      if (tid == 0) {
        const int t = cs.piv[r];
        cs.piv[r] = cs.piv[jm];
        cs.piv[jm] = t;
      }
    }
    __syncthreads();
    if (w == 0) {
      double xn = 0.0;
      for (int i = r + 1 + lane; i < K; i += 32) xn += M[i + (int64_t)r * TR_KT] * M[i + (int64_t)r * TR_KT];
      xn = warp_sum(xn);
      const double alpha = M[r + (int64_t)r * TR_KT];
      double tau = 0.0, sc = 0.0, beta = alpha;
      if (xn > 0.0) {
        beta = -copysign(sqrt(alpha * alpha + xn), alpha);
        tau = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
      }
      if (tau != 0.0)
        for (int i = r + 1 + lane; i < K; i += 32) M[i + (int64_t)r * TR_KT] *= sc;
      if (lane == 0) {
        M[r + (int64_t)r * TR_KT] = beta;
        cs.tauq[r] = tau;
      }
    }
    __syncthreads();
    const double tau = cs.tauq[r];
    if (tau != 0.0) {
      for (int l = r + 1 + w; l < K; l += nw) {
        double p = 0.0;
        for (int i = r + 1 + lane; i < K; i += 32) p += M[i + (int64_t)r * TR_KT] * M[i + (int64_t)l * TR_KT];
        p = warp_sum(p);
        const double wv = tau * (p + M[r + (int64_t)l * TR_KT]);
        for (int i = r + 1 + lane; i < K; i += 32) M[i + (int64_t)l * TR_KT] -= wv * M[i + (int64_t)r * TR_KT];
        if (lane == 0) M[r + (int64_t)l * TR_KT] -= wv;
      }
    }
    __syncthreads();
  }
  const int rank = r;
  (void)ref;
  (void)X;
  if (rank == 0) {
    if (tid == 0) cs.k = 0;
    __syncthreads();
    return;
  }
  // B = (R P^T)^T (K x rank) into W
  for (int e = tid; e < K * rank; e += blockDim.x) {
    const int j = e % K, i = e / K;  // R(i, j) -> B(piv[j], i)
    W[cs.piv[j] + (int64_t)i * TR_KT] = (i <= j) ? M[i + (int64_t)j * TR_KT] : 0.0;
  }
  __syncthreads();
  // Householder QR of B (K x rank): B = Q_B R_B; the one-sided Jacobi then
  // works on the rank x rank triangle R_B (QR preconditioning of the Jacobi
  // SVD), and the left vectors of B are Q_B times those of R_B.
  for (int q = 0; q < rank; ++q) {
    if (w == 0) {
      double xn = 0.0;
      for (int i = q + 1 + lane; i < K; i += 32) xn += W[i + (int64_t)q * TR_KT] * W[i + (int64_t)q * TR_KT];
      xn = warp_sum(xn);
      const double alpha = W[q + (int64_t)q * TR_KT];
      double tau = 0.0, sc = 0.0, beta = alpha;
      if (xn > 0.0) {
        beta = -copysign(sqrt(alpha * alpha + xn), alpha);
        tau = (beta - alpha) / beta;
        sc = 1.0 / (alpha - beta);
      }
      if (tau != 0.0)
        for (int i = q + 1 + lane; i < K; i += 32) W[i + (int64_t)q * TR_KT] *= sc;
      if (lane == 0) {
        W[q + (int64_t)q * TR_KT] = beta;
        cs.cn[q] = tau;  // tau of the B reflectors
      }
    }
    __syncthreads();
    const double tau = cs.cn[q];
    if (tau != 0.0) {
      for (int l = q + 1 + w; l < rank; l += nw) {
        double p = 0.0;
        for (int i = q + 1 + lane; i < K; i += 32) p += W[i + (int64_t)q * TR_KT] * W[i + (int64_t)l * TR_KT];
        p = warp_sum(p);
        const double wv = tau * (p + W[q + (int64_t)l * TR_KT]);
        for (int i = q + 1 + lane; i < K; i += 32) W[i + (int64_t)l * TR_KT] -= wv * W[i + (int64_t)q * TR_KT];
        if (lane == 0) W[q + (int64_t)l * TR_KT] -= wv;
      }
    }
    __syncthreads();
  }
  // R_B (upper triangle of W's first rank rows) becomes the Jacobi matrix A
  // (X region); J accumulates its rotations.
  double* A = X;
  for (int e = tid; e < rank * rank; e += blockDim.x) {
    const int i = e % rank, j = e / rank;
    A[i + (int64_t)j * TR_KT] = (i <= j) ? W[i + (int64_t)j * TR_KT] : 0.0;
    J[i + (int64_t)j * TR_KT] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // one-sided Jacobi on the rank columns of A, round-robin pairs
  double fro2 = 0.0;
  for (int e = tid; e < rank * rank; e += blockDim.x) {
    const double v = A[(e % rank) + (int64_t)(e / rank) * TR_KT];
    fro2 += v * v;
  }
  fro2 = block_sum(fro2, cs.red + 1);
  const double tiny = 1e-34 * fro2;
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
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < rank; i += 32) {
          const double x = A[i + (int64_t)a * TR_KT], y = A[i + (int64_t)b * TR_KT];
          al += x * x;
          be += y * y;
          ga += x * y;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (al <= tiny && be <= tiny) continue;
        if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        for (int i = lane; i < rank; i += 32) {
          const double x = A[i + (int64_t)a * TR_KT], y = A[i + (int64_t)b * TR_KT];
          A[i + (int64_t)a * TR_KT] = c * x - sn * y;
          A[i + (int64_t)b * TR_KT] = sn * x + c * y;
          const double jx = J[i + (int64_t)a * TR_KT], jy = J[i + (int64_t)b * TR_KT];
          J[i + (int64_t)a * TR_KT] = c * jx - sn * jy;
          J[i + (int64_t)b * TR_KT] = sn * jx + c * jy;
        }
        if (lane == 0) cs.rot = 1;
      }
      __syncthreads();
    }
    if (!cs.rot) break;
    __syncthreads();
  }
  // singular values, order (ties: smaller index first), truncation rank
  for (int j = w; j < rank; j += nw) {
    double s = 0.0;
    for (int i = lane; i < rank; i += 32) s += A[i + (int64_t)j * TR_KT] * A[i + (int64_t)j * TR_KT];
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
    const double smax = cs.sv[cs.order[0]];
    int k = 0;
    if (smax > 0.0)
      while (k < rank && cs.sv[cs.order[k]] > eps * smax) ++k;
    if (!(smax == smax)) {
      record_error(status, DEV_BAD, 1);
      k = 0;
    }
    if (k > kcap) {
      record_error(status, DEV_RANK, k);
      k = kcap;
    }
    cs.k = k;
  }
  __syncthreads();
  const int k = cs.k;
  // With B = P R^T = Q_B A J^T... the Jacobi gives A J = Wa (orthogonal
  // columns), so B = Q_B Wa J^T and M = Q R P^T = Q B^T = (Q J) S (Q_B Wa_n)^T:
  //   left vectors of M:  x_c = Q [J(:, j_c); 0]      (reflectors of the pivoted QR, in M)
  //   right vectors of M: y_c = Q_B [Wa_n(:, j_c); 0]  (reflectors of the QR of B, in W)
  // Both are built in the Cu/Cv regions' columns (K x k each) before the
  // coefficients overwrite them: x_c in Cv, y_c in Cu.
  for (int c = w; c < k; c += nw) {
    const int j = cs.order[c];
    const double sv = cs.sv[j];
    double* x = Cv + (int64_t)c * TR_KT;
    double* y = Cu + (int64_t)c * TR_KT;
    for (int i = lane; i < K; i += 32) {
      x[i] = i < rank ? J[i + (int64_t)j * TR_KT] : 0.0;
      y[i] = i < rank ? A[i + (int64_t)j * TR_KT] / sv : 0.0;
    }
    __syncwarp();
    for (int q = rank - 1; q >= 0; --q) {
      const double tq = cs.tauq[q], tb = cs.cn[q];
      double p = 0.0, pb = 0.0;
      for (int i = q + lane; i < K; i += 32) {
        p += (i == q ? 1.0 : M[i + (int64_t)q * TR_KT]) * x[i];
        pb += (i == q ? 1.0 : W[i + (int64_t)q * TR_KT]) * y[i];
      }
      p = warp_sum(p);
      pb = warp_sum(pb);
      for (int i = q + lane; i < K; i += 32) {
        if (tq != 0.0) x[i] -= tq * p * (i == q ? 1.0 : M[i + (int64_t)q * TR_KT]);
        if (tb != 0.0) y[i] -= tb * pb * (i == q ? 1.0 : W[i + (int64_t)q * TR_KT]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // Cu = R_v^T y_c / s^0.5 ; Cv = R_u^T x_c / s^0.5 (in place: column c of
  // Cu / Cv holds y_c / x_c; each thread finishes a whole column)
  for (int c = tid; c < k; c += blockDim.x) {
    const double isq = 1.0 / sqrt(cs.sv[cs.order[c]]);
    double* y = Cu + (int64_t)c * TR_KT;
    double* x = Cv + (int64_t)c * TR_KT;
    for (int col = K - 1; col >= 0; --col) {  // R^T is lower: row col needs entries p <= col
      double a = 0.0, b = 0.0;
      for (int p = 0; p <= col; ++p) {
        a += (double)Rv[p + (int64_t)col * TR_KT] * y[p];
        b += (double)Ru[p + (int64_t)col * TR_KT] * x[p];
      }
      y[col] = a * isq;
      x[col] = b * isq;
    }
  }
  __syncthreads();
}

// Rows [r0, r1) of one side: out(row, c) = sum_col cat(row, col) C(col, c).
template <class T>
__device__ void tr_apply(const Bases& B, const OpTrunc& op, const TrCat& cat, int side, int r0, int r1, int K,
                         int k, const double* C, T* stage) {
  const int tid = threadIdx.x;
  const int ld = side == 0 ? op.m : op.n;
  double* out = side == 0 ? B.buf[op.U.buf] + op.U.off : B.buf[op.V.buf] + op.V.off;
  T* so = stage + tid * TR_OUT_LD;
  for (int base = r0; base < r1; base += blockDim.x) {
    const int r = base + tid;
    if (r < r1) {
      for (int c = 0; c < k; ++c) so[c] = T(0);
      for (int col = 0; col < K; ++col) {
        const T v = (T)cat_value(B, op, cat, side, r, col);
        if (v != T(0))
          for (int c = 0; c < k; ++c) so[c] += v * (T)C[col + (int64_t)c * TR_KT];
      }
    }
    __syncthreads();
    if (r < r1)
      for (int c = 0; c < k; ++c) out[r + (int64_t)c * ld] = (double)so[c];
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
      c += term_cols(tl[t], ranks);
    }
    cat.col0[t1 - t0] = c;
  }
  __syncthreads();
  *t1out = t1;
  return kacc + kb;
}

template <class T>
__global__ void __launch_bounds__(TR_THREADS) k_trunc(const OpTrunc* ops, int64_t count, const TermD* terms,
                                                       Bases B) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sC = reinterpret_cast<T*>(smraw);
  __shared__ TrCat cat;
  __shared__ CoreShared cs;
  __shared__ double sh[2];
  double* scr = B.scratch + (int64_t)blockIdx.x * TR_SCRATCH;
  T* Pu = reinterpret_cast<T*>(scr);
  T* Pv = reinterpret_cast<T*>(scr + TR_REG);
  double* M = scr + 2 * TR_REG;
  double* W = scr + 3 * TR_REG;
  double* J = scr + 4 * TR_REG;
  double* X = scr + TR_OFF_X;
  double* Cu = scr + TR_OFF_CU;
  double* Cv = scr + TR_OFF_CV;
  T* stage = reinterpret_cast<T*>(scr + TR_OFF_STAGE);
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) {
    const OpTrunc op = ops[o];
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
      qr_stream<T>([&](int r, int c) { return cat_value(B, op, cat, 0, r, c); }, op.m, K, Pu, sC, sh);
      qr_stream<T>([&](int r, int c) { return cat_value(B, op, cat, 1, r, c); }, op.n, K, Pv, sC, sh);
      tr_core<T>(Pu, Pv, K, op.eps, op.kcap, M, W, J, X, Cu, Cv, cs, B.status);
      const int k = cs.k;
      // algorithmic flops of the batch: two streamed R factors and the apply
      if (B.flops && threadIdx.x == 0)
        atomicAdd(B.flops + OP_TRUNC, 2.0 * K * K * (double)(op.m + op.n) + 2.0 * K * (double)k * (op.m + op.n));
      tr_apply<T>(B, op, cat, 0, 0, op.m, K, k, Cu, stage);
      tr_apply<T>(B, op, cat, 1, 0, op.n, K, k, Cv, stage);
      kacc = k;
      __syncthreads();
    }
    if (threadIdx.x == 0) B.ranks[op.slot] = kacc;
    __syncthreads();
  }
}

// Cluster variant for large targets: the TR_CL CTAs of a cluster share one op.
template <class T>
__global__ void __cluster_dims__(TR_CL, 1, 1) __launch_bounds__(TR_THREADS)
    k_trunc_cl(const OpTrunc* ops, int64_t count, const TermD* terms, Bases B) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sC = reinterpret_cast<T*>(smraw);
  __shared__ TrCat cat;
  __shared__ CoreShared cs;
  __shared__ double sh[2];
  cg::cluster_group cluster = cg::this_cluster();
  const int rk = (int)cluster.block_rank();
  const int64_t cid = blockIdx.x / TR_CL, ncl = gridDim.x / TR_CL;
  const int64_t base_cta = cid * TR_CL;  // first CTA of this cluster
  auto scr_of = [&](int r) { return B.scratch + (base_cta + r) * TR_SCRATCH; };
  double* scr = scr_of(rk);
  T* Pu = reinterpret_cast<T*>(scr);
  T* Pv = reinterpret_cast<T*>(scr + TR_REG);
  double* M = scr + 2 * TR_REG;
  double* W = scr + 3 * TR_REG;
  double* J = scr + 4 * TR_REG;
  double* X = scr + TR_OFF_X;
  double* Cu0 = scr_of(0) + TR_OFF_CU;  // coefficients live with CTA 0
  double* Cv0 = scr_of(0) + TR_OFF_CV;
  int* flag0 = reinterpret_cast<int*>(scr_of(0) + TR_OFF_FLAG);
  T* stage = reinterpret_cast<T*>(scr + TR_OFF_STAGE);
  for (int64_t o = cid; o < count; o += ncl) {
    const OpTrunc op = ops[o];
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
      // 1. partial R factors of this CTA's rows
      qr_stream<T>([&](int r, int c) { return cat_value(B, op, cat, 0, mu0 + r, c); }, mu1 - mu0, K, Pu, sC, sh);
      qr_stream<T>([&](int r, int c) { return cat_value(B, op, cat, 1, nv0 + r, c); }, nv1 - nv0, K, Pv, sC, sh);
      __threadfence();
      cluster.sync();
      // 2. CTA 0 combines the U partials into its J region, CTA 1 the V partials
      if (rk < 2) {
        const int64_t poff = rk == 0 ? 0 : TR_REG;
        T* fin = reinterpret_cast<T*>(J);
        qr_stream<T>(
            [&](int r, int c) {
              const T* P = reinterpret_cast<const T*>(scr_of(r / K) + poff);
              const int i = r % K;
              return i <= c ? (double)P[i + (int64_t)c * TR_KT] : 0.0;
            },
            TR_CL * K, K, fin, sC, sh);
      }
      __threadfence();
      cluster.sync();
      // 3. CTA 0: core from R_u (own J) and R_v (CTA 1's J)
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
        tr_core<T>(Ru, Rv, K, op.eps, op.kcap, M, W, J, X, Cu0, Cv0, cs, B.status);
        if (threadIdx.x == 0) flag0[0] = cs.k;
      }
      __threadfence();
      cluster.sync();
      const int k = reinterpret_cast<const volatile int*>(flag0)[0];
      if (B.flops && threadIdx.x == 0 && rk == 0)
        atomicAdd(B.flops + OP_TRUNC_BIG,
                  2.0 * K * K * (double)(op.m + op.n) + 2.0 * K * (double)k * (op.m + op.n));
      // 4. all CTAs apply to their rows
      tr_apply<T>(B, op, cat, 0, mu0, mu1, K, k, Cu0, stage);
      tr_apply<T>(B, op, cat, 1, nv0, nv1, K, k, Cv0, stage);
      kacc = k;
      __threadfence();
      cluster.sync();
    }
    if (threadIdx.x == 0 && rk == 0) B.ranks[op.slot] = kacc;
    __threadfence();
    cluster.sync();
  }
}

static size_t smem_bytes(bool f32) {
  return f32 ? (size_t)TrCh<float>::value * TR_KT * sizeof(float) : (size_t)TrCh<double>::value * TR_KT * sizeof(double);
}

int configure_trunc() {
  int bad = 0;
  bad |= cudaFuncSetAttribute(k_trunc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(false)) !=
         cudaSuccess;
  bad |= cudaFuncSetAttribute(k_trunc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(true)) !=
         cudaSuccess;
  bad |= cudaFuncSetAttribute(k_trunc_cl<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes(false)) != cudaSuccess;
  bad |= cudaFuncSetAttribute(k_trunc_cl<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem_bytes(true)) != cudaSuccess;
  return bad ? -1 : 0;
}

void launch_trunc(const OpTrunc* ops, int64_t count, const TermD* terms, const Bases& B, bool big,
                  cudaStream_t st) {
  if (count <= 0) return;
  const int cap = max_trunc_ctas();
  if (!big) {
    const int grid = (int)(count < cap ? count : cap);
    if (B.mixed)
      k_trunc<float><<<grid, TR_THREADS, smem_bytes(true), st>>>(ops, count, terms, B);
    else
      k_trunc<double><<<grid, TR_THREADS, smem_bytes(false), st>>>(ops, count, terms, B);
  } else {
    const int64_t ncl = count < cap / TR_CL ? count : cap / TR_CL;
    const int grid = (int)(ncl * TR_CL);
    if (B.mixed)
      k_trunc_cl<float><<<grid, TR_THREADS, smem_bytes(true), st>>>(ops, count, terms, B);
    else
      k_trunc_cl<double><<<grid, TR_THREADS, smem_bytes(false), st>>>(ops, count, terms, B);
  }
}

}  // namespace hlc
