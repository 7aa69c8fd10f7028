// kernels.cu -- sm_103a kernels of the H-matrix likelihood (FP64 path).
//
//   k_dense_asm   dense inadmissible leaves of C~ (eq. 3 + nugget, Sec. 4.1)
//   k_aca         ACA with partial pivoting for admissible leaves (App. B)
//   k_potrf       Cholesky of dense diagonal leaves (eq. 2)
//   k_trsm        triangular solves with dense diagonal leaves
//   k_gemm        strided multiply-add of dense views (H-arithmetic, Table 1)
//   k_trunc       truncated low-rank sums: QR of both factors, SVD of the
//                 core, keep sigma_i > eps sigma_1 (Remark A.1)
//   reductions    log det = 2 sum log L_ii, dot products (fixed order)
//
// Op kernels take a list of descriptors produced by the planner and loop
// over it grid-stride, one op per CTA at a time.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hlc_internal.h"
#include "kernels.h"
#include "matern.cuh"

namespace hlc {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dimv(const Dim& d, const int* ranks) {
  if (d.slot < 0) return d.n;
  const int r = ranks[d.slot];
  return r < d.n ? r : d.n;
}

__device__ __forceinline__ double* vptr(const Bases& B, const Mv& v) { return B.buf[v.buf] + v.off; }

__device__ void record_error(int* status, int code, int detail) {
  if (atomicCAS(status, 0, code) == 0) status[1] = detail;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; all threads get the result.  `red` needs 33 doubles.
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// Block-wide argmax of |value| with ties to the smaller index; returns the
// index (or -1 when every candidate is excluded) and the value in *best.
__device__ int block_argmax(double v, int idx, double* redv, int* redi, double* best) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) {
      v = ov;
      idx = oi;
    }
  }
  __syncthreads();
  if (lane == 0) {
    redv[w] = v;
    redi[w] = idx;
  }
  __syncthreads();
  if (w == 0) {
    v = lane < nw ? redv[lane] : -1.0;
    idx = lane < nw ? redi[lane] : -1;
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) {
        v = ov;
        idx = oi;
      }
    }
    if (lane == 0) {
      redv[32] = v;
      redi[32] = idx;
    }
  }
  __syncthreads();
  *best = redv[32];
  return redi[32];
}

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
__global__ void __launch_bounds__(ACA_THREADS) k_aca(const LrAsm* blks, int64_t count, double* arena,
                                                      const double* px, const double* py, MaternDev mp,
                                                      double eps, int* ranks) {
  __shared__ double s_ui[64], s_vj[64];
  __shared__ double s_cu[64][8], s_cv[64][8];
  __shared__ int used_r[128], used_c[64];
  __shared__ double redv[33];
  __shared__ int redi[33];
  const int tid = threadIdx.x;
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) {
    const LrAsm b = blks[o];
    const int m = b.m, n = b.n, kcap = b.kcap;
    double* U = arena + b.offU;
    double* V = arena + b.offV;
    int k = 0, next = 0, zero_tries = 0, nur = 0, nuc = 0;
    double s2 = 0.0;
    while (k < kcap && nur < 128) {
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
        double v = matern_f64(dist_f64(xi, yi, px[b.c0 + j], py[b.c0 + j]), mp);
        for (int l = 0; l < k; ++l) v -= s_ui[l] * V[j + (int64_t)l * n];
        V[j + (int64_t)k * n] = v;
        bool used = false;
        for (int q = 0; q < nuc; ++q) used |= (used_c[q] == j);
        const double a = fabs(v);
        if (!used && (a > best || (a == best && (bj < 0 || j < bj)))) {
          best = a;
          bj = j;
        }
      }
      double bval;
      const int jp = block_argmax(best, bj, redv, redi, &bval);
      if (jp < 0) break;
      if (bval == 0.0) {
        if (++zero_tries > 3) break;
        // first unused row
        int nx = -1;
        for (int t = 0; t < m && nx < 0; ++t) {
          bool u = false;
          for (int q = 0; q < nur; ++q) u |= (used_r[q] == t);
          if (!u) nx = t;
        }
        if (nx < 0) break;
        next = nx;
        continue;
      }
      zero_tries = 0;
      __syncthreads();
      const double piv = V[jp + (int64_t)k * n];
      __syncthreads();
      for (int j = tid; j < n; j += blockDim.x) V[j + (int64_t)k * n] /= piv;
      if (tid < k) s_vj[tid] = V[jp + (int64_t)tid * n];
      if (tid == 0) used_c[nuc] = jp;
      __syncthreads();
      ++nuc;
      // residual column jp into U[:, k]
      const double xj = px[b.c0 + jp], yj = py[b.c0 + jp];
      for (int t = tid; t < m; t += blockDim.x) {
        double u = matern_f64(dist_f64(px[b.r0 + t], py[b.r0 + t], xj, yj), mp);
        for (int l = 0; l < k; ++l) u -= U[t + (int64_t)l * m] * s_vj[l];
        U[t + (int64_t)k * m] = u;
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
      if (sqrt(uu) * sqrt(vv) <= eps * sqrt(fmax(s2, 0.0))) break;
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
      if (ip < 0) break;
      next = ip;
    }
    __syncthreads();
    if (tid == 0) ranks[b.slot] = k;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// POTRF: dense lower Cholesky of a diagonal leaf (n <= 128), right-looking.
// ---------------------------------------------------------------------------
__global__ void k_potrf(const OpPotrf* ops, int64_t count, Bases B) {
  extern __shared__ double sm[];
  __shared__ double dg[128];
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) {
    const OpPotrf op = ops[o];
    const int n = op.n;
    double* A = vptr(B, op.A);
    const int64_t ld = op.A.cs;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e % n, j = e / n;
      sm[e] = A[i + j * ld];
    }
    __syncthreads();
    // diagonal before this block's elimination (pivot tolerance reference)
    for (int j = threadIdx.x; j < n; j += blockDim.x) dg[j] = sm[j + j * n];
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      if (threadIdx.x == 0) {
        double d = sm[j + j * n];
        // a pivot at rounding level (<= 64 u of its starting diagonal) is
        // the non-positive pivot of an exactly singular block
        if (!(d > 64.0 * 1.1102230246251565e-16 * dg[j])) {
          record_error(B.status, DEV_NOT_SPD, op.row0 + j);
          d = nan("");
        }
        sm[j + j * n] = sqrt(d);
      }
      __syncthreads();
      const double dj = sm[j + j * n];
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) sm[i + j * n] /= dj;
      __syncthreads();
      const int cnt = n - j - 1;
      for (int e = threadIdx.x; e < cnt * cnt; e += blockDim.x) {
        const int ii = e % cnt, ll = e / cnt;
        if (ii >= ll) {
          const int i = j + 1 + ii, l = j + 1 + ll;
          sm[i + l * n] -= sm[i + j * n] * sm[l + j * n];
        }
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e % n, j = e / n;
      if (i >= j) A[i + j * ld] = sm[e];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// TRSM: X (n x c) := L^-1 X or L^-T X, L dense lower n x n (n <= 128).
// One warp per column of X; lane i holds rows i, i+32, i+64, i+96.
// ---------------------------------------------------------------------------
__global__ void k_trsm(const OpTrsm* ops, int64_t count, Bases B) {
  extern __shared__ double sL[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) {
    const OpTrsm op = ops[o];
    const int n = op.n;
    const int c = dimv(op.c, B.ranks);
    const double* L = vptr(B, op.L);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e % n, j = e / n;
      sL[e] = L[i * op.L.rs + j * op.L.cs];
    }
    __syncthreads();
    double* X = vptr(B, op.X);
    for (int col = w; col < c; col += nw) {
      double* xc = X + col * op.X.cs;
      double x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = lane + 32 * q;
        x[q] = r < n ? xc[r * op.X.rs] : 0.0;
      }
      if (!op.trans) {
        for (int i = 0; i < n; ++i) {
          const int owner = i & 31, qi = i >> 5;
          double mine = qi == 0 ? x[0] : qi == 1 ? x[1] : qi == 2 ? x[2] : x[3];
          if (lane == owner) mine /= sL[i + i * n];
          const double xi = __shfl_sync(0xffffffffu, mine, owner);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int r = lane + 32 * q;
            if (r == i) x[q] = xi;
            else if (r > i && r < n) x[q] -= sL[r + i * n] * xi;
          }
        }
      } else {
        for (int i = n - 1; i >= 0; --i) {
          const int owner = i & 31, qi = i >> 5;
          double mine = qi == 0 ? x[0] : qi == 1 ? x[1] : qi == 2 ? x[2] : x[3];
          if (lane == owner) mine /= sL[i + i * n];
          const double xi = __shfl_sync(0xffffffffu, mine, owner);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int r = lane + 32 * q;
            if (r == i) x[q] = xi;
            else if (r < i) x[q] -= sL[i + r * n] * xi;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = lane + 32 * q;
        if (r < n) xc[r * op.X.rs] = x[q];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// GEMM: Y = beta Y + alpha A B on strided views, 64 x 32 output tiles,
// 16 x 16 threads with 4 x 2 outputs each.
// ---------------------------------------------------------------------------
constexpr int GB_M = 64, GB_N = 32, GB_K = 16;

__global__ void __launch_bounds__(256) k_gemm(const OpGemm* ops, int64_t count, Bases B) {
  __shared__ double As[GB_K][GB_M + 1];
  __shared__ double Bs[GB_K][GB_N + 1];
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) {
    const OpGemm op = ops[o];
    const int m = dimv(op.m, B.ranks), k = dimv(op.k, B.ranks), c = dimv(op.c, B.ranks);
    if (m <= 0 || c <= 0) continue;
    double* Y = vptr(B, op.Y);
    const double* A = vptr(B, op.A);
    if (op.B.buf < 0) {  // Y = beta Y + alpha A
      for (int64_t e = tid; e < (int64_t)m * c; e += blockDim.x) {
        const int64_t i = e % m, j = e / m;
        double* y = Y + i * op.Y.rs + j * op.Y.cs;
        const double a = op.alpha * A[i * op.A.rs + j * op.A.cs];
        *y = op.beta ? *y + a : a;
      }
      continue;
    }
    const double* Bm = vptr(B, op.B);
    for (int ti = 0; ti < m; ti += GB_M) {
      for (int tj = 0; tj < c; tj += GB_N) {
        double acc[4][2];
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = 0.0;
        for (int kk = 0; kk < k; kk += GB_K) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int e = tid + q * 256;
            const int kq = e / GB_M, iq = e % GB_M;
            const int gi = ti + iq, gk = kk + kq;
            As[kq][iq] = (gi < m && gk < k) ? A[(int64_t)gi * op.A.rs + (int64_t)gk * op.A.cs] : 0.0;
          }
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int e = tid + q * 256;
            const int kq = e / GB_N, jq = e % GB_N;
            const int gj = tj + jq, gk = kk + kq;
            Bs[kq][jq] = (gj < c && gk < k) ? Bm[(int64_t)gk * op.B.rs + (int64_t)gj * op.B.cs] : 0.0;
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < GB_K; ++q) {
            double a[4], b[2];
#pragma unroll
            for (int x = 0; x < 4; ++x) a[x] = As[q][tr * 4 + x];
            b[0] = Bs[q][tc * 2];
            b[1] = Bs[q][tc * 2 + 1];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
              acc[x][0] += a[x] * b[0];
              acc[x][1] += a[x] * b[1];
            }
          }
          __syncthreads();
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 2; ++y) {
            const int gi = ti + tr * 4 + x, gj = tj + tc * 2 + y;
            if (gi < m && gj < c) {
              double* yp = Y + (int64_t)gi * op.Y.rs + (int64_t)gj * op.Y.cs;
              const double v = op.alpha * acc[x][y];
              *yp = op.beta ? *yp + v : v;
            }
          }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// TRUNC: target := trunc(target + sum of terms) (Remark A.1), in batches of
// at most TR_KB new columns: acc := trunc(acc + batch).
//
// For K = rank(acc) + batch columns with concatenated factors Ucat (m x K),
// Vcat (n x K):
//   1. R_u, R_v: R factors of Ucat and Vcat by Householder QR streamed over
//      row chunks of TR_CH rows ([R; chunk] -> R), Q never formed;
//   2. M = R_u R_v^T (K x K), one-sided Jacobi: M J = W, sigma_j = |W_j|;
//   3. keep sigma_j > eps sigma_max (sorted), k columns;
//   4. U_new = Ucat R_v^T J_k S_k^-1/2,  V_new = Vcat R_u^T W_k S_k^-3/2,
//      so that U_new V_new^T = Q_u X_k S_k Y_k^T Q_v^T (the truncated SVD)
//      and both factors carry S_k^1/2.
// ---------------------------------------------------------------------------
constexpr int TR_KB = 64;
constexpr int TR_KT = 192;  // rank capacity (<= 64) + one batch (<= 64 columns, or one dense term <= 128)
constexpr int TR_CH = 64;
constexpr int TR_THREADS = 256;
constexpr int TR_OUT_LD = 65;
constexpr int64_t TR_SCRATCH = 4LL * TR_KT * TR_KT + 2LL * TR_KT * 64 + 4LL * TR_KT;

size_t trunc_smem_bytes() {
  const size_t a = (size_t)TR_CH * TR_KT, b = (size_t)TR_THREADS * TR_OUT_LD;
  return (a > b ? a : b) * sizeof(double);
}
int64_t trunc_scratch_doubles() { return TR_SCRATCH; }

struct TrCat {
  // column map of the current concatenation
  int kacc;           // leading columns from the target itself
  int nt;             // terms in the batch
  const TermD* terms; // batch terms
  int col0[65];       // first concatenated column of each batch term (col0[nt] = K)
};

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

// R factor (K x K, ld TR_KT) of the M x K concatenation of one side.
__device__ void tr_qr(const Bases& B, const OpTrunc& op, const TrCat& cat, int side, int M, int K, double* R,
                      double* sC, double* sTau) {
  const int tid = threadIdx.x;
  for (int e = tid; e < K * K; e += blockDim.x) R[(e % K) + (int64_t)(e / K) * TR_KT] = 0.0;
  __syncthreads();
  for (int r0 = 0; r0 < M; r0 += TR_CH) {
    const int rows = min(TR_CH, M - r0);
    for (int e = tid; e < rows * K; e += blockDim.x) {
      const int i = e % rows, c = e / rows;
      sC[i + c * TR_CH] = cat_value(B, op, cat, side, r0 + i, c);
    }
    __syncthreads();
    for (int j = 0; j < K; ++j) {
      if (tid == 0) {
        const double alpha = R[j + (int64_t)j * TR_KT];
        double xn = 0.0;
        for (int i = 0; i < rows; ++i) xn += sC[i + j * TR_CH] * sC[i + j * TR_CH];
        double tau = 0.0;
        if (xn > 0.0) {
          const double beta = -copysign(sqrt(alpha * alpha + xn), alpha);
          tau = (beta - alpha) / beta;
          const double sc = 1.0 / (alpha - beta);
          for (int i = 0; i < rows; ++i) sC[i + j * TR_CH] *= sc;
          R[j + (int64_t)j * TR_KT] = beta;
        }
        sTau[0] = tau;
      }
      __syncthreads();
      const double tau = sTau[0];
      if (tau != 0.0) {
        for (int l = j + 1 + tid; l < K; l += blockDim.x) {
          double w = R[j + (int64_t)l * TR_KT];
          for (int i = 0; i < rows; ++i) w += sC[i + j * TR_CH] * sC[i + l * TR_CH];
          w *= tau;
          R[j + (int64_t)l * TR_KT] -= w;
          for (int i = 0; i < rows; ++i) sC[i + l * TR_CH] -= w * sC[i + j * TR_CH];
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(TR_THREADS) k_trunc(const OpTrunc* ops, int64_t count, const TermD* terms,
                                                       Bases B) {
  extern __shared__ double sm[];
  __shared__ TrCat cat;
  __shared__ double sTau[2];
  __shared__ double red[33];
  __shared__ int s_rot, s_k, s_order[TR_KT];
  __shared__ double s_sv[TR_KT];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  double* scr = B.scratch + (int64_t)blockIdx.x * TR_SCRATCH;
  double* Ru = scr;
  double* Rv = Ru + TR_KT * TR_KT;
  double* M = Rv + TR_KT * TR_KT;
  double* J = M + TR_KT * TR_KT;
  double* Cu = J + TR_KT * TR_KT;
  double* Cv = Cu + TR_KT * 64;
  for (int64_t o = blockIdx.x; o < count; o += gridDim.x) {
    const OpTrunc op = ops[o];
    const TermD* tl = terms + op.term0;
    int kacc = op.keep ? B.ranks[op.slot] : 0;
    int t0 = 0;
    bool first = true;
    while (first || t0 < op.nterms) {
      first = false;
      // batch [t0, t1)
      int t1 = t0, kb = 0;
      while (t1 < op.nterms) {
        const int kt = (tl[t1].flags & 1) ? tl[t1].urows : (tl[t1].flags & 2) ? tl[t1].vrows
                                                                              : dimv(tl[t1].k, B.ranks);
        if (kb != 0 && kb + kt > TR_KB) break;
        if (t1 - t0 >= 64) break;
        kb += kt;
        ++t1;
      }
      const int K = kacc + kb;
      __syncthreads();
      if (tid == 0) {
        cat.kacc = kacc;
        cat.nt = t1 - t0;
        cat.terms = tl + t0;
        int c = kacc;
        for (int t = t0; t < t1; ++t) {
          cat.col0[t - t0] = c;
          c += (tl[t].flags & 1) ? tl[t].urows : (tl[t].flags & 2) ? tl[t].vrows : dimv(tl[t].k, B.ranks);
        }
        cat.col0[t1 - t0] = c;
      }
      __syncthreads();
      t0 = t1;
      if (K == 0) {
        kacc = 0;
        continue;
      }
      if (K > TR_KT) {
        if (tid == 0) record_error(B.status, DEV_RANK, K);
        kacc = 0;
        break;
      }
      tr_qr(B, op, cat, 0, op.m, K, Ru, sm, sTau);
      tr_qr(B, op, cat, 1, op.n, K, Rv, sm, sTau);
      // M = Ru Rv^T ; J = I
      for (int e = tid; e < K * K; e += blockDim.x) {
        const int i = e % K, j = e / K;
        double s = 0.0;
        for (int c = max(i, j); c < K; ++c) s += Ru[i + (int64_t)c * TR_KT] * Rv[j + (int64_t)c * TR_KT];
        M[i + (int64_t)j * TR_KT] = s;
        J[i + (int64_t)j * TR_KT] = (i == j) ? 1.0 : 0.0;
      }
      __syncthreads();
      // one-sided Jacobi, round-robin pairs
      double fro2 = 0.0;
      for (int e = tid; e < K * K; e += blockDim.x) {
        const double v = M[(e % K) + (int64_t)(e / K) * TR_KT];
        fro2 += v * v;
      }
      fro2 = block_sum(fro2, red);
      const double tiny = 1e-34 * fro2;
      const int Kp = K + (K & 1);
      for (int sweep = 0; sweep < 80; ++sweep) {
        if (tid == 0) s_rot = 0;
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
            if (b >= K) continue;
            double al = 0.0, be = 0.0, ga = 0.0;
            for (int r = lane; r < K; r += 32) {
              const double x = M[r + (int64_t)a * TR_KT], y = M[r + (int64_t)b * TR_KT];
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
            const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
            for (int r = lane; r < K; r += 32) {
              const double x = M[r + (int64_t)a * TR_KT], y = M[r + (int64_t)b * TR_KT];
              M[r + (int64_t)a * TR_KT] = cs * x - sn * y;
              M[r + (int64_t)b * TR_KT] = sn * x + cs * y;
              const double jx = J[r + (int64_t)a * TR_KT], jy = J[r + (int64_t)b * TR_KT];
              J[r + (int64_t)a * TR_KT] = cs * jx - sn * jy;
              J[r + (int64_t)b * TR_KT] = sn * jx + cs * jy;
            }
            if (lane == 0) s_rot = 1;
          }
          __syncthreads();
        }
        if (!s_rot) break;
        __syncthreads();
      }
      // singular values, order (ties: smaller index first), truncation rank
      for (int j = tid; j < K; j += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < K; ++r) s += M[r + (int64_t)j * TR_KT] * M[r + (int64_t)j * TR_KT];
        s_sv[j] = sqrt(s);
      }
      __syncthreads();
      for (int j = tid; j < K; j += blockDim.x) {
        int rank = 0;
        for (int i = 0; i < K; ++i) rank += (s_sv[i] > s_sv[j]) || (s_sv[i] == s_sv[j] && i < j);
        s_order[rank] = j;
      }
      __syncthreads();
      if (tid == 0) {
        const double smax = s_sv[s_order[0]];
        int k = 0;
        if (smax > 0.0)
          while (k < K && s_sv[s_order[k]] > op.eps * smax) ++k;
        if (!(smax == smax)) {
          record_error(B.status, DEV_BAD, 1);
          k = 0;
        }
        if (k > op.kcap) {
          record_error(B.status, DEV_RANK, k);
          k = op.kcap;
        }
        s_k = k;
      }
      __syncthreads();
      const int k = s_k;
      // coefficients
      for (int e = tid; e < K * k; e += blockDim.x) {
        const int col = e % K, c = e / K;
        const int j = s_order[c];
        const double sv = s_sv[j], isq = 1.0 / sqrt(sv);
        double a = 0.0, b = 0.0;
        for (int p = 0; p <= col; ++p) {
          a += Rv[p + (int64_t)col * TR_KT] * J[p + (int64_t)j * TR_KT];
          b += Ru[p + (int64_t)col * TR_KT] * M[p + (int64_t)j * TR_KT];
        }
        Cu[col + (int64_t)c * TR_KT] = a * isq;
        Cv[col + (int64_t)c * TR_KT] = b * isq / sv;
      }
      __syncthreads();
      // apply, row-local and in place
      for (int side = 0; side < 2; ++side) {
        const int rows = side == 0 ? op.m : op.n;
        const double* C = side == 0 ? Cu : Cv;
        double* out = side == 0 ? B.buf[op.U.buf] + op.U.off : B.buf[op.V.buf] + op.V.off;
        double* so = sm + tid * TR_OUT_LD;
        for (int r0 = 0; r0 < rows; r0 += blockDim.x) {
          const int r = r0 + tid;
          if (r < rows) {
            for (int c = 0; c < k; ++c) so[c] = 0.0;
            for (int col = 0; col < K; ++col) {
              const double v = cat_value(B, op, cat, side, r, col);
              if (v != 0.0)
                for (int c = 0; c < k; ++c) so[c] += v * C[col + (int64_t)c * TR_KT];
            }
          }
          __syncthreads();
          if (r < rows)
            for (int c = 0; c < k; ++c) out[r + (int64_t)c * rows] = so[c];
          __syncthreads();
        }
      }
      kacc = k;
      __syncthreads();
    }
    if (tid == 0) B.ranks[op.slot] = kacc;
    __syncthreads();
  }
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
                const MaternDev& mp, double eps, int* ranks, cudaStream_t st) {
  if (count <= 0) return;
  k_aca<<<grid_for(count, 152 * 8), ACA_THREADS, 0, st>>>(d, count, arena, px, py, mp, eps, ranks);
}

int max_trunc_ctas() { return 152 * 2; }

void launch_ops(int type, const void* ops, int64_t count, const TermD* terms, const Bases& B, int max_dense,
                cudaStream_t st) {
  if (count <= 0) return;
  switch (type) {
    case OP_POTRF:
      k_potrf<<<grid_for(count, 152 * 8), 128, (size_t)max_dense * max_dense * sizeof(double), st>>>(
          (const OpPotrf*)ops, count, B);
      break;
    case OP_TRSM:
      k_trsm<<<grid_for(count, 152 * 8), 256, (size_t)max_dense * max_dense * sizeof(double), st>>>(
          (const OpTrsm*)ops, count, B);
      break;
    case OP_GEMM:
      k_gemm<<<grid_for(count, 152 * 16), 256, 0, st>>>((const OpGemm*)ops, count, B);
      break;
    case OP_TRUNC:
      k_trunc<<<grid_for(count, max_trunc_ctas()), TR_THREADS, trunc_smem_bytes(), st>>>((const OpTrunc*)ops,
                                                                                         count, terms, B);
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
  cudaError_t e2 = cudaFuncSetAttribute(k_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
  cudaError_t e3 =
      cudaFuncSetAttribute(k_trunc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trunc_smem_bytes());
  return (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess) ? 0 : -1;
}

}  // namespace hlc
