// ops.cuh -- device bodies of the primitive ops of a plan (POTRF, TRSM,
// GEMM/GEMV), each run by one whole CTA; shared by the per-type kernels, the
// persistent solve kernels and the dependency-driven factorisation kernel.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "devutil.cuh"
#include "hlc_internal.h"

namespace hlc {

// loads staged through registers per thread before their stores to shared
// memory (independent loads in flight)
constexpr int LD_BATCH = 16;

// ---------------------------------------------------------------------------
// POTRF: dense lower Cholesky of a diagonal leaf (n <= 128), right-looking.
// ---------------------------------------------------------------------------
// One POTRF op by the whole CTA; sm: n x n doubles of shared memory.
inline __device__ void do_potrf(const OpPotrf& op, const Bases& B, double* sm) {
  __shared__ double dg[128];
  const int n = op.n;
  if (B.flops && threadIdx.x == 0) atomicAdd(B.flops + OP_POTRF, (double)n * n * n / 3.0);
  double* A = vptr(B, op.A);
  const int64_t ld = op.A.cs;
  for (int e0 = threadIdx.x; e0 < n * n; e0 += LD_BATCH * blockDim.x) {
    double v[LD_BATCH];
#pragma unroll
    for (int u = 0; u < LD_BATCH; ++u) {
      const int e = e0 + u * blockDim.x;
      v[u] = e < n * n ? A[(e % n) + (e / n) * ld] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < LD_BATCH; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < n * n) sm[e] = v[u];
    }
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

// ---------------------------------------------------------------------------
// TRSM: X (n x c) := L^-1 X or L^-T X, L dense lower n x n (n <= 128), in
// arithmetic type T (FP32 in the mixed modes: the solves are panel operations
// and preconditioner applications there; FP64 otherwise).
// One warp per column of X; lane i holds rows i, i+32, i+64, i+96.  The
// reciprocals of the diagonal are formed once, in parallel, so that the
// sequential substitution chain multiplies instead of dividing.
// sL: n * n + n entries of T.
// ---------------------------------------------------------------------------
// The block L and the reciprocals of its diagonal into shared memory (does
// not touch X: in a solve, where L is final, it may run before X is).
template <class T>
__device__ void trsm_load(const OpTrsm& op, const Bases& B, T* sL) {
  const int n = op.n;
  const double* L = vptr(B, op.L);
  T* sInv = sL + n * n;
  // the block through registers, LD_BATCH loads in flight per thread
  for (int e0 = threadIdx.x; e0 < n * n; e0 += LD_BATCH * blockDim.x) {
    T v[LD_BATCH];
#pragma unroll
    for (int u = 0; u < LD_BATCH; ++u) {
      const int e = e0 + u * blockDim.x;
      v[u] = e < n * n ? (T)L[(e % n) * op.L.rs + (e / n) * op.L.cs] : T(0);
    }
#pragma unroll
    for (int u = 0; u < LD_BATCH; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < n * n) sL[e] = v[u];
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) sInv[i] = T(1) / (T)L[i * op.L.rs + i * op.L.cs];
  __syncthreads();
}

// The substitution (or product) against X with L already in shared memory.
template <class T>
__device__ void trsm_apply(const OpTrsm& op, const Bases& B, const T* sL) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int n = op.n;
  const int c = dimv(op.c, B.ranks);
  if (B.flops && threadIdx.x == 0) atomicAdd(B.flops + OP_TRSM, (double)n * n * c);
  const T* sInv = sL + n * n;
  double* X = vptr(B, op.X);
  for (int col = w; col < c; col += nw) {
    double* xc = X + col * op.X.cs;
    T x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = lane + 32 * q;
      x[q] = r < n ? (T)xc[r * op.X.rs] : T(0);
    }
    if (op.trans >= 2) {
      // multiplication by the lower triangle (trans 2) or its transpose
      // (trans 3): y_r = sum_{i <= r} L_ri x_i, resp. sum_{i >= r} L_ir x_i,
      // accumulated in a fixed order (increasing i)
      T acc[4] = {T(0), T(0), T(0), T(0)};
      for (int i = 0; i < n; ++i) {
        const int owner = i & 31, qi = i >> 5;
        const T mine = qi == 0 ? x[0] : qi == 1 ? x[1] : qi == 2 ? x[2] : x[3];
        const T xi = __shfl_sync(0xffffffffu, mine, owner);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = lane + 32 * q;
          if (r < n) {
            if (op.trans == 2 && r >= i) acc[q] += sL[r + i * n] * xi;
            if (op.trans == 3 && r <= i) acc[q] += sL[i + r * n] * xi;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = acc[q];
    } else if (!op.trans) {
      for (int i = 0; i < n; ++i) {
        const int owner = i & 31, qi = i >> 5;
        T mine = qi == 0 ? x[0] : qi == 1 ? x[1] : qi == 2 ? x[2] : x[3];
        if (lane == owner) mine *= sInv[i];
        const T xi = __shfl_sync(0xffffffffu, mine, owner);
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
        T mine = qi == 0 ? x[0] : qi == 1 ? x[1] : qi == 2 ? x[2] : x[3];
        if (lane == owner) mine *= sInv[i];
        const T xi = __shfl_sync(0xffffffffu, mine, owner);
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
      if (r < n) xc[r * op.X.rs] = (double)x[q];
    }
  }
  __syncthreads();
}

template <class T>
__device__ void do_trsm(const OpTrsm& op, const Bases& B, T* sL) {
  trsm_load<T>(op, B, sL);
  trsm_apply<T>(op, B, sL);
}



// ---------------------------------------------------------------------------
// GEMM: Y = beta Y + alpha A B on strided views, 64 x 32 output tiles,
// 16 x 16 threads with 4 x 2 outputs each.
// ---------------------------------------------------------------------------
constexpr int GB_M = 64, GB_N = 32, GB_K = 16;

template <class T>
struct GemmSmem {
  T As[GB_K][GB_M + 1];
  T Bs[GB_K][GB_N + 1];
};

// Y (m x 1) = beta Y + alpha A x, in a fixed summation order.  Where the
// rows of A are contiguous, a warp per row (lanes stride along the row).
// Otherwise (column-major A) a thread per (row, part): the CTA takes R rows
// at a time (R = m rounded up to a warp, at most the CTA) and splits the
// inner dimension into P = blockDim / R interleaved parts; every thread
// issues GV_UNROLL independent loads before it uses them, so that a product
// over a block in HBM waits for a few memory latencies instead of one per
// column.  With P > 1 the parts are added in part order through shared
// memory.
constexpr int GV_UNROLL = 8;

template <class T>
__device__ void do_gemv(const OpGemm& op, const Bases& B, int m, int k, double* Y, const double* A) {
  __shared__ T gv_red[256];
  const bool ones = op.B.buf == MV_ONES;
  const double* x = ones ? nullptr : vptr(B, op.B);
  const int64_t xs = op.B.rs;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  if (op.A.cs == 1 && op.A.rs != 1) {
    for (int i = w; i < m; i += nw) {
      const double* a = A + (int64_t)i * op.A.rs;
      T acc = T(0);
      if (ones)
        for (int q = lane; q < k; q += 32) acc += (T)a[q];
      else
        for (int q = lane; q < k; q += 32) acc += (T)a[q] * (T)x[q * xs];
      acc = warp_sum(acc);
      if (lane == 0) {
        double* yp = Y + (int64_t)i * op.Y.rs;
        const double v = op.alpha * (double)acc;
        *yp = op.beta ? *yp + v : v;
      }
    }
    return;
  }
  const int nt = (int)blockDim.x;
  const int R = min(nt, (m + 31) & ~31);
  const int P = nt / R;
  const int r = tid % R, p = tid / R;
  for (int r0 = 0; r0 < m; r0 += R) {
    const int i = r0 + r;
    T acc = T(0);
    if (i < m && p < P) {
      const double* a = A + (int64_t)i * op.A.rs;
      for (int q0 = p; q0 < k; q0 += GV_UNROLL * P) {
        T av[GV_UNROLL], xv[GV_UNROLL];
#pragma unroll
        for (int u = 0; u < GV_UNROLL; ++u) {
          const int q = q0 + u * P;
          av[u] = q < k ? (T)a[(int64_t)q * op.A.cs] : T(0);
          xv[u] = q < k ? (ones ? T(1) : (T)x[(int64_t)q * xs]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < GV_UNROLL; ++u) acc += av[u] * xv[u];
      }
    }
    if (P > 1) {
      __syncthreads();
      if (p < P) gv_red[p * R + r] = acc;
      __syncthreads();
      if (p == 0 && i < m) {
        T s = T(0);
        for (int q = 0; q < P; ++q) s += gv_red[q * R + r];
        acc = s;
      }
    }
    if (p == 0 && i < m) {
      double* yp = Y + (int64_t)i * op.Y.rs;
      const double v = op.alpha * (double)acc;
      *yp = op.beta ? *yp + v : v;
    }
  }
  if (P > 1) __syncthreads();
}

// Prefetch for the dependency-driven solves: the A operand of a product
// with one column (a block of the factor or of C~, final while a solve or
// matvec runs) into shared memory as T, sA[i + q m], before the op's
// producers are done.  Returns whether it did (m k <= cap entries, A in a
// matrix arena); the CTA then runs do_gemv_pre after the wait, which adds
// in exactly do_gemv's order.
template <class T>
__device__ bool gemv_prefetch(const OpGemm& op, const Bases& B, T* sA, int64_t cap) {
  if (op.B.buf == MV_IDENTITY || (op.A.buf != BUF_L && op.A.buf != BUF_C)) return false;
  const int m = dimv(op.m, B.ranks), k = dimv(op.k, B.ranks), c = dimv(op.c, B.ranks);
  if (m <= 0 || k <= 0 || (c != 1 && op.B.buf != MV_ONES) || (int64_t)m * k > cap) return false;
  const double* A = vptr(B, op.A);
  const int n = m * k;
  for (int e0 = threadIdx.x; e0 < n; e0 += LD_BATCH * blockDim.x) {
    T v[LD_BATCH];
#pragma unroll
    for (int u = 0; u < LD_BATCH; ++u) {
      const int e = e0 + u * blockDim.x;
      v[u] = e < n ? (T)A[(int64_t)(e % m) * op.A.rs + (int64_t)(e / m) * op.A.cs] : T(0);
    }
#pragma unroll
    for (int u = 0; u < LD_BATCH; ++u) {
      const int e = e0 + u * blockDim.x;
      if (e < n) sA[e] = v[u];
    }
  }
  __syncthreads();
  return true;
}

// do_gemv with A prefetched (gemv_prefetch): the same threads add the same
// products in the same order.
template <class T>
__device__ void do_gemv_pre(const OpGemm& op, const Bases& B, const T* sA) {
  __shared__ T gp_red[256];
  const int m = dimv(op.m, B.ranks), k = dimv(op.k, B.ranks);
  if (B.flops && threadIdx.x == 0) atomicAdd(B.flops + OP_GEMM, 2.0 * m * (double)k);
  double* Y = vptr(B, op.Y);
  const bool ones = op.B.buf == MV_ONES;
  const double* x = ones ? nullptr : vptr(B, op.B);
  const int64_t xs = op.B.rs;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
  if (op.A.cs == 1 && op.A.rs != 1) {
    for (int i = w; i < m; i += nw) {
      T acc = T(0);
      if (ones)
        for (int q = lane; q < k; q += 32) acc += sA[i + q * m];
      else
        for (int q = lane; q < k; q += 32) acc += sA[i + q * m] * (T)x[q * xs];
      acc = warp_sum(acc);
      if (lane == 0) {
        double* yp = Y + (int64_t)i * op.Y.rs;
        const double v = op.alpha * (double)acc;
        *yp = op.beta ? *yp + v : v;
      }
    }
    __syncthreads();
    return;
  }
  const int nt = (int)blockDim.x;
  const int R = min(nt, (m + 31) & ~31);
  const int P = nt / R;
  const int r = tid % R, p = tid / R;
  for (int r0 = 0; r0 < m; r0 += R) {
    const int i = r0 + r;
    T acc = T(0);
    if (i < m && p < P) {
      for (int q0 = p; q0 < k; q0 += GV_UNROLL * P) {
        T av[GV_UNROLL], xv[GV_UNROLL];
#pragma unroll
        for (int u = 0; u < GV_UNROLL; ++u) {
          const int q = q0 + u * P;
          av[u] = q < k ? sA[i + q * m] : T(0);
          xv[u] = q < k ? (ones ? T(1) : (T)x[(int64_t)q * xs]) : T(0);
        }
#pragma unroll
        for (int u = 0; u < GV_UNROLL; ++u) acc += av[u] * xv[u];
      }
    }
    if (P > 1) {
      __syncthreads();
      if (p < P) gp_red[p * R + r] = acc;
      __syncthreads();
      if (p == 0 && i < m) {
        T s = T(0);
        for (int q = 0; q < P; ++q) s += gp_red[q * R + r];
        acc = s;
      }
    }
    if (p == 0 && i < m) {
      double* yp = Y + (int64_t)i * op.Y.rs;
      const double v = op.alpha * (double)acc;
      *yp = op.beta ? *yp + v : v;
    }
  }
  __syncthreads();
}

template <class T>
__device__ void do_gemm(const OpGemm& op, const Bases& B, GemmSmem<T>& sm) {
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  const int m = dimv(op.m, B.ranks), k = dimv(op.k, B.ranks), c = dimv(op.c, B.ranks);
  if (m <= 0 || c <= 0) return;
  if (B.flops && threadIdx.x == 0)
    atomicAdd(B.flops + OP_GEMM, op.B.buf == MV_IDENTITY ? (double)m * c : 2.0 * m * (double)k * c);
  double* Y = vptr(B, op.Y);
  const double* A = vptr(B, op.A);
  if (op.B.buf == MV_IDENTITY) {  // Y = beta Y + alpha A
    for (int64_t e = tid; e < (int64_t)m * c; e += blockDim.x) {
      const int64_t i = e % m, j = e / m;
      double* y = Y + i * op.Y.rs + j * op.Y.cs;
      const double a = op.alpha * A[i * op.A.rs + j * op.A.cs];
      *y = op.beta ? *y + a : a;
    }
    return;
  }
  if (c == 1 || op.B.buf == MV_ONES) {
    if (k > 0) do_gemv<T>(op, B, m, k, Y, A);
    return;
  }
  const double* Bm = vptr(B, op.B);
  for (int ti = 0; ti < m; ti += GB_M) {
    for (int tj = 0; tj < c; tj += GB_N) {
      T acc[4][2];
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a][0] = acc[a][1] = T(0);
      for (int kk = 0; kk < k; kk += GB_K) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int e = tid + q * 256;
          const int kq = e / GB_M, iq = e % GB_M;
          const int gi = ti + iq, gk = kk + kq;
          sm.As[kq][iq] = (gi < m && gk < k) ? (T)A[(int64_t)gi * op.A.rs + (int64_t)gk * op.A.cs] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int e = tid + q * 256;
          const int kq = e / GB_N, jq = e % GB_N;
          const int gj = tj + jq, gk = kk + kq;
          sm.Bs[kq][jq] = (gj < c && gk < k) ? (T)Bm[(int64_t)gk * op.B.rs + (int64_t)gj * op.B.cs] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GB_K; ++q) {
          T a[4], b[2];
#pragma unroll
          for (int x = 0; x < 4; ++x) a[x] = sm.As[q][tr * 4 + x];
          b[0] = sm.Bs[q][tc * 2];
          b[1] = sm.Bs[q][tc * 2 + 1];
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
            const double v = op.alpha * (double)acc[x][y];
            *yp = op.beta ? *yp + v : v;
          }
        }
    }
  }
}

// dynamic shared memory of a TRSM or POTRF on blocks of up to max_dense rows
// (the block and the inverted diagonal)
inline size_t trsm_smem(int max_dense) { return ((size_t)max_dense * max_dense + max_dense) * sizeof(double); }

}  // namespace hlc
