// tree.cu -- device build of the cluster tree and the block-cluster tree
// (Sec. 2.2, Def. 2.2, App. A):
//
//   1. global bounding box (reduction), Morton keys: each coordinate
//      quantised to 32 bits over the box, bits interleaved with x in the even
//      positions;
//   2. stable LSD radix sort of the 64-bit keys (8 passes of 8 bits), so that
//      equal keys keep the callers' index order;
//   3. bisection level by level: per cluster the tight bounding box (block
//      reduction) and its longest axis (x on ties); the geometric rule puts
//      the coordinates <= the axis midpoint to the left, the cardinality rule
//      the floor(size/2) smallest coordinates (ties in position order);
//      both partitions are stable; clusters of at most `leaf` points, or
//      whose split would leave a side empty, are leaves; children are
//      numbered breadth-first;
//   4. block-cluster tree level by level over the lower triangle: a diagonal
//      pair of a non-leaf splits into (1,1), (2,1), (2,2); an off-diagonal pair
//      is admissible (low-rank) under the chosen rule -- dist > 0 and
//      min(diam) <= eta dist of the tight boxes (standard), dist > 0 and
//      max(diam) <= eta dist, or always (weak) -- else dense when one side is
//      a leaf, else split into its four child pairs.
//
// The floating-point geometry uses explicitly rounded operations so that the
// tree is bit-identical to the host build of the same rules.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "devutil.cuh"
#include "hlc_internal.h"
#include "kernels.h"

namespace hlc {

// ---------------------------------------------------------------------------
// 1. bounding box and Morton keys
// ---------------------------------------------------------------------------
__global__ void k_bbox_part(const double* xy, int64_t n, double* part) {
  double mn0 = INFINITY, mn1 = INFINITY, mx0 = -INFINITY, mx1 = -INFINITY;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = xy[2 * i], y = xy[2 * i + 1];
    mn0 = fmin(mn0, x);
    mx0 = fmax(mx0, x);
    mn1 = fmin(mn1, y);
    mx1 = fmax(mx1, y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn0 = fmin(mn0, __shfl_xor_sync(0xffffffffu, mn0, o));
    mn1 = fmin(mn1, __shfl_xor_sync(0xffffffffu, mn1, o));
    mx0 = fmax(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
    mx1 = fmax(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
  }
  __shared__ double s[4][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    s[0][w] = mn0;
    s[1][w] = mn1;
    s[2][w] = mx0;
    s[3][w] = mx1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < nw; ++q) {
      s[0][0] = fmin(s[0][0], s[0][q]);
      s[1][0] = fmin(s[1][0], s[1][q]);
      s[2][0] = fmax(s[2][0], s[2][q]);
      s[3][0] = fmax(s[3][0], s[3][q]);
    }
    for (int q = 0; q < 4; ++q) part[4 * blockIdx.x + q] = s[q][0];
  }
}

__global__ void k_bbox_final(const double* part, int nb, double* bb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double r[4] = {INFINITY, INFINITY, -INFINITY, -INFINITY};
  for (int b = 0; b < nb; ++b) {
    r[0] = fmin(r[0], part[4 * b + 0]);
    r[1] = fmin(r[1], part[4 * b + 1]);
    r[2] = fmax(r[2], part[4 * b + 2]);
    r[3] = fmax(r[3], part[4 * b + 3]);
  }
  for (int q = 0; q < 4; ++q) bb[q] = r[q];
}

__device__ __forceinline__ uint32_t quantise_dev(double c, double lo, double hi) {
  const double range = __dsub_rn(hi, lo);
  if (!(range > 0.0)) return 0u;
  const double t = __dmul_rn(__ddiv_rn(__dsub_rn(c, lo), range), 4294967295.0);
  return (uint32_t)floor(t);
}

__device__ __forceinline__ uint64_t spread_bits(uint32_t v) {
  uint64_t x = v;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

__global__ void k_morton(const double* xy, int64_t n, const double* bb, uint64_t* key, int32_t* idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t qx = quantise_dev(xy[2 * i], bb[0], bb[2]);
    const uint32_t qy = quantise_dev(xy[2 * i + 1], bb[1], bb[3]);
    key[i] = spread_bits(qx) | (spread_bits(qy) << 1);
    idx[i] = (int32_t)i;
  }
}

// ---------------------------------------------------------------------------
// 2. stable LSD radix sort, 8-bit digits
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_TILE = 4096;  // elements per block

__global__ void k_rs_hist(const uint64_t* key, int64_t n, int shift, uint32_t* hist, int nb) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
  const int64_t t1 = t0 + RS_TILE < n ? t0 + RS_TILE : n;
  for (int64_t i = t0 + threadIdx.x; i < t1; i += blockDim.x) atomicAdd(&cnt[(key[i] >> shift) & 255u], 1u);
  __syncthreads();
  hist[(int64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// exclusive scan of `total` counts (single CTA of 1024 threads)
__global__ void k_rs_scan(uint32_t* a, int64_t total) {
  __shared__ uint32_t part[1024];
  const int64_t per = (total + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = threadIdx.x * per, b1 = b0 + per < total ? b0 + per : total;
  uint32_t s = 0;
  for (int64_t i = b0; i < b1; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int q = 0; q < (int)blockDim.x; ++q) {
      const uint32_t v = part[q];
      part[q] = run;
      run += v;
    }
  }
  __syncthreads();
  uint32_t run = part[threadIdx.x];
  for (int64_t i = b0; i < b1; ++i) {
    const uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
}

__global__ void k_rs_scatter(const uint64_t* kin, const int32_t* iin, uint64_t* kout, int32_t* iout, int64_t n,
                             int shift, const uint32_t* offs, int nb) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wc[RS_THREADS / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  base[tid] = offs[(int64_t)tid * nb + blockIdx.x];
  const int64_t t0 = (int64_t)blockIdx.x * RS_TILE;
  const int64_t t1 = t0 + RS_TILE < n ? t0 + RS_TILE : n;
  for (int64_t c0 = t0; c0 < t1; c0 += RS_THREADS) {
    for (int q = tid; q < (RS_THREADS / 32) * 256; q += RS_THREADS) (&wc[0][0])[q] = 0;
    __syncthreads();
    const int64_t i = c0 + tid;
    const bool valid = i < t1;
    uint64_t k = 0;
    int32_t id = 0;
    uint32_t d = 256 + lane;  // distinct dummy digits for idle lanes
    if (valid) {
      k = kin[i];
      id = iin[i];
      d = (uint32_t)((k >> shift) & 255u);
    }
    const uint32_t mask = __match_any_sync(0xffffffffu, d);
    const uint32_t lt = (1u << lane) - 1u;
    const int rank = __popc(mask & lt);
    if (valid && (mask & lt) == 0) wc[w][d] = __popc(mask);
    __syncthreads();
    if (valid) {
      uint32_t off = base[d];
      for (int q = 0; q < w; ++q) off += wc[q][d];
      kout[off + rank] = k;
      iout[off + rank] = id;
    }
    __syncthreads();
    uint32_t add = 0;
    for (int q = 0; q < RS_THREADS / 32; ++q) add += wc[q][tid];
    base[tid] += add;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// 3. bisection, one level per round
// ---------------------------------------------------------------------------
struct DevCluster {
  int64_t lo, hi;
  double bmin[2], bmax[2];
  int32_t child[2];
  int32_t level;
  int32_t pad;
};

constexpr int BS_THREADS = 256;

__device__ __forceinline__ double block_min(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = red[0];
    for (int q = 1; q < nw; ++q) r = fmin(r, red[q]);
    red[32] = r;
  }
  __syncthreads();
  return red[32];
}

// Monotone 64-bit key of a double: a < b iff key(a) < key(b) (finite values,
// -0 below +0).
__device__ __forceinline__ uint64_t order_key(double v) {
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// bbox, split decision and left count of every frontier cluster; for the
// cardinality rule also the key of the median coordinate (thr) and how many
// points with exactly that key go left (need)
__global__ void k_bis_measure(DevCluster* cl, const int32_t* front, const double* px, const double* py, int leaf,
                              int split_rule, int32_t* split, int64_t* nleft, int32_t* axis, double* mid,
                              uint64_t* thr, int64_t* need) {
  __shared__ double red[33];
  const int32_t c = front[blockIdx.x];
  DevCluster C = cl[c];
  double mn0 = INFINITY, mn1 = INFINITY, mx0 = -INFINITY, mx1 = -INFINITY;
  for (int64_t i = C.lo + threadIdx.x; i < C.hi; i += blockDim.x) {
    mn0 = fmin(mn0, px[i]);
    mx0 = fmax(mx0, px[i]);
    mn1 = fmin(mn1, py[i]);
    mx1 = fmax(mx1, py[i]);
  }
  mn0 = block_min(mn0, red);
  mn1 = block_min(mn1, red);
  mx0 = -block_min(-mx0, red);
  mx1 = -block_min(-mx1, red);
  const int64_t size = C.hi - C.lo;
  int ax = 0;
  double md = 0.0;
  if (size > leaf) {
    const double ex = __dsub_rn(mx0, mn0), ey = __dsub_rn(mx1, mn1);
    ax = ex >= ey ? 0 : 1;
    md = ax == 0 ? __dmul_rn(0.5, __dadd_rn(mn0, mx0)) : __dmul_rn(0.5, __dadd_rn(mn1, mx1));
  }
  double cntl = 0.0;
  uint64_t t_key = 0;
  int64_t t_need = 0;
  if (size > leaf && split_rule == HLC_SPLIT_GEOMETRIC) {
    const double* co = ax == 0 ? px : py;
    for (int64_t i = C.lo + threadIdx.x; i < C.hi; i += blockDim.x) cntl += (co[i] <= md) ? 1.0 : 0.0;
    cntl = block_sum(cntl, red);
  } else if (size > leaf) {
    // the k-th smallest key, k = floor(size / 2): the smallest t with
    // #{key <= t} >= k, found bit by bit from the top
    const double* co = ax == 0 ? px : py;
    const int64_t k = size / 2;
    uint64_t t = 0;
    for (int b = 63; b >= 0; --b) {
      const uint64_t cand = t | ((1ull << b) - 1);  // t with the lower bits set: is #{key <= cand} >= k ?
      double c = 0.0;
      for (int64_t i = C.lo + threadIdx.x; i < C.hi; i += blockDim.x) c += order_key(co[i]) <= cand ? 1.0 : 0.0;
      c = block_sum(c, red);
      if (!(c >= (double)k)) t |= (1ull << b);  // the k-th key has bit b set
    }
    double below = 0.0;
    for (int64_t i = C.lo + threadIdx.x; i < C.hi; i += blockDim.x) below += order_key(co[i]) < t ? 1.0 : 0.0;
    below = block_sum(below, red);
    t_key = t;
    t_need = k - (int64_t)below;
    cntl = (double)k;
  }
  if (threadIdx.x == 0) {
    C.bmin[0] = mn0;
    C.bmin[1] = mn1;
    C.bmax[0] = mx0;
    C.bmax[1] = mx1;
    cl[c].bmin[0] = mn0;
    cl[c].bmin[1] = mn1;
    cl[c].bmax[0] = mx0;
    cl[c].bmax[1] = mx1;
    const int64_t nl = (int64_t)cntl;
    const int sp = (size > leaf) && nl > 0 && nl < size;
    split[blockIdx.x] = sp;
    nleft[blockIdx.x] = nl;
    axis[blockIdx.x] = ax;
    mid[blockIdx.x] = md;
    thr[blockIdx.x] = t_key;
    need[blockIdx.x] = t_need;
  }
}

// exclusive scan of split flags -> first child id of every splitting cluster
__global__ void k_bis_scan(const int32_t* split, int nf, int32_t next_id, int32_t* child0, int32_t* nsplit) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int32_t run = 0;
  for (int i = 0; i < nf; ++i) {
    child0[i] = next_id + 2 * run;
    run += split[i];
  }
  *nsplit = run;
}

// stable partition of every splitting cluster (through tmp), children records
__global__ void k_bis_split(DevCluster* cl, const int32_t* front, const int32_t* split, const int64_t* nleft,
                            const int32_t* axis, const double* mid, const uint64_t* thr, const int64_t* need,
                            int split_rule, const int32_t* child0, double* px, double* py, int32_t* perm, double* tx,
                            double* ty, int32_t* tp, int32_t* next_front) {
  __shared__ int sc[BS_THREADS];
  __shared__ int64_t run_l, run_r, run_eq;
  if (!split[blockIdx.x]) return;
  const int32_t c = front[blockIdx.x];
  const DevCluster C = cl[c];
  const int64_t nl = nleft[blockIdx.x];
  const int ax = axis[blockIdx.x];
  const double md = mid[blockIdx.x];
  const uint64_t tk = thr[blockIdx.x];
  const int64_t nd = need[blockIdx.x];
  const double* co = ax == 0 ? px : py;
  if (threadIdx.x == 0) {
    run_l = 0;
    run_r = 0;
    run_eq = 0;
  }
  __syncthreads();
  for (int64_t c0 = C.lo; c0 < C.hi; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    int f;
    if (split_rule == HLC_SPLIT_GEOMETRIC) {
      f = (i < C.hi && co[i] <= md) ? 1 : 0;
    } else {
      // below the median key: left; equal to it: left while fewer than
      // `need` equal keys came before (position order); above: right
      const uint64_t key = i < C.hi ? order_key(co[i]) : ~0ull;
      const int eq = (i < C.hi && key == tk) ? 1 : 0;
      sc[threadIdx.x] = eq;
      __syncthreads();
      for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        const int v = threadIdx.x >= o ? sc[threadIdx.x - o] : 0;
        __syncthreads();
        sc[threadIdx.x] += v;
        __syncthreads();
      }
      const int64_t eq_before = run_eq + sc[threadIdx.x] - eq;
      const int eq_tot = sc[blockDim.x - 1];
      f = (i < C.hi && (key < tk || (eq && eq_before < nd))) ? 1 : 0;
      __syncthreads();
      if (threadIdx.x == 0) run_eq += eq_tot;
    }
    sc[threadIdx.x] = f;
    __syncthreads();
    // inclusive scan (Hillis-Steele) over the chunk
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
      const int v = threadIdx.x >= o ? sc[threadIdx.x - o] : 0;
      __syncthreads();
      sc[threadIdx.x] += v;
      __syncthreads();
    }
    const int incl = sc[threadIdx.x];
    const int tot = sc[blockDim.x - 1];
    if (i < C.hi) {
      const int64_t t = threadIdx.x;
      const int64_t excl = incl - f;
      const int64_t dst = f ? C.lo + run_l + excl : C.lo + nl + run_r + (t - excl);
      tx[dst] = px[i];
      ty[dst] = py[i];
      tp[dst] = perm[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int64_t chunk = (C.hi - c0) < (int64_t)blockDim.x ? (C.hi - c0) : (int64_t)blockDim.x;
      run_l += tot;
      run_r += chunk - tot;
    }
    __syncthreads();
  }
  for (int64_t i = C.lo + threadIdx.x; i < C.hi; i += blockDim.x) {
    px[i] = tx[i];
    py[i] = ty[i];
    perm[i] = tp[i];
  }
  if (threadIdx.x == 0) {
    const int32_t a = child0[blockIdx.x];
    DevCluster L{}, R{};
    L.lo = C.lo;
    L.hi = C.lo + nl;
    R.lo = C.lo + nl;
    R.hi = C.hi;
    L.level = R.level = C.level + 1;
    L.child[0] = L.child[1] = R.child[0] = R.child[1] = -1;
    cl[a] = L;
    cl[a + 1] = R;
    cl[c].child[0] = a;
    cl[c].child[1] = a + 1;
    // position in the next frontier = child id - first id of that level
    next_front[2 * ((a - child0[0]) / 2)] = a;
    next_front[2 * ((a - child0[0]) / 2) + 1] = a + 1;
  }
}

// ---------------------------------------------------------------------------
// 4. block-cluster tree, one level per round
// ---------------------------------------------------------------------------
struct DevBlock {
  int32_t r, s, type, diag;
  int32_t ch[4];
};

__device__ __forceinline__ double diam_dev(const DevCluster& c) {
  const double ex = __dsub_rn(c.bmax[0], c.bmin[0]), ey = __dsub_rn(c.bmax[1], c.bmin[1]);
  return __dsqrt_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)));
}

__device__ __forceinline__ double dist_dev(const DevCluster& a, const DevCluster& b) {
  double g[2];
  for (int d = 0; d < 2; ++d) g[d] = fmax(0.0, fmax(__dsub_rn(a.bmin[d], b.bmax[d]), __dsub_rn(b.bmin[d], a.bmax[d])));
  return __dsqrt_rn(__dadd_rn(__dmul_rn(g[0], g[0]), __dmul_rn(g[1], g[1])));
}

// type and child count of every frontier block
__global__ void k_blk_classify(DevBlock* bl, const int32_t* front, int nf, const DevCluster* cl, double eta,
                               int adm_rule, int32_t* nchild) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  DevBlock& B = bl[front[i]];
  const DevCluster& R = cl[B.r];
  const DevCluster& S = cl[B.s];
  const bool lr = R.child[0] < 0, ls = S.child[0] < 0;
  int nc = 0;
  if (B.r == B.s) {
    B.diag = 1;
    if (lr) {
      B.type = BT_DENSE;
    } else {
      B.type = BT_SUB;
      nc = 3;
    }
  } else {
    B.diag = 0;
    const double d = dist_dev(R, S);
    bool adm;
    if (adm_rule == HLC_ADM_WEAK)
      adm = true;
    else if (adm_rule == HLC_ADM_MAXDIAM)
      adm = d > 0.0 && fmax(diam_dev(R), diam_dev(S)) <= __dmul_rn(eta, d);
    else
      adm = d > 0.0 && fmin(diam_dev(R), diam_dev(S)) <= __dmul_rn(eta, d);
    if (adm) {
      B.type = BT_LR;
    } else if (lr || ls) {
      B.type = BT_DENSE;
    } else {
      B.type = BT_SUB;
      nc = 4;
    }
  }
  nchild[i] = nc;
}

__global__ void k_blk_scan(const int32_t* nchild, int nf, int32_t next_id, int32_t* first, int32_t* total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int32_t run = 0;
  for (int i = 0; i < nf; ++i) {
    first[i] = next_id + run;
    run += nchild[i];
  }
  *total = run;
}

__global__ void k_blk_expand(DevBlock* bl, const int32_t* front, int nf, const DevCluster* cl, const int32_t* nchild,
                             const int32_t* first, int32_t next_id, int32_t* next_front) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf || nchild[i] == 0) return;
  DevBlock& B = bl[front[i]];
  const DevCluster& R = cl[B.r];
  const DevCluster& S = cl[B.s];
  const int32_t f = first[i];
  int32_t kid[4];
  int nk = 0;
  if (B.diag) {
    kid[0] = f;
    kid[1] = -1;
    kid[2] = f + 1;
    kid[3] = f + 2;
    DevBlock a{R.child[0], R.child[0], 0, 0, {-1, -1, -1, -1}};
    DevBlock b{R.child[1], R.child[0], 0, 0, {-1, -1, -1, -1}};
    DevBlock c{R.child[1], R.child[1], 0, 0, {-1, -1, -1, -1}};
    bl[f] = a;
    bl[f + 1] = b;
    bl[f + 2] = c;
    nk = 3;
  } else {
    for (int p = 0; p < 2; ++p)
      for (int q = 0; q < 2; ++q) {
        DevBlock x{R.child[p], S.child[q], 0, 0, {-1, -1, -1, -1}};
        bl[f + 2 * p + q] = x;
        kid[2 * p + q] = f + 2 * p + q;
      }
    nk = 4;
  }
  for (int q = 0; q < 4; ++q) B.ch[q] = kid[q];
  for (int q = 0; q < nk; ++q) next_front[f - next_id + q] = f + q;
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
#define TCK(x)                                 \
  do {                                         \
    if ((x) != cudaSuccess) return -1;         \
  } while (0)

int device_tree_build(const double* d_xy, int64_t n, int leaf, double eta, int adm, int split_rule, cudaStream_t st,
                      std::vector<int32_t>& perm, std::vector<Cluster>& clusters, std::vector<Block>& blocks,
                      int* depth) {
  const int nb_box = 304;
  double *d_part = nullptr, *d_bb = nullptr;
  uint64_t *k0 = nullptr, *k1 = nullptr;
  int32_t *i0 = nullptr, *i1 = nullptr;
  uint32_t* hist = nullptr;
  const int nb = (int)((n + RS_TILE - 1) / RS_TILE);
  int rc = 0;
  double *px = nullptr, *py = nullptr, *tx = nullptr, *ty = nullptr, *dmid = nullptr;
  int32_t *tp = nullptr, *front = nullptr, *nfront = nullptr, *dsplit = nullptr, *daxis = nullptr, *dchild0 = nullptr,
          *dn = nullptr;
  int64_t* dnl = nullptr;
  int64_t* dneed = nullptr;
  uint64_t* dthr = nullptr;
  DevCluster* dcl = nullptr;
  DevBlock* dbl = nullptr;
  const int64_t maxcl = 2 * n + 1;
  do {
    if (cudaMalloc(&d_part, nb_box * 4 * sizeof(double)) || cudaMalloc(&d_bb, 4 * sizeof(double)) ||
        cudaMalloc(&k0, n * 8) || cudaMalloc(&k1, n * 8) || cudaMalloc(&i0, n * 4) || cudaMalloc(&i1, n * 4) ||
        cudaMalloc(&hist, (size_t)256 * nb * 4)) {
      rc = -1;
      break;
    }
    k_bbox_part<<<nb_box, 256, 0, st>>>(d_xy, n, d_part);
    k_bbox_final<<<1, 32, 0, st>>>(d_part, nb_box, d_bb);
    k_morton<<<nb_box * 4, 256, 0, st>>>(d_xy, n, d_bb, k0, i0);
    for (int pass = 0; pass < 8; ++pass) {
      const int shift = 8 * pass;
      k_rs_hist<<<nb, RS_THREADS, 0, st>>>(k0, n, shift, hist, nb);
      k_rs_scan<<<1, 1024, 0, st>>>(hist, (int64_t)256 * nb);
      k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(k0, i0, k1, i1, n, shift, hist, nb);
      std::swap(k0, k1);
      std::swap(i0, i1);
    }
    // sorted coordinates
    if (cudaMalloc(&px, n * 8) || cudaMalloc(&py, n * 8) || cudaMalloc(&tx, n * 8) || cudaMalloc(&ty, n * 8) ||
        cudaMalloc(&tp, n * 4) || cudaMalloc(&dcl, maxcl * sizeof(DevCluster)) ||
        cudaMalloc(&front, maxcl * 4) || cudaMalloc(&nfront, maxcl * 4) || cudaMalloc(&dsplit, maxcl * 4) ||
        cudaMalloc(&daxis, maxcl * 4) || cudaMalloc(&dchild0, maxcl * 4) || cudaMalloc(&dmid, maxcl * 8) ||
        cudaMalloc(&dnl, maxcl * 8) || cudaMalloc(&dn, 8) || cudaMalloc(&dthr, maxcl * 8) ||
        cudaMalloc(&dneed, maxcl * 8)) {
      rc = -1;
      break;
    }
    launch_points(d_xy, i0, px, py, n, st);
    DevCluster root{};
    root.lo = 0;
    root.hi = n;
    root.child[0] = root.child[1] = -1;
    root.level = 0;
    cudaMemcpyAsync(dcl, &root, sizeof(root), cudaMemcpyHostToDevice, st);
    int32_t zero = 0;
    cudaMemcpyAsync(front, &zero, 4, cudaMemcpyHostToDevice, st);
    int32_t nf = 1, ncl = 1, lev = 0;
    while (nf > 0) {
      k_bis_measure<<<nf, BS_THREADS, 0, st>>>(dcl, front, px, py, leaf, split_rule, dsplit, dnl, daxis, dmid, dthr,
                                             dneed);
      k_bis_scan<<<1, 1, 0, st>>>(dsplit, nf, ncl, dchild0, dn);
      k_bis_split<<<nf, BS_THREADS, 0, st>>>(dcl, front, dsplit, dnl, daxis, dmid, dthr, dneed, split_rule, dchild0, px,
                                           py, i0, tx, ty, tp, nfront);
      int32_t ns = 0;
      cudaMemcpyAsync(&ns, dn, 4, cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess) {
        rc = -1;
        break;
      }
      if (ns > 0) ++lev;
      ncl += 2 * ns;
      nf = 2 * ns;
      std::swap(front, nfront);
    }
    if (rc) break;
    *depth = lev;
    // block tree
    std::vector<DevCluster> hcl(ncl);
    TCK(cudaMemcpy(hcl.data(), dcl, ncl * sizeof(DevCluster), cudaMemcpyDeviceToHost));
    const int64_t maxbl = std::max<int64_t>(64, 16 * (int64_t)ncl * 8);
    if (cudaMalloc(&dbl, maxbl * sizeof(DevBlock))) {
      rc = -1;
      break;
    }
    cudaFree(front);
    cudaFree(nfront);
    front = nfront = nullptr;
    if (cudaMalloc(&front, maxbl * 4) || cudaMalloc(&nfront, maxbl * 4)) {
      rc = -1;
      break;
    }
    DevBlock rb{0, 0, 0, 1, {-1, -1, -1, -1}};
    cudaMemcpyAsync(dbl, &rb, sizeof(rb), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(front, &zero, 4, cudaMemcpyHostToDevice, st);
    int32_t nbl = 1;
    nf = 1;
    int32_t* nchild = dsplit;  // reuse (maxcl >= frontier sizes is not guaranteed: realloc)
    int32_t* first = dchild0;
    cudaFree(nchild);
    cudaFree(first);
    dsplit = dchild0 = nullptr;
    if (cudaMalloc(&dsplit, maxbl * 4) || cudaMalloc(&dchild0, maxbl * 4)) {
      rc = -1;
      break;
    }
    nchild = dsplit;
    first = dchild0;
    while (nf > 0) {
      k_blk_classify<<<(nf + 255) / 256, 256, 0, st>>>(dbl, front, nf, dcl, eta, adm, nchild);
      k_blk_scan<<<1, 1, 0, st>>>(nchild, nf, nbl, first, dn);
      int32_t tot = 0;
      cudaMemcpyAsync(&tot, dn, 4, cudaMemcpyDeviceToHost, st);
      if (cudaStreamSynchronize(st) != cudaSuccess || nbl + (int64_t)tot > maxbl) {
        rc = -1;
        break;
      }
      k_blk_expand<<<(nf + 255) / 256, 256, 0, st>>>(dbl, front, nf, dcl, nchild, first, nbl, nfront);
      nbl += tot;
      nf = tot;
      std::swap(front, nfront);
    }
    if (rc) break;
    std::vector<DevBlock> hbl(nbl);
    TCK(cudaMemcpy(hbl.data(), dbl, nbl * sizeof(DevBlock), cudaMemcpyDeviceToHost));
    perm.resize(n);
    TCK(cudaMemcpy(perm.data(), i0, n * 4, cudaMemcpyDeviceToHost));
    clusters.resize(ncl);
    for (int32_t c = 0; c < ncl; ++c) {
      Cluster& C = clusters[c];
      C.lo = hcl[c].lo;
      C.hi = hcl[c].hi;
      for (int d = 0; d < 2; ++d) {
        C.bmin[d] = hcl[c].bmin[d];
        C.bmax[d] = hcl[c].bmax[d];
      }
      C.child[0] = hcl[c].child[0];
      C.child[1] = hcl[c].child[1];
      C.level = hcl[c].level;
    }
    blocks.resize(nbl);
    for (int32_t b = 0; b < nbl; ++b) {
      Block& B = blocks[b];
      B = Block{};
      B.r = hbl[b].r;
      B.s = hbl[b].s;
      B.type = hbl[b].type;
      B.diag = hbl[b].diag;
      for (int q = 0; q < 4; ++q) B.ch[q] = hbl[b].ch[q];
      B.m = clusters[B.r].size();
      B.n = clusters[B.s].size();
      B.slot = -1;
      B.leaf_index = -1;
    }
  } while (0);
  cudaFree(d_part);
  cudaFree(d_bb);
  cudaFree(k0);
  cudaFree(k1);
  cudaFree(i0);
  cudaFree(i1);
  cudaFree(hist);
  cudaFree(px);
  cudaFree(py);
  cudaFree(tx);
  cudaFree(ty);
  cudaFree(tp);
  cudaFree(front);
  cudaFree(nfront);
  cudaFree(dsplit);
  cudaFree(daxis);
  cudaFree(dchild0);
  cudaFree(dmid);
  cudaFree(dnl);
  cudaFree(dthr);
  cudaFree(dneed);
  cudaFree(dn);
  cudaFree(dcl);
  cudaFree(dbl);
  return rc;
}

}  // namespace hlc
