// kernels.h -- launchers of the device kernels (kernels.cu).
#pragma once

#include "hlc_internal.h"
#include "matern.cuh"

namespace hlc {

int64_t trunc_scratch_doubles();
int max_trunc_ctas();
int configure_trunc();
void launch_trunc(const OpTrunc* ops, int64_t count, const TermD* terms, const Bases& B, bool big,
                  cudaStream_t st);
int configure_kernels(int max_dense);

void launch_dense_asm(const DenseAsm* d, int64_t count, double* arena, const double* px, const double* py,
                      const MaternDev& mp, cudaStream_t st);
// ACA of every admissible leaf; a leaf that reaches its rank capacity before
// the stopping test holds (and is not full rank) records DEV_RANK in status.
// kfix > 0 (fixed-rank mode): at most kfix crosses, without an error.
void launch_aca(const LrAsm* d, int64_t count, double* arena, const double* px, const double* py,
                const MaternDev& mp, double eps, int kfix, int* ranks, int* status, cudaStream_t st);
void launch_ops(int type, const void* ops, int64_t count, const TermD* terms, const ChainTab& ct, const Bases& B,
                int max_dense, cudaStream_t st);
// One cooperative launch executing all waves of a TRSM/GEMM/chain plan with
// per_sm CTAs per SM (0 or more than fit: as many as fit); -1 when the
// cooperative launch is unavailable (the caller then launches wave by wave).
int launch_waves(const WaveRange* waves, int nwaves, const OpTrsm* trsm, const OpGemm* gemm, const OpChain* chain,
                 const ChainTab& ct, const Bases& B, GridBar* gb, int max_dense, int per_sm, cudaStream_t st);
int waves_max_per_sm(int max_dense);
// One cooperative launch executing a TRSM/GEMM plan in dataflow order (every
// op once its producers have signalled); count: nops ints of scratch.  -1
// when the cooperative launch is unavailable.
// The whole factorisation plan (its dataflow form) as one dependency-driven
// cooperative launch; -1 when the launch is unavailable.
int launch_factor(const Plan& P, const Bases& B, GridBar* gb, int max_dense, FactorTrace* trace,
                  cudaStream_t st);
int launch_flow(const FlowOp* flow, int64_t nops, const int32_t* npred, const int64_t* succ_off, const int32_t* succ,
                int32_t* count, const OpTrsm* trsm, const OpGemm* gemm, const Bases& B, GridBar* gb, int max_dense,
                int per_sm, FactorTrace* trace, cudaStream_t st);
// Two CTAs wait at a grid barrier that expects one arrival more than the
// grid has; the wait ends by its time limit with DEV_TIMEOUT in *status.
int launch_barrier_probe(GridBar* gb, int* status, cudaStream_t st);
// y = C x with the exact (dense, on the fly) covariance of the points in
// tree order; O(n^2) kernel evaluations (accuracy diagnostics only)
void launch_exact_matvec(const double* px, const double* py, const double* x, double* y, int64_t n,
                         const MaternDev& mp, cudaStream_t st);
void launch_gather(const double* src, const int32_t* perm, double* dst, int64_t n, cudaStream_t st);
void launch_scatter(const double* src, const int32_t* perm, double* dst, int64_t n, cudaStream_t st);
void launch_points(const double* xy, const int32_t* perm, double* px, double* py, int64_t n, cudaStream_t st);
void launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t st);
void launch_sub(const double* x, const double* y, double* z, int64_t n, cudaStream_t st);
void launch_dot(const double* x, const double* y, int64_t n, double* part, double* out, cudaStream_t st);
void launch_logdet(const int64_t* offs, const int32_t* dims, int64_t count, const double* arena, double* part,
                   double* out, cudaStream_t st);

// Device build of the cluster tree and block-cluster tree (tree.cu); returns
// 0 or -1 on a CUDA failure.
// adm: HLC_ADM_* admissibility rule; split: HLC_SPLIT_* bisection rule.
int device_tree_build(const double* d_xy, int64_t n, int leaf, double eta, int adm, int split, cudaStream_t st,
                      std::vector<int32_t>& perm, std::vector<Cluster>& clusters, std::vector<Block>& blocks,
                      int* depth);

}  // namespace hlc
