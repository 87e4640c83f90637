// Device side of the many-geometry solve: the outer iterations of every member problem
// (each its own hierarchy and grid size) advance inside one CUDA graph launch.
//
// The graph is a WHILE conditional node whose body holds one IF conditional node per member
// (the member's outer iteration: FP32 V-cycles, the FP64 update and residual, or FP64
// V-cycles) and, after all of them, k_group_decide.  That kernel reads every active member's
// residual max-norm, stores its relative residual, retires the members that reached their
// tolerance (or their iteration limit, or a non-finite residual, or a timed-out wait) by
// clearing their IF condition, and clears the WHILE condition when no member is left.
// k_group_init runs once before the loop on the initial residuals.  The decisions are the
// ones the single-problem solve takes on the host, per member.
#pragma once

#include <cuda_runtime.h>

namespace ccm {
namespace dev {

constexpr int GROUP_HIST = 64;   // relative residuals kept per member (ccm_stats.history)

struct GroupArgs {
  int n;                                         // members
  const unsigned long long* const* norm;         // per member: bits of its residual max-norm
  const int* const* err;                         // per member: its device error word
  const unsigned long long* rnorm;               // per member: bits of ||r_hat||_inf
  const double* rtol;
  const int* max_iter;
  const cudaGraphConditionalHandle* hk;          // per member: its IF condition
  cudaGraphConditionalHandle hw;                 // the WHILE condition
  int* act;                                      // per member: still iterating
  int* iters;                                    // per member: outer iterations done
  int* failed;                                   // per member: a bounded wait ran out
  double* rel;                                   // per member: last relative residual
  double* hist;                                  // [n][GROUP_HIST]
  int* it;                                       // outer iterations of the loop so far
};

__device__ __forceinline__ double bits_to_double(unsigned long long b) { return __longlong_as_double((long long)b); }

__device__ __forceinline__ double group_rel(const GroupArgs& A, int k) {
  double r0 = bits_to_double(A.rnorm[k]);
  if (r0 == 0.0) r0 = 1.0;
  return bits_to_double(*A.norm[k]) / r0;
}

// one block; the conditional values are written by thread 0 alone (concurrent writes of
// conditional values are not allowed)
__global__ void k_group_init(GroupArgs A) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < A.n; k += blockDim.x) {
    const double r = group_rel(A, k);
    A.rel[k] = r;
    A.hist[(long)k * GROUP_HIST] = r;
    A.iters[k] = 0;
    A.failed[k] = 0;
    const int a = (r == r && r <= 1.7976931348623157e308 && r > A.rtol[k] && A.max_iter[k] > 0) ? 1 : 0;
    A.act[k] = a;
    if (a) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *A.it = 0;
    for (int k = 0; k < A.n; ++k) cudaGraphSetConditional(A.hk[k], (unsigned)A.act[k]);
    cudaGraphSetConditional(A.hw, (unsigned)any);
  }
}

__global__ void k_group_decide(GroupArgs A) {
  __shared__ int any;
  const int it = *A.it + 1;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < A.n; k += blockDim.x) {
    if (!A.act[k]) continue;
    const double r = group_rel(A, k);
    A.rel[k] = r;
    A.iters[k] = it;
    if (it < GROUP_HIST) A.hist[(long)k * GROUP_HIST + it] = r;
    const int bad = *A.err[k] != 0;
    if (bad) A.failed[k] = 1;
    const int a = (!bad && r == r && r <= 1.7976931348623157e308 && r > A.rtol[k] && it < A.max_iter[k]) ? 1 : 0;
    A.act[k] = a;
    if (a) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *A.it = it;
    for (int k = 0; k < A.n; ++k) cudaGraphSetConditional(A.hk[k], (unsigned)A.act[k]);
    cudaGraphSetConditional(A.hw, (unsigned)any);
  }
}

}  // namespace dev
}  // namespace ccm
