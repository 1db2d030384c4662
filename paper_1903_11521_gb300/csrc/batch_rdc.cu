// The persistent batch kernel (see batch_kernel.cuh).  Separately compiled (-rdc): the
// per-degree tile functions live in the generated units ader_o<N>_<p>_batch_rdc.cu.
#include <cuda_runtime.h>

#include "batch_kernel.cuh"

namespace yt {

#define YT_BATCH_DECLARE(N, P)                                                              \
  __device__ void batch_local_o##N##_##P(const BatchGroup* g, const StarPattern* SP, size_t tile); \
  __device__ void batch_neigh_o##N##_##P(const BatchGroup* g, const FaceGroups* G, size_t tile);
YT_BATCH_DECLARE(1, f64)
YT_BATCH_DECLARE(2, f64)
YT_BATCH_DECLARE(3, f64)
YT_BATCH_DECLARE(4, f64)
YT_BATCH_DECLARE(5, f64)
YT_BATCH_DECLARE(6, f64)
YT_BATCH_DECLARE(1, f32)
YT_BATCH_DECLARE(2, f32)
YT_BATCH_DECLARE(3, f32)
YT_BATCH_DECLARE(4, f32)
YT_BATCH_DECLARE(5, f32)
YT_BATCH_DECLARE(6, f32)
#undef YT_BATCH_DECLARE

namespace {

__device__ __forceinline__ uint64_t batch_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a co-resident grid: one arrival per CTA on a counter that starts at
// zero in every launch; the wait is bounded (kBarrierWaitNs), after which the CTA records
// YT_ERR_TIMEOUT and returns false (it then skips the neighbour phase: no hang, the
// outputs of that step are incomplete and yt_batch_status reports it).
__device__ bool grid_barrier(int* count, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(count, 1);
    ok = 1;
    const uint64_t t0 = batch_timer();
    while (*(volatile int*)count < (int)gridDim.x) {
      if (batch_timer() - t0 > kBarrierWaitNs) {
        ok = 0;
        atomicExch(status, 7);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <bool F32>
__device__ void run_item(int phase, const BatchGroup* g, const StarPattern* SP, const FaceGroups* G,
                         size_t tile) {
#define YT_BATCH_CASE(N)                                                   \
  case N:                                                                  \
    if (F32) {                                                             \
      if (phase == 0) batch_local_o##N##_f32(g, SP, tile);                 \
      else batch_neigh_o##N##_f32(g, G, tile);                             \
    } else {                                                               \
      if (phase == 0) batch_local_o##N##_f64(g, SP, tile);                 \
      else batch_neigh_o##N##_f64(g, G, tile);                             \
    }                                                                      \
    break;
  switch (g->N) {
    YT_BATCH_CASE(1)
    YT_BATCH_CASE(2)
    YT_BATCH_CASE(3)
    YT_BATCH_CASE(4)
    YT_BATCH_CASE(5)
    YT_BATCH_CASE(6)
  }
#undef YT_BATCH_CASE
}

template <bool F32>
__global__ void __launch_bounds__(kNq * kTile, 1) k_batch_step(BatchArgs A) {
  __shared__ int claim;
  const StarPattern SP = A.SP;
  const FaceGroups G = A.faces;
  for (int phase = 0; phase < 2; ++phase) {
    const int2* items = A.items + (phase == 0 ? 0 : A.n_items[0]);
    const int n = A.n_items[phase];
    for (;;) {
      if (threadIdx.x == 0) claim = atomicAdd(A.counters + phase, A.chunk);
      __syncthreads();
      const int i0 = claim;
      __syncthreads();                 // every thread has read the claim before the next one
      if (i0 >= n) break;
      const int i1 = min(i0 + A.chunk, n);
      for (int i = i0; i < i1; ++i) {
        const int2 it = items[i];
        run_item<F32>(phase, A.groups + it.x, &SP, &G, (size_t)it.y);
      }
    }
    if (phase == 0 && !grid_barrier(A.counters + 2, A.status)) return;
  }
}

}  // namespace

int batch_persistent_prepare(bool f32, size_t smem) {
  const void* fn = f32 ? (const void*)k_batch_step<true> : (const void*)k_batch_step<false>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return -1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kNq * kTile, smem) != cudaSuccess) return -1;
  return per_sm;
}

cudaError_t batch_persistent_launch(bool f32, const BatchArgs& A, unsigned grid, size_t smem,
                                    cudaStream_t st, bool cooperative) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kNq * kTile);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = cooperative ? 1 : 0;
  BatchArgs a = A;
  void* args[] = {&a};
  const void* fn = f32 ? (const void*)k_batch_step<true> : (const void*)k_batch_step<false>;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace yt
