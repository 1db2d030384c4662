// Batched executor of a plan's binary contraction tree (device side).
//
// A plan is compiled on the host into a list of operations.  Every operation writes one
// tensor (a temporary or the per-element result) as
//     C[oc] = scalar * sum_t A[oa_t] * B[ob_t]  (+ C[oc] if accumulating)
// where the (oa_t, ob_t) pairs of each output entry oc enumerate exactly the non-zero
// products of the equivalent sparsity patterns (Sec. 4.2): the executed flops are the
// strength-reduced non-zero flops of Sec. 4.3.  Unary operations (copy / early
// summation of one operand) have no B.
//
// Mapping: a warp processes 32 elements (one per lane) through the whole operation list
// with warp-uniform control flow; temporaries live in a scratch buffer laid out
// [warp slot][entry][32 lanes] (coalesced), reused by every tile the warp processes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace yt {

enum OperandKind : int { kOpTemp = 0, kOpTensor = 1, kOpConst = 2, kOpNone = 3 };
enum OpKind : int { kOpProduct = 0, kOpUnary = 1, kOpZero = 2 };

struct ExecOp {
  int kind;
  int out_kind, out_ref, out_size;   // temp: ref = entry offset; tensor: ref = slot
  int a_kind, a_ref, a_size;
  int b_kind, b_ref, b_size;
  int nrows, rows_off, rp_off, pairs_off;
  double scalar;
  int accumulate;
};

constexpr int kMaxExecTensors = 16;

template <typename Real>
struct ExecPtrs {
  Real* p[kMaxExecTensors];
};

template <typename Real>
__device__ __forceinline__ Real exec_load(int kind, int ref, int size, int off,
                                          const Real* __restrict__ consts,
                                          const ExecPtrs<Real>& T, const Real* tmp, int64_t e,
                                          bool valid, int lane) {
  if (kind == kOpTemp) return tmp[(size_t)(ref + off) * 32 + lane];
  if (kind == kOpConst) return __ldg(consts + ref + off);
  if (kind == kOpTensor) return valid ? T.p[ref][e * size + off] : Real(0);
  return Real(1);
}

// grid: any number of 128-thread blocks; warp slots = gridDim.x * 4.
template <typename Real>
__global__ void __launch_bounds__(128)
k_execute(const ExecOp* __restrict__ ops, int nops, const int* __restrict__ prog,
          const Real* __restrict__ consts, ExecPtrs<Real> T, Real* __restrict__ scratch,
          int temp_entries, int64_t n_elements) {
  const int lane = threadIdx.x & 31;
  const int64_t warp_slot = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t n_slots = (int64_t)gridDim.x * (blockDim.x >> 5);
  Real* tmp = scratch + (size_t)warp_slot * temp_entries * 32;
  const int64_t n_tiles = (n_elements + 31) / 32;
  for (int64_t tile = warp_slot; tile < n_tiles; tile += n_slots) {
    const int64_t e = tile * 32 + lane;
    const bool valid = e < n_elements;
    for (int o = 0; o < nops; ++o) {
      const ExecOp op = ops[o];
      if (op.kind == kOpZero) {
        if (valid)
          for (int i = 0; i < op.out_size; ++i) T.p[op.out_ref][e * op.out_size + i] = Real(0);
        continue;
      }
      for (int r = 0; r < op.nrows; ++r) {
        const int oc = __ldg(prog + op.rows_off + r);
        const int b = __ldg(prog + op.rp_off + r), en = __ldg(prog + op.rp_off + r + 1);
        Real acc = Real(0);
        for (int t = b; t < en; ++t) {
          const int oa = __ldg(prog + op.pairs_off + 2 * t);
          const int ob = __ldg(prog + op.pairs_off + 2 * t + 1);
          const Real va = exec_load<Real>(op.a_kind, op.a_ref, op.a_size, oa, consts, T, tmp, e, valid, lane);
          const Real vb = exec_load<Real>(op.b_kind, op.b_ref, op.b_size, ob, consts, T, tmp, e, valid, lane);
          acc = fma(va, vb, acc);
        }
        if (op.scalar != 1.0) acc *= (Real)op.scalar;
        if (op.out_kind == kOpTemp) {
          tmp[(size_t)(op.out_ref + oc) * 32 + lane] = acc;
        } else if (valid) {
          Real* dst = T.p[op.out_ref] + e * op.out_size + oc;
          *dst = op.accumulate ? *dst + acc : acc;
        }
      }
    }
  }
}

// Element-per-warp variant: a warp takes one element at a time (grid-stride over the
// elements), its lanes share out the output entries (rows) of each operation, and the
// temporaries live in the warp's slice of shared memory ([warp][temp_entries]).  The
// element's own tensors are contiguous in global memory, so the gathers of one warp stay
// in L1.  Lanes exchange temporaries between operations, hence a __syncwarp after each.
template <typename Real>
__device__ __forceinline__ Real ew_load(int kind, int ref, int off, const Real* __restrict__ consts,
                                        const ExecPtrs<Real>& T, const Real* tmp, int64_t base) {
  if (kind == kOpTemp) return tmp[ref + off];
  if (kind == kOpConst) return __ldg(consts + ref + off);
  if (kind == kOpTensor) return T.p[ref][base + off];
  return Real(1);
}

// grid: any number of blocks of kEwWarps warps; dynamic shared memory kEwWarps *
// temp_entries * sizeof(Real) (GTMP: none; the temporaries in `scratch`, [warp][entries],
// for plans whose temporaries exceed the shared-memory cap: each warp's slice stays in
// L1 / L2 while the warp works on its element).
constexpr int kEwWarps = 4;
// plans whose four warps' temporaries fit this much shared memory use k_execute_ew (two
// blocks per SM at least)
constexpr int kEwSmemCap = 96 * 1024;
template <typename Real, bool GTMP = false>
__global__ void __launch_bounds__(kEwWarps * 32)
k_execute_ew(const ExecOp* __restrict__ ops, int nops, const int* __restrict__ prog,
             const Real* __restrict__ consts, ExecPtrs<Real> T, int temp_entries, int64_t n_elements,
             Real* __restrict__ scratch = nullptr) {
  extern __shared__ __align__(16) unsigned char ew_smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  Real* tmp = GTMP ? scratch + ((size_t)blockIdx.x * kEwWarps + wib) * temp_entries
                   : reinterpret_cast<Real*>(ew_smem) + (size_t)wib * temp_entries;
  const int64_t n_warps = (int64_t)gridDim.x * kEwWarps;
  for (int64_t e = (int64_t)blockIdx.x * kEwWarps + wib; e < n_elements; e += n_warps) {
    for (int o = 0; o < nops; ++o) {
      const ExecOp op = ops[o];
      if (op.kind == kOpZero) {
        Real* dst = T.p[op.out_ref] + e * op.out_size;
        for (int i = lane; i < op.out_size; i += 32) dst[i] = Real(0);
        __syncwarp();
        continue;
      }
      const int64_t abase = e * op.a_size, bbase = e * op.b_size;
      for (int r = lane; r < op.nrows; r += 32) {
        const int oc = __ldg(prog + op.rows_off + r);
        const int b = __ldg(prog + op.rp_off + r), en = __ldg(prog + op.rp_off + r + 1);
        Real acc = Real(0);
#pragma unroll 4
        for (int t = b; t < en; ++t) {
          const int oa = __ldg(prog + op.pairs_off + 2 * t);
          const int ob = __ldg(prog + op.pairs_off + 2 * t + 1);
          const Real va = ew_load<Real>(op.a_kind, op.a_ref, oa, consts, T, tmp, abase);
          const Real vb = ew_load<Real>(op.b_kind, op.b_ref, ob, consts, T, tmp, bbase);
          acc = fma(va, vb, acc);
        }
        if (op.scalar != 1.0) acc *= (Real)op.scalar;
        if (op.out_kind == kOpTemp) {
          tmp[op.out_ref + oc] = acc;
        } else {
          Real* dst = T.p[op.out_ref] + e * op.out_size + oc;
          *dst = op.accumulate ? *dst + acc : acc;
        }
      }
      __syncwarp();
    }
  }
}

}  // namespace yt
