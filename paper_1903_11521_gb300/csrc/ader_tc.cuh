// Tensor-core form of the ADER-DG step (precision YT_BF16X3_F32ACC): the products with
// the global matrices (CK derivatives Ktilde^x, volume Khat^x, face projections R^sT,
// lifting Rhat^s; Sec. 5.1.1 of the paper) run on the 5th-generation tensor cores as
// element-batched GEMMs, the per-element 9x9 products (star matrices, flux solvers) and
// the time-integral accumulation stay on the CUDA cores.
//
// Split precision.  Each operand value x is carried as two bfloat16 numbers,
// x_hi = bf16(x) and x_lo = bf16(x - x_hi) (together 16 significant bits), and a product
// a x is formed from the three tensor-core products a_hi x_hi + a_hi x_lo + a_lo x_hi
// with FP32 accumulation in tensor memory (the dropped a_lo x_lo term is below 2^-16 of
// |a x|).  The global matrices are split once on the host; element data are split by
// the threads that produce them.
//
// GEMM orientation.  For a tile of 32 elements, the M dimension is the (quantity,
// element) pair: the element operand has 288 rows r(q, e) and K = basis functions; the
// global matrix (transposed) is the N x K operand with N = output basis functions.  The
// 288 rows form three M = 128 groups: quantities 0-3 (rows 32..159), 4-7 (rows
// 160..287) and quantity 8 (rows 0..31; the group's rows 32..127 overlap the first group
// and give accumulator lanes that are never read).  Thread (warp q, lane e) therefore
// writes its own operand row and reads its own accumulator lane: warp q's TMEM lane
// quarter is q mod 4, which is where row (q, e) of its group lands.
//
// Shared-memory operands use the K-major, unswizzled canonical layout: 8 x 8 bf16 core
// matrices of 128 contiguous bytes (a row's 8 K-consecutive values in 16 bytes),
// K-adjacent core matrices 128 bytes apart, groups of 8 rows kp * 16 bytes apart.
//
// Synchronisation.  One elected thread per accumulator group issues that group's MMAs of
// a pass and commits them to an mbarrier; all threads wait for it (bounded, see tc_wait)
// before reading the accumulators with tcgen05.ld.  Every device-side wait gives up after kTcWaitNs and
// reports YT_ERR_TIMEOUT through the status word; the kernel then issues no further MMA,
// finishes its tile, waits (bounded) for what it issued and frees its tensor memory.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ader_kernels.cuh"
#include "fp_convert.cuh"

namespace yt {
namespace tc {

constexpr int kRows = kNq * kTile;                 // 288 element-operand rows
constexpr unsigned long long kTcWaitNs = 1000000000ull;   // 1 s
constexpr int kStatusTimeout = 7;                  // YT_ERR_TIMEOUT

__host__ __device__ constexpr int up8(int x) { return (x + 7) / 8 * 8; }
__host__ __device__ constexpr int up16(int x) { return (x + 15) / 16 * 16; }
__host__ __device__ constexpr int max2(int a, int b) { return a > b ? a : b; }

// Byte offset of entry (row r, k) of a canonical operand with K capacity kp.
__host__ __device__ constexpr int op_offset(int r, int k, int kp) {
  return (r / 8) * (kp * 16) + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
}
// Element-operand row of (quantity q, element e) and first row of each M = 128 group.
__host__ __device__ constexpr int op_row(int q, int e) { return q == 8 ? e : 32 + 32 * q + e; }
__host__ __device__ constexpr int group_first_row(int g) { return g == 0 ? 32 : (g == 1 ? 160 : 0); }
__host__ __device__ constexpr int group_of(int q) { return q < 4 ? 0 : (q < 8 ? 1 : 2); }

// Passes of the two kernels of degree N.  A pass is one set of MMAs into the three
// accumulator groups (N columns each, K = kp): k_local runs the CK derivatives (columns
// x * R8 + k - row0 for the output rows k of the pass), NV volume passes over row chunks
// (columns x * R8 + k - k0) and the face projections (columns s * BT8 + m); k_neigh runs
// the lifting (columns k, K = s * BT8 + m).  When the first derivative's three directions
// would need more than 160 accumulator columns per group (order 7: 3 x 56), it runs as
// two passes over its rows [0, 32) and [32, C(N+2,3)): derivative passes p < ND, with
// derivative tc_delta(p), first row tc_row0(p) and tc_rows(p) rows.
constexpr int kSplitRows = 32;
template <int N>
__host__ __device__ constexpr bool tc_split0() { return 3 * up8(Dims<N>::nd(1)) > 160; }
template <int N>
__host__ __device__ constexpr int tc_nderiv() { return N + (tc_split0<N>() ? 1 : 0); }
template <int N>
__host__ __device__ constexpr int tc_delta(int p) { return tc_split0<N>() ? (p == 0 ? 0 : p - 1) : p; }
template <int N>
__host__ __device__ constexpr int tc_row0(int p) { return (tc_split0<N>() && p == 1) ? kSplitRows : 0; }
template <int N>
__host__ __device__ constexpr int tc_rows(int p) {
  return (tc_split0<N>() && p == 0) ? kSplitRows
                                    : ((tc_split0<N>() && p == 1) ? Dims<N>::nd(1) - kSplitRows
                                                                  : Dims<N>::nd(tc_delta<N>(p) + 1));
}
template <int N>
__host__ __device__ constexpr int tc_nv() {
  int n = 1;
  while (up16(3 * up8((Dims<N>::B + n - 1) / n)) > 160) ++n;
  return n;
}
template <int N>
__host__ __device__ constexpr int tc_vr() { return up8((Dims<N>::B + tc_nv<N>() - 1) / tc_nv<N>()); }
template <int N>
__host__ __device__ constexpr int tc_vrows(int v) {
  return (Dims<N>::B - v * tc_vr<N>()) < tc_vr<N>() ? (Dims<N>::B - v * tc_vr<N>()) : tc_vr<N>();
}
template <int N>
__host__ __device__ constexpr int tc_r8(int p) {
  return p < tc_nderiv<N>() ? up8(tc_rows<N>(p))
                            : (p < tc_nderiv<N>() + tc_nv<N>() ? up8(tc_vrows<N>(p - tc_nderiv<N>())) : up8(Dims<N>::BT));
}
template <int N>
__host__ __device__ constexpr int tc_np(int p) {
  return p < tc_nderiv<N>() + tc_nv<N>() ? up16(3 * tc_r8<N>(p)) : up16(4 * up8(Dims<N>::BT));
}
template <int N>
__host__ __device__ constexpr int tc_kp(int p) {
  return p < tc_nderiv<N>() ? up16(Dims<N>::nd(tc_delta<N>(p)))
                            : (p < tc_nderiv<N>() + tc_nv<N>() ? up16(Dims<N>::nd(1)) : up16(Dims<N>::B));
}
template <int N>
__host__ __device__ constexpr int tc_size(int p) { return 2 * tc_np<N>(p) * tc_kp<N>(p) * 2; }
template <int N>
__host__ __device__ constexpr int tc_off(int p) { return p == 0 ? 0 : tc_off<N>(p - 1) + tc_size<N>(p - 1); }
template <int N>
__host__ __device__ constexpr int tc_cs() {
  int c = 0;
  for (int p = 0; p < tc_nderiv<N>() + tc_nv<N>() + 1; ++p) c = max2(c, tc_np<N>(p));
  return c;
}
template <int N>
__host__ __device__ constexpr int tc_pass_max() {
  int c = 0;
  for (int p = 0; p < tc_nderiv<N>() + tc_nv<N>() + 1; ++p) c = max2(c, tc_size<N>(p));
  return c;
}
constexpr size_t kSmemCap = 232448;      // dynamic shared memory of one CTA (227 KB)

// first scratch row of D~^d (d >= 1): rows C(N-d+3,3) of every earlier derivative
template <int N>
__host__ __device__ constexpr int tc_srow(int d) { return d <= 1 ? 0 : tc_srow<N>(d - 1) + Dims<N>::nd(d - 1); }

template <int N>
struct Layout {
  using D = Dims<N>;
  static constexpr int B = D::B, BT = D::BT, BT8 = up8(BT), NI = D::nd(1);
  static constexpr int KPA = up16(B);                  // K capacity, k_local element operand
  static constexpr int NV = tc_nv<N>();
  static constexpr int VR = tc_vr<N>();               // rows per volume pass
  static constexpr bool SPLIT0 = tc_split0<N>();
  static constexpr int ND = tc_nderiv<N>();            // derivative passes
  static constexpr int NPASS = ND + NV + 1;
  __host__ __device__ static constexpr int vrows(int v) { return tc_vrows<N>(v); }
  __host__ __device__ static constexpr int r8(int p) { return tc_r8<N>(p); }
  __host__ __device__ static constexpr int np(int p) { return tc_np<N>(p); }
  __host__ __device__ static constexpr int kp(int p) { return tc_kp<N>(p); }
  __host__ __device__ static constexpr int off(int p) { return tc_off<N>(p); }
  __host__ __device__ static constexpr int size(int p) { return tc_size<N>(p); }
  static constexpr int BLOB = tc_off<N>(NPASS);
  static constexpr int CS = tc_cs<N>();               // TMEM columns per group
  // rows of the scaled derivatives D~^1..D~^N kept for the time integral (per-CTA scratch)
  static constexpr int SROWS = tc_srow<N>(N + 1);
  static constexpr int OPA_SPLIT = kRows * KPA * 2;    // bytes of one split
  // exchange buffer: 3 directions (mixing) or BT8 / 8 chunks (face projections) of
  // [9][2][32][4] floats
  static constexpr int XS_CHUNKS = max2(3, BT8 / 8);
  static constexpr int XS_FLOATS = XS_CHUNKS * kNq * 2 * kTile * 4;
  // the global-matrix operands of all passes stay in shared memory when they fit beside
  // the element operand; otherwise (order 7) each pass's operand is loaded into one
  // buffer while the previous pass's accumulators are mixed (STREAM)
  static constexpr bool STREAM = (size_t)2 * OPA_SPLIT + BLOB + XS_FLOATS * 4 + 64 > kSmemCap;
  static constexpr int OPB_BYTES = STREAM ? tc_pass_max<N>() : BLOB;
  static constexpr size_t SMEM = (size_t)2 * OPA_SPLIT + OPB_BYTES + XS_FLOATS * 4 + 64;
  // k_neigh: the lifting with K = the four faces' W stacked, or (order 7, LIFT2) two
  // passes of two faces each (K = 2 BT8), accumulated in tensor memory, so that the
  // element operand holds two faces only
  static constexpr int KPN = up16(4 * BT8);            // K of the Rhat operand (all faces)
  static constexpr int NPL = up16(B);
  static constexpr int BLOB_N = 2 * NPL * KPN * 2;
  static constexpr int STAGE_FLOATS = BT8 * kNq * kTile;     // one face of gathered projections
  static constexpr bool LIFT2 = (size_t)2 * kRows * KPN * 2 + BLOB_N + 3 * STAGE_FLOATS * 4 + 64 > kSmemCap;
  static constexpr int KPE = LIFT2 ? up16(2 * BT8) : KPN;      // K of the element operand
  static constexpr int OPN_SPLIT = kRows * KPE * 2;
  static constexpr int XSN_FLOATS = LIFT2 ? (BT + 3) / 4 * 4 * kNq * kTile : STAGE_FLOATS;
  static constexpr size_t SMEM_N = (size_t)2 * OPN_SPLIT + BLOB_N + 2 * STAGE_FLOATS * 4 + XSN_FLOATS * 4 + 64;
  // k_local_tc converts with the integer units (fp_convert.cuh) except at degree 5, where
  // the extra registers cost more than the FP64-pipe slots they save (measured)
  static constexpr bool INT_CVT_LOCAL = N <= 4;
  // the time integral widens its binary32 derivative terms on the integer units at every
  // degree (measured at order 6: k_local_tc 14.4 -> 13.1 ms; narrowing I or Q the same
  // way was slower: 15.5 / 16.5 ms)
  static constexpr bool INT_WIDEN_TI = true;
  // the 8-row chunk loops of k_local_tc's volume mixing and face projections run as
  // loops (one copy of the body per chunk parity) instead of fully unrolled: at order 7
  // the unrolled kernel waits on instruction fetch first (measured at 1M tets: 25.2 ->
  // 23.8 ms).  The derivative mixing stays unrolled: as a loop it spills (ptxas: 132 ->
  // 320 bytes of spill stores), which cost what the smaller code saved (25.3 ms).
  static constexpr bool ROLL = N >= 6;
  static_assert(3 * CS <= 512 && 3 * NPL <= 512, "accumulators exceed tensor memory");
  static_assert(BT8 / 8 <= XS_CHUNKS, "face basis too large for the exchange buffer");
  static_assert(SMEM <= kSmemCap && SMEM_N <= kSmemCap, "shared memory of one CTA exceeded");
  static_assert(!SPLIT0 || (kSplitRows % 8 == 0 && NI > kSplitRows), "split of the first derivative");
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Shared-memory matrix descriptor: start, LBO = 128 (K-adjacent core matrices), SBO
// (row-group stride), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 accumulator,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Generic-proxy shared-memory writes become visible to the tensor cores (async proxy).
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bulk (TMA) copy global -> shared, completion counted in bytes on `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait for phase `parity` of `bar`: false after `limit_ns` (default kTcWaitNs).
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns = kTcWaitNs) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = global_timer();
  while (global_timer() - t0 < limit_ns)
    if (mbar_try(bar, parity)) return true;
  return false;
}
// 8 consecutive FP32 accumulator columns of this thread's lane (32x32b shape).
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&r)[8]) {
  uint32_t u[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) r[i] = __uint_as_float(u[i]);
}
// 3 x 8 accumulator columns without waiting: the values are valid only after tmem_wait24
// (which takes the registers as operands, so no use can move above it).
__device__ __forceinline__ void tmem_ld3x8_async(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t (&u)[24]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
        "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]),
        "=r"(u[16]), "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23])
      : "r"(a0), "r"(a1), "r"(a2)
      : "memory");
}
__device__ __forceinline__ void tmem_wait24(uint32_t (&u)[24]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n"
               : "+r"(u[0]), "+r"(u[1]), "+r"(u[2]), "+r"(u[3]), "+r"(u[4]), "+r"(u[5]), "+r"(u[6]), "+r"(u[7]),
                 "+r"(u[8]), "+r"(u[9]), "+r"(u[10]), "+r"(u[11]), "+r"(u[12]), "+r"(u[13]), "+r"(u[14]),
                 "+r"(u[15]), "+r"(u[16]), "+r"(u[17]), "+r"(u[18]), "+r"(u[19]), "+r"(u[20]), "+r"(u[21]),
                 "+r"(u[22]), "+r"(u[23])
               :
               : "memory");
}

// Stores 8 K-consecutive values of one operand row as hi and lo bf16 parts.
__device__ __forceinline__ void store_split8(unsigned char* op, int split_bytes, int off, const float (&v)[8]) {
  uint32_t hi[4], lo[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
    hi[i] = *reinterpret_cast<const uint32_t*>(&h);
    lo[i] = *reinterpret_cast<const uint32_t*>(&l);
  }
  *reinterpret_cast<uint4*>(op + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4*>(op + split_bytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
}

// Calls body(k0, odd) for the 8-row chunks k0 = 0, 8, .., 8 (NCH - 1) of a pass, odd =
// integral_constant<bool, chunk index odd>, so that the body picks its double-buffered
// register arrays at compile time.  ROLL: a loop over chunk pairs (one copy of the body
// per parity), else fully unrolled (k0 folds to a constant).
template <int NCH, bool ROLL, typename F>
__device__ __forceinline__ void for_chunk_pairs(F&& body) {
  if constexpr (ROLL && NCH > 2) {
#pragma unroll 1
    for (int c = 0; c < NCH; c += 2) {
      body(8 * c, std::false_type{});
      if (c + 1 < NCH) body(8 * c + 8, std::true_type{});
    }
  } else {
    static_for<0, NCH>([&](auto cc) {
      constexpr int c = decltype(cc)::value;
      body(8 * c, std::integral_constant<bool, (c & 1) != 0>{});
    });
  }
}
// Calls body(c) for c = 0 .. NC - 1: a loop (ROLL) or fully unrolled.
template <int NC, bool ROLL, typename F>
__device__ __forceinline__ void for_chunks(F&& body) {
  if constexpr (ROLL && NC > 1) {
#pragma unroll 1
    for (int c = 0; c < NC; ++c) body(c);
  } else {
    static_for<0, NC>([&](auto cc) { body((int)decltype(cc)::value); });
  }
}

// The MMAs of one pass for accumulator group g (K steps of 16 x three products), issued
// by one elected thread per group (lane 0 of warps 0..2: the three groups' MMAs are
// independent and issue in parallel) and committed to `bar` (expected count 3).  The
// descriptors of step j differ from step 0 only in the start address (+256 B, i.e. +16
// in the address field, which cannot carry: shared addresses are below 256 KB).
// The MMAs of accumulator group g over `ksteps` K-steps of 16: A (element operand, K
// capacity kpa, lo part a_split bytes after hi), B (global-matrix operand, K capacity kpb
// for its row-group stride, lo part b_split bytes after hi; b_base may point into its
// K range).  The first product starts the accumulator unless `acc` (continue it).
__device__ __forceinline__ void issue_group_k(int g, uint32_t tmem, int cs, uint32_t a_base, int a_split,
                                              int kpa, uint32_t b_base, int b_split, int np, int kpb,
                                              int ksteps, bool acc, uint32_t bar) {
  const uint32_t idesc = idesc_bf16(np);
  const uint32_t sbo_a = (uint32_t)kpa * 16, sbo_b = (uint32_t)kpb * 16;
  const uint32_t a_hi = a_base + (uint32_t)(group_first_row(g) / 8) * sbo_a;
  const uint64_t dah = smem_desc(a_hi, sbo_a), dal = smem_desc(a_hi + (uint32_t)a_split, sbo_a);
  const uint64_t dbh = smem_desc(b_base, sbo_b), dbl = smem_desc(b_base + (uint32_t)b_split, sbo_b);
  const uint32_t d = tmem + (uint32_t)(g * cs);
  for (int j = 0; j < ksteps; ++j) {
    const uint64_t dk = (uint64_t)(j * 16);
    mma_bf16(d, dah + dk, dbh + dk, idesc, (acc || j > 0) ? 1u : 0u);
    mma_bf16(d, dah + dk, dbl + dk, idesc, 1);
    mma_bf16(d, dal + dk, dbh + dk, idesc, 1);
  }
  mma_commit(bar);
}
__device__ __forceinline__ void issue_group(int g, uint32_t tmem, int cs, uint32_t a_base, int a_split,
                                            int kpa, uint32_t b_base, int np, int kp, uint32_t bar) {
  issue_group_k(g, tmem, cs, a_base, a_split, kpa, b_base, np * kp * 2, np, kp, kp / 16, false, bar);
}

struct TcStep {
  double dt;
  double invfact[8];
  int expire_first_wait;     // diagnostics: the operand load is not issued and its wait
                             // gives up after kDiagWaitNs (nothing is in flight then)
};
constexpr unsigned long long kDiagWaitNs = 1000000ull;    // 1 ms

// Per-CTA resources: tensor memory, two mbarriers (operand load, MMA completion).
struct TcShared {
  uint64_t bar[2];
  uint32_t tmem;
  int ok;
};

// Allocation of `ncols` tensor-memory columns by warp 0 (written to ts->tmem).
template <int NCOLS>
__device__ __forceinline__ void tmem_alloc(TcShared* ts) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ts->tmem)),
               "n"(NCOLS)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int NCOLS>
__device__ __forceinline__ void tmem_free(uint32_t tmem) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(NCOLS) : "memory");
}

// Loads `bytes` of pre-split global-matrix operands into shared memory with bulk copies
// (elected thread; chunks of at most 32 KB, all counted on bar).
__device__ __forceinline__ void load_operands(unsigned char* dst, const unsigned char* src, int bytes,
                                              uint32_t bar) {
  mbar_expect_tx(bar, (uint32_t)bytes);
  for (int o = 0; o < bytes; o += 32768) {
    const int n = bytes - o < 32768 ? bytes - o : 32768;
    bulk_load(smem_u32(dst + o), src + o, (uint32_t)n, bar);
  }
}

// 16-byte global -> shared copy bypassing the registers (L2 only), grouped per face.
__device__ __forceinline__ void cp_async16(float* dst_shared, const float* src_global) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst_shared)), "l"(src_global)
               : "memory");
}

// ------------------------------------------------------------------------- K_local
// Derivatives, time integral, volume, face projections and local flux products of tiles
// of 32 elements; persistent CTAs (grid <= number of tiles) stride over the tiles.
// Outputs and layouts as k_local<N, false, float>: I, Wloc [tile][4][9][BT][32] =
// (R^sT I) Aloc_s^T, except that the face projections Pface are [element][4][9][BT8] (rows
// padded to 8 floats: 16-byte copies in k_neigh_tc) and that the volume increment is not
// added to Q here but written to Vol [tile][9][B][32] (binary32): k_neigh_tc adds it with
// the lifting in one binary64 update of Q (one read-modify-write of Q per step instead
// of two).  VE: Q gets the volume and the stress rows' source here.
// The scaled derivatives D~^d (binary32, as produced) go to this CTA's scratch rows
// [SROWS][9][32] (L2-resident, reused tile after tile); the time integral is summed from
// them in binary64, in the order d = 0..N, once the derivatives are done.  Keeping the
// binary64 accumulator in registers instead spills (168-register cap of 9-warp CTAs).
//
// VE: 27-quantity (viscoelastic-shaped) step, Q and I [tile][27][B][32].  The source
// couples the stress rows with the anelastic functions theta^l_i at every row, so every
// derivative has all B rows: each one is the pass (or the two row blocks) of the first
// derivative, K = B, for the rows of degree < N; the stress rows get the feedback
// -sum_l theta^l_i, the rows of degree N only that.  The anelastic functions of stress
// warp i (theta^l_i, l = 0..2) are advanced on the CUDA cores from the velocity columns
// of the same accumulator chunks (their star rows have the stress rows' slots):
// D~^{d+1}_theta = dt (sum_x sum_q Astar^x_theta,q X^x_q - omega_l D~^d_theta), their
// scaled state in V.theta.  The time integral of all 27 quantities accumulates in binary64
// in I as the derivatives are produced (I = c0 Q first).  The volume adds the source of the
// stress rows, -sum_l I_theta; the anelastic rows' volume, source and fluxes are k_theta's.
template <int N, bool VE = false>
__global__ void __launch_bounds__(kRows, 1)
k_local_tc(double* Q, double* __restrict__ Iout, float* __restrict__ Pface, float* __restrict__ Wloc,
           const float* __restrict__ star, const float* __restrict__ floc,
           const unsigned char* __restrict__ blob, float* __restrict__ scratch, TcStep T, StarPattern SP,
           VeTables<float> V, float* __restrict__ Vol, int64_t ntiles, int* __restrict__ status) {
  using L = Layout<N>;
  using Dm = Dims<N>;
  constexpr int B = L::B, BT = L::BT, BT8 = L::BT8, KPA = L::KPA, NI = L::NI, CS = L::CS, NV = L::NV;
  constexpr int NQT = VE ? kNqVe : kNq;                  // quantities per element in Q and I
  constexpr size_t LS = (size_t)6 * B * kTile;           // VE: mechanism stride of theta and I
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* opa = smem_raw;                                  // [hi | lo] 288 x KPA
  unsigned char* opb = opa + 2 * L::OPA_SPLIT;                    // global-matrix passes
  float* xs = reinterpret_cast<float*>(opb + L::OPB_BYTES);       // [XS_CHUNKS][9][2][32][4]
  TcShared* ts = reinterpret_cast<TcShared*>(xs + L::XS_FLOATS);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool leader = threadIdx.x == 0;
  const uint32_t bar_ld = smem_u32(&ts->bar[0]), bar_mma = smem_u32(&ts->bar[1]);

  // zero the element operand once: padding columns are read (times zero) by every pass
  for (int i = threadIdx.x; i < 2 * L::OPA_SPLIT / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(opa)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (w == 0) tmem_alloc<512>(ts);
  if (leader) {
    mbar_init(bar_ld, 1);
    mbar_init(bar_mma, 3);
    mbar_fence_init();
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = ts->tmem;
  const bool issuer = lane == 0 && w < 3;          // issues accumulator group w
  // all passes' operands at once, or (STREAM) the first pass's
  if (leader && !T.expire_first_wait) load_operands(opb, blob, L::STREAM ? L::size(0) : L::BLOB, bar_ld);
  bool ok = __syncthreads_and(tc_wait(bar_ld, 0, T.expire_first_wait ? kDiagWaitNs : kTcWaitNs)) != 0;
  uint32_t phase = 0;
  bool pending = false;              // a commit whose wait timed out
  uint32_t pending_phase = 0;
  uint32_t ld_phase = 1;             // STREAM: phase of the next operand load
  bool ld_out = false;               // STREAM: an operand load is in flight

  const uint32_t opa_s = smem_u32(opa), opb_s = smem_u32(opb);
  const int g = group_of(w);
  const uint32_t my_tmem = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(g * CS);
  const int my_row = op_row(w, lane);
  float* my_scr = scratch + (size_t)blockIdx.x * L::SROWS * kRows + w * kTile + lane;
  const int s0 = SP.start[w], cnt = SP.start[w + 1] - s0;
  int scol[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) scol[s] = (s < cnt) ? SP.col[s0 + s] : 0;
  const double dt = T.dt;
  const float dtf = (float)dt;

  // STREAM: the operand of pass p into the single operand buffer (issued only after the
  // MMAs reading that buffer have completed), and the wait for it before the pass
  auto load_pass = [&](int p) {
    if constexpr (L::STREAM) {
      if (ok) {
        if (leader) load_operands(opb, blob + L::off(p), L::size(p), bar_ld);
        ld_out = true;
      }
    }
  };
  auto pass_ready = [&]() {
    if constexpr (L::STREAM) {
      if (ld_out && ok) {
        const bool all = __syncthreads_and(tc_wait(bar_ld, ld_phase)) != 0;
        if (all) {
          ld_phase ^= 1u;
          ld_out = false;
        } else {
          ok = false;                // the final bounded wait covers the load in flight
        }
      }
    }
  };
  // MMAs are issued only while ok (block-uniform), so every issued pass is waited for
  auto issue = [&](int p) {
    pass_ready();
    if (issuer && ok) {
      fence_after_sync();
      issue_group(w, tmem, CS, opa_s, L::OPA_SPLIT, KPA, opb_s + (uint32_t)(L::STREAM ? 0 : L::off(p)), L::np(p),
                  L::kp(p), bar_mma);
    }
  };
  // waits for the pass in flight; STREAM: then loads the operand of pass `next` (< 0: none)
  auto wait_pass = [&](int next) {
    const bool was_ok = ok;
    const bool done = was_ok ? tc_wait(bar_mma, phase) : false;
    ok = __syncthreads_and(done) != 0;
    if (was_ok && !ok) {
      pending = true;
      pending_phase = phase;
    }
    phase ^= 1u;
    fence_after_sync();
    if (next >= 0) load_pass(next);
  };
  // publishes this thread's operand writes and TMEM reads before the next MMA issue
  auto sync_for_mma = [&]() {
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
  };
  // star product of an 8-row chunk held in xs: v[i] = sum_x sum_q Astar^x_pq X^x[k0+i][q]
  auto mix_star = [&](const float (&sc)[3][3], float (&v)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = 0.0f;
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int s = 0; s < 3; ++s)
        if (s < cnt) {
          const float4* src = reinterpret_cast<const float4*>(xs) + ((x * kNq + scol[s]) * 2) * kTile + lane;
          const float4 a = src[0], b = src[kTile];
          const float c = sc[x][s];
          v[0] = fmaf(c, a.x, v[0]);
          v[1] = fmaf(c, a.y, v[1]);
          v[2] = fmaf(c, a.z, v[2]);
          v[3] = fmaf(c, a.w, v[3]);
          v[4] = fmaf(c, b.x, v[4]);
          v[5] = fmaf(c, b.y, v[5]);
          v[6] = fmaf(c, b.z, v[6]);
          v[7] = fmaf(c, b.w, v[7]);
        }
  };
  // 3 x 8 accumulator columns (plane stride r8) of this thread's lane into xs
  // accumulator chunks: columns col0 + x * r8 + 0..7 (x = 0..2) of this thread's lane;
  // the load of chunk c + 1 is issued before chunk c is mixed and waited for after it
  auto load_chunk = [&](int col0, int r8, uint32_t (&u)[24]) {
    tmem_ld3x8_async(my_tmem + col0, my_tmem + col0 + r8, my_tmem + col0 + 2 * r8, u);
  };
  auto put_chunk = [&](uint32_t (&u)[24]) {
    tmem_wait24(u);
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      float4* dst = reinterpret_cast<float4*>(xs) + ((x * kNq + w) * 2) * kTile + lane;
      dst[0] = make_float4(__uint_as_float(u[8 * x]), __uint_as_float(u[8 * x + 1]),
                           __uint_as_float(u[8 * x + 2]), __uint_as_float(u[8 * x + 3]));
      dst[kTile] = make_float4(__uint_as_float(u[8 * x + 4]), __uint_as_float(u[8 * x + 5]),
                               __uint_as_float(u[8 * x + 6]), __uint_as_float(u[8 * x + 7]));
    }
  };

  for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
    const double* Qt = Q + tile * (NQT * B * kTile);
    double* Qo = Q + tile * (NQT * B * kTile);
    double* It = Iout + tile * (NQT * B * kTile);
    float sc[3][3];
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int s = 0; s < 3; ++s)
        sc[x][s] = (s < cnt) ? __ldg(star + ((tile * 3 + x) * kStarSlots + s0 + s) * kTile + lane) : 0.0f;
    // VE: relaxation rates of this stress warp's mechanisms; D~^0 of its anelastic
    // functions into their scratch and I = c0 Q of them
    float om[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (VE) {
      if (w < 6) {
#pragma unroll
        for (int l = 0; l < 3; ++l) om[l] = __ldg(V.om + (tile * 3 + l) * kTile + lane);
        float* th = V.theta + ((tile * kNTheta + w) * B) * kTile + lane;
        const double* qth = Qt + ((size_t)(9 + w) * B) * kTile + lane;
        double* ith = It + ((size_t)(9 + w) * B) * kTile + lane;
        // four rows of the three mechanisms loaded before they are stored
        static_for<0, (B + 3) / 4>([&](auto cc) {
          constexpr int k0 = decltype(cc)::value * 4;
          double q[3][4];
#pragma unroll
          for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int i = 0; i < 4; ++i) q[l][i] = (k0 + i < B) ? __ldg(qth + l * LS + (k0 + i < B ? k0 + i : 0) * kTile) : 0.0;
#pragma unroll
          for (int l = 0; l < 3; ++l)
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (k0 + i < B) {
                th[l * LS + (k0 + i) * kTile] = from_f64<float, L::INT_CVT_LOCAL>(q[l][i]);
                ith[l * LS + (k0 + i) * kTile] = dt * T.invfact[0] * q[l][i];
              }
        });
      }
    }

    // D~^0 = Q as operand (two chunks of loads in flight at a time); VE: I = c0 Q
    static_for<0, (up8(B) / 8 + 1) / 2>([&](auto cc) {
      constexpr int k0 = decltype(cc)::value * 16;
      float v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = k0 + i;
        const double q = k < B ? __ldg(Qt + (w * B + (k < B ? k : 0)) * kTile + lane) : 0.0;
        v[i] = k < B ? from_f64<float, L::INT_CVT_LOCAL>(q) : 0.0f;
        if constexpr (VE) {
          if (k < B) It[(w * B + k) * kTile + lane] = dt * T.invfact[0] * q;
        }
      }
      store_split8(opa, L::OPA_SPLIT, op_offset(my_row, k0, KPA), *reinterpret_cast<float(*)[8]>(v));
      if constexpr (k0 + 8 < up8(B))
        store_split8(opa, L::OPA_SPLIT, op_offset(my_row, k0 + 8, KPA), *reinterpret_cast<float(*)[8]>(v + 8));
    });
    sync_for_mma();
    issue(0);

    // CK derivatives: D~^{delta+1} = dt sum_x (Ktilde^x D~^delta) Astar^xT, in the operand.
    // Mixing of derivative pass P: its rows ROW0 + k (k < R) from accumulator columns
    // x * R8 + k, into the scratch and (TO_OPA) the operand.
    auto mix_deriv = [&](auto pp, auto to_opa) {
      constexpr int P = decltype(pp)::value;
      constexpr bool TO_OPA = decltype(to_opa)::value;
      constexpr int DELTA = tc_delta<N>(P), R = tc_rows<N>(P), R8 = up8(R), ROW0 = tc_row0<N>(P);
      uint32_t ua[24], ub[24];       // chunk c in ua (c even) or ub (c odd)
      load_chunk(0, R8, ua);
      for_chunk_pairs<R8 / 8, false>([&](int k0, auto odd) {
        uint32_t (&cur)[24] = decltype(odd)::value ? ub : ua;
        uint32_t (&nxt)[24] = decltype(odd)::value ? ua : ub;
        put_chunk(cur);
        if (k0 + 8 < R8) load_chunk(k0 + 8, R8, nxt);
        __syncthreads();
        float v[8];
        mix_star(sc, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = k0 + i;
          if (k < R) {
            v[i] *= dtf;
            my_scr[(tc_srow<N>(DELTA + 1) + ROW0 + k) * kRows] = v[i];
          } else {
            v[i] = 0.0f;
          }
        }
        if constexpr (TO_OPA) store_split8(opa, L::OPA_SPLIT, op_offset(my_row, ROW0 + k0, KPA), v);
        if (k0 + 8 < R8) __syncthreads();
      });
    };
    // VE: the anelastic functions of the 8 rows kb..kb+7 of stress warp w and the source
    // feedback into v (the stress row's star product, unscaled); HASX: the rows have
    // accumulator chunks in xs (degree < N), else only the relaxation acts
    // (the loads of each mechanism's rows are issued together, ahead of its stores: a
    // store to the scratch could alias them otherwise and serialise every row on the
    // memory latency)
    auto ve_chunk = [&](int kb, float (&v)[8], double cw, auto hasx) {
      constexpr bool HASX = decltype(hasx)::value;
      float* th = V.theta + ((tile * kNTheta + w) * B + kb) * kTile + lane;
      double* ith = It + ((size_t)(9 + w) * B + kb) * kTile + lane;
      float t[3][8];
#pragma unroll
      for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int i = 0; i < 8; ++i) t[l][i] = (kb + i < B) ? th[l * LS + (kb + i < B ? i : 0) * kTile] : 0.0f;
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] -= (t[0][i] + t[1][i]) + t[2][i];     // E_{sigma_i, theta^l_i} = -1
#pragma unroll
      for (int l = 0; l < 3; ++l) {
        double ti[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) ti[i] = (kb + i < B) ? ith[l * LS + (size_t)(kb + i < B ? i : 0) * kTile] : 0.0;
        float u[8];
        if constexpr (HASX) {
          float c[3][3];
#pragma unroll
          for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int q = 0; q < 3; ++q)
              c[x][q] = (q < cnt) ? __ldg(V.cth + (((tile * 3 + l) * 3 + x) * kStressSlots + s0 + q) * kTile + lane)
                                  : 0.0f;
          mix_star(c, u);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) u[i] = 0.0f;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          u[i] = fmaf(-om[l], t[l][i], u[i]) * dtf;                          // E_{theta, theta} = -omega_l
          if (kb + i < B) {
            const size_t o = l * LS + (size_t)(kb + i < B ? i : 0) * kTile;
            th[o] = u[i];
            ith[o] = fma(cw, to_f64<float, L::INT_CVT_LOCAL>(u[i]), ti[i]);
          }
        }
      }
    };
    // VE: one derivative pass (row block PB of the first derivative's passes): rows
    // ROW0 + k of D~^{d+1} from the accumulator chunks, accumulated into I, into the
    // operand (TO_OPA) or the scratch (a first row block, while the second block's pass
    // still reads D~^d)
    auto mix_ve = [&](auto pb, auto to_opa, double cw) {
      constexpr int PB = decltype(pb)::value;
      constexpr bool TO_OPA = decltype(to_opa)::value;
      constexpr int R = tc_rows<N>(PB), R8 = up8(R), ROW0 = tc_row0<N>(PB);
      uint32_t ua[24], ub[24];
      load_chunk(0, R8, ua);
      for_chunk_pairs<R8 / 8, false>([&](int k0, auto odd) {
        uint32_t (&cur)[24] = decltype(odd)::value ? ub : ua;
        uint32_t (&nxt)[24] = decltype(odd)::value ? ua : ub;
        put_chunk(cur);
        if (k0 + 8 < R8) load_chunk(k0 + 8, R8, nxt);
        // I of this chunk's rows, loaded ahead of the anelastic stores
        double iv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = ROW0 + k0 + i;
          iv[i] = (k < B) ? It[(w * B + (k < B ? k : 0)) * kTile + lane] : 0.0;
        }
        __syncthreads();
        float v[8];
        mix_star(sc, v);
        if (w < 6) ve_chunk(ROW0 + k0, v, cw, std::true_type{});
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = ROW0 + k0 + i;
          if (k < B) {
            v[i] *= dtf;
            It[(w * B + k) * kTile + lane] = fma(cw, to_f64<float, L::INT_CVT_LOCAL>(v[i]), iv[i]);
            if constexpr (!TO_OPA) my_scr[(ROW0 + k0 + i) * kRows] = v[i];
          } else {
            v[i] = 0.0f;
          }
        }
        if constexpr (TO_OPA) store_split8(opa, L::OPA_SPLIT, op_offset(my_row, ROW0 + k0, KPA), v);
        if (k0 + 8 < R8) __syncthreads();
      });
    };

    if constexpr (VE) {
      // the rows past the last accumulator chunk (degree N): the stress rows' feedback
      // and the anelastic functions' relaxation only; velocity rows zero
      constexpr int PL = L::SPLIT0 ? 1 : 0;                       // last row block
      constexpr int KS = tc_row0<N>(PL) + up8(tc_rows<N>(PL));    // first row without a chunk
#pragma unroll 1
      for (int d = 0; d < N; ++d) {
        const double cw = dt * T.invfact[d + 1];
        const bool last = d + 1 == N;
        if constexpr (L::SPLIT0) {
          wait_pass(1);
          mix_ve(std::integral_constant<int, 0>{}, std::false_type{}, cw);
          sync_for_mma();
          issue(1);
          wait_pass(last ? L::ND : 0);
          mix_ve(std::integral_constant<int, 1>{}, std::true_type{}, cw);
          static_for<0, kSplitRows / 8>([&](auto cc) {
            constexpr int k0 = decltype(cc)::value * 8;
            float v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = my_scr[(k0 + i) * kRows];
            store_split8(opa, L::OPA_SPLIT, op_offset(my_row, k0, KPA), v);
          });
        } else {
          wait_pass(last ? L::ND : 0);
          mix_ve(std::integral_constant<int, 0>{}, std::true_type{}, cw);
        }
        static_for<0, (up8(B) - KS) / 8>([&](auto cc) {
          constexpr int k0 = KS + decltype(cc)::value * 8;
          float v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = 0.0f;
          if (w < 6) {
            double iv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) iv[i] = (k0 + i < B) ? It[(w * B + (k0 + i < B ? k0 + i : 0)) * kTile + lane] : 0.0;
            ve_chunk(k0, v, cw, std::false_type{});
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              if (k0 + i < B) {
                v[i] *= dtf;
                It[(w * B + (k0 + i < B ? k0 + i : 0)) * kTile + lane] = fma(cw, to_f64<float, L::INT_CVT_LOCAL>(v[i]), iv[i]);
              } else {
                v[i] = 0.0f;
              }
            }
          }
          store_split8(opa, L::OPA_SPLIT, op_offset(my_row, k0, KPA), v);
        });
        if (!last) {
          sync_for_mma();
          issue(0);
        }
      }
    } else {
    static_for<0, N>([&](auto dd) {
      constexpr int DELTA = decltype(dd)::value;
      if constexpr (L::SPLIT0 && DELTA == 0) {
        // first derivative in two row blocks: the first block's rows go to the scratch
        // only, since the second pass still reads D~^0 from the operand; once it is done
        // its rows and then the first block's (from the scratch) go into the operand
        wait_pass(1);
        mix_deriv(std::integral_constant<int, 0>{}, std::false_type{});
        sync_for_mma();
        issue(1);
        wait_pass(2 < L::ND ? 2 : L::ND);
        mix_deriv(std::integral_constant<int, 1>{}, std::true_type{});
        static_for<0, kSplitRows / 8>([&](auto cc) {
          constexpr int k0 = decltype(cc)::value * 8;
          float v[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = my_scr[(tc_srow<N>(1) + k0 + i) * kRows];
          store_split8(opa, L::OPA_SPLIT, op_offset(my_row, k0, KPA), v);
        });
        sync_for_mma();
        if constexpr (2 < L::ND) issue(2);
      } else {
        constexpr int P = DELTA + (L::SPLIT0 ? 1 : 0);   // the pass of this derivative
        wait_pass(P + 1 < L::ND ? P + 1 : L::ND);       // then the next pass's operand
        mix_deriv(std::integral_constant<int, P>{}, std::true_type{});
        sync_for_mma();
        if constexpr (P + 1 < L::ND) issue(P + 1);
      }
    });
    }

    // time integral I = sum_d (dt / (d+1)!) D~^d in binary64: HBM and operand.  All loads
    // of a chunk are issued before its stores (a store to I could alias them otherwise,
    // which serialises every row on the L2 latency).  VE: I is complete; operand only.
    if constexpr (VE) {
      static_for<0, up8(B) / 8>([&](auto cc) {
        constexpr int k0 = decltype(cc)::value * 8;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
          v[i] = (k0 + i < B) ? from_f64<float, L::INT_CVT_LOCAL>(It[(w * B + (k0 + i < B ? k0 + i : 0)) * kTile + lane])
                              : 0.0f;
        store_split8(opa, L::OPA_SPLIT, op_offset(my_row, k0, KPA), v);
      });
    } else
    static_for<0, up8(B) / 8>([&](auto cc) {
      constexpr int k0 = decltype(cc)::value * 8;
      double qv[8];
      float sv[N][8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        qv[i] = (k0 + i < B) ? Qt[(w * B + (k0 + i < B ? k0 + i : 0)) * kTile + lane] : 0.0;
#pragma unroll
        for (int d = 1; d <= N; ++d)
          sv[d - 1][i] = (k0 + i < Dm::nd(d)) ? my_scr[(tc_srow<N>(d) + k0 + i) * kRows] : 0.0f;
      }
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k0 + i;
        if (k < B) {
          double ik = dt * T.invfact[0] * qv[i];
#pragma unroll
          for (int d = 1; d <= N; ++d)
            if (k < Dm::nd(d)) ik = fma(dt * T.invfact[d], to_f64<float, L::INT_WIDEN_TI>(sv[d - 1][i]), ik);
          It[(w * B + k) * kTile + lane] = ik;
          v[i] = from_f64<float, L::INT_CVT_LOCAL>(ik);
        } else {
          v[i] = 0.0f;
        }
      }
      store_split8(opa, L::OPA_SPLIT, op_offset(my_row, k0, KPA), v);
    });
    sync_for_mma();
    issue(L::ND);

    // volume: Q[k][p] += sum_x sum_q Astar^x_pq (Khat^x I)[k][q], row chunks of VR
    static_for<0, NV>([&](auto vv) {
      constexpr int V = decltype(vv)::value;
      constexpr int R = L::vrows(V), R8 = up8(R), KB0 = V * L::VR;
      wait_pass(L::ND + V + 1);       // the next volume pass or the face projections
      uint32_t ua[24], ub[24];
      double qa[8], qb[8];           // VE: Q of chunk c in qa (c even) or qb (c odd), loaded one chunk ahead
      load_chunk(0, R8, ua);
      if constexpr (VE) {
#pragma unroll
        for (int i = 0; i < 8; ++i) qa[i] = (i < R) ? Qt[(w * B + KB0 + (i < R ? i : 0)) * kTile + lane] : 0.0;
      }
      float* Vt = VE ? nullptr : Vol + tile * (kNq * B * kTile);
      for_chunk_pairs<R8 / 8, L::ROLL>([&](int k0, auto odd) {
        constexpr bool ODD = decltype(odd)::value;
        uint32_t (&cur)[24] = ODD ? ub : ua;
        uint32_t (&nxt)[24] = ODD ? ua : ub;
        double (&qc)[8] = ODD ? qb : qa;
        double (&qn)[8] = ODD ? qa : qb;
        put_chunk(cur);
        if (k0 + 8 < R8) {
          load_chunk(k0 + 8, R8, nxt);
          if constexpr (VE) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              qn[i] = (k0 + 8 + i < R) ? Qt[(w * B + KB0 + (k0 + 8 + i < R ? k0 + 8 + i : 0)) * kTile + lane] : 0.0;
          }
        }
        __syncthreads();
        float v[8];
        mix_star(sc, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = KB0 + k0 + i;
          if (k0 + i < R) {
            if constexpr (VE) {
              double src = 0.0;                // (I E^T)_{k, sigma_i} = -sum_l I[k][theta^l_i]
              if (w < 6) {
                const double* ith = It + ((size_t)(9 + w) * B + k) * kTile + lane;
                src = -((ith[0] + ith[LS]) + ith[2 * LS]);
              }
              Qo[(w * B + k) * kTile + lane] = qc[i] + to_f64<float, L::INT_CVT_LOCAL>(v[i]) + src;
            } else {
              Vt[(w * B + k) * kTile + lane] = v[i];
            }
          }
        }
        if (k0 + 8 < R8) __syncthreads();
      });
      fence_before_sync();
      __syncthreads();
      issue(L::ND + V + 1);
    });

    // face projections P^s = R^sT I -> Pface; local flux products W = P^s Aloc_s^T -> Wloc
    // (the flux-solver rows of all four faces are loaded while the pass runs)
    const float* Ft = floc + tile * (4 * kNq * kNq * kTile);
    float af[4][kNq];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int q = 0; q < kNq; ++q) af[f][q] = __ldg(Ft + ((f * kNq + w) * kNq + q) * kTile + lane);
    wait_pass(tile + gridDim.x < ntiles ? 0 : -1);   // then the next tile's first operand
    float* Pe = Pface + (tile * kTile + lane) * (4 * kNq * BT8);
    float* Wt = Wloc + tile * (4 * kNq * BT * kTile);
    static_for<0, 4>([&](auto face) {
      constexpr int s = decltype(face)::value;
      for_chunks<BT8 / 8, L::ROLL>([&](int c) {
        float r[8];
        tmem_ld8(my_tmem + s * BT8 + 8 * c, r);
        float4* pe = reinterpret_cast<float4*>(Pe + (s * kNq + w) * BT8 + 8 * c);
        pe[0] = make_float4(r[0], r[1], r[2], r[3]);
        pe[1] = make_float4(r[4], r[5], r[6], r[7]);
        float4* dst = reinterpret_cast<float4*>(xs) + ((c * kNq + w) * 2) * kTile + lane;
        dst[0] = make_float4(r[0], r[1], r[2], r[3]);
        dst[kTile] = make_float4(r[4], r[5], r[6], r[7]);
      });
      const float (&a)[kNq] = af[s];
      __syncthreads();
      for_chunks<BT8 / 8, L::ROLL>([&](int c) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = 0.0f;
#pragma unroll
        for (int q = 0; q < kNq; ++q) {
          const float4* src = reinterpret_cast<const float4*>(xs) + ((c * kNq + q) * 2) * kTile + lane;
          const float4 x0 = src[0], x1 = src[kTile];
          v[0] = fmaf(a[q], x0.x, v[0]);
          v[1] = fmaf(a[q], x0.y, v[1]);
          v[2] = fmaf(a[q], x0.z, v[2]);
          v[3] = fmaf(a[q], x0.w, v[3]);
          v[4] = fmaf(a[q], x1.x, v[4]);
          v[5] = fmaf(a[q], x1.y, v[5]);
          v[6] = fmaf(a[q], x1.z, v[6]);
          v[7] = fmaf(a[q], x1.w, v[7]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (8 * c + i < BT) Wt[((s * kNq + w) * BT + 8 * c + i) * kTile + lane] = v[i];
      });
      fence_before_sync();
      __syncthreads();
    });
  }
  // after a timeout: one more bounded wait for the pass and the operand load in flight,
  // then free
  if (pending) (void)tc_wait(bar_mma, pending_phase);
  if (ld_out) (void)tc_wait(bar_ld, ld_phase);
  if (!ok && leader) atomicExch(status, kStatusTimeout);
  fence_before_sync();
  __syncthreads();
  if (w == 0) {
    fence_after_sync();
    tmem_free<512>(tmem);
  }
}

// ------------------------------------------------------------------------- K_neigh
// Flux lifting of tiles of 32 elements: W^s = [Wloc^s] + [f^h (R^jT I_nb) Anb_s^T] per
// face (CUDA cores, as k_neigh<N, ..., float>), then Q += sum_s Rhat^s W^s as one
// tensor-core pass with K = the four faces' W stacked (s * BT8 + m).
//   WITH_LOCAL: add the local flux products written by k_local_tc
//   WITH_NEIGH: add the neighbour contributions (gathered face projections)
//   NQT: quantities per element of Q (27: the elastic rows of a 27-quantity step)
template <int N, bool WITH_LOCAL, bool WITH_NEIGH, int NQT = kNq>
__global__ void __launch_bounds__(kRows, 1)
k_neigh_tc(double* Q, const float* __restrict__ Pface, const float* __restrict__ Wloc,
           const float* __restrict__ Vol, const float* __restrict__ fnb, const int* __restrict__ conn,
           const float* __restrict__ fmat, const unsigned char* __restrict__ blob, int64_t ntiles,
           int* __restrict__ status) {
  using L = Layout<N>;
  constexpr int B = L::B, BT = L::BT, BT8 = L::BT8, KPN = L::KPN, NPL = L::NPL, KPE = L::KPE;
  constexpr int NM4 = L::LIFT2 ? (BT + 3) / 4 : BT8 / 4;        // float4 rows of the exchange
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* opa = smem_raw;                                  // [hi | lo] 288 x KPE
  unsigned char* opb = opa + 2 * L::OPN_SPLIT;                    // Rhat operand (K = KPN)
  float* stage = reinterpret_cast<float*>(opb + L::BLOB_N);       // 2 x [9][32][BT8] gathered
  float* xs = stage + 2 * L::STAGE_FLOATS;                        // [NM4][9][32][4]
  TcShared* ts = reinterpret_cast<TcShared*>(xs + L::XSN_FLOATS);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool leader = threadIdx.x == 0;
  const uint32_t bar_ld = smem_u32(&ts->bar[0]), bar_mma = smem_u32(&ts->bar[1]);
  constexpr int NCOLS = (3 * NPL <= 128) ? 128 : ((3 * NPL <= 256) ? 256 : 512);

  for (int i = threadIdx.x; i < 2 * L::OPN_SPLIT / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(opa)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (w == 0) tmem_alloc<NCOLS>(ts);
  if (leader) {
    mbar_init(bar_ld, 1);
    mbar_init(bar_mma, 3);
    mbar_fence_init();
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = ts->tmem;
  const bool issuer = lane == 0 && w < 3;
  if (leader) load_operands(opb, blob, L::BLOB_N, bar_ld);
  bool ok = __syncthreads_and(tc_wait(bar_ld, 0)) != 0;
  uint32_t phase = 0;
  bool pending = false;
  uint32_t pending_phase = 0;
  const int g = group_of(w);
  const uint32_t my_tmem = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(g * NPL);
  const int my_row = op_row(w, lane);
  const uint32_t opa_s = smem_u32(opa), opb_s = smem_u32(opb);

  // lifting pass h: faces h * FH .. of the element operand against their K range of the
  // Rhat operand (LIFT2: two passes of two faces, the second continuing the accumulator)
  constexpr int FH = L::LIFT2 ? 2 : 4;
  auto issue_lift = [&](int h) {
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    if (issuer && ok) {
      fence_after_sync();
      issue_group_k(w, tmem, NPL, opa_s, L::OPN_SPLIT, KPE, opb_s + (uint32_t)(h * (KPE / 8) * 128),
                    NPL * KPN * 2, NPL, KPN, KPE / 16, h > 0, bar_mma);
    }
  };
  auto wait_lift = [&]() {
    const bool was_ok = ok;
    const bool done = was_ok ? tc_wait(bar_mma, phase) : false;
    ok = __syncthreads_and(done) != 0;
    if (was_ok && !ok) {
      pending = true;
      pending_phase = phase;
    }
    phase ^= 1u;
    fence_after_sync();
  };

  for (int64_t tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
    const size_t e = (size_t)tile * kTile + lane;
    const float* Ft = fnb + tile * (4 * kNq * kNq * kTile);
    // the neighbour's projection row (its face j, quantity w) into this thread's column
    // of the face's staging slot; issued one face ahead
    auto prefetch = [&](auto face) {
      constexpr int s = decltype(face)::value;
      const int c = __ldg(conn + e * 4 + s);
      const size_t nb = (size_t)(c >> 7);
      const int j = (c >> 2) & 3;
      const float* P = Pface + ((nb * 4 + j) * kNq + w) * (size_t)BT8;
      float* dst = stage + (s & 1) * L::STAGE_FLOATS + (w * kTile + lane) * BT8;
#pragma unroll
      for (int n = 0; n < BT8; n += 4) cp_async16(dst + n, P + n);
      cp_async_commit();
    };
    if constexpr (WITH_NEIGH) prefetch(std::integral_constant<int, 0>{});
    static_for<0, 4>([&](auto face) {
      constexpr int s = decltype(face)::value;
      // LIFT2: the first two faces' W are in the element operand: their pass runs while
      // the third face's W is formed
      if constexpr (L::LIFT2 && s == 2) issue_lift(0);
      float Wr[BT];
#pragma unroll
      for (int m = 0; m < BT; ++m)
        Wr[m] = WITH_LOCAL ? __ldg(Wloc + ((tile * 4 + s) * kNq * BT + w * BT + m) * kTile + lane) : 0.0f;
      if constexpr (WITH_NEIGH) {
        const int h = __ldg(conn + e * 4 + s) & 3;
        if constexpr (s < 3) {
          prefetch(std::integral_constant<int, s + 1>{});
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        float Pn[BT8];
        const float4* own = reinterpret_cast<const float4*>(stage + (s & 1) * L::STAGE_FLOATS +
                                                            (w * kTile + lane) * BT8);
#pragma unroll
        for (int n4 = 0; n4 < BT8 / 4; ++n4) {
          const float4 t = own[n4];
          Pn[4 * n4] = t.x;
          Pn[4 * n4 + 1] = t.y;
          Pn[4 * n4 + 2] = t.z;
          Pn[4 * n4 + 3] = t.w;
        }
        const float* fh = fmat + (size_t)h * BT * BT;
        // V[m][q] = sum_n f^h_mn Pn[n], f^h block-diagonal by polynomial degree
        float V[BT8];
#pragma unroll
        for (int m = BT; m < BT8; ++m) V[m] = 0.0f;
#pragma unroll
        for (int d = 0; d <= N; ++d) {
          const int lo = d * (d + 1) / 2, hi = (d + 1) * (d + 2) / 2;
#pragma unroll
          for (int m = lo; m < hi; ++m) {
            float v = 0.0f;
#pragma unroll
            for (int n = lo; n < hi; ++n) v = fmaf(__ldg(fh + m + n * BT), Pn[n], v);
            V[m] = v;
          }
        }
        float4* xw = reinterpret_cast<float4*>(xs) + w * kTile + lane;
#pragma unroll
        for (int m4 = 0; m4 < NM4; ++m4)
          xw[m4 * kNq * kTile] = make_float4(V[4 * m4], V[4 * m4 + 1], V[4 * m4 + 2], V[4 * m4 + 3]);
        float a[kNq];
#pragma unroll
        for (int q = 0; q < kNq; ++q) a[q] = __ldg(Ft + ((s * kNq + w) * kNq + q) * kTile + lane);
        __syncthreads();
#pragma unroll
        for (int m4 = 0; m4 < NM4; ++m4) {
#pragma unroll
          for (int q = 0; q < kNq; ++q) {
            const float4 x = reinterpret_cast<const float4*>(xs)[(m4 * kNq + q) * kTile + lane];
            if (4 * m4 < BT) Wr[4 * m4 < BT ? 4 * m4 : 0] = fmaf(a[q], x.x, Wr[4 * m4 < BT ? 4 * m4 : 0]);
            if (4 * m4 + 1 < BT) Wr[4 * m4 + 1 < BT ? 4 * m4 + 1 : 0] = fmaf(a[q], x.y, Wr[4 * m4 + 1 < BT ? 4 * m4 + 1 : 0]);
            if (4 * m4 + 2 < BT) Wr[4 * m4 + 2 < BT ? 4 * m4 + 2 : 0] = fmaf(a[q], x.z, Wr[4 * m4 + 2 < BT ? 4 * m4 + 2 : 0]);
            if (4 * m4 + 3 < BT) Wr[4 * m4 + 3 < BT ? 4 * m4 + 3 : 0] = fmaf(a[q], x.w, Wr[4 * m4 + 3 < BT ? 4 * m4 + 3 : 0]);
          }
        }
        __syncthreads();
      }
      // LIFT2: the element operand is free again once the first pass has completed
      if constexpr (L::LIFT2 && s == 2) wait_lift();
      // W^s into the element operand at K = (s mod FH) * BT8 + m
      static_for<0, BT8 / 8>([&](auto cc) {
        constexpr int c = decltype(cc)::value;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = (8 * c + i < BT) ? Wr[(8 * c + i < BT) ? 8 * c + i : 0] : 0.0f;
        store_split8(opa, L::OPN_SPLIT, op_offset(my_row, (s % FH) * BT8 + 8 * c, KPE), v);
      });
    });
    issue_lift(L::LIFT2 ? 1 : 0);
    wait_lift();
    double* Qt = Q + tile * (NQT * B * kTile);
    // WITH_LOCAL (9 quantities): the local kernel's volume increment joins the lifting in
    // the one binary64 update of Q
    constexpr bool ADD_VOL = WITH_LOCAL && NQT == kNq;
    const float* Vt = ADD_VOL ? Vol + tile * (kNq * B * kTile) : nullptr;
    static_for<0, up8(B) / 8>([&](auto cc) {
      constexpr int k0 = decltype(cc)::value * 8;
      float vv[8];
      if constexpr (ADD_VOL) {
#pragma unroll
        for (int i = 0; i < 8; ++i) vv[i] = (k0 + i < B) ? __ldg(Vt + (w * B + (k0 + i < B ? k0 + i : 0)) * kTile + lane) : 0.0f;
      }
      float r[8];
      tmem_ld8(my_tmem + k0, r);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (k0 + i < B) Qt[(w * B + k0 + i) * kTile + lane] += f2d_int(ADD_VOL ? r[i] + vv[i] : r[i]);
    });
    fence_before_sync();
    __syncthreads();
  }
  if (pending) (void)tc_wait(bar_mma, pending_phase);
  if (!ok && leader) atomicExch(status, kStatusTimeout);
  fence_before_sync();
  __syncthreads();
  if (w == 0) {
    fence_after_sync();
    tmem_free<NCOLS>(tmem);
  }
}

// ------------------------------------------------------------------ launch helpers
struct TcLaunch {
  int64_t ntiles;
  int64_t tile0;             // first tile of the launch (per-tile pointers are offset to it)
  unsigned grid;             // persistent CTAs
  double *Q, *I;
  float *Pface, *Wloc;       // Pface: all elements (k_local_tc writes at tile0 onwards)
  const float *star, *floc, *fnb, *f;
  const int* conn;
  const unsigned char *blob_local, *blob_neigh;
  float* scratch;            // grid x Layout<N>::SROWS x 288 floats
  float* vol;                // [tile][9][B][32] volume increments (9-quantity steps)
  VeTables<float> ve;        // 27-quantity steps: anelastic scratch, star rows, rates
  double dt;
  StarPattern SP;
  int* status;
  int expire_first_wait;     // diagnostics (YT_SCHEME_DIAG_EXPIRE_WAIT)
  cudaStream_t stream;
};

}  // namespace tc

// Entry points of the tensor-core kernels (ader_tc.cu): shared-memory sizes, host
// construction of the split global-matrix operands, attributes and launches.
size_t tc_smem_local(int N);
size_t tc_smem_neigh(int N);
size_t tc_scratch_floats(int N, unsigned grid);
void tc_operands_local(int N, std::vector<unsigned char>& out);
void tc_operands_neigh(int N, std::vector<unsigned char>& out);
void tc_set_attributes(int N);
void tc_launch_local(int N, const tc::TcLaunch& L);
// variant 0: local + neighbour products (fused step), 1: neighbour only, 2: local only
void tc_launch_neigh(int N, const tc::TcLaunch& L, int variant);
// 27-quantity step (ader_tc_ve.cu): k_local_tc<N, true>, then the fused lifting of the
// elastic rows
tc::TcStep tc_step_of(const tc::TcLaunch& L);       // dt and 1/(d+1)! of a launch
void tc_set_attributes_ve(int N);
void tc_launch_local_ve(int N, const tc::TcLaunch& L);
void tc_launch_neigh_ve(int N, const tc::TcLaunch& L);

}  // namespace yt
