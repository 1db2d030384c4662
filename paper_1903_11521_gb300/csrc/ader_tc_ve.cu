// Host side of the tensor-core form of the 27-quantity (viscoelastic-shaped) step:
// attributes and launches of k_local_tc<N, true> and of the fused lifting of the elastic
// rows (k_neigh_tc<N, true, true, 27>), degrees N = 1..6.  The global-matrix operands
// are those of the elastic form (every derivative uses the first derivative's passes).
#include "ader_tc.cuh"
#include "common.h"

namespace yt {
namespace {

template <int N>
void set_attributes_ve() {
  using L = tc::Layout<N>;
  cudaFuncSetAttribute(tc::k_local_tc<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM);
  cudaFuncSetAttribute(tc::k_neigh_tc<N, true, true, kNqVe>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)L::SMEM_N);
}

template <int N>
void launch_local_ve(const tc::TcLaunch& L) {
  float* P = L.Pface + (size_t)L.tile0 * kTile * 4 * kNq * tc::Layout<N>::BT8;
  tc::k_local_tc<N, true><<<L.grid, tc::kRows, tc::Layout<N>::SMEM, L.stream>>>(
      L.Q, L.I, P, L.Wloc, L.star, L.floc, L.blob_local, L.scratch, tc_step_of(L), L.SP, L.ve, nullptr,
      L.ntiles, L.status);
}

template <int N>
void launch_neigh_ve(const tc::TcLaunch& L) {
  tc::k_neigh_tc<N, true, true, kNqVe><<<L.grid, tc::kRows, tc::Layout<N>::SMEM_N, L.stream>>>(
      L.Q, L.Pface, L.Wloc, nullptr, L.fnb, L.conn, L.f, L.blob_neigh, L.ntiles, L.status);
}

}  // namespace

#define YT_TC_VE_SWITCH(N, CALL)                                                            \
  switch (N) {                                                                              \
    case 1: CALL(1); break;                                                                 \
    case 2: CALL(2); break;                                                                 \
    case 3: CALL(3); break;                                                                 \
    case 4: CALL(4); break;                                                                 \
    case 5: CALL(5); break;                                                                 \
    case 6: CALL(6); break;                                                                 \
    default: throw Error(YT_ERR_UNSUPPORTED, "tensor-core 27-quantity step: orders 2..7");  \
  }

void tc_set_attributes_ve(int N) {
#define YT_C(n) set_attributes_ve<n>()
  YT_TC_VE_SWITCH(N, YT_C);
#undef YT_C
}
void tc_launch_local_ve(int N, const tc::TcLaunch& L) {
#define YT_C(n) launch_local_ve<n>(L)
  YT_TC_VE_SWITCH(N, YT_C);
#undef YT_C
}
void tc_launch_neigh_ve(int N, const tc::TcLaunch& L) {
#define YT_C(n) launch_neigh_ve<n>(L)
  YT_TC_VE_SWITCH(N, YT_C);
#undef YT_C
}

}  // namespace yt
