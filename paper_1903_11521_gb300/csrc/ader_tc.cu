// Host side of the tensor-core step (precision YT_BF16X3_F32ACC): the split-bf16 global
// matrices in the kernels' canonical shared-memory layout, kernel attributes and
// launches for degrees N = 1..6.
#include <cstring>
#include <vector>

#include "ader_tc.cuh"
#include "common.h"
#include "tables.h"

namespace yt {
namespace {

// bfloat16 by round-to-nearest-even of a binary32 value (finite inputs)
uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

// Entry (n, k) of a pass with N x K = np x kp at byte offset `base`: hi part, then lo.
void put_split(std::vector<unsigned char>& out, int base, int np, int kp, int n, int k, double v) {
  const uint16_t hi = bf16_rn((float)v);
  const uint16_t lo = bf16_rn((float)(v - bf16_value(hi)));
  const size_t o = (size_t)base + tc::op_offset(n, k, kp);
  std::memcpy(&out[o], &hi, 2);
  std::memcpy(&out[o + (size_t)np * kp * 2], &lo, 2);
}

template <int N>
void operands_local(std::vector<unsigned char>& out) {
  using L = tc::Layout<N>;
  const RefMatrices& R = reference_matrices(N);
  const int B = R.B, BT = R.BT;
  out.assign(L::BLOB, 0);
  // CK derivative passes: Ktilde^x of derivative delta restricted to the staircase (rows
  // < nd(delta+1), columns < nd(delta), as in the sparse kernels), each pass holding its
  // block of output rows [row0, row0 + rows) at columns x * r8 + k - row0
  for (int p = 0; p < L::ND; ++p) {
    const int d = tc::tc_delta<N>(p), row0 = tc::tc_row0<N>(p), rows = tc::tc_rows<N>(p);
    const int nin = Dims<N>::nd(d), r8 = L::r8(p);
    for (int x = 0; x < 3; ++x)
      for (int k = row0; k < row0 + rows; ++k)
        for (int l = 0; l < nin; ++l) {
          const double v = R.Ktilde[(size_t)x * B * B + k + (size_t)l * B];
          if (v != 0.0) put_split(out, L::off(p), L::np(p), L::kp(p), x * r8 + (k - row0), l, v);
        }
  }
  // volume: Khat^x, columns l < C(N+2,3) (the others are zero: equivalent sparsity)
  for (int v = 0; v < L::NV; ++v) {
    const int p = L::ND + v, k0 = v * L::VR, r8 = L::r8(p);
    for (int x = 0; x < 3; ++x)
      for (int k = k0; k < k0 + L::vrows(v); ++k)
        for (int l = 0; l < B; ++l) {
          const double val = R.Khat[(size_t)x * B * B + k + (size_t)l * B];
          if (val == 0.0) continue;
          YT_REQUIRE(l < L::NI, YT_ERR_INVALID, "volume matrix outside its zero-block pattern");
          put_split(out, L::off(p), L::np(p), L::kp(p), x * r8 + (k - k0), l, val);
        }
  }
  // face projections R^sT: column s * BT8 + m, K = l
  const int pp = L::ND + L::NV;
  for (int s = 0; s < 4; ++s)
    for (int m = 0; m < BT; ++m)
      for (int l = 0; l < B; ++l) {
        const double v = R.R[(size_t)s * B * BT + l + (size_t)m * B];
        if (v != 0.0) put_split(out, L::off(pp), L::np(pp), L::kp(pp), s * L::BT8 + m, l, v);
      }
}

template <int N>
void operands_neigh(std::vector<unsigned char>& out) {
  using L = tc::Layout<N>;
  const RefMatrices& R = reference_matrices(N);
  const int B = R.B, BT = R.BT;
  out.assign(L::BLOB_N, 0);
  // lifting Rhat^s: column k, K = s * BT8 + m
  for (int s = 0; s < 4; ++s)
    for (int k = 0; k < B; ++k)
      for (int m = 0; m < BT; ++m) {
        const double v = R.Rhat[(size_t)s * B * BT + k + (size_t)m * B];
        if (v != 0.0) put_split(out, 0, L::NPL, L::KPN, k, s * L::BT8 + m, v);
      }
}

template <int N>
void set_attributes() {
  using L = tc::Layout<N>;
  cudaFuncSetAttribute(tc::k_local_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM);
  cudaFuncSetAttribute(tc::k_neigh_tc<N, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM_N);
  cudaFuncSetAttribute(tc::k_neigh_tc<N, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM_N);
  cudaFuncSetAttribute(tc::k_neigh_tc<N, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM_N);
}

}  // namespace

tc::TcStep tc_step_of(const tc::TcLaunch& L) {
  tc::TcStep T;
  T.dt = L.dt;
  T.expire_first_wait = L.expire_first_wait;
  double f = 1.0;
  for (int i = 0; i < 8; ++i) {
    f *= (i + 1.0);
    T.invfact[i] = 1.0 / f;
  }
  return T;
}

namespace {

tc::TcStep step_of(const tc::TcLaunch& L) { return tc_step_of(L); }

template <int N>
void launch_local(const tc::TcLaunch& L) {
  float* P = L.Pface + (size_t)L.tile0 * kTile * 4 * kNq * tc::Layout<N>::BT8;
  tc::k_local_tc<N><<<L.grid, tc::kRows, tc::Layout<N>::SMEM, L.stream>>>(
      L.Q, L.I, P, L.Wloc, L.star, L.floc, L.blob_local, L.scratch, step_of(L), L.SP, VeTables<float>{},
      L.vol, L.ntiles, L.status);
}

template <int N>
void launch_neigh(const tc::TcLaunch& L, int variant) {
  const size_t sm = tc::Layout<N>::SMEM_N;
  if (variant == 0)
    tc::k_neigh_tc<N, true, true><<<L.grid, tc::kRows, sm, L.stream>>>(
        L.Q, L.Pface, L.Wloc, L.vol, L.fnb, L.conn, L.f, L.blob_neigh, L.ntiles, L.status);
  else if (variant == 1)
    tc::k_neigh_tc<N, false, true><<<L.grid, tc::kRows, sm, L.stream>>>(
        L.Q, L.Pface, L.Wloc, L.vol, L.fnb, L.conn, L.f, L.blob_neigh, L.ntiles, L.status);
  else
    tc::k_neigh_tc<N, true, false><<<L.grid, tc::kRows, sm, L.stream>>>(
        L.Q, L.Pface, L.Wloc, L.vol, L.fnb, L.conn, L.f, L.blob_neigh, L.ntiles, L.status);
}

}  // namespace

#define YT_TC_SWITCH(N, CALL)                                                  \
  switch (N) {                                                                 \
    case 1: CALL(1); break;                                                    \
    case 2: CALL(2); break;                                                    \
    case 3: CALL(3); break;                                                    \
    case 4: CALL(4); break;                                                    \
    case 5: CALL(5); break;                                                    \
    case 6: CALL(6); break;                                                    \
    default: throw Error(YT_ERR_UNSUPPORTED, "tensor-core step: orders 2..7"); \
  }

size_t tc_smem_local(int N) {
  size_t r = 0;
#define YT_C(n) r = tc::Layout<n>::SMEM
  YT_TC_SWITCH(N, YT_C);
#undef YT_C
  return r;
}
size_t tc_smem_neigh(int N) {
  size_t r = 0;
#define YT_C(n) r = tc::Layout<n>::SMEM_N
  YT_TC_SWITCH(N, YT_C);
#undef YT_C
  return r;
}
size_t tc_scratch_floats(int N, unsigned grid) {
  size_t r = 0;
#define YT_C(n) r = (size_t)grid * tc::Layout<n>::SROWS * tc::kRows
  YT_TC_SWITCH(N, YT_C);
#undef YT_C
  return r;
}
void tc_operands_local(int N, std::vector<unsigned char>& out) {
#define YT_C(n) operands_local<n>(out)
  YT_TC_SWITCH(N, YT_C);
#undef YT_C
}
void tc_operands_neigh(int N, std::vector<unsigned char>& out) {
#define YT_C(n) operands_neigh<n>(out)
  YT_TC_SWITCH(N, YT_C);
#undef YT_C
}
void tc_set_attributes(int N) {
#define YT_C(n) set_attributes<n>()
  YT_TC_SWITCH(N, YT_C);
#undef YT_C
}
void tc_launch_local(int N, const tc::TcLaunch& L) {
#define YT_C(n) launch_local<n>(L)
  YT_TC_SWITCH(N, YT_C);
#undef YT_C
}
void tc_launch_neigh(int N, const tc::TcLaunch& L, int variant) {
#define YT_C(n) launch_neigh<n>(L, variant)
  YT_TC_SWITCH(N, YT_C);
#undef YT_C
}

}  // namespace yt

// Host-only: the split global-matrix operands of the tensor-core kernels (diagnostics).
extern "C" yt_status yt_tc_operands(int32_t order, int32_t kernel, unsigned char* out, int64_t* bytes) {
  return yt::guarded([&] {
    YT_REQUIRE(bytes, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(order >= 2 && order <= 7, YT_ERR_UNSUPPORTED, "tensor-core operands: orders 2..7");
    YT_REQUIRE(kernel == 0 || kernel == 1, YT_ERR_INVALID, "kernel must be 0 (local) or 1 (neighbour)");
    std::vector<unsigned char> v;
    if (kernel == 0) yt::tc_operands_local(order - 1, v);
    else yt::tc_operands_neigh(order - 1, v);
    *bytes = (int64_t)v.size();
    if (out) std::memcpy(out, v.data(), v.size());
  });
}
