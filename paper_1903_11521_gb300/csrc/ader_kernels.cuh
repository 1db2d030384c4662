// Device kernels of one elastic ADER-DG step on tetrahedra (Sec. 5.1 of the paper).
//
// Work decomposition.  Elements are processed in tiles of 32.  A CTA has 9 warps: warp w
// owns quantity w (as the column q of the contractions with global matrices, and as the
// row p of the per-element 9x9 star / flux-solver products), lane l owns element l of the
// tile.  Every lane of a warp therefore executes the same sparse loop over the same
// global-matrix non-zeros (warp-uniform control flow, broadcast loads of the global
// values) while its operands differ (its own element).  Products with the per-element
// 9x9 matrices mix the quantities of one element; they exchange data through shared
// memory between the two halves of a contraction.
//
// Data layout in HBM ("element-blocked"): every per-element array is stored as
// [tile][...entries...][32 lanes], so a warp's access to one entry of 32 elements is one
// contiguous 256-byte segment.
//
// Sparse products with the global matrices are straight-line code generated per degree
// (codegen.py): every non-zero of the list is one fma with its value read at a fixed
// offset of the solver's value array and its operand at a fixed shared-memory offset, so
// structural zeros and the equivalent-sparsity zero blocks (Sec. 4.2, 5.1.2) are never
// multiplied:
//   CK derivative delta: Ktilde^x restricted to rows < C(N-delta+2,3), columns
//                        < C(N-delta+3,3) (the derivative staircase);
//   volume:              Khat^x (zero columns l >= C(N+2,3) are absent);
//   face projection:     R^sT (rows m < Btilde, columns l < B);
//   lifting:             Rhat^s (rows k < B, columns m < Btilde);
//   orientation:         f^h (dense block-diagonal by polynomial degree, per lane).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace yt {

namespace gen {
// Row<N, LIST, ROW>::dot(v, x) = sum over the non-zeros (l, value offset o) of row ROW of
// sparse list LIST of v[o] * x[l * 9 * 32]; specialisations are generated per degree N
// (codegen.py) with every non-zero unrolled.  Lists: 3*delta + x = derivative delta,
// direction x; 18 + x = volume Khat^x; 21 + s = R^sT; 25 + s = Rhat^s.
template <int N, int LIST, int ROW>
struct Row;
}  // namespace gen

template <int Begin, int End, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  if constexpr (Begin < End) {
    f(std::integral_constant<int, Begin>{});
    static_for<Begin + 1, End>(f);
  }
}

constexpr int kTile = 32;
constexpr int kNq = 9;
constexpr int kStarSlots = 24;

// Non-zero slots of every star matrix: the union of the patterns of A, B and C of the
// velocity-stress system; slots are grouped by row p.
struct StarPattern {
  int start[kNq + 1];
  int col[kStarSlots];
};

template <int N>
struct Dims {
  static constexpr int B = (N + 1) * (N + 2) * (N + 3) / 6;
  static constexpr int BT = (N + 1) * (N + 2) / 2;
  static constexpr int BM = N * (N + 1) * (N + 2) / 6;
  static constexpr int KC = (BT / 3) > 0 ? (BT / 3) : 1;  // rows per mixing chunk
  static constexpr int XR = (3 * KC > BT) ? 3 * KC : BT;  // rows of the exchange buffer
  __host__ __device__ static constexpr int nd(int delta) {
    return (N - delta + 3) * (N - delta + 2) * (N - delta + 1) / 6;
  }
};

// Offsets of the CSR lists in the table buffers (all row-pointer arrays share `rp`).
struct StepTables {
  const int* rp;
  const uint16_t* col;
  const double* val;
  const double* f;      // 3 x BT x BT dense, column-major (f[h][m + n*BT])
  int ck[6][3];         // rp offset of the CK list for derivative delta, direction x
  int vol[3];
  int rT[4];
  int rhat[4];
  double coeff[8];      // dt^{d+1} / (d+1)!
};

// ------------------------------------------------------------------- CK derivatives
// One derivative step delta -> delta+1, in place in Dsh (see the degree argument in the
// solver's design notes: output row k only reads rows of higher polynomial degree, which
// are overwritten later), accumulating the time integral in registers.
template <int N, int DELTA>
__device__ __forceinline__ void ck_step(const StepTables& T, const int (&scol)[3], int cnt,
                                        double* __restrict__ Dsh, double* __restrict__ Xsh,
                                        const double (&sc)[3][3], double (&Icol)[Dims<N>::B],
                                        int w, int lane) {
  using Dm = Dims<N>;
  if constexpr (DELTA < N) {
    constexpr int nout = Dm::nd(DELTA + 1);
    constexpr int KC = Dm::KC;
    const double* xcol = Dsh + w * kTile + lane;
    static_for<0, (nout + KC - 1) / KC>([&](auto chunk) {
      constexpr int k0 = decltype(chunk)::value * KC;
      // X^x[k][q] = sum_l Ktilde^x_kl D[l][q]  (this thread: column q = w)
      static_for<0, KC>([&](auto kkc) {
        constexpr int kk = decltype(kkc)::value;
        if constexpr (k0 + kk < nout) {
          Xsh[((0 * KC + kk) * kNq + w) * kTile + lane] = gen::Row<N, DELTA * 3 + 0, k0 + kk>::dot(T.val, xcol);
          Xsh[((1 * KC + kk) * kNq + w) * kTile + lane] = gen::Row<N, DELTA * 3 + 1, k0 + kk>::dot(T.val, xcol);
          Xsh[((2 * KC + kk) * kNq + w) * kTile + lane] = gen::Row<N, DELTA * 3 + 2, k0 + kk>::dot(T.val, xcol);
        }
      });
      __syncthreads();
      // D^{delta+1}[k][p] = sum_x sum_q Astar^x_pq X^x[k][q]  (this thread: row p = w)
      static_for<0, KC>([&](auto kkc) {
        constexpr int kk = decltype(kkc)::value;
        if constexpr (k0 + kk < nout) {
          double v = 0.0;
#pragma unroll
          for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int s = 0; s < 3; ++s)
              if (s < cnt) v = fma(sc[x][s], Xsh[((x * KC + kk) * kNq + scol[s]) * kTile + lane], v);
          Dsh[((k0 + kk) * kNq + w) * kTile + lane] = v;
          Icol[k0 + kk] = fma(T.coeff[DELTA + 1], v, Icol[k0 + kk]);
        }
      });
      __syncthreads();
    });
    ck_step<N, DELTA + 1>(T, scol, cnt, Dsh, Xsh, sc, Icol, w, lane);
  }
}

// ------------------------------------------------------------------------- K_local
// Derivatives, time integral, volume and local flux of one tile of 32 elements.
//   Q, Qout : [tile][9][B][32]   (may alias)
//   Iout    : [tile][9][B][32]
//   Pface   : [tile][4][9][BT][32]   projections R^sT I of the four faces
//   star    : [tile][3][24][32]      non-zero slots of Astar^x
//   floc    : [tile][4][9][9][32]    local flux solvers (row p, column q)
//   Wloc    : [tile][4][9][BT][32]   (R^sT I) Aloc_s^T per face, written when LIFT is
//                                    false (the full step lifts it together with the
//                                    neighbour contribution in k_neigh)
// LIFT = true applies the local flux here (Q is then the complete local update).
template <int N, bool LIFT>
__global__ void __launch_bounds__(kNq * kTile, 1)
k_local(const double* Q, double* Qout, double* __restrict__ Iout,
        double* __restrict__ Pface, double* __restrict__ Wloc, const double* __restrict__ star,
        const double* __restrict__ floc, StepTables T, StarPattern SP) {
  using Dm = Dims<N>;
  constexpr int B = Dm::B, BT = Dm::BT, KC = Dm::KC;
  extern __shared__ double smem[];
  double* Dsh = smem;                           // B rows x 9 x 32
  double* Xsh = smem + B * kNq * kTile;         // XR rows x 9 x 32
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const size_t tile = blockIdx.x;
  const double* Qt = Q + tile * (kNq * B * kTile);

  // star coefficients of row p = w
  const int s0 = SP.start[w], cnt = SP.start[w + 1] - s0;
  int scol[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) scol[s] = (s < cnt) ? SP.col[s0 + s] : 0;
  double sc[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int s = 0; s < 3; ++s)
      sc[x][s] = (s < cnt) ? __ldg(star + ((tile * 3 + x) * kStarSlots + s0 + s) * kTile + lane) : 0.0;

  double Icol[B];
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const double q = __ldg(Qt + (w * B + k) * kTile + lane);
    Dsh[(k * kNq + w) * kTile + lane] = q;
    Icol[k] = T.coeff[0] * q;
  }
  // (own column only is read before the first barrier)
  ck_step<N, 0>(T, scol, cnt, Dsh, Xsh, sc, Icol, w, lane);

  // publish I: shared (own column) and HBM
  double* It = Iout + tile * (kNq * B * kTile);
#pragma unroll
  for (int k = 0; k < B; ++k) {
    Dsh[(k * kNq + w) * kTile + lane] = Icol[k];
    It[(w * B + k) * kTile + lane] = Icol[k];
  }

  // With LIFT the local flux is added to every row after the volume term, so the update
  // is accumulated in registers; without it the volume term completes each row of Q,
  // which is written as soon as its chunk is done.
  double dQ[LIFT ? B : 1];
  double* Qo = Qout + tile * (kNq * B * kTile);

  // volume: dQ[k][p] += sum_x sum_q Astar^x_pq (Khat^x I)[k][q]
  const double* icol = Dsh + w * kTile + lane;
  static_for<0, (B + KC - 1) / KC>([&](auto chunk) {
    constexpr int k0 = decltype(chunk)::value * KC;
    static_for<0, KC>([&](auto kkc) {
      constexpr int kk = decltype(kkc)::value;
      if constexpr (k0 + kk < B) {
        Xsh[((0 * KC + kk) * kNq + w) * kTile + lane] = gen::Row<N, 18, k0 + kk>::dot(T.val, icol);
        Xsh[((1 * KC + kk) * kNq + w) * kTile + lane] = gen::Row<N, 19, k0 + kk>::dot(T.val, icol);
        Xsh[((2 * KC + kk) * kNq + w) * kTile + lane] = gen::Row<N, 20, k0 + kk>::dot(T.val, icol);
      }
    });
    __syncthreads();
    static_for<0, KC>([&](auto kkc) {
      constexpr int kk = decltype(kkc)::value;
      if constexpr (k0 + kk < B) {
        constexpr int k = k0 + kk;
        double v = 0.0;
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
          for (int s = 0; s < 3; ++s)
            if (s < cnt) v = fma(sc[x][s], Xsh[((x * KC + kk) * kNq + scol[s]) * kTile + lane], v);
        if constexpr (LIFT) dQ[k] = v;
        else Qo[(w * B + k) * kTile + lane] = Qt[(w * B + k) * kTile + lane] + v;
      }
    });
    __syncthreads();
  });

  // local flux: dQ += Rhat^s ((R^sT I) Aloc_s^T)
  double* Pt = Pface + tile * (4 * kNq * BT * kTile);
  const double* Ft = floc + tile * (4 * kNq * kNq * kTile);
  static_for<0, 4>([&](auto face) {
    constexpr int s = decltype(face)::value;
    static_for<0, BT>([&](auto mm) {
      constexpr int m = decltype(mm)::value;
      const double z = gen::Row<N, 21 + s, m>::dot(T.val, icol);
      Xsh[(m * kNq + w) * kTile + lane] = z;
      Pt[((s * kNq + w) * BT + m) * kTile + lane] = z;
    });
    double a[kNq];
#pragma unroll
    for (int q = 0; q < kNq; ++q) a[q] = __ldg(Ft + ((s * kNq + w) * kNq + q) * kTile + lane);
    __syncthreads();
    double Wr[BT];
#pragma unroll
    for (int m = 0; m < BT; ++m) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < kNq; ++q) v = fma(a[q], Xsh[(m * kNq + q) * kTile + lane], v);
      Wr[m] = v;
    }
    __syncthreads();
    if constexpr (LIFT) {
#pragma unroll
      for (int m = 0; m < BT; ++m) Xsh[(m * kNq + w) * kTile + lane] = Wr[m];
      const double* wcol = Xsh + w * kTile + lane;
      static_for<0, B>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        dQ[k] += gen::Row<N, 25 + s, k>::dot(T.val, wcol);
      });
    } else {
      double* Wt = Wloc + tile * (4 * kNq * BT * kTile);
#pragma unroll
      for (int m = 0; m < BT; ++m) Wt[((s * kNq + w) * BT + m) * kTile + lane] = Wr[m];
    }
  });

  if constexpr (LIFT) {
#pragma unroll
    for (int k = 0; k < B; ++k) Qo[(w * B + k) * kTile + lane] = Qt[(w * B + k) * kTile + lane] + dQ[k];
  }
}

// ------------------------------------------------------------------------- K_neigh
// Neighbour flux of one tile: dQ += Rhat^s f^h (R^jT I_nb) Anb_s^T, with R^jT I_nb read
// from the neighbour's face projections written by k_local.
//   conn : [E_pad][4] packed (neighbour << 4) | (j << 2) | h
// WITH_LOCAL: add the local flux terms Wloc written by k_local<N, false> before lifting,
// so that Rhat^s is applied once per face to the sum of both flux contributions.
template <int N, bool WITH_LOCAL>
__global__ void __launch_bounds__(kNq * kTile, 1)
k_neigh(double* Q, const double* __restrict__ Pface, const double* __restrict__ Wloc,
        const double* __restrict__ fnb, const int* __restrict__ conn, StepTables T) {
  using Dm = Dims<N>;
  constexpr int B = Dm::B, BT = Dm::BT;
  extern __shared__ double smem[];
  double* Xsh = smem;                           // BT rows x 9 x 32
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const size_t tile = blockIdx.x;
  const size_t e = tile * kTile + lane;

  double dQ[B];
#pragma unroll
  for (int k = 0; k < B; ++k) dQ[k] = 0.0;
  const double* Ft = fnb + tile * (4 * kNq * kNq * kTile);

  static_for<0, 4>([&](auto face) {
    constexpr int s = decltype(face)::value;
    const int c = __ldg(conn + e * 4 + s);
    const size_t nb = (size_t)(c >> 4);
    const int j = (c >> 2) & 3, h = c & 3;
    const double* P = Pface + ((((nb / kTile) * 4 + j) * kNq + w) * BT) * kTile + (nb % kTile);
    double Pn[BT];
#pragma unroll
    for (int n = 0; n < BT; ++n) Pn[n] = __ldg(P + n * kTile);
    const double* fh = T.f + (size_t)h * BT * BT;
    // V[m][q] = sum_n f^h_mn Pn[n], f^h block-diagonal by polynomial degree
#pragma unroll
    for (int d = 0; d <= N; ++d) {
      const int lo = d * (d + 1) / 2, hi = (d + 1) * (d + 2) / 2;
#pragma unroll
      for (int m = lo; m < hi; ++m) {
        double v = 0.0;
#pragma unroll
        for (int n = lo; n < hi; ++n) v = fma(__ldg(fh + m + n * BT), Pn[n], v);
        Xsh[(m * kNq + w) * kTile + lane] = v;
      }
    }
    double a[kNq];
#pragma unroll
    for (int q = 0; q < kNq; ++q) a[q] = __ldg(Ft + ((s * kNq + w) * kNq + q) * kTile + lane);
    __syncthreads();
    double Wr[BT];
#pragma unroll
    for (int m = 0; m < BT; ++m) {
      double v = 0.0;
      if constexpr (WITH_LOCAL) v = __ldg(Wloc + ((tile * 4 + s) * kNq * BT + w * BT + m) * kTile + lane);
#pragma unroll
      for (int q = 0; q < kNq; ++q) v = fma(a[q], Xsh[(m * kNq + q) * kTile + lane], v);
      Wr[m] = v;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < BT; ++m) Xsh[(m * kNq + w) * kTile + lane] = Wr[m];
    const double* wcol = Xsh + w * kTile + lane;
    static_for<0, B>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      dQ[k] += gen::Row<N, 25 + s, k>::dot(T.val, wcol);
    });
  });
  double* Qt = Q + tile * (kNq * B * kTile);
#pragma unroll
  for (int k = 0; k < B; ++k) Qt[(w * B + k) * kTile + lane] += dQ[k];
}

// ------------------------------------------------------------------ launch helpers
struct AderLaunch {
  int64_t ntiles;
  size_t smem_local, smem_neigh;
  double *Q, *I, *Pface, *Wloc;
  const double *star, *floc, *fnb;
  const int* conn;
  StepTables T;
  StarPattern SP;
  cudaStream_t stream;
};

template <int N>
void ader_set_attributes(size_t smem_local, size_t smem_neigh) {
  cudaFuncSetAttribute(k_local<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_local);
  cudaFuncSetAttribute(k_local<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_local);
  cudaFuncSetAttribute(k_neigh<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_neigh);
  cudaFuncSetAttribute(k_neigh<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_neigh);
}

// fused = true: the local half of the full step (local flux lifted in k_neigh)
template <int N>
void ader_launch_local(const AderLaunch& L, bool fused) {
  const unsigned grid = (unsigned)L.ntiles;
  if (fused)
    k_local<N, false><<<grid, kNq * kTile, L.smem_local, L.stream>>>(L.Q, L.Q, L.I, L.Pface, L.Wloc,
                                                                       L.star, L.floc, L.T, L.SP);
  else
    k_local<N, true><<<grid, kNq * kTile, L.smem_local, L.stream>>>(L.Q, L.Q, L.I, L.Pface, L.Wloc,
                                                                      L.star, L.floc, L.T, L.SP);
}

template <int N>
void ader_launch_neigh(const AderLaunch& L, bool fused) {
  const unsigned grid = (unsigned)L.ntiles;
  if (fused)
    k_neigh<N, true><<<grid, kNq * kTile, L.smem_neigh, L.stream>>>(L.Q, L.Pface, L.Wloc, L.fnb,
                                                                      L.conn, L.T);
  else
    k_neigh<N, false><<<grid, kNq * kTile, L.smem_neigh, L.stream>>>(L.Q, L.Pface, L.Wloc, L.fnb,
                                                                       L.conn, L.T);
}

// per-degree instantiations live in generated translation units
void ader_set_attributes_o1(size_t, size_t);
void ader_set_attributes_o2(size_t, size_t);
void ader_set_attributes_o3(size_t, size_t);
void ader_set_attributes_o4(size_t, size_t);
void ader_set_attributes_o5(size_t, size_t);
void ader_launch_local_o1(const AderLaunch&, bool);
void ader_launch_local_o2(const AderLaunch&, bool);
void ader_launch_local_o3(const AderLaunch&, bool);
void ader_launch_local_o4(const AderLaunch&, bool);
void ader_launch_local_o5(const AderLaunch&, bool);
void ader_launch_neigh_o1(const AderLaunch&, bool);
void ader_launch_neigh_o2(const AderLaunch&, bool);
void ader_launch_neigh_o3(const AderLaunch&, bool);
void ader_launch_neigh_o4(const AderLaunch&, bool);
void ader_launch_neigh_o5(const AderLaunch&, bool);
int ader_generated_nnz_o1();
int ader_generated_nnz_o2();
int ader_generated_nnz_o3();
int ader_generated_nnz_o4();
int ader_generated_nnz_o5();

}  // namespace yt
