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
// contiguous segment.
//
// Precision: Real is the type of the bulk contractions (double, or float for the
// precision form).  The DOFs Q, the time integral I and its accumulation over the
// derivatives stay in double in both cases; the star matrices and flux solvers are set up
// in double and stored as Real.
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

#include "fp_convert.cuh"

namespace yt {

// Conversions between the contraction type and binary64: identities for double; for
// float either the hardware conversions or the integer-unit ones of fp_convert.cuh (INT),
// which leave the FP64 pipe (the scarce resource of these kernels' binary64 parts) to the
// arithmetic but cost registers: the kernels use them where they compile without spills.
template <typename Real, bool INT>
__device__ __forceinline__ double to_f64(Real x) {
  if constexpr (sizeof(Real) == 4 && INT) return f2d_int(x);
  else return (double)x;
}
template <typename Real, bool INT>
__device__ __forceinline__ Real from_f64(double x) {
  if constexpr (sizeof(Real) == 4 && INT) return d2f_int(x);
  else return (Real)x;
}

// Resident CTAs per SM requested from the compiler (__launch_bounds__): the FP64 kernels
// run one 9-warp CTA per SM (168 registers); the FP32 neighbour kernels and the FP32
// local kernels of degree <= 4 fit 96 registers without spilling and run two CTAs per SM
// (18 warps) to hide shared-memory and dependency latency.
template <int N, typename Real, bool LOCAL>
struct MinBlocks {
  static constexpr int value = (sizeof(Real) == 4 && (!LOCAL || N <= 4)) ? 2 : 1;
  // integer-unit conversions where they fit the registers (the two-CTA variants)
  static constexpr bool int_cvt = value == 2;
};

namespace gen {
// Row<N, LIST, ROW>::dot<Real>(v, x) = sum over the non-zeros (l, value offset o) of row
// ROW of sparse list LIST of v[o] * x[l * 9 * 32]; specialisations are generated per
// degree N (codegen.py) with every non-zero unrolled.  Lists: 3*delta + x = derivative
// delta, direction x; 18 + x = volume Khat^x; 21 + s = R^sT; 25 + s = Rhat^s.
template <int N, int LIST, int ROW>
struct Row;
}  // namespace gen

// Sparse row of a list.  FP64: one accumulator chain (Row::dot1; the FP64 pipe is the
// limit and nine warps supply enough independent chains, while every extra accumulator
// costs an add to combine).  FP32: four accumulators (Row::dot; latency is the limit),
// values of degrees <= 5 from constant memory (Row::dotc, one constant-bank operand per
// fma).  row_dot_acc continues an accumulation (one chain across several rows in FP64).
template <int N, int LIST, int ROW, typename Real>
__device__ __forceinline__ Real row_dot(const Real* __restrict__ v, const Real* __restrict__ x) {
  if constexpr (sizeof(Real) == 8)
    return gen::Row<N, LIST, ROW>::dot1(v, x, Real(0));
  else if constexpr (N <= 5)
    return gen::Row<N, LIST, ROW>::dotc(x);
  else
    return gen::Row<N, LIST, ROW>::dot(v, x);
}
template <int N, int LIST, int ROW, typename Real>
__device__ __forceinline__ Real row_dot_acc(const Real* __restrict__ v, const Real* __restrict__ x, Real a) {
  if constexpr (sizeof(Real) == 8)
    return gen::Row<N, LIST, ROW>::dot1(v, x, a);
  else
    return a + row_dot<N, LIST, ROW, Real>(v, x);
}

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

// Face projections of the element groups a neighbour may belong to (one group per
// polynomial degree in a p-adaptive mesh; a single group otherwise): base pointer of the
// group's [element][4][9][BT] array and its face-basis size BT.
constexpr int kMaxGroups = 8;
struct FaceGroups {
  const void* base[kMaxGroups];
  int bt[kMaxGroups];
};

// Global data of the step: the packed non-zero values of the sparse lists, the f^h
// matrices (3 x BT x BT, column-major f[h][m + n*BT]), the time step and 1/(d+1)!.
// The derivatives are carried scaled, D~^d = dt^d D^d:
// D~^{d+1} = dt sum_x Ktilde^x D~^d Astar^xT (the factor dt is applied to each mixed
// row), and I = sum_d (dt / (d+1)!) D~^d = sum_d dt^{d+1}/(d+1)! D^d.  Magnitudes of D~
// stay near those of Q (by the CFL condition), which keeps FP32 clear of overflow.
template <typename Real>
struct StepTables {
  const Real* val;
  const Real* f;
  double dt;
  double invfact[8];
};

// One CTA's tile in a launch shared by several independent problems (serving): the
// problem's buffers, the tile's index within them and the problem's time step.  With a
// null table a launch covers one problem, tile = blockIdx.x.
struct TileRef {
  double* Q;
  double* I;
  void* Pface;
  void* Wloc;
  const void* star;
  const void* floc;
  const void* fnb;
  const int* conn;
  int64_t tile;
  double dt;
};

// ------------------------------------------------------------------- CK derivatives
// One derivative step delta -> delta+1, in place in Dsh: output row k only reads rows of
// strictly higher polynomial degree (K~_kl != 0 only if deg phi_k < deg phi_l), so rows
// processed in increasing order overwrite rows that are no longer needed.  The time
// integral accumulates in double registers; only the C(N+2,3) rows that receive
// derivative terms need one (rows of degree N hold c0 Q alone).
template <int N, int DELTA, typename Real>
__device__ __forceinline__ void ck_step(const StepTables<Real>& T, double dt, const int (&scol)[3], int cnt,
                                        Real* __restrict__ Dsh, Real* __restrict__ Xsh,
                                        const Real (&sc)[3][3], double (&Icol)[Dims<N>::nd(1)],
                                        int w, int lane) {
  using Dm = Dims<N>;
  if constexpr (DELTA < N) {
    constexpr int nout = Dm::nd(DELTA + 1);
    constexpr int KC = Dm::KC;
    const Real* xcol = Dsh + w * kTile + lane;
    const Real dtr = (Real)dt;
    static_for<0, (nout + KC - 1) / KC>([&](auto chunk) {
      constexpr int k0 = decltype(chunk)::value * KC;
      // X^x[k][q] = sum_l Ktilde^x_kl D[l][q]  (this thread: column q = w)
      static_for<0, KC>([&](auto kkc) {
        constexpr int kk = decltype(kkc)::value;
        if constexpr (k0 + kk < nout) {
          Xsh[((0 * KC + kk) * kNq + w) * kTile + lane] = row_dot<N, DELTA * 3 + 0, k0 + kk>(T.val, xcol);
          Xsh[((1 * KC + kk) * kNq + w) * kTile + lane] = row_dot<N, DELTA * 3 + 1, k0 + kk>(T.val, xcol);
          Xsh[((2 * KC + kk) * kNq + w) * kTile + lane] = row_dot<N, DELTA * 3 + 2, k0 + kk>(T.val, xcol);
        }
      });
      __syncthreads();
      // D^{delta+1}[k][p] = sum_x sum_q Astar^x_pq X^x[k][q]  (this thread: row p = w)
      static_for<0, KC>([&](auto kkc) {
        constexpr int kk = decltype(kkc)::value;
        if constexpr (k0 + kk < nout) {
          Real v = Real(0);
#pragma unroll
          for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int s = 0; s < 3; ++s)
              if (s < cnt) v = fma(sc[x][s], Xsh[((x * KC + kk) * kNq + scol[s]) * kTile + lane], v);
          v *= dtr;
          Dsh[((k0 + kk) * kNq + w) * kTile + lane] = v;
          Icol[k0 + kk] = fma(dt * T.invfact[DELTA + 1], to_f64<Real, MinBlocks<N, Real, true>::int_cvt>(v),
                              Icol[k0 + kk]);
        }
      });
      __syncthreads();
    });
    ck_step<N, DELTA + 1, Real>(T, dt, scol, cnt, Dsh, Xsh, sc, Icol, w, lane);
  }
}

// ------------------------------------------------------------------------- K_local
// Derivatives, time integral, volume and local flux of one tile of 32 elements.
//   Q, Qout : [tile][9][B][32] double   (may alias)
//   Iout    : [tile][9][B][32] double
//   Pface   : [element][4][9][BT]       projections R^sT I of the four faces, contiguous per
//                                       element so that a neighbour's face block is read
//                                       whole (the only per-element array gathered at random)
//   star    : [tile][3][24][32]         non-zero slots of Astar^x
//   floc    : [tile][4][9][9][32]       local flux solvers (row p, column q)
//   Wloc    : [tile][4][9][BT][32]      (R^sT I) Aloc_s^T per face, written when LIFT is
//                                       false (the full step lifts it together with the
//                                       neighbour contribution in k_neigh)
// LIFT = true applies the local flux here (Q is then the complete local update).
template <int N, bool LIFT, typename Real>
__global__ void __launch_bounds__(kNq * kTile, (MinBlocks<N, Real, true>::value))
k_local(const double* Q, double* Qout, double* Iout, Real* Pface, Real* Wloc, const Real* star,
        const Real* floc, StepTables<Real> T, StarPattern SP, const TileRef* __restrict__ refs) {
  using Dm = Dims<N>;
  constexpr int B = Dm::B, BT = Dm::BT, KC = Dm::KC;
  constexpr bool CVT = MinBlocks<N, Real, true>::int_cvt;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Dsh = reinterpret_cast<Real*>(smem_raw);  // B rows x 9 x 32
  Real* Xsh = Dsh + B * kNq * kTile;               // XR rows x 9 x 32
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  size_t tile = blockIdx.x;
  double dt = T.dt;
  if (refs) {
    const TileRef& r = refs[blockIdx.x];
    Q = r.Q;
    Qout = r.Q;
    Iout = r.I;
    Pface = static_cast<Real*>(r.Pface);
    Wloc = static_cast<Real*>(r.Wloc);
    star = static_cast<const Real*>(r.star);
    floc = static_cast<const Real*>(r.floc);
    tile = (size_t)r.tile;
    dt = r.dt;
  }
  const double* Qt = Q + tile * (kNq * B * kTile);

  // star coefficients of row p = w
  const int s0 = SP.start[w], cnt = SP.start[w + 1] - s0;
  int scol[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) scol[s] = (s < cnt) ? SP.col[s0 + s] : 0;
  Real sc[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int s = 0; s < 3; ++s)
      sc[x][s] = (s < cnt) ? __ldg(star + ((tile * 3 + x) * kStarSlots + s0 + s) * kTile + lane) : Real(0);

  constexpr int NI = Dm::nd(1);
  double Icol[NI];
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const double q = __ldg(Qt + (w * B + k) * kTile + lane);
    Dsh[(k * kNq + w) * kTile + lane] = from_f64<Real, CVT>(q);
    if (k < NI) Icol[k < NI ? k : 0] = dt * T.invfact[0] * q;
  }
  // (own column only is read before the first barrier)
  ck_step<N, 0, Real>(T, dt, scol, cnt, Dsh, Xsh, sc, Icol, w, lane);

  // publish I: shared (own column) and HBM
  double* It = Iout + tile * (kNq * B * kTile);
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const double ik = k < NI ? Icol[k < NI ? k : 0] : dt * T.invfact[0] * Qt[(w * B + k) * kTile + lane];
    Dsh[(k * kNq + w) * kTile + lane] = from_f64<Real, CVT>(ik);
    It[(w * B + k) * kTile + lane] = ik;
  }

  // The volume term is added to each row of Q as soon as its chunk is done; with LIFT the
  // local flux is then added face by face (every row of an element column belongs to
  // one thread, so these read-modify-writes need no synchronisation).
  double* Qo = Qout + tile * (kNq * B * kTile);

  // volume: dQ[k][p] += sum_x sum_q Astar^x_pq (Khat^x I)[k][q]
  const Real* icol = Dsh + w * kTile + lane;
  static_for<0, (B + KC - 1) / KC>([&](auto chunk) {
    constexpr int k0 = decltype(chunk)::value * KC;
    static_for<0, KC>([&](auto kkc) {
      constexpr int kk = decltype(kkc)::value;
      if constexpr (k0 + kk < B) {
        Xsh[((0 * KC + kk) * kNq + w) * kTile + lane] = row_dot<N, 18, k0 + kk>(T.val, icol);
        Xsh[((1 * KC + kk) * kNq + w) * kTile + lane] = row_dot<N, 19, k0 + kk>(T.val, icol);
        Xsh[((2 * KC + kk) * kNq + w) * kTile + lane] = row_dot<N, 20, k0 + kk>(T.val, icol);
      }
    });
    __syncthreads();
    static_for<0, KC>([&](auto kkc) {
      constexpr int kk = decltype(kkc)::value;
      if constexpr (k0 + kk < B) {
        constexpr int k = k0 + kk;
        Real v = Real(0);
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
          for (int s = 0; s < 3; ++s)
            if (s < cnt) v = fma(sc[x][s], Xsh[((x * KC + kk) * kNq + scol[s]) * kTile + lane], v);
        Qo[(w * B + k) * kTile + lane] = Qt[(w * B + k) * kTile + lane] + to_f64<Real, CVT>(v);
      }
    });
    __syncthreads();
  });

  // local flux: dQ += Rhat^s ((R^sT I) Aloc_s^T)
  Real* Pt = Pface + (tile * kTile + lane) * (4 * kNq * BT);
  const Real* Ft = floc + tile * (4 * kNq * kNq * kTile);
  static_for<0, 4>([&](auto face) {
    constexpr int s = decltype(face)::value;
    static_for<0, BT>([&](auto mm) {
      constexpr int m = decltype(mm)::value;
      const Real z = row_dot<N, 21 + s, m>(T.val, icol);
      Xsh[(m * kNq + w) * kTile + lane] = z;
      Pt[(s * kNq + w) * BT + m] = z;
    });
    Real a[kNq];
#pragma unroll
    for (int q = 0; q < kNq; ++q) a[q] = __ldg(Ft + ((s * kNq + w) * kNq + q) * kTile + lane);
    __syncthreads();
    Real Wr[BT];
#pragma unroll
    for (int m = 0; m < BT; ++m) {
      Real v = Real(0);
#pragma unroll
      for (int q = 0; q < kNq; ++q) v = fma(a[q], Xsh[(m * kNq + q) * kTile + lane], v);
      Wr[m] = v;
    }
    __syncthreads();
    if constexpr (LIFT) {
#pragma unroll
      for (int m = 0; m < BT; ++m) Xsh[(m * kNq + w) * kTile + lane] = Wr[m];
      const Real* wcol = Xsh + w * kTile + lane;
      static_for<0, B>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        Qo[(w * B + k) * kTile + lane] += to_f64<Real, CVT>(row_dot<N, 25 + s, k>(T.val, wcol));
      });
    } else {
      Real* Wt = Wloc + tile * (4 * kNq * BT * kTile);
#pragma unroll
      for (int m = 0; m < BT; ++m) Wt[((s * kNq + w) * BT + m) * kTile + lane] = Wr[m];
    }
  });

}

// ------------------------------------------------------------- asynchronous copies
// Global -> shared copy of one element (4 or 8 bytes) that bypasses the registers
// (cp.async), grouped and waited for per face.
template <typename Real>
__device__ __forceinline__ void cp_async_elem(Real* dst_shared, const Real* src_global) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(dst_shared);
  if constexpr (sizeof(Real) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src_global) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src_global) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory"); }

// ------------------------------------------------------------------------- K_neigh
// Neighbour flux of one tile: dQ += Rhat^s f^h (R^jT I_nb) Anb_s^T, with R^jT I_nb read
// from the neighbour's face projections written by k_local.
//   conn : [E_pad][4] packed (neighbour << 7) | (group << 4) | (j << 2) | h, the neighbour
//          index counted within its group; a neighbour whose face basis is smaller
//          contributes zeros above its size, a larger one is truncated to this degree
//          (the face basis is hierarchical and orthogonal, so truncation is the L2
//          projection onto this element's face space)
// WITH_LOCAL: add the local flux terms Wloc written by k_local<N, false> before lifting,
// so that Rhat^s is applied once per face to the sum of both flux contributions.
// The four faces' W (BT x 9 each) stay in shared memory; every row k of Q is then
// updated once with sum_s Rhat^s_k. W^s (no per-row accumulator array).
template <int N, bool WITH_LOCAL, typename Real>
__global__ void __launch_bounds__(kNq * kTile, (MinBlocks<N, Real, false>::value))
k_neigh(double* Q, FaceGroups G, const Real* Wloc, const Real* fnb, const int* conn,
        StepTables<Real> T, const TileRef* __restrict__ refs) {
  using Dm = Dims<N>;
  constexpr int B = Dm::B, BT = Dm::BT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Wsh = reinterpret_cast<Real*>(smem_raw);  // 4 faces x BT rows x 9 x 32
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  size_t tile = blockIdx.x;
  if (refs) {
    const TileRef& r = refs[blockIdx.x];
    Q = r.Q;
    Wloc = static_cast<const Real*>(r.Wloc);
    fnb = static_cast<const Real*>(r.fnb);
    conn = r.conn;
    G.base[0] = r.Pface;        // neighbours lie in the same problem (group 0)
    tile = (size_t)r.tile;
  }
  const size_t e = tile * kTile + lane;
  const Real* Ft = fnb + tile * (4 * kNq * kNq * kTile);

  // The neighbour's projection for face s is copied asynchronously into this thread's
  // column of face s's slot of Wsh (free until face s is processed); the copy for face
  // s + 1 is issued before face s is computed, so the gather overlaps computation.
  auto prefetch = [&](auto face) {
    constexpr int s = decltype(face)::value;
    const int c = __ldg(conn + e * 4 + s);
    const size_t nb = (size_t)(c >> 7);
    const int g = (c >> 4) & 7, j = (c >> 2) & 3;
    const int btn = G.bt[g];
    const Real* P = static_cast<const Real*>(G.base[g]) + ((nb * 4 + j) * kNq + w) * (size_t)btn;
    Real* dst = Wsh + s * BT * kNq * kTile + w * kTile + lane;
#pragma unroll
    for (int n = 0; n < BT; ++n) {
      if (n < btn) cp_async_elem(dst + n * kNq * kTile, P + n);
      else dst[n * kNq * kTile] = Real(0);
    }
    cp_async_commit();
  };
  prefetch(std::integral_constant<int, 0>{});
  static_for<0, 4>([&](auto face) {
    constexpr int s = decltype(face)::value;
    Real* Xsh = Wsh + s * BT * kNq * kTile;
    const int h = __ldg(conn + e * 4 + s) & 3;
    if constexpr (s < 3) {
      prefetch(std::integral_constant<int, s + 1>{});
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    Real Pn[BT];
#pragma unroll
    for (int n = 0; n < BT; ++n) Pn[n] = Xsh[(n * kNq + w) * kTile + lane];
    const Real* fh = T.f + (size_t)h * BT * BT;
    // V[m][q] = sum_n f^h_mn Pn[n], f^h block-diagonal by polynomial degree
#pragma unroll
    for (int d = 0; d <= N; ++d) {
      const int lo = d * (d + 1) / 2, hi = (d + 1) * (d + 2) / 2;
#pragma unroll
      for (int m = lo; m < hi; ++m) {
        Real v = Real(0);
#pragma unroll
        for (int n = lo; n < hi; ++n) v = fma(__ldg(fh + m + n * BT), Pn[n], v);
        Xsh[(m * kNq + w) * kTile + lane] = v;
      }
    }
    Real a[kNq];
#pragma unroll
    for (int q = 0; q < kNq; ++q) a[q] = __ldg(Ft + ((s * kNq + w) * kNq + q) * kTile + lane);
    __syncthreads();
    Real Wr[BT];
#pragma unroll
    for (int m = 0; m < BT; ++m) {
      Real v = Real(0);
      if constexpr (WITH_LOCAL) v = __ldg(Wloc + ((tile * 4 + s) * kNq * BT + w * BT + m) * kTile + lane);
#pragma unroll
      for (int q = 0; q < kNq; ++q) v = fma(a[q], Xsh[(m * kNq + q) * kTile + lane], v);
      Wr[m] = v;
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < BT; ++m) Xsh[(m * kNq + w) * kTile + lane] = Wr[m];
  });
  // every thread reads only its own columns of Wsh below: no barrier needed
  double* Qt = Q + tile * (kNq * B * kTile);
  static_for<0, B>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const Real* wcol = Wsh + w * kTile + lane;
    // the four faces' lifted rows summed in the contraction type (FP64: one chain), then
    // one binary64 update
    Real dq = row_dot<N, 25, k>(T.val, wcol);
    dq = row_dot_acc<N, 26, k>(T.val, wcol + 1 * BT * kNq * kTile, dq);
    dq = row_dot_acc<N, 27, k>(T.val, wcol + 2 * BT * kNq * kTile, dq);
    dq = row_dot_acc<N, 28, k>(T.val, wcol + 3 * BT * kNq * kTile, dq);
    Qt[(w * B + k) * kTile + lane] += to_f64<Real, MinBlocks<N, Real, false>::int_cvt>(dq);
  });
}

// ------------------------------------------------------------------ launch helpers
// Buffers typed by the contraction type are passed untyped and cast by the per-degree,
// per-precision launch functions.
struct AderLaunch {
  int64_t ntiles;
  size_t smem_local, smem_neigh;
  double *Q, *I;
  void *Pface, *Wloc;
  const void *star, *floc, *fnb, *val, *f;
  const int* conn;
  FaceGroups groups;
  double dt;
  StarPattern SP;
  const TileRef* refs;     // null: one problem, grid = ntiles; else grid = ntiles entries
  cudaStream_t stream;
};

template <typename Real>
StepTables<Real> step_tables(const AderLaunch& L) {
  StepTables<Real> T;
  T.val = static_cast<const Real*>(L.val);
  T.f = static_cast<const Real*>(L.f);
  T.dt = L.dt;
  double f = 1.0;
  for (int i = 0; i < 8; ++i) {
    f *= (i + 1.0);
    T.invfact[i] = 1.0 / f;
  }
  return T;
}

// Launch functions of one kernel variant (LOCAL: k_local<N, !FUSED>; else
// k_neigh<N, FUSED>); the generated translation units instantiate one variant each.
template <int N, typename Real, bool LOCAL, bool FUSED>
void ader_set_attribute(size_t smem) {
  if constexpr (LOCAL)
    cudaFuncSetAttribute(k_local<N, !FUSED, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else
    cudaFuncSetAttribute(k_neigh<N, FUSED, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <int N, typename Real, bool LOCAL, bool FUSED>
void ader_launch(const AderLaunch& L) {
  const unsigned grid = (unsigned)L.ntiles;
  const StepTables<Real> T = step_tables<Real>(L);
  if constexpr (LOCAL) {
    k_local<N, !FUSED, Real><<<grid, kNq * kTile, L.smem_local, L.stream>>>(
        L.Q, L.Q, L.I, static_cast<Real*>(L.Pface), static_cast<Real*>(L.Wloc),
        static_cast<const Real*>(L.star), static_cast<const Real*>(L.floc), T, L.SP, L.refs);
  } else {
    k_neigh<N, FUSED, Real><<<grid, kNq * kTile, L.smem_neigh, L.stream>>>(
        L.Q, L.groups, static_cast<const Real*>(L.Wloc), static_cast<const Real*>(L.fnb), L.conn, T, L.refs);
  }
}

// Per-degree, per-precision, per-variant instantiations live in generated translation
// units (ader_o<N>_<f64|f32>_<variant>.cu, variant = lf: local fused, ll: local lifted,
// nf: neighbour fused, np: neighbour plain).  Degree 6 exists in f32 only: its FP64
// shared-memory footprint (258 KB) exceeds the 227 KB a CTA may use.
#define YT_DECLARE_ADER_VARIANT(N, P, V)                  \
  void ader_set_attribute_o##N##_##P##_##V(size_t);      \
  void ader_launch_o##N##_##P##_##V(const AderLaunch&);  \
  int ader_upload_o##N##_##P##_##V(const float*, size_t);
#define YT_DECLARE_ADER_UNIT(N, P)     \
  YT_DECLARE_ADER_VARIANT(N, P, lf)    \
  YT_DECLARE_ADER_VARIANT(N, P, ll)    \
  YT_DECLARE_ADER_VARIANT(N, P, nf)    \
  YT_DECLARE_ADER_VARIANT(N, P, np)
YT_DECLARE_ADER_UNIT(1, f64)
YT_DECLARE_ADER_UNIT(2, f64)
YT_DECLARE_ADER_UNIT(3, f64)
YT_DECLARE_ADER_UNIT(4, f64)
YT_DECLARE_ADER_UNIT(5, f64)
YT_DECLARE_ADER_UNIT(1, f32)
YT_DECLARE_ADER_UNIT(2, f32)
YT_DECLARE_ADER_UNIT(3, f32)
YT_DECLARE_ADER_UNIT(4, f32)
YT_DECLARE_ADER_UNIT(5, f32)
YT_DECLARE_ADER_UNIT(6, f32)
#undef YT_DECLARE_ADER_UNIT
#undef YT_DECLARE_ADER_VARIANT
int ader_generated_nnz(int N);

}  // namespace yt
