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
// offset of the solver's value array (FP32: of constant memory) and its operand a fixed
// register or shared-memory element of the thread's operand column, so structural zeros
// and the equivalent-sparsity zero blocks (Sec. 4.2, 5.1.2) are never multiplied:
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

// The same with the operand column in a register array x[0..S).
template <int N, int LIST, int ROW, typename Real, int S>
__device__ __forceinline__ Real row_dotr(const Real* __restrict__ v, const Real (&x)[S]) {
  if constexpr (sizeof(Real) == 4 && N <= 5)
    return gen::Row<N, LIST, ROW>::dotrc(x);
  else
    return gen::Row<N, LIST, ROW>::template dotr1<Real, S>(v, x, Real(0));
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

// Where k_local keeps the operand column of its sparse products (D~^delta, then I): rows
// in registers make every non-zero one fma with a register operand (the binary64
// time-integral accumulator then lives in shared memory, touched once per row and
// derivative); rows in shared memory cost one load per fma.
// Rows of the operand column held in registers (the rest in shared memory).  The FP64
// column of degree 5 (56 doubles) does not fit beside the rest of the kernel under the
// 168-register cap of a 9-warp CTA: its C(N+2,3) = 35 rows of degree < 5 (read by every
// list) are registers, its 21 rows of degree 5 (read only by the first derivative and the
// face projections) shared memory.  Degree 6 in FP64 is not built.
template <int N, typename Real>
struct LocalRegRows {
  static constexpr int value = (sizeof(Real) == 8 && N >= 5) ? Dims<N>::nd(1) : Dims<N>::B;
};
// Exchange rows of k_local.  FP64 at degree 6 (order 7) mixes the derivatives in chunks
// of 5 rows (15 exchange rows of their own) and runs the exchange of the volume and flux
// phases (up to max(3 KC, BT) = 28 rows) in the time-integral accumulator rows, which
// are free once I is published: (28 + 15) operand / exchange rows + 56 accumulator rows
// of 9 x 32 doubles = 228 KB, where separate buffers would need 258 KB.
template <int N, typename Real>
struct LocalExchange {
  static constexpr bool alias = sizeof(Real) == 8 && N >= 6;
  static constexpr int KCK = alias ? 5 : Dims<N>::KC;        // rows per derivative chunk
  static constexpr int XR = alias ? 3 * KCK : Dims<N>::XR;   // exchange rows of their own
};
// Shared memory of k_local ([rows][9][32] each): operand rows not in registers, the
// exchange buffer, and the binary64 time-integral accumulator when any operand row is
// in registers (it is in registers otherwise).
template <int N, typename Real>
constexpr size_t local_smem_bytes() {
  using Dm = Dims<N>;
  constexpr int RS = LocalRegRows<N, Real>::value;
  return (size_t)sizeof(Real) * (Dm::B - RS + LocalExchange<N, Real>::XR) * kNq * kTile +
         (RS > 0 ? (size_t)8 * Dm::nd(1) * kNq * kTile : 0);
}
// Face slots of k_neigh's shared memory ([slot][BT][9][32]): four (the four faces lifted
// together), or three for FP64 at degree 6, where four slots (258 KB) exceed one CTA's
// shared memory: faces 0 and 1 are lifted after face 1, faces 2 and 3 after face 3, and
// face 3 reuses slot 0.
template <int N, typename Real>
struct NeighSlots {
  static constexpr int value = (sizeof(Real) == 8 && N >= 6) ? 3 : 4;
  static constexpr int slot(int s) { return (value == 4 || s < 3) ? s : 0; }
};
template <int N, typename Real>
constexpr size_t neigh_smem_bytes() {
  return (size_t)sizeof(Real) * NeighSlots<N, Real>::value * Dims<N>::BT * kNq * kTile;
}
// Sparse row with the operand column split at RS: rows < RS in D (registers), rows >= RS
// in shared memory at xs (that part of this thread's column, stride 9 x 32).
template <int N, int LIST, int ROW, int RS, typename Real, int S>
__device__ __forceinline__ Real row_op(const Real* __restrict__ v, const Real (&D)[S], const Real* __restrict__ xs) {
  if constexpr (RS == 0)
    return row_dot<N, LIST, ROW, Real>(v, xs);
  else if constexpr (RS >= Dims<N>::B)
    return row_dotr<N, LIST, ROW, Real>(v, D);
  else
    return gen::Row<N, LIST, ROW>::template dotrh<Real, S>(v, D, xs, Real(0));
}

// ------------------------------------------------------------------- CK derivatives
// One derivative step delta -> delta+1, in place in Dsh: output row k only reads rows of
// strictly higher polynomial degree (K~_kl != 0 only if deg phi_k < deg phi_l), so rows
// processed in increasing order overwrite rows that are no longer needed.  The time
// integral accumulates in double registers; only the C(N+2,3) rows that receive
// derivative terms need one (rows of degree N hold c0 Q alone).
template <int N, int DELTA, typename Real, int RS, int S>
__device__ __forceinline__ void ck_step(const StepTables<Real>& T, double dt, const int (&scol)[3], int cnt,
                                        Real* __restrict__ Dsh, Real (&D)[S], Real* __restrict__ Xsh,
                                        const Real (&sc)[3][3], double (&Icol)[Dims<N>::nd(1)],
                                        double* __restrict__ Ish, int w, int lane) {
  using Dm = Dims<N>;
  if constexpr (DELTA < N) {
    constexpr int nout = Dm::nd(DELTA + 1);
    constexpr int KC = LocalExchange<N, Real>::KCK;
    constexpr bool CVT = MinBlocks<N, Real, true>::int_cvt;
    const Real* xcol = Dsh + w * kTile + lane;
    const Real dtr = (Real)dt;
    const double cw = dt * T.invfact[DELTA + 1];
    static_for<0, (nout + KC - 1) / KC>([&](auto chunk) {
      constexpr int k0 = decltype(chunk)::value * KC;
      // X^x[k][q] = sum_l Ktilde^x_kl D[l][q]  (this thread: column q = w)
      static_for<0, KC>([&](auto kkc) {
        constexpr int kk = decltype(kkc)::value;
        if constexpr (k0 + kk < nout) {
          Xsh[((0 * KC + kk) * kNq + w) * kTile + lane] = row_op<N, DELTA * 3 + 0, k0 + kk, RS>(T.val, D, xcol);
          Xsh[((1 * KC + kk) * kNq + w) * kTile + lane] = row_op<N, DELTA * 3 + 1, k0 + kk, RS>(T.val, D, xcol);
          Xsh[((2 * KC + kk) * kNq + w) * kTile + lane] = row_op<N, DELTA * 3 + 2, k0 + kk, RS>(T.val, D, xcol);
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
          if constexpr (RS > 0) {
            static_assert(nout <= RS, "derivative rows must be register rows");
            D[k0 + kk] = v;
            double* ip = Ish + ((k0 + kk) * kNq + w) * kTile + lane;
            *ip = fma(cw, to_f64<Real, CVT>(v), *ip);
          } else {
            Dsh[((k0 + kk) * kNq + w) * kTile + lane] = v;
            Icol[k0 + kk] = fma(cw, to_f64<Real, CVT>(v), Icol[k0 + kk]);
          }
        }
      });
      __syncthreads();
    });
    ck_step<N, DELTA + 1, Real, RS, S>(T, dt, scol, cnt, Dsh, D, Xsh, sc, Icol, Ish, w, lane);
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
  constexpr int XR = LocalExchange<N, Real>::XR;
  constexpr bool ALIAS = LocalExchange<N, Real>::alias;
  constexpr bool CVT = MinBlocks<N, Real, true>::int_cvt;
  constexpr int RS = LocalRegRows<N, Real>::value;   // operand rows in registers
  constexpr int SD = RS > 0 ? RS : 1;
  static_assert(!ALIAS || (RS > 0 && sizeof(Real) == 8 && Dm::nd(1) >= Dm::XR),
                "the volume / flux exchange must fit the accumulator rows");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // [B - RS operand rows][XR exchange rows][NI accumulator rows (double), when RS > 0]
  Real* Dsh = reinterpret_cast<Real*>(smem_raw);
  Real* Xsh = Dsh + (B - RS) * kNq * kTile;
  double* Ish = RS > 0 ? reinterpret_cast<double*>(Xsh + XR * kNq * kTile) : nullptr;
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
  Real D[SD];           // operand rows < RS
  double Icol[NI];      // time-integral accumulator (RS == 0)
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const double q = __ldg(Qt + (w * B + k) * kTile + lane);
    if (k < RS) D[k < RS ? k : 0] = from_f64<Real, CVT>(q);
    else Dsh[((k - RS) * kNq + w) * kTile + lane] = from_f64<Real, CVT>(q);
    if constexpr (RS > 0) {
      if (k < NI) Ish[(k * kNq + w) * kTile + lane] = dt * T.invfact[0] * q;
    } else {
      if (k < NI) Icol[k < NI ? k : 0] = dt * T.invfact[0] * q;
    }
  }
  // (own column only is read before the first barrier)
  const Real* xcol = Dsh + w * kTile + lane;      // this thread's shared operand rows
  ck_step<N, 0, Real, RS, SD>(T, dt, scol, cnt, Dsh, D, Xsh, sc, Icol, Ish, w, lane);

  // publish I: operand column (own) and HBM
  double* It = Iout + tile * (kNq * B * kTile);
#pragma unroll
  for (int k = 0; k < B; ++k) {
    double ik;
    if constexpr (RS > 0)
      ik = k < NI ? Ish[(k * kNq + w) * kTile + lane] : dt * T.invfact[0] * Qt[(w * B + k) * kTile + lane];
    else
      ik = k < NI ? Icol[k < NI ? k : 0] : dt * T.invfact[0] * Qt[(w * B + k) * kTile + lane];
    if (k < RS) D[k < RS ? k : 0] = from_f64<Real, CVT>(ik);
    else Dsh[((k - RS) * kNq + w) * kTile + lane] = from_f64<Real, CVT>(ik);
    It[(w * B + k) * kTile + lane] = ik;
  }

  // The volume term is added to each row of Q as soon as its chunk is done; with LIFT the
  // local flux is then added face by face (every row of an element column belongs to
  // one thread, so these read-modify-writes need no synchronisation).
  double* Qo = Qout + tile * (kNq * B * kTile);
  // exchange of the volume and flux phases: the accumulator rows when ALIAS (each thread
  // has read its own accumulator column above and writes only its own column before the
  // next barrier)
  if constexpr (ALIAS) Xsh = reinterpret_cast<Real*>(Ish);

  // volume: dQ[k][p] += sum_x sum_q Astar^x_pq (Khat^x I)[k][q]
  static_for<0, (B + KC - 1) / KC>([&](auto chunk) {
    constexpr int k0 = decltype(chunk)::value * KC;
    static_for<0, KC>([&](auto kkc) {
      constexpr int kk = decltype(kkc)::value;
      if constexpr (k0 + kk < B) {
        Xsh[((0 * KC + kk) * kNq + w) * kTile + lane] = row_op<N, 18, k0 + kk, RS>(T.val, D, xcol);
        Xsh[((1 * KC + kk) * kNq + w) * kTile + lane] = row_op<N, 19, k0 + kk, RS>(T.val, D, xcol);
        Xsh[((2 * KC + kk) * kNq + w) * kTile + lane] = row_op<N, 20, k0 + kk, RS>(T.val, D, xcol);
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
      const Real z = row_op<N, 21 + s, m, RS>(T.val, D, xcol);
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
  using Slots = NeighSlots<N, Real>;
  constexpr int B = Dm::B, BT = Dm::BT;
  constexpr int SLOT = BT * kNq * kTile;
  constexpr bool CVT = MinBlocks<N, Real, false>::int_cvt;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Wsh = reinterpret_cast<Real*>(smem_raw);  // slots x BT rows x 9 x 32
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
    Real* dst = Wsh + Slots::slot(s) * SLOT + w * kTile + lane;
#pragma unroll
    for (int n = 0; n < BT; ++n) {
      if (n < btn) cp_async_elem(dst + n * kNq * kTile, P + n);
      else dst[n * kNq * kTile] = Real(0);
    }
    cp_async_commit();
  };
  // lifting of faces F0 .. F0 + NF - 1: every row k of Q gets the sum over these faces of
  // Rhat^s_k. W^s, summed in the contraction type (FP64: one chain), then one binary64
  // update (each thread reads only its own columns of Wsh)
  double* Qt = Q + tile * (kNq * B * kTile);
  auto lift = [&](auto f0, auto nf) {
    constexpr int F0 = decltype(f0)::value, NF = decltype(nf)::value;
    const Real* wcol = Wsh + w * kTile + lane;
    static_for<0, B>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      Real dq = row_dot<N, 25 + F0, k>(T.val, wcol + Slots::slot(F0) * SLOT);
      if constexpr (NF > 1) dq = row_dot_acc<N, 26 + F0, k>(T.val, wcol + Slots::slot(F0 + 1) * SLOT, dq);
      if constexpr (NF > 2) dq = row_dot_acc<N, 27 + F0, k>(T.val, wcol + Slots::slot(F0 + 2) * SLOT, dq);
      if constexpr (NF > 3) dq = row_dot_acc<N, 28 + F0, k>(T.val, wcol + Slots::slot(F0 + 3) * SLOT, dq);
      Qt[(w * B + k) * kTile + lane] += to_f64<Real, CVT>(dq);
    });
  };
  prefetch(std::integral_constant<int, 0>{});
  static_for<0, 4>([&](auto face) {
    constexpr int s = decltype(face)::value;
    Real* Xsh = Wsh + Slots::slot(s) * SLOT;
    const int h = __ldg(conn + e * 4 + s) & 3;
    // with three slots, face 3's slot (0) is free only once every thread has lifted faces
    // 0 and 1: its copy is issued after face 2's first barrier
    constexpr bool late = Slots::value == 3 && s == 2;
    if constexpr (s < 3 && !late) {
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
    if constexpr (late) prefetch(std::integral_constant<int, 3>{});
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
    if constexpr (Slots::value == 3 && s == 1) lift(std::integral_constant<int, 0>{}, std::integral_constant<int, 2>{});
  });
  // every thread reads only its own columns of Wsh below: no barrier needed
  if constexpr (Slots::value == 4)
    lift(std::integral_constant<int, 0>{}, std::integral_constant<int, 4>{});
  else
    lift(std::integral_constant<int, 2>{}, std::integral_constant<int, 2>{});
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

// Shared memory of k_local for a runtime degree (1..6) and contraction type.
inline size_t ader_local_smem(int N, bool f32) {
  switch (N * 2 + (f32 ? 1 : 0)) {
    case 2: return local_smem_bytes<1, double>();
    case 3: return local_smem_bytes<1, float>();
    case 4: return local_smem_bytes<2, double>();
    case 5: return local_smem_bytes<2, float>();
    case 6: return local_smem_bytes<3, double>();
    case 7: return local_smem_bytes<3, float>();
    case 8: return local_smem_bytes<4, double>();
    case 9: return local_smem_bytes<4, float>();
    case 10: return local_smem_bytes<5, double>();
    case 11: return local_smem_bytes<5, float>();
    case 12: return local_smem_bytes<6, double>();
    case 13: return local_smem_bytes<6, float>();
  }
  return 0;
}
inline size_t ader_neigh_smem(int N, bool f32) {
  if (N == 6) return f32 ? neigh_smem_bytes<6, float>() : neigh_smem_bytes<6, double>();
  return (f32 ? 4 : 8) * (size_t)(4 * ((N + 1) * (N + 2) / 2)) * kNq * kTile;
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
// nf: neighbour fused, np: neighbour plain).
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
YT_DECLARE_ADER_UNIT(6, f64)
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
