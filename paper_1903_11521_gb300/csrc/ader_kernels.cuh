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

// FP32 values of degrees <= 5 come from constant memory (one copy per translation unit),
// except in the translation units of the persistent batch kernel, which are linked into
// one device module (YT_ROWS_GLOBAL): the constant bank could not hold every degree's
// values at once, so they read the values from global memory.
#ifdef YT_ROWS_GLOBAL
constexpr bool kConstValues = false;
#else
constexpr bool kConstValues = true;
#endif

// Sparse row of a list.  FP64: one accumulator chain (Row::dot1; the FP64 pipe is the
// limit and nine warps supply enough independent chains, while every extra accumulator
// costs an add to combine).  FP32: four accumulators (Row::dot; latency is the limit),
// values of degrees <= 5 from constant memory (Row::dotc, one constant-bank operand per
// fma).  row_dot_acc continues an accumulation (one chain across several rows in FP64).
template <int N, int LIST, int ROW, typename Real>
__device__ __forceinline__ Real row_dot(const Real* __restrict__ v, const Real* __restrict__ x) {
  if constexpr (sizeof(Real) == 8)
    return gen::Row<N, LIST, ROW>::dot1(v, x, Real(0));
  else if constexpr (N <= 5 && kConstValues)
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
  if constexpr (sizeof(Real) == 4 && N <= 5 && kConstValues)
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

// 27-quantity (viscoelastic-shaped) steps: q = (9 elastic quantities, theta^l_i at
// 9 + 6 l + i for three mechanisms l and six components i).  The anelastic functions
// carry no flux (their columns of the Jacobians are zero) and are driven by the
// velocities through the rows of the star matrices Astar^x_{theta,q}, which have the
// slot pattern of the stress rows (columns 6..8); the source E couples them:
// d sigma_i/dt -= sum_l theta^l_i, d theta^l_i/dt -= omega_l theta^l_i.  Warp i < 6 (the
// stress row i) owns theta^l_i of its lane's element in k_local.
constexpr int kNqVe = 27;
constexpr int kNTheta = 18;
constexpr int kStressSlots = 15;       // star slots of the six stress rows
template <typename Real>
struct VeTables {
  Real* theta;          // [tile][18][B][32] current scaled derivative D~^d of theta (scratch)
  const Real* cth;      // [tile][3 mech][3 dir][15 stress slots][32] Astar^x rows of theta^l
  const Real* om;       // [tile][3][32] omega_l
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
// One row K of a derivative of a 27-quantity step, stress warp w: the feedback of the
// anelastic functions into the stress (E_{sigma_i, theta^l_i} = -1) is added to v, and
// D~^{d+1}[K][theta^l_w] = dt (sum_x sum_q Astar^x_{theta,q} X^x[K][q] - omega_l D~^d[K][theta^l_w])
// replaces D~^d in the scratch, its time-integral term accumulated in binary64 in It.
template <int N, typename Real, bool CVT, bool HASX, int KC, int K>
__device__ __forceinline__ Real ve_row(const VeTables<Real>& V, size_t tile, int w, int lane, int kk,
                                       const Real* __restrict__ Xsh, const int (&scol)[3], int cnt, int s0,
                                       const Real (&om)[3], Real dtr, double cw, double* __restrict__ It, Real v) {
  constexpr int B = Dims<N>::B;
  constexpr size_t LS = (size_t)6 * B * kTile;         // mechanism stride (theta scratch and I)
  Real* th = V.theta + ((tile * kNTheta + w) * B + K) * kTile + lane;
  double* ith = It + ((size_t)(9 + w) * B + K) * kTile + lane;
  // the row's state and accumulators, loaded together ahead of the stores (a store to
  // the scratch could alias the accumulators otherwise: one memory latency each)
  const Real t[3] = {th[0], th[LS], th[2 * LS]};
  const double ti[3] = {ith[0], ith[LS], ith[2 * LS]};
  v -= (t[0] + t[1]) + t[2];                             // E_{sigma_i, theta^l_i} = -1
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    Real u = Real(0);
    if constexpr (HASX) {
      const Real* c = V.cth + (((tile * 3 + l) * 3) * kStressSlots + s0) * kTile + lane;
#pragma unroll
      for (int x = 0; x < 3; ++x)
#pragma unroll
        for (int s = 0; s < 3; ++s)
          if (s < cnt) u = fma(__ldg(c + (x * kStressSlots + s) * kTile), Xsh[((x * KC + kk) * kNq + scol[s]) * kTile + lane], u);
    }
    u = fma(-om[l], t[l], u);                            // E_{theta, theta} = -omega_l
    u *= dtr;
    th[l * LS] = u;
    ith[l * LS] = fma(cw, to_f64<Real, CVT>(u), ti[l]);
  }
  return v;
}

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

// 27 quantities: every derivative runs the same unrestricted lists (those of delta = 0:
// the source term keeps all B rows of D^delta non-zero), so the derivatives are a runtime
// loop around one unrolled body (N times less code than unrolling them).  Each
// derivative mixes all B rows: rows of degree < N as above; the stress warps add the
// feedback -sum_l theta^l_i and advance their anelastic functions (ve_row); the stress
// rows of degree N (only the feedback reaches them) accumulate their time integral in
// the output array It itself; the velocity rows of degree N stay zero.  The operand
// column D (registers, rows >= RS in shared memory) holds all B rows.
template <int N, typename Real, int RS, int S>
__device__ __forceinline__ void ck_ve(const StepTables<Real>& T, double dt, const int (&scol)[3], int cnt,
                                      Real* __restrict__ Dsh, Real (&D)[S], Real* __restrict__ Xsh,
                                      const Real (&sc)[3][3], double* __restrict__ Ish, int w, int lane,
                                      const VeTables<Real>& V, size_t tile, int s0, const Real (&om)[3],
                                      double* __restrict__ It) {
  using Dm = Dims<N>;
  constexpr int B = Dm::B, NI = Dm::nd(1);
  constexpr int KC = LocalExchange<N, Real>::KCK;
  constexpr bool CVT = MinBlocks<N, Real, true>::int_cvt;
  static_assert(RS > 0, "the time-integral accumulator is in shared memory");
  const Real* xcol = Dsh + w * kTile + lane;
  const Real dtr = (Real)dt;
#pragma unroll 1
  for (int delta = 0; delta < N; ++delta) {
    const double cw = dt * T.invfact[delta + 1];
    static_for<0, (B + KC - 1) / KC>([&](auto chunk) {
      constexpr int k0 = decltype(chunk)::value * KC;
      if constexpr (k0 < NI) {
        static_for<0, KC>([&](auto kkc) {
          constexpr int kk = decltype(kkc)::value;
          if constexpr (k0 + kk < NI) {
            Xsh[((0 * KC + kk) * kNq + w) * kTile + lane] = row_op<N, 0, k0 + kk, RS>(T.val, D, xcol);
            Xsh[((1 * KC + kk) * kNq + w) * kTile + lane] = row_op<N, 1, k0 + kk, RS>(T.val, D, xcol);
            Xsh[((2 * KC + kk) * kNq + w) * kTile + lane] = row_op<N, 2, k0 + kk, RS>(T.val, D, xcol);
          }
        });
        __syncthreads();
      }
      static_for<0, KC>([&](auto kkc) {
        constexpr int kk = decltype(kkc)::value;
        constexpr int k = k0 + kk;
        if constexpr (k < B) {
          Real v = Real(0);
          if constexpr (k < NI) {
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
              for (int s = 0; s < 3; ++s)
                if (s < cnt) v = fma(sc[x][s], Xsh[((x * KC + kk) * kNq + scol[s]) * kTile + lane], v);
          }
          // stress rows of degree N: their accumulator in I, loaded before ve_row's stores
          double* ipn = It + ((size_t)w * B + k) * kTile + lane;
          const double in_old = (k >= NI && w < 6) ? *ipn : 0.0;
          if (w < 6) v = ve_row<N, Real, CVT, (k < NI), KC, k>(V, tile, w, lane, kk, Xsh, scol, cnt, s0, om, dtr, cw, It, v);
          v *= dtr;
          if constexpr (k < RS) D[k < RS ? k : 0] = v;
          else Dsh[((k - RS) * kNq + w) * kTile + lane] = v;
          if constexpr (k < NI) {
            double* ip = Ish + (k * kNq + w) * kTile + lane;
            *ip = fma(cw, to_f64<Real, CVT>(v), *ip);
          } else if (w < 6) {
            *ipn = fma(cw, to_f64<Real, CVT>(v), in_old);
          }
        }
      });
      if constexpr (k0 < NI) __syncthreads();
    });
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
// VE: 27 quantities (Q, Qout, Iout are [tile][27][B][32]); the elastic rows as above
// with the source terms, the anelastic functions' derivatives and time integral by the
// stress warps (their volume, source and flux terms are k_theta's).
// local_tile: the work of one tile (tile index and time step given), shared by the
// kernel below and the persistent batch kernel.
template <int N, bool LIFT, typename Real, bool VE>
__device__ __forceinline__ void local_tile(const double* Q, double* Qout, double* Iout, Real* Pface,
                                           Real* Wloc, const Real* star, const Real* floc,
                                           StepTables<Real> T, StarPattern SP, VeTables<Real> V,
                                           size_t tile, double dt) {
  using Dm = Dims<N>;
  constexpr int NQT = VE ? kNqVe : kNq;      // quantities per element in Q and I
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
  const double* Qt = Q + tile * (NQT * B * kTile);
  // VE: this tile's I, read and accumulated during the derivatives (the elastic path
  // forms its pointer only where it publishes I, so nothing extra lives through the CK)
  double* Ive = VE ? Iout + tile * (NQT * B * kTile) : nullptr;

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
  Real om[3] = {Real(0), Real(0), Real(0)};
  if constexpr (VE) {
    if (w < 6) {
      // D~^0 of this warp's anelastic functions and their time-integral accumulators;
      // the accumulators of the stress rows of degree N (fed by the source) in I itself
      constexpr size_t LS = (size_t)6 * B * kTile;
#pragma unroll
      for (int l = 0; l < 3; ++l) om[l] = __ldg(V.om + (tile * 3 + l) * kTile + lane);
      Real* th = V.theta + ((tile * kNTheta + w) * B) * kTile + lane;
      const double* qth = Qt + ((size_t)(9 + w) * B) * kTile + lane;
      double* ith = Ive + ((size_t)(9 + w) * B) * kTile + lane;
      // four rows of the three mechanisms loaded before they are stored (the stores could
      // alias the loads otherwise: one memory latency per value)
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
              th[l * LS + (k0 + i) * kTile] = from_f64<Real, CVT>(q[l][i]);
              ith[l * LS + (k0 + i) * kTile] = dt * T.invfact[0] * q[l][i];
            }
      });
      static_for<0, (B - NI + 3) / 4>([&](auto cc) {
        constexpr int k0 = NI + decltype(cc)::value * 4;
        double q[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) q[i] = (k0 + i < B) ? __ldg(Qt + (w * B + (k0 + i < B ? k0 + i : 0)) * kTile + lane) : 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (k0 + i < B) Ive[((size_t)w * B + k0 + i) * kTile + lane] = dt * T.invfact[0] * q[i];
      });
    }
  }
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
  if constexpr (VE) ck_ve<N, Real, RS, SD>(T, dt, scol, cnt, Dsh, D, Xsh, sc, Ish, w, lane, V, tile, s0, om, Ive);
  else ck_step<N, 0, Real, RS, SD>(T, dt, scol, cnt, Dsh, D, Xsh, sc, Icol, Ish, w, lane);

  // publish I: operand column (own) and HBM
  double* It = Iout + tile * (NQT * B * kTile);
#pragma unroll
  for (int k = 0; k < B; ++k) {
    double ik;
    if (VE && w < 6 && k >= NI)
      ik = It[(w * B + k) * kTile + lane];
    else if constexpr (RS > 0)
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
  double* Qo = Qout + tile * (NQT * B * kTile);
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
        if constexpr (VE) {
          double src = 0.0;                      // (I E^T)_{k, sigma_i} = -sum_l I[k][theta^l_i]
          if (w < 6) {
            const double* ith = It + ((size_t)(9 + w) * B + k) * kTile + lane;
            src = -((ith[0] + ith[(size_t)6 * B * kTile]) + ith[(size_t)12 * B * kTile]);
          }
          Qo[(w * B + k) * kTile + lane] = Qt[(w * B + k) * kTile + lane] + to_f64<Real, CVT>(v) + src;
        } else {
          Qo[(w * B + k) * kTile + lane] = Qt[(w * B + k) * kTile + lane] + to_f64<Real, CVT>(v);
        }
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

template <int N, bool LIFT, typename Real, bool VE = false>
__global__ void __launch_bounds__(kNq * kTile, (MinBlocks<N, Real, true>::value))
k_local(const double* Q, double* Qout, double* Iout, Real* Pface, Real* Wloc, const Real* star,
        const Real* floc, StepTables<Real> T, StarPattern SP, const TileRef* __restrict__ refs,
        VeTables<Real> V) {
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
  local_tile<N, LIFT, Real, VE>(Q, Qout, Iout, Pface, Wloc, star, floc, T, SP, V, tile, dt);
}

// ------------------------------------------------------------ K_local, small meshes
// The local update with the local flux lifted (k_local<N, true, Real>) for meshes of few
// tiles, where one CTA per 32 elements leaves most SMs idle and a tile's work on one SM
// sets the time: one CTA per 8 elements of a tile, thread (slot q, element e) = column q
// of element e (q = 0..8; slots 9..11 shadow quantity 8 so that every warp runs the same
// code, and write nothing to global memory).  Same arithmetic and order of operations as
// k_local (operand column in registers, binary64 time-integral accumulator in shared
// memory); the lifting reads the face's flux products from registers.  Degrees whose
// operand column fits the registers (FP64 N <= 4, FP32).
constexpr int kSmallElems = 8;                          // elements per CTA
constexpr int kSmallSlots = 12;                         // quantity slots
constexpr int kSmallThreads = kSmallElems * kSmallSlots;
template <int N, typename Real>
constexpr size_t small_smem_bytes() {
  using Dm = Dims<N>;
  return (size_t)sizeof(Real) * Dm::XR * kSmallSlots * kSmallElems +
         (size_t)8 * Dm::nd(1) * kSmallSlots * kSmallElems;
}

template <int N, typename Real>
__global__ void __launch_bounds__(kSmallThreads, 1)
k_local_small(const double* Q, double* Qout, double* __restrict__ Iout, Real* __restrict__ Pface,
              const Real* __restrict__ star, const Real* __restrict__ floc, StepTables<Real> T, StarPattern SP) {
  using Dm = Dims<N>;
  constexpr int B = Dm::B, BT = Dm::BT, KC = Dm::KC, NI = Dm::nd(1);
  constexpr int QS = kSmallSlots, TS = kSmallElems;
  constexpr bool CVT = MinBlocks<N, Real, true>::int_cvt;
  static_assert(LocalRegRows<N, Real>::value == B, "the operand column must be register rows");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Xsh = reinterpret_cast<Real*>(smem_raw);                          // [XR][QS][TS]
  double* Ish = reinterpret_cast<double*>(Xsh + Dm::XR * QS * TS);       // [NI][QS][TS]
  const int q = threadIdx.x / TS, e = threadIdx.x % TS;
  const bool act = q < kNq;
  const int p = act ? q : kNq - 1;
  const size_t tile = blockIdx.x / (kTile / TS);
  const int lane = (int)(blockIdx.x % (kTile / TS)) * TS + e;           // the element's lane in its tile
  auto xs = [&](int r, int slot) -> Real& { return Xsh[(r * QS + slot) * TS + e]; };
  auto is = [&](int r) -> double& { return Ish[(r * QS + q) * TS + e]; };
  const double dt = T.dt;
  const double* Qt = Q + tile * (kNq * B * kTile);
  double* Qo = Qout + tile * (kNq * B * kTile);
  double* It = Iout + tile * (kNq * B * kTile);
  const int s0 = SP.start[p], cnt = SP.start[p + 1] - s0;
  int scol[3];
#pragma unroll
  for (int s = 0; s < 3; ++s) scol[s] = (s < cnt) ? SP.col[s0 + s] : 0;
  Real sc[3][3];
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int s = 0; s < 3; ++s)
      sc[x][s] = (s < cnt) ? __ldg(star + ((tile * 3 + x) * kStarSlots + s0 + s) * kTile + lane) : Real(0);
  auto mix = [&](int kk) {
    Real v = Real(0);
#pragma unroll
    for (int x = 0; x < 3; ++x)
#pragma unroll
      for (int s = 0; s < 3; ++s)
        if (s < cnt) v = fma(sc[x][s], xs(x * KC + kk, scol[s]), v);
    return v;
  };

  Real D[B];
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const double qv = __ldg(Qt + (p * B + k) * kTile + lane);
    D[k] = from_f64<Real, CVT>(qv);
    if (k < NI) is(k) = dt * T.invfact[0] * qv;
  }
  // CK derivatives in place (output row k reads rows of higher degree only)
  const Real dtr = (Real)dt;
  static_for<0, N>([&](auto dd) {
    constexpr int DELTA = decltype(dd)::value;
    constexpr int nout = Dm::nd(DELTA + 1);
    const double cw = dt * T.invfact[DELTA + 1];
    static_for<0, (nout + KC - 1) / KC>([&](auto chunk) {
      constexpr int k0 = decltype(chunk)::value * KC;
      static_for<0, KC>([&](auto kkc) {
        constexpr int kk = decltype(kkc)::value;
        if constexpr (k0 + kk < nout) {
          xs(0 * KC + kk, q) = row_dotr<N, DELTA * 3 + 0, k0 + kk, Real, B>(T.val, D);
          xs(1 * KC + kk, q) = row_dotr<N, DELTA * 3 + 1, k0 + kk, Real, B>(T.val, D);
          xs(2 * KC + kk, q) = row_dotr<N, DELTA * 3 + 2, k0 + kk, Real, B>(T.val, D);
        }
      });
      __syncthreads();
      static_for<0, KC>([&](auto kkc) {
        constexpr int kk = decltype(kkc)::value;
        if constexpr (k0 + kk < nout) {
          const Real v = mix(kk) * dtr;
          D[k0 + kk] = v;
          is(k0 + kk) = fma(cw, to_f64<Real, CVT>(v), is(k0 + kk));
        }
      });
      __syncthreads();
    });
  });
  // publish I: operand column and global memory
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const double ik = k < NI ? is(k < NI ? k : 0) : dt * T.invfact[0] * Qt[(p * B + k) * kTile + lane];
    D[k] = from_f64<Real, CVT>(ik);
    if (act) It[(p * B + k) * kTile + lane] = ik;
  }
  // volume: Q[k][p] += sum_x sum_q Astar^x_pq (Khat^x I)[k][q]
  static_for<0, (B + KC - 1) / KC>([&](auto chunk) {
    constexpr int k0 = decltype(chunk)::value * KC;
    static_for<0, KC>([&](auto kkc) {
      constexpr int kk = decltype(kkc)::value;
      if constexpr (k0 + kk < B) {
        xs(0 * KC + kk, q) = row_dotr<N, 18, k0 + kk, Real, B>(T.val, D);
        xs(1 * KC + kk, q) = row_dotr<N, 19, k0 + kk, Real, B>(T.val, D);
        xs(2 * KC + kk, q) = row_dotr<N, 20, k0 + kk, Real, B>(T.val, D);
      }
    });
    __syncthreads();
    static_for<0, KC>([&](auto kkc) {
      constexpr int kk = decltype(kkc)::value;
      constexpr int k = k0 + kk;
      if constexpr (k < B) {
        const Real v = mix(kk);
        if (act) Qo[(p * B + k) * kTile + lane] = Qt[(p * B + k) * kTile + lane] + to_f64<Real, CVT>(v);
      }
    });
    __syncthreads();
  });
  // local flux: Q += Rhat^s ((R^sT I) Aloc_s^T), face by face
  Real* Pt = Pface + (tile * kTile + lane) * (4 * kNq * BT);
  const Real* Ft = floc + tile * (4 * kNq * kNq * kTile);
  static_for<0, 4>([&](auto face) {
    constexpr int s = decltype(face)::value;
    static_for<0, BT>([&](auto mm) {
      constexpr int m = decltype(mm)::value;
      const Real z = row_dotr<N, 21 + s, m, Real, B>(T.val, D);
      xs(m, q) = z;
      if (act) Pt[(s * kNq + p) * BT + m] = z;
    });
    Real a[kNq];
#pragma unroll
    for (int c = 0; c < kNq; ++c) a[c] = __ldg(Ft + ((s * kNq + p) * kNq + c) * kTile + lane);
    __syncthreads();
    Real Wr[BT];
#pragma unroll
    for (int m = 0; m < BT; ++m) {
      Real v = Real(0);
#pragma unroll
      for (int c = 0; c < kNq; ++c) v = fma(a[c], xs(m, c), v);
      Wr[m] = v;
    }
    __syncthreads();
    static_for<0, B>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const Real dq = row_dotr<N, 25 + s, k, Real, BT>(T.val, Wr);
      if (act) Qo[(p * B + k) * kTile + lane] += to_f64<Real, CVT>(dq);
    });
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
// NQT: quantities per element of Q (27 for the elastic rows of a 27-quantity step).
template <int N, bool WITH_LOCAL, typename Real, int NQT>
__device__ __forceinline__ void neigh_tile(double* Q, const FaceGroups& G, const Real* Wloc, const Real* fnb,
                                           const int* conn, StepTables<Real> T, size_t tile) {
  using Dm = Dims<N>;
  using Slots = NeighSlots<N, Real>;
  constexpr int B = Dm::B, BT = Dm::BT;
  constexpr int SLOT = BT * kNq * kTile;
  constexpr bool CVT = MinBlocks<N, Real, false>::int_cvt;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Wsh = reinterpret_cast<Real*>(smem_raw);  // slots x BT rows x 9 x 32
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
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
  double* Qt = Q + tile * (NQT * B * kTile);
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

template <int N, bool WITH_LOCAL, typename Real, int NQT = kNq>
__global__ void __launch_bounds__(kNq * kTile, (MinBlocks<N, Real, false>::value))
k_neigh(double* Q, FaceGroups G, const Real* Wloc, const Real* fnb, const int* conn,
        StepTables<Real> T, const TileRef* __restrict__ refs) {
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
  neigh_tile<N, WITH_LOCAL, Real, NQT>(Q, G, Wloc, fnb, conn, T, tile);
}

// ------------------------------------------------------------------------- K_theta
// faces whose staged projections k_theta holds at once
template <typename Real>
struct ThetaFacesPerPass {
  static constexpr int value = sizeof(Real) == 4 ? 2 : 1;
};
// The anelastic rows of a 27-quantity step (after k_local<N, false, Real, true>, beside
// k_neigh<N, true, Real, 27>, which updates only the elastic rows): for each anelastic
// function t = (l, i) of mechanism l and component i,
//   Q[k][t] += sum_x sum_q Astar^x_tq (Khat^x I)[k][q] - omega_l I[k][t]      (volume, source)
//            + sum_s Rhat^s_k. ((R^sT I) Aloc_s,t^T + f^h (R^jT I_nb) Anb_s,t^T) (fluxes)
// The star rows of theta^l_i have the slots of stress row i (velocity columns only), so
// the volume needs Khat^x I for the three velocity columns: warp w forms the three
// directions of velocity column 6 + w % 3 for the rows k = w / 3 (mod 3).  The flux
// terms need the face projections of this element and of its neighbours (written by
// k_local): both are staged per face in shared memory, then every warp mixes them into
// the flux products of its two anelastic functions t = w, w + 9 (registers) and lifts
// them into Q (one binary64 update of the column per face).
//   Q, I   : [tile][27][B][32] double
//   Pown   : [element][4][9][PS]  R^sT I of the elastic quantities of this launch's tiles
//            (rows of PS >= BT values: BT, or padded to 8 in the tensor-core form)
//   Pface  : the same for all elements (gathered by neighbour index)
//   fthl, fthn : [tile][4][18][9][32] anelastic rows of the local / neighbour flux solvers
template <int N, typename Real>
__global__ void __launch_bounds__(kNq * kTile, 1)
k_theta(double* Q, const double* __restrict__ I, const Real* __restrict__ Pown, const Real* __restrict__ Pface,
        int PS, const int* __restrict__ conn, const Real* __restrict__ fthl, const Real* __restrict__ fthn,
        StepTables<Real> T, StarPattern SP, VeTables<Real> V) {
  using Dm = Dims<N>;
  constexpr int B = Dm::B, BT = Dm::BT, KC = Dm::KC;
  // the volume's operand column in shared memory: in registers it left too few for the
  // face phase, which then spilled (kilobytes of local memory per thread)
  constexpr int RS = 0;
  constexpr int SD = 1;
  constexpr bool CVT = MinBlocks<N, Real, true>::int_cvt;
  constexpr size_t TQ = (size_t)kNqVe * B * kTile;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Real* Dsh = reinterpret_cast<Real*>(smem_raw);            // volume operand rows [B][9][32]
  Real* Xsh = Dsh + B * kNq * kTile;                        // volume exchange [KC][9][32]
  Real* Xf = Dsh;                                           // then the faces [2 FP][BT][9][32]
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const size_t tile = blockIdx.x;
  const size_t e = tile * kTile + lane;
  double* Qt = Q + tile * TQ;
  const double* It = I + tile * TQ;

  // this warp's anelastic functions t = w, w + 9 -> (mechanism, component), star slots
  int tl[2], ti[2], ts0[2], tcnt[2], tcol[2][3];
  Real tom[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int t = w + 9 * c;
    tl[c] = t / 6;
    ti[c] = t % 6;
    ts0[c] = SP.start[ti[c]];
    tcnt[c] = SP.start[ti[c] + 1] - ts0[c];
#pragma unroll
    for (int s = 0; s < 3; ++s) tcol[c][s] = (s < tcnt[c]) ? SP.col[ts0[c] + s] - 6 : 0;
    tom[c] = __ldg(V.om + (tile * 3 + tl[c]) * kTile + lane);
  }

  // ---- volume and source
  const int qv = 6 + w % 3, rc = w / 3;
  Real D[SD];
#pragma unroll
  for (int k = 0; k < B; ++k) {
    const Real v = from_f64<Real, CVT>(It[(qv * B + k) * kTile + lane]);
    if (k < RS) D[k < RS ? k : 0] = v;
    else Dsh[((k - RS) * kNq + w) * kTile + lane] = v;
  }
  const Real* xcol = Dsh + w * kTile + lane;
  static_for<0, (B + KC - 1) / KC>([&](auto chunk) {
    constexpr int k0 = decltype(chunk)::value * KC;
    static_for<0, KC>([&](auto kkc) {
      constexpr int kk = decltype(kkc)::value;
      constexpr int k = k0 + kk;
      if constexpr (k < B) {
        if (k % 3 == rc) {
          Xsh[(kk * kNq + 0 + (qv - 6)) * kTile + lane] = row_op<N, 18, k, RS>(T.val, D, xcol);
          Xsh[(kk * kNq + 3 + (qv - 6)) * kTile + lane] = row_op<N, 19, k, RS>(T.val, D, xcol);
          Xsh[(kk * kNq + 6 + (qv - 6)) * kTile + lane] = row_op<N, 20, k, RS>(T.val, D, xcol);
        }
      }
    });
    __syncthreads();
    static_for<0, KC>([&](auto kkc) {
      constexpr int kk = decltype(kkc)::value;
      constexpr int k = k0 + kk;
      if constexpr (k < B) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int t = w + 9 * c;
          const Real* cc = V.cth + (((tile * 3 + tl[c]) * 3) * kStressSlots + ts0[c]) * kTile + lane;
          Real u = Real(0);
#pragma unroll
          for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int s = 0; s < 3; ++s)
              if (s < tcnt[c]) u = fma(__ldg(cc + (x * kStressSlots + s) * kTile), Xsh[(kk * kNq + 3 * x + tcol[c][s]) * kTile + lane], u);
          const size_t o = ((size_t)(9 + t) * B + k) * kTile + lane;
          Qt[o] += to_f64<Real, CVT>(u) - (double)tom[c] * It[o];
        }
      }
    });
    __syncthreads();
  });

  // ---- fluxes, FP faces per pass (FP32: two, so that the anelastic rows of Q are
  // read-modify-written twice instead of four times; FP64: one, two faces' staged
  // projections do not fit beside the shared operand rows)
  constexpr int FP = ThetaFacesPerPass<Real>::value;
  static_for<0, 4 / FP>([&](auto pass) {
    constexpr int f0 = decltype(pass)::value * FP;
    // own projections Yl [BT][9][32] and the neighbour's with f^h applied Yn, per face
    static_for<0, FP>([&](auto ff) {
      constexpr int sf = f0 + decltype(ff)::value;
      Real* Yl = Xf + (2 * decltype(ff)::value) * BT * kNq * kTile;
      Real* Yn = Yl + BT * kNq * kTile;
      const Real* P = Pown + ((e * 4 + sf) * kNq + w) * (size_t)PS;
      const int cn = __ldg(conn + e * 4 + sf);
      const size_t nb = (size_t)(cn >> 7);
      const int j = (cn >> 2) & 3, h = cn & 3;
      const Real* Pn = Pface + ((nb * 4 + j) * kNq + w) * (size_t)PS;
      Real pn[BT];
#pragma unroll
      for (int m = 0; m < BT; ++m) {
        Yl[(m * kNq + w) * kTile + lane] = P[m];
        pn[m] = Pn[m];
      }
      const Real* fh = T.f + (size_t)h * BT * BT;
#pragma unroll
      for (int d = 0; d <= N; ++d) {
        const int lo = d * (d + 1) / 2, hi = (d + 1) * (d + 2) / 2;
#pragma unroll
        for (int m = lo; m < hi; ++m) {
          Real v = Real(0);
#pragma unroll
          for (int n = lo; n < hi; ++n) v = fma(__ldg(fh + m + n * BT), pn[n], v);
          Yn[(m * kNq + w) * kTile + lane] = v;
        }
      }
    });
    __syncthreads();
    // one column after the other (unrolled, the two columns' lifting sequences were
    // interleaved and spilled kilobytes per thread)
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const int t = w + 9 * c;
      // W^s = (R^sT I) Aloc_s,t^T + (f^h R^jT I_nb) Anb_s,t^T of the pass's faces
      Real Wr[FP][BT];
      static_for<0, FP>([&](auto ff) {
        constexpr int fi = decltype(ff)::value, sf = f0 + fi;
        const Real* Yl = Xf + (2 * fi) * BT * kNq * kTile;
        const Real* Yn = Yl + BT * kNq * kTile;
        const Real* al = fthl + (((tile * 4 + sf) * kNTheta + t) * kNq) * kTile + lane;
        const Real* an = fthn + (((tile * 4 + sf) * kNTheta + t) * kNq) * kTile + lane;
        Real a[kNq], b[kNq];
#pragma unroll
        for (int q = 0; q < kNq; ++q) {
          a[q] = __ldg(al + q * kTile);
          b[q] = __ldg(an + q * kTile);
        }
#pragma unroll
        for (int m = 0; m < BT; ++m) {
          Real v = Real(0);
#pragma unroll
          for (int q = 0; q < kNq; ++q) {
            v = fma(a[q], Yl[(m * kNq + q) * kTile + lane], v);
            v = fma(b[q], Yn[(m * kNq + q) * kTile + lane], v);
          }
          Wr[fi][m] = v;
        }
      });
      // Q += sum_s Rhat^s W^s, eight rows at a time: their loads issued together ahead of
      // the stores
      double* qc = Qt + ((size_t)(9 + t) * B) * kTile + lane;
      static_for<0, (B + 7) / 8>([&](auto kc) {
        constexpr int k0 = decltype(kc)::value * 8;
        double qv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) qv[i] = (k0 + i < B) ? qc[(k0 + i < B ? k0 + i : 0) * kTile] : 0.0;
        static_for<0, 8>([&](auto ii) {
          constexpr int i = decltype(ii)::value;
          if constexpr (k0 + i < B) {
            Real dq = row_dotr<N, 25 + f0, k0 + i, Real, BT>(T.val, Wr[0]);
            if constexpr (FP == 2) dq += row_dotr<N, 25 + f0 + 1, k0 + i, Real, BT>(T.val, Wr[FP - 1]);
            qc[(k0 + i) * kTile] = qv[i] + to_f64<Real, CVT>(dq);
          }
        });
      });
    }
    __syncthreads();
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
  // 27-quantity steps
  void* theta;
  const void *cth, *om, *fthl, *fthn;
  size_t smem_theta;
  int pstride;             // values per face-projection row (0: BT)
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
        static_cast<const Real*>(L.star), static_cast<const Real*>(L.floc), T, L.SP, L.refs, VeTables<Real>{});
  } else {
    k_neigh<N, FUSED, Real><<<grid, kNq * kTile, L.smem_neigh, L.stream>>>(
        L.Q, L.groups, static_cast<const Real*>(L.Wloc), static_cast<const Real*>(L.fnb), L.conn, T, L.refs);
  }
}

// The small-mesh local update (k_local_small): 4 CTAs of 8 elements per tile.
template <int N, typename Real>
void ader_set_attribute_small(size_t) {
  cudaFuncSetAttribute(k_local_small<N, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)small_smem_bytes<N, Real>());
}
template <int N, typename Real>
void ader_launch_small(const AderLaunch& L) {
  k_local_small<N, Real><<<(unsigned)(L.ntiles * (kTile / kSmallElems)), kSmallThreads,
                           small_smem_bytes<N, Real>(), L.stream>>>(
      L.Q, L.Q, L.I, static_cast<Real*>(L.Pface), static_cast<const Real*>(L.star),
      static_cast<const Real*>(L.floc), step_tables<Real>(L), L.SP);
}

// Kernels of a 27-quantity step: WHICH 0 = k_local (VE, fused step), 1 = k_neigh on the
// elastic rows (fused step), 2 = k_theta.
// Shared memory of k_theta: the volume's operand rows and exchange, then (aliased) the
// staged projections of the faces of one pass.
inline size_t ader_theta_smem(int N, bool f32) {
  const int B = (N + 1) * (N + 2) * (N + 3) / 6, BT = (N + 1) * (N + 2) / 2;
  const int KC = BT / 3 > 0 ? BT / 3 : 1;
  const int fp = f32 ? ThetaFacesPerPass<float>::value : ThetaFacesPerPass<double>::value;
  const int rows = (B + KC) > 2 * fp * BT ? (B + KC) : 2 * fp * BT;
  return (size_t)(f32 ? 4 : 8) * rows * kNq * kTile;
}
template <int N, typename Real, int WHICH>
void ader_set_attribute_ve(size_t smem) {
  if constexpr (WHICH == 0)
    cudaFuncSetAttribute(k_local<N, false, Real, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else if constexpr (WHICH == 1)
    cudaFuncSetAttribute(k_neigh<N, true, Real, kNqVe>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  else
    cudaFuncSetAttribute(k_theta<N, Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template <int N, typename Real, int WHICH>
void ader_launch_ve(const AderLaunch& L) {
  const unsigned grid = (unsigned)L.ntiles;
  const StepTables<Real> T = step_tables<Real>(L);
  VeTables<Real> V;
  V.theta = static_cast<Real*>(L.theta);
  V.cth = static_cast<const Real*>(L.cth);
  V.om = static_cast<const Real*>(L.om);
  if constexpr (WHICH == 0) {
    k_local<N, false, Real, true><<<grid, kNq * kTile, L.smem_local, L.stream>>>(
        L.Q, L.Q, L.I, static_cast<Real*>(L.Pface), static_cast<Real*>(L.Wloc),
        static_cast<const Real*>(L.star), static_cast<const Real*>(L.floc), T, L.SP, nullptr, V);
  } else if constexpr (WHICH == 1) {
    k_neigh<N, true, Real, kNqVe><<<grid, kNq * kTile, L.smem_neigh, L.stream>>>(
        L.Q, L.groups, static_cast<const Real*>(L.Wloc), static_cast<const Real*>(L.fnb), L.conn, T, nullptr);
  } else {
    k_theta<N, Real><<<grid, kNq * kTile, L.smem_theta, L.stream>>>(
        L.Q, L.I, static_cast<const Real*>(L.Pface), static_cast<const Real*>(L.groups.base[0]),
        L.pstride > 0 ? L.pstride : Dims<N>::BT, L.conn, static_cast<const Real*>(L.fthl),
        static_cast<const Real*>(L.fthn), T, L.SP, V);
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
  YT_DECLARE_ADER_VARIANT(N, P, np)    \
  YT_DECLARE_ADER_VARIANT(N, P, vl)    \
  YT_DECLARE_ADER_VARIANT(N, P, vn)    \
  YT_DECLARE_ADER_VARIANT(N, P, vt)
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
#define YT_DECLARE_ADER_SMALL(N, P)                           \
  void ader_set_attribute_o##N##_##P##_ls(size_t);           \
  void ader_launch_o##N##_##P##_ls(const AderLaunch&);       \
  int ader_upload_o##N##_##P##_ls(const float*, size_t);
YT_DECLARE_ADER_SMALL(1, f64)
YT_DECLARE_ADER_SMALL(2, f64)
YT_DECLARE_ADER_SMALL(3, f64)
YT_DECLARE_ADER_SMALL(4, f64)
YT_DECLARE_ADER_SMALL(1, f32)
YT_DECLARE_ADER_SMALL(2, f32)
YT_DECLARE_ADER_SMALL(3, f32)
YT_DECLARE_ADER_SMALL(4, f32)
#undef YT_DECLARE_ADER_SMALL
#undef YT_DECLARE_ADER_UNIT
#undef YT_DECLARE_ADER_VARIANT
int ader_generated_nnz(int N);

}  // namespace yt
