// Elastic ADER-DG solver: device buffers, setup kernel, layout conversion and the C ABI
// entry points yt_solver_* / yt_step* (Sec. 5.1 of the paper).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "ader_kernels.cuh"
#include "ader_tc.cuh"
#include "batch_kernel.cuh"
#include "common.h"
#include "solver_internal.h"
#include "tables.h"

using namespace yt;

namespace {

// Elastic Jacobians A^j (j = x, y, z) of the velocity-stress system
// q = (sxx, syy, szz, sxy, syz, sxz, u, v, w): eight entries each.
// kind 0: -(lambda + 2 mu), 1: -lambda, 2: -mu, 3: -1/rho.
struct JacEntry { int8_t p, q, kind; };
__constant__ JacEntry c_jac[3][8] = {
    {{0, 6, 0}, {1, 6, 1}, {2, 6, 1}, {3, 7, 2}, {5, 8, 2}, {6, 0, 3}, {7, 3, 3}, {8, 5, 3}},
    {{0, 7, 1}, {1, 7, 0}, {2, 7, 1}, {3, 6, 2}, {4, 8, 2}, {6, 3, 3}, {7, 1, 3}, {8, 4, 3}},
    {{0, 8, 1}, {1, 8, 1}, {2, 8, 0}, {4, 7, 2}, {5, 6, 2}, {6, 5, 3}, {7, 4, 3}, {8, 2, 3}}};
// Star slots grouped by row (union of the three patterns): row p owns slots
// [start[p], start[p+1]) with columns col[slot].
const StarPattern kStar = {{0, 3, 6, 9, 11, 13, 15, 18, 21, 24},
                           {6, 7, 8, 6, 7, 8, 6, 7, 8, 6, 7, 7, 8, 6, 8, 0, 3, 5, 1, 3, 4, 2, 4, 5}};
__constant__ StarPattern c_star;

const int kFaceVerts[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};
__constant__ int c_face_verts[4][3];

__device__ void mat9_mul(const double* a, const double* b, double* c) {
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j) {
      double s = 0.0;
      for (int k = 0; k < 9; ++k) s = fma(a[i * 9 + k], b[k * 9 + j], s);
      c[i * 9 + j] = s;
    }
}

// Setup (not part of a step): star matrices Astar^x = sum_j (dxi_x/dx_j) A^j and upwind
// flux solvers -(2|S|/|J|)(A_n +- |A_n|)/2.  |A_n| = alpha A_n^2 + beta A_n^4 is the even
// polynomial interpolating |lambda| on the spectrum {0, +-c_s, +-c_p} of the
// diagonalisable A_n: alpha = (cp^2 + cp cs + cs^2) / (cp cs (cp + cs)),
// beta = -1 / (cp cs (cp + cs)).  One thread per element.
__global__ void k_setup(const double* __restrict__ material, const double* __restrict__ jac,
                        int64_t E, int64_t Epad, double* __restrict__ star,
                        double* __restrict__ floc, double* __restrict__ fnb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Epad) return;
  const int64_t tile = e / kTile;
  const int lane = (int)(e % kTile);
  if (e >= E) {
    for (int i = 0; i < 3 * kStarSlots; ++i) star[(tile * 3 * kStarSlots + i) * kTile + lane] = 0.0;
    for (int i = 0; i < 4 * 81; ++i) {
      floc[(tile * 4 * 81 + i) * kTile + lane] = 0.0;
      fnb[(tile * 4 * 81 + i) * kTile + lane] = 0.0;
    }
    return;
  }
  const double rho = material[e * 3 + 0], lam = material[e * 3 + 1], mu = material[e * 3 + 2];
  double J[9];
  for (int i = 0; i < 9; ++i) J[i] = jac[e * 9 + i];       // J[i + 3c] = dx_i / dxi_c
  auto Jm = [&](int i, int c) { return J[i + 3 * c]; };
  const double det = Jm(0, 0) * (Jm(1, 1) * Jm(2, 2) - Jm(1, 2) * Jm(2, 1)) -
                     Jm(0, 1) * (Jm(1, 0) * Jm(2, 2) - Jm(1, 2) * Jm(2, 0)) +
                     Jm(0, 2) * (Jm(1, 0) * Jm(2, 1) - Jm(1, 1) * Jm(2, 0));
  // G[d][j] = dxi_d / dx_j = (J^-1)_{dj} via the adjugate
  double G[3][3];
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < 3; ++j) {
      const int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (d + 1) % 3, c1 = (d + 2) % 3;
      G[d][j] = (Jm(r0, c0) * Jm(r1, c1) - Jm(r0, c1) * Jm(r1, c0)) / det;
    }
  const double val[4] = {-(lam + 2.0 * mu), -lam, -mu, -1.0 / rho};
  double A[3][81];
  for (int j = 0; j < 3; ++j) {
    for (int i = 0; i < 81; ++i) A[j][i] = 0.0;
    for (int t = 0; t < 8; ++t) A[j][c_jac[j][t].p * 9 + c_jac[j][t].q] = val[c_jac[j][t].kind];
  }
  for (int d = 0; d < 3; ++d)
    for (int p = 0; p < kNq; ++p)
      for (int s = c_star.start[p]; s < c_star.start[p + 1]; ++s) {
        const int q = c_star.col[s];
        double v = 0.0;
        for (int j = 0; j < 3; ++j) v = fma(G[d][j], A[j][p * 9 + q], v);
        star[((tile * 3 + d) * kStarSlots + s) * kTile + lane] = v;
      }
  const double cp = sqrt((lam + 2.0 * mu) / rho), cs = sqrt(mu / rho);
  const double alpha = (cp * cp + cp * cs + cs * cs) / (cp * cs * (cp + cs));
  const double beta = -1.0 / (cp * cs * (cp + cs));
  const double V[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int s = 0; s < 4; ++s) {
    double X[3][3];
    for (int v = 0; v < 3; ++v)
      for (int i = 0; i < 3; ++i) {
        const double* r = V[c_face_verts[s][v]];
        X[v][i] = Jm(i, 0) * r[0] + Jm(i, 1) * r[1] + Jm(i, 2) * r[2];
      }
    double u[3], t[3], c[3];
    for (int i = 0; i < 3; ++i) { u[i] = X[1][i] - X[0][i]; t[i] = X[2][i] - X[0][i]; }
    c[0] = u[1] * t[2] - u[2] * t[1];
    c[1] = u[2] * t[0] - u[0] * t[2];
    c[2] = u[0] * t[1] - u[1] * t[0];
    const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double area = 0.5 * len;
    double An[81], A2[81], A4[81];
    for (int i = 0; i < 81; ++i) An[i] = (c[0] * A[0][i] + c[1] * A[1][i] + c[2] * A[2][i]) / len;
    mat9_mul(An, An, A2);
    mat9_mul(A2, A2, A4);
    const double scale = -(2.0 * area / det) * 0.5;
    for (int i = 0; i < 81; ++i) {
      const double absA = alpha * A2[i] + beta * A4[i];
      floc[((tile * 4 + s) * 81 + i) * kTile + lane] = scale * (An[i] + absA);
      fnb[((tile * 4 + s) * 81 + i) * kTile + lane] = scale * (An[i] - absA);
    }
  }
}

// Setup of the anelastic rows of a 27-quantity solver (FP64, one thread per element):
//   star slots of theta^l_i:  sum_j (dxi_x/dx_j) omega_l A^j_{sigma_i, v}(Y^lambda_l, Y^mu_l)
//                             in the slots of stress row i (velocity columns);
//   omega_l;
//   flux-solver rows: the 27 x 27 A_n = [[A_e, 0], [C, 0]] (C = its anelastic rows, velocity
//   columns only) is diagonalisable with the spectrum of A_e plus zeros, so |A_n| is the
//   same even polynomial alpha A_n^2 + beta A_n^4, whose anelastic rows are
//   C (alpha A_e + beta A_e^3); Aloc / Anb rows = -(2|S|/|J|)(C +- C (alpha A_e + beta A_e^3))/2.
// att: [e][l][omega, Y^lambda, Y^mu]; outputs [tile][...][32] as the kernels read them.
__global__ void k_setup_theta(const double* __restrict__ material, const double* __restrict__ jac,
                              const double* __restrict__ att, int64_t E, int64_t Epad,
                              double* __restrict__ cth, double* __restrict__ om,
                              double* __restrict__ fthl, double* __restrict__ fthn) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Epad) return;
  const int64_t tile = e / kTile;
  const int lane = (int)(e % kTile);
  if (e >= E) {
    for (int i = 0; i < 3 * 3 * kStressSlots; ++i) cth[(tile * 3 * 3 * kStressSlots + i) * kTile + lane] = 0.0;
    for (int i = 0; i < 3; ++i) om[(tile * 3 + i) * kTile + lane] = 0.0;
    for (int i = 0; i < 4 * kNTheta * kNq; ++i) {
      fthl[(tile * 4 * kNTheta * kNq + i) * kTile + lane] = 0.0;
      fthn[(tile * 4 * kNTheta * kNq + i) * kTile + lane] = 0.0;
    }
    return;
  }
  const double rho = material[e * 3 + 0], lam = material[e * 3 + 1], mu = material[e * 3 + 2];
  double J[9];
  for (int i = 0; i < 9; ++i) J[i] = jac[e * 9 + i];
  auto Jm = [&](int i, int c) { return J[i + 3 * c]; };
  const double det = Jm(0, 0) * (Jm(1, 1) * Jm(2, 2) - Jm(1, 2) * Jm(2, 1)) -
                     Jm(0, 1) * (Jm(1, 0) * Jm(2, 2) - Jm(1, 2) * Jm(2, 0)) +
                     Jm(0, 2) * (Jm(1, 0) * Jm(2, 1) - Jm(1, 1) * Jm(2, 0));
  double G[3][3];
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < 3; ++j) {
      const int r0 = (j + 1) % 3, r1 = (j + 2) % 3, c0 = (d + 1) % 3, c1 = (d + 2) % 3;
      G[d][j] = (Jm(r0, c0) * Jm(r1, c1) - Jm(r0, c1) * Jm(r1, c0)) / det;
    }
  const double val[4] = {-(lam + 2.0 * mu), -lam, -mu, -1.0 / rho};
  double A[3][81];
  for (int j = 0; j < 3; ++j) {
    for (int i = 0; i < 81; ++i) A[j][i] = 0.0;
    for (int t = 0; t < 8; ++t) A[j][c_jac[j][t].p * 9 + c_jac[j][t].q] = val[c_jac[j][t].kind];
  }
  // anelastic Jacobian rows: Ath[l][j][i][v] (stress component i, velocity v)
  double Ath[3][3][6][3];
  for (int l = 0; l < 3; ++l) {
    const double w = att[(e * 3 + l) * 3 + 0], yl = att[(e * 3 + l) * 3 + 1], ym = att[(e * 3 + l) * 3 + 2];
    const double vy[3] = {-(yl + 2.0 * ym), -yl, -ym};
    om[(tile * 3 + l) * kTile + lane] = w;
    for (int j = 0; j < 3; ++j) {
      for (int i = 0; i < 6; ++i)
        for (int v = 0; v < 3; ++v) Ath[l][j][i][v] = 0.0;
      for (int t = 0; t < 8; ++t)
        if (c_jac[j][t].p < 6) Ath[l][j][c_jac[j][t].p][c_jac[j][t].q - 6] = w * vy[c_jac[j][t].kind];
    }
    for (int d = 0; d < 3; ++d)
      for (int p = 0; p < 6; ++p)
        for (int s = c_star.start[p]; s < c_star.start[p + 1]; ++s) {
          const int v = c_star.col[s] - 6;
          double x = 0.0;
          for (int j = 0; j < 3; ++j) x = fma(G[d][j], Ath[l][j][p][v], x);
          cth[(((tile * 3 + l) * 3 + d) * kStressSlots + s) * kTile + lane] = x;
        }
  }
  const double cp = sqrt((lam + 2.0 * mu) / rho), cs = sqrt(mu / rho);
  const double alpha = (cp * cp + cp * cs + cs * cs) / (cp * cs * (cp + cs));
  const double beta = -1.0 / (cp * cs * (cp + cs));
  const double V[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int s = 0; s < 4; ++s) {
    double X[3][3];
    for (int v = 0; v < 3; ++v)
      for (int i = 0; i < 3; ++i) {
        const double* r = V[c_face_verts[s][v]];
        X[v][i] = Jm(i, 0) * r[0] + Jm(i, 1) * r[1] + Jm(i, 2) * r[2];
      }
    double u[3], t[3], c[3];
    for (int i = 0; i < 3; ++i) { u[i] = X[1][i] - X[0][i]; t[i] = X[2][i] - X[0][i]; }
    c[0] = u[1] * t[2] - u[2] * t[1];
    c[1] = u[2] * t[0] - u[0] * t[2];
    c[2] = u[0] * t[1] - u[1] * t[0];
    const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double area = 0.5 * len;
    double An[81], A2[81], A3[81], qa[81];
    for (int i = 0; i < 81; ++i) An[i] = (c[0] * A[0][i] + c[1] * A[1][i] + c[2] * A[2][i]) / len;
    mat9_mul(An, An, A2);
    mat9_mul(An, A2, A3);
    for (int i = 0; i < 81; ++i) qa[i] = alpha * An[i] + beta * A3[i];
    const double scale = -(2.0 * area / det) * 0.5;
    for (int l = 0; l < 3; ++l)
      for (int i = 0; i < 6; ++i) {
        double Cn[9];
        for (int q = 0; q < 9; ++q) Cn[q] = 0.0;
        for (int v = 0; v < 3; ++v)
          Cn[6 + v] = (c[0] * Ath[l][0][i][v] + c[1] * Ath[l][1][i][v] + c[2] * Ath[l][2][i][v]) / len;
        for (int q = 0; q < 9; ++q) {
          double a = 0.0;
          for (int r = 6; r < 9; ++r) a = fma(Cn[r], qa[r * 9 + q], a);
          const size_t o = ((((size_t)tile * 4 + s) * kNTheta + 6 * l + i) * kNq + q) * kTile + lane;
          fthl[o] = scale * (Cn[q] + a);
          fthn[o] = scale * (Cn[q] - a);
        }
      }
  }
}

// canonical [e][q][k] <-> element-blocked [tile][q][k][lane], P quantities per element
__global__ void k_to_blocked(const double* __restrict__ in, double* __restrict__ out,
                             int64_t E, int64_t Epad, int B, int P) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = Epad * P * B;
  if (i >= total) return;
  const int lane = (int)(i % kTile);
  const int64_t rest = i / kTile;
  const int k = (int)(rest % B);
  const int q = (int)((rest / B) % P);
  const int64_t tile = rest / ((int64_t)B * P);
  const int64_t e = tile * kTile + lane;
  out[i] = e < E ? in[(e * P + q) * B + k] : 0.0;
}
__global__ void k_from_blocked(const double* __restrict__ in, double* __restrict__ out,
                               int64_t E, int B, int P) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E * P * B) return;
  const int k = (int)(i % B);
  const int q = (int)((i / B) % P);
  const int64_t e = i / ((int64_t)B * P);
  out[i] = in[(((e / kTile) * P + q) * B + k) * kTile + (e % kTile)];
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

// --------------------------------------------------------------------- host helpers
struct Csr {
  std::vector<int> rp;
  std::vector<uint16_t> col;
  std::vector<double> val;
  // Appends the CSR of a rows x cols view; `at(r, c)` gives the entry.  Returns the rp
  // offset.  Flops of the lists are accumulated by the caller.
  // Values are stored multiplied by `scale`; the pattern is that of the unscaled entries.
  template <typename F>
  int add(int rows, int cols, F at, double scale = 1.0) {
    const int off = static_cast<int>(rp.size());
    for (int r = 0; r < rows; ++r) {
      rp.push_back(static_cast<int>(col.size()));
      for (int c = 0; c < cols; ++c) {
        const double v = at(r, c);
        if (v != 0.0) {
          col.push_back(static_cast<uint16_t>(c));
          val.push_back(v * scale);
        }
      }
    }
    rp.push_back(static_cast<int>(col.size()));
    return off;
  }
  int64_t row_nnz(int off, int r) const { return rp[off + r + 1] - rp[off + r]; }
};

// Allocation mode of the calling thread (solver_create_stream_ordered sets it while it
// creates a solver): stream-ordered allocations on that stream, each followed by a
// synchronisation of that stream so that the memory is ready for any stream.
struct AllocMode {
  bool async = false;
  cudaStream_t stream = nullptr;
};
thread_local AllocMode t_alloc;

template <typename T>
T* dalloc(size_t n) {
  T* p = nullptr;
  if (t_alloc.async) {
    cuda_check(cudaMallocAsync(reinterpret_cast<void**>(&p), n * sizeof(T) + 16, t_alloc.stream), "cudaMallocAsync");
    cuda_check(cudaStreamSynchronize(t_alloc.stream), "allocation sync");
  } else {
    cuda_check(cudaMalloc(&p, n * sizeof(T) + 16), "cudaMalloc");
  }
  return p;
}
// Allocation in the mode of solver s (its buffers created after yt_solver_create).
template <typename T>
T* sdalloc(const yt_solver* s, size_t n) {
  const AllocMode saved = t_alloc;
  t_alloc.async = s->alloc_async;
  t_alloc.stream = s->alloc_stream;
  T* p = nullptr;
  try {
    p = dalloc<T>(n);
  } catch (...) {
    t_alloc = saved;
    throw;
  }
  t_alloc = saved;
  return p;
}
void dfree_temp(void* p) {
  if (!p) return;
  if (t_alloc.async) cudaFreeAsync(p, t_alloc.stream);
  else cudaFree(p);
}

}  // namespace

namespace {

AderLaunch launch_args(yt_solver* s, cudaStream_t st) {
  AderLaunch L;
  L.ntiles = s->ntiles;
  L.smem_local = s->smem_local;
  L.smem_neigh = s->smem_neigh;
  L.Q = s->Q;
  L.I = s->I;
  L.Pface = s->Pface;
  L.Wloc = s->Wloc;
  L.star = s->star_r;
  L.floc = s->floc_r;
  L.fnb = s->fnb_r;
  L.conn = s->conn;
  L.groups = FaceGroups{};
  L.groups.base[0] = s->Pface;
  L.groups.bt[0] = s->BT;
  L.groups.base[1] = s->halo;      // partitioned solves: remote face projections
  L.groups.bt[1] = s->BT;
  const bool f32 = s->prec != YT_F64;
  L.val = f32 ? (const void*)s->d_val32 : (const void*)s->d_val;
  L.f = f32 ? (const void*)s->d_f32 : (const void*)s->d_f;
  L.dt = s->dt;
  L.refs = nullptr;
  L.SP = kStar;
  L.theta = s->theta;
  L.cth = s->cth_r;
  L.om = s->om_r;
  L.fthl = s->fthl_r;
  L.fthn = s->fthn_r;
  L.smem_theta = s->smem_theta;
  L.pstride = s->prec == YT_BF16X3_F32ACC ? tc::up8(s->BT) : s->BT;
  L.stream = st;
  return L;
}

#define YT_VARIANT_SWITCH(FN, V, ...)                                          \
  do {                                                                         \
    switch (s->N * 2 + (s->prec == YT_F32 ? 1 : 0)) {                          \
      case 2: FN##_o1_f64_##V(__VA_ARGS__); break;                            \
      case 3: FN##_o1_f32_##V(__VA_ARGS__); break;                            \
      case 4: FN##_o2_f64_##V(__VA_ARGS__); break;                            \
      case 5: FN##_o2_f32_##V(__VA_ARGS__); break;                            \
      case 6: FN##_o3_f64_##V(__VA_ARGS__); break;                            \
      case 7: FN##_o3_f32_##V(__VA_ARGS__); break;                            \
      case 8: FN##_o4_f64_##V(__VA_ARGS__); break;                            \
      case 9: FN##_o4_f32_##V(__VA_ARGS__); break;                            \
      case 10: FN##_o5_f64_##V(__VA_ARGS__); break;                           \
      case 11: FN##_o5_f32_##V(__VA_ARGS__); break;                           \
      case 12: FN##_o6_f64_##V(__VA_ARGS__); break;                           \
      case 13: FN##_o6_f32_##V(__VA_ARGS__); break;                           \
      default: throw Error(YT_ERR_UNSUPPORTED, "no kernel for this order and precision"); \
    }                                                                          \
  } while (0)

// The small-mesh local kernel of degree N <= 4 and the solver's contraction type
#define YT_SMALL_SWITCH(FN, ...)                                               \
  do {                                                                         \
    switch (s->N * 2 + (s->prec == YT_F32 ? 1 : 0)) {                          \
      case 2: FN##_o1_f64_ls(__VA_ARGS__); break;                             \
      case 3: FN##_o1_f32_ls(__VA_ARGS__); break;                             \
      case 4: FN##_o2_f64_ls(__VA_ARGS__); break;                             \
      case 5: FN##_o2_f32_ls(__VA_ARGS__); break;                             \
      case 6: FN##_o3_f64_ls(__VA_ARGS__); break;                             \
      case 7: FN##_o3_f32_ls(__VA_ARGS__); break;                             \
      case 8: FN##_o4_f64_ls(__VA_ARGS__); break;                             \
      case 9: FN##_o4_f32_ls(__VA_ARGS__); break;                             \
      default: throw Error(YT_ERR_UNSUPPORTED, "no small-mesh kernel for this order"); \
    }                                                                          \
  } while (0)

// k_theta of the FP32 contraction type whatever the solver's precision (the anelastic
// rows of a tensor-core 27-quantity step run on the CUDA cores in FP32)
#define YT_THETA_F32_SWITCH(FN, ...)                                           \
  do {                                                                         \
    switch (s->N) {                                                            \
      case 1: FN##_o1_f32_vt(__VA_ARGS__); break;                             \
      case 2: FN##_o2_f32_vt(__VA_ARGS__); break;                             \
      case 3: FN##_o3_f32_vt(__VA_ARGS__); break;                             \
      case 4: FN##_o4_f32_vt(__VA_ARGS__); break;                             \
      case 5: FN##_o5_f32_vt(__VA_ARGS__); break;                             \
      case 6: FN##_o6_f32_vt(__VA_ARGS__); break;                             \
      default: throw Error(YT_ERR_UNSUPPORTED, "no kernel for this order");    \
    }                                                                          \
  } while (0)

// Shared memory of the two kernels of degree N: k_local holds the operand rows not kept
// in registers, the exchange buffer and (with register operands) the time-integral
// accumulator; k_neigh the four faces' flux products.
void set_smem(yt_solver* s) {
  const int N = s->N;
  if (s->prec == YT_BF16X3_F32ACC) {
    s->smem_local = tc_smem_local(N);
    s->smem_neigh = tc_smem_neigh(N);
    int dev = 0, optin = 0;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    cuda_check(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "device attribute");
    YT_REQUIRE(s->smem_local <= (size_t)optin && s->smem_neigh <= (size_t)optin, YT_ERR_UNSUPPORTED,
               "tensor-core step: shared memory of this order exceeds the device limit");
    tc_set_attributes(N);
    if (s->P == kNqVe) {
      tc_set_attributes_ve(N);
      s->smem_theta = ader_theta_smem(N, true);
      YT_REQUIRE(s->smem_theta <= (size_t)optin, YT_ERR_UNSUPPORTED, "order too high for this precision");
      YT_THETA_F32_SWITCH(ader_set_attribute, s->smem_theta);
    }
    cuda_check(cudaGetLastError(), "cudaFuncSetAttribute");
    return;
  }
  s->smem_local = ader_local_smem(N, s->prec != YT_F64);
  s->smem_neigh = ader_neigh_smem(N, s->prec != YT_F64);
  YT_REQUIRE(s->smem_local <= 227 * 1024 && s->smem_neigh <= 227 * 1024, YT_ERR_UNSUPPORTED,
             "order too high for this precision");
  if (s->P == kNqVe) {
    s->smem_theta = ader_theta_smem(N, s->prec != YT_F64);
    YT_REQUIRE(s->smem_theta <= 227 * 1024, YT_ERR_UNSUPPORTED, "order too high for this precision");
    YT_VARIANT_SWITCH(ader_set_attribute, vl, s->smem_local);
    YT_VARIANT_SWITCH(ader_set_attribute, vn, s->smem_neigh);
    YT_VARIANT_SWITCH(ader_set_attribute, vt, s->smem_theta);
    cuda_check(cudaGetLastError(), "cudaFuncSetAttribute");
    return;
  }
  YT_VARIANT_SWITCH(ader_set_attribute, lf, s->smem_local);
  YT_VARIANT_SWITCH(ader_set_attribute, ll, s->smem_local);
  YT_VARIANT_SWITCH(ader_set_attribute, nf, s->smem_neigh);
  YT_VARIANT_SWITCH(ader_set_attribute, np, s->smem_neigh);
  // small meshes: the local update on 8-element CTAs when the tiles do not fill the SMs
  int dev = 0, sms = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  s->small_local = N <= 4 && s->ntiles <= sms;
  if (s->small_local) YT_SMALL_SWITCH(ader_set_attribute, 0);
  cuda_check(cudaGetLastError(), "cudaFuncSetAttribute");
}

tc::TcLaunch tc_args(yt_solver* s, cudaStream_t st, int64_t t0 = 0, int64_t nt = -1) {
  tc::TcLaunch L;
  if (nt < 0) nt = s->ntiles;
  const size_t e0 = (size_t)t0 * kTile;
  L.ntiles = nt;
  L.tile0 = t0;
  L.grid = (unsigned)std::min<int64_t>(nt, s->tc_grid);
  L.Q = s->Q + e0 * s->P * s->B;
  L.I = s->I + e0 * s->P * s->B;
  L.Pface = static_cast<float*>(s->Pface);             // gathered by absolute index
  L.Wloc = static_cast<float*>(s->Wloc) + e0 * 4 * kNq * s->BT;
  L.star = static_cast<const float*>(s->star_r) + e0 * 3 * kStarSlots;
  L.floc = static_cast<const float*>(s->floc_r) + e0 * 4 * 81;
  L.fnb = static_cast<const float*>(s->fnb_r) + e0 * 4 * 81;
  L.f = s->d_f32;
  L.conn = s->conn + e0 * 4;
  L.blob_local = s->d_tc_local;
  L.scratch = s->d_tc_scratch;
  L.vol = s->d_tc_vol ? s->d_tc_vol + e0 * kNq * s->B : nullptr;
  L.blob_neigh = s->d_tc_neigh;
  L.ve = VeTables<float>{};
  if (s->P == kNqVe) {
    L.ve.theta = static_cast<float*>(s->theta) + e0 * kNTheta * s->B;
    L.ve.cth = static_cast<const float*>(s->cth_r) + e0 * 3 * 3 * kStressSlots;
    L.ve.om = static_cast<const float*>(s->om_r) + e0 * 3;
  }
  L.dt = s->dt;
  L.SP = kStar;
  L.status = s->d_status;
  L.expire_first_wait = s->diag_expire_wait ? 1 : 0;
  L.stream = st;
  return L;
}

// Launch arguments restricted to tiles [t0, t0 + nt): every per-tile array is offset;
// the neighbour kernel still gathers face projections of all elements (groups.base).
AderLaunch chunk_args(const AderLaunch& F, const yt_solver* s, int64_t t0, int64_t nt) {
  AderLaunch L = F;
  const size_t rb = s->real_bytes;
  L.ntiles = nt;
  L.Q += (size_t)t0 * s->P * s->B * kTile;
  L.I += (size_t)t0 * s->P * s->B * kTile;
  if (s->P == kNqVe) {
    L.theta = static_cast<unsigned char*>(L.theta) + (size_t)t0 * kNTheta * s->B * kTile * rb;
    L.cth = static_cast<const unsigned char*>(L.cth) + (size_t)t0 * 3 * 3 * kStressSlots * kTile * rb;
    L.om = static_cast<const unsigned char*>(L.om) + (size_t)t0 * 3 * kTile * rb;
    L.fthl = static_cast<const unsigned char*>(L.fthl) + (size_t)t0 * 4 * kNTheta * kNq * kTile * rb;
    L.fthn = static_cast<const unsigned char*>(L.fthn) + (size_t)t0 * 4 * kNTheta * kNq * kTile * rb;
  }
  L.Pface = static_cast<unsigned char*>(L.Pface) + (size_t)t0 * kTile * 4 * kNq * L.pstride * rb;
  L.Wloc = static_cast<unsigned char*>(L.Wloc) + (size_t)t0 * kTile * 4 * kNq * s->BT * rb;
  L.star = static_cast<const unsigned char*>(L.star) + (size_t)t0 * 3 * kStarSlots * kTile * rb;
  L.floc = static_cast<const unsigned char*>(L.floc) + (size_t)t0 * 4 * 81 * kTile * rb;
  L.fnb = static_cast<const unsigned char*>(L.fnb) + (size_t)t0 * 4 * 81 * kTile * rb;
  L.conn += (size_t)t0 * kTile * 4;
  return L;
}

// Tensor-core form, fused step over tiles [t0, t0 + nt): phase 0 k_local_tc, phase 1 the
// lifting kernel (local and neighbour products through Rhat^s); 27 quantities: the
// elastic rows so, and k_theta (FP32 CUDA cores) for the anelastic rows after them.
void dispatch_tc_fused(yt_solver* s, cudaStream_t st, int phase, int64_t t0, int64_t nt) {
  const tc::TcLaunch T = tc_args(s, st, t0, nt);
  if (s->P == kNqVe) {
    if (phase == 0) {
      tc_launch_local_ve(s->N, T);
    } else {
      tc_launch_neigh_ve(s->N, T);
      const AderLaunch L = chunk_args(launch_args(s, st), s, t0, T.ntiles);
      YT_THETA_F32_SWITCH(ader_launch, L);
    }
  } else if (phase == 0) {
    tc_launch_local(s->N, T);
  } else {
    tc_launch_neigh(s->N, T, 0);
  }
}

// Tensor-core form: k_local_tc writes the local flux products, and the lifting kernel
// adds them (fused step: with the neighbour products) through Rhat^s.
void dispatch_local(yt_solver* s, cudaStream_t st, bool fused) {
  if (s->prec == YT_BF16X3_F32ACC) {
    if (fused) {
      dispatch_tc_fused(s, st, 0, 0, -1);
    } else {
      YT_REQUIRE(s->P == kNq, YT_ERR_UNSUPPORTED, "27-quantity solvers: fused step only (yt_step, yt_step_phase)");
      const tc::TcLaunch T = tc_args(s, st);
      tc_launch_local(s->N, T);
      tc_launch_neigh(s->N, T, 2);
    }
    cuda_check(cudaGetLastError(), "k_local_tc launch");
    return;
  }
  const AderLaunch L = launch_args(s, st);
  if (s->P == kNqVe) {
    YT_REQUIRE(fused, YT_ERR_UNSUPPORTED, "27-quantity solvers: fused step only (yt_step, yt_step_phase)");
    YT_VARIANT_SWITCH(ader_launch, vl, L);
  } else if (fused) {
    YT_VARIANT_SWITCH(ader_launch, lf, L);
  } else if (s->small_local) {
    YT_SMALL_SWITCH(ader_launch, L);
  } else {
    YT_VARIANT_SWITCH(ader_launch, ll, L);
  }
  cuda_check(cudaGetLastError(), "k_local launch");
}
void dispatch_neigh(yt_solver* s, cudaStream_t st, bool fused) {
  if (s->prec == YT_BF16X3_F32ACC) {
    if (fused) {
      dispatch_tc_fused(s, st, 1, 0, -1);
    } else {
      YT_REQUIRE(s->P == kNq, YT_ERR_UNSUPPORTED, "27-quantity solvers: fused step only (yt_step, yt_step_phase)");
      tc_launch_neigh(s->N, tc_args(s, st), 1);
    }
    cuda_check(cudaGetLastError(), "k_neigh_tc launch");
    return;
  }
  const AderLaunch L = launch_args(s, st);
  if (s->P == kNqVe) {
    YT_REQUIRE(fused, YT_ERR_UNSUPPORTED, "27-quantity solvers: fused step only (yt_step, yt_step_phase)");
    YT_VARIANT_SWITCH(ader_launch, vn, L);
    YT_VARIANT_SWITCH(ader_launch, vt, L);
  } else if (fused) {
    YT_VARIANT_SWITCH(ader_launch, nf, L);
  } else {
    YT_VARIANT_SWITCH(ader_launch, np, L);
  }
  cuda_check(cudaGetLastError(), "k_neigh launch");
}

// Packs the non-zero values of the sparse lists of one order (in the order the generated
// kernels read them) and counts the flops / bytes of the two kernels.
void build_tables(yt_solver* s) {
  const RefMatrices& R = reference_matrices(s->N);
  const int N = s->N, B = R.B, BT = R.BT;
  Csr csr;
  auto nd = [N](int delta) { return (N - delta + 3) * (N - delta + 2) * (N - delta + 1) / 6; };
  // Non-zero flops per element in the convention of Sec. 4.9: an entry that is a sum of n
  // non-zero products costs 2n - 1 flops when assigned and 2n when added to an existing
  // value; a scaling costs 1.  The derivatives' factor dt (an implementation choice that
  // keeps their magnitude bounded) is not counted.
  auto assigned = [&](int off, int rows) {
    double f = 0.0;
    for (int r = 0; r < rows; ++r) {
      const int n = csr.row_nnz(off, r);
      if (n > 0) f += 9.0 * (2.0 * n - 1.0);
    }
    return f;
  };
  auto nnz_total = [&](int off, int rows) {
    double n = 0.0;
    for (int r = 0; r < rows; ++r) n += csr.row_nnz(off, r);
    return n;
  };
  // mixing with the three star matrices: entry p sums 3 * cnt_p products (cnt_p = non-zeros
  // of star row p, 24 per matrix): assigned sum_p (6 cnt_p - 1) = 135, added 144 per row
  const double mix_assigned = 6.0 * kStarSlots - 9.0, mix_added = 6.0 * kStarSlots;
  double fl = 9.0 * B;                                     // I = c0 Q
  int off_kt0[3] = {0, 0, 0}, off_kh[3] = {0, 0, 0};
  for (int delta = 0; delta < N; ++delta) {
    const int nin = nd(delta), nout = nd(delta + 1);
    for (int x = 0; x < 3; ++x) {
      const double* K = R.Ktilde.data() + (size_t)x * B * B;
      const int off = csr.add(nout, nin, [&](int r, int c) { return K[r + (size_t)c * B]; });
      if (delta == 0) off_kt0[x] = off;
      fl += assigned(off, nout);                           // X^x = Ktilde^x D
    }
    fl += nout * (mix_assigned + 2.0 * 9);                 // D' = sum_x X^x A^xT; I += c D'
  }
  double fkh = 0.0;
  for (int x = 0; x < 3; ++x) {
    const double* K = R.Khat.data() + (size_t)x * B * B;
    off_kh[x] = csr.add(B, B, [&](int r, int c) { return K[r + (size_t)c * B]; });
    fkh += assigned(off_kh[x], B);                         // X^x = Khat^x I
  }
  fl += fkh + B * mix_added;                               // Q += sum_x X^x A^xT
  double fn = 0.0, lift_total = 0.0, fproj = 0.0, ftheta_faces = 0.0;
  for (int f = 0; f < 4; ++f) {
    const double* Rs = R.R.data() + (size_t)f * B * BT;
    const double* Rh = R.Rhat.data() + (size_t)f * B * BT;
    const int off_rt = csr.add(BT, B, [&](int r, int c) { return Rs[c + (size_t)r * B]; });
    const int off_rh = csr.add(B, BT, [&](int r, int c) { return Rh[r + (size_t)c * B]; });
    fproj += assigned(off_rt, BT) + BT * 9.0 * 17.0;      // P = R^T I; Wloc = P Aloc^T
    const double lift = 9.0 * 2.0 * nnz_total(off_rh, B);  // Q += Rhat W (per face)
    lift_total += lift;
    double blocks = 0.0;                                   // V = f^h P_nb, block-diagonal
    for (int d = 0; d <= N; ++d) blocks += (d + 1.0) * (2.0 * (d + 1.0) - 1.0);
    fn += 9.0 * blocks + BT * 9.0 * 18.0 + lift;           // W = Wloc + V Anb^T; lifting
    // anelastic rows (27 quantities, k_theta): V as above; W of 18 functions from the 9
    // local and 9 neighbour projections (18 products each); their lifting
    ftheta_faces += 9.0 * blocks + BT * 18.0 * 35.0 + 2.0 * lift;
  }
  fl += fproj;
  if (s->P == kNqVe) {
    // 27 quantities.  k_local: every derivative uses the unrestricted lists of delta = 0
    // and writes all B rows: elastic rows of degree < N as above; per row the stress
    // feedback -sum_l theta^l_i (3 per stress row), the stress rows of degree N (scaling,
    // accumulation: 3); the anelastic functions: rows of degree < N mix 3 cnt_i products
    // plus -omega theta (6 cnt_i + 1), scaling 1, accumulation 2; rows of degree N 4.
    const int NI = nd(1);
    double kt0 = 0.0;
    for (int x = 0; x < 3; ++x) kt0 += assigned(off_kt0[x], NI);
    const double per_deriv = kt0 + NI * (mix_assigned + 2.0 * 9) + B * 18.0 + (B - NI) * 6 * 3.0 +
                             NI * 3.0 * (6.0 * 15 + 6 * (1.0 + 1.0 + 2.0)) + (B - NI) * 3.0 * 6 * 4.0;
    // I = c0 Q (27 quantities); volume of the elastic rows and their source (3 per stress row)
    fl = 27.0 * B + N * per_deriv + fkh + B * mix_added + B * 18.0 + fproj;
    // k_theta: Khat^x on the three velocity columns; per row and anelastic function the
    // mixing (6 cnt_i - 1), the source -omega I and the update (3); the faces as above
    fn += fkh / 3.0 + B * 3.0 * (6.0 * 15 + 6 * 2.0) + ftheta_faces;
  }
  // yt_step runs k_local without the local lifting and k_neigh with the sum of both flux
  // products lifted once (the flops of the lifting are the same as lifting them one by
  // one: every non-zero product is added to Q); the unfused pair lifts the local products
  // in k_local and computes W = V Anb^T (17 per entry) in k_neigh
  s->flops_local = fl;
  s->flops_neigh = fn;
  s->flops_local_unfused = fl + lift_total;
  const double rb = (double)s->real_bytes;
  const double qb = 8.0 * 9 * B, pb = rb * 4 * 9 * BT;
  s->bytes_local = 3 * qb + 2 * pb + rb * (3 * kStarSlots + 4 * 81);   // + Wloc written
  s->bytes_neigh = 2 * qb + 2 * pb + rb * 4 * 81 + 16.0;               // + Wloc read
  if (s->P == kNqVe) {
    // k_local: Q read (27 quantities), elastic rows of Q written, I written (27), the
    // anelastic coefficients read; k_theta: anelastic rows of Q read and written, I of
    // the velocities and anelastic functions read, own and neighbour projections, the
    // anelastic rows of both flux solvers
    const double qt = 8.0 * 18 * B;
    s->bytes_local += 2 * qt + rb * (3 * 3 * kStressSlots + 3);
    s->bytes_neigh += 2 * qt + 8.0 * 21 * B + 2 * pb + rb * (2 * 4 * kNTheta * kNq + 3 * 3 * kStressSlots + 3);
  }
  if (csr.col.size() > 0x7fffffff) throw Error(YT_ERR_UNSUPPORTED, "tables too large");
  s->n_values = (int64_t)csr.val.size();
  s->d_val = dalloc<double>(csr.val.size());
  s->d_f = dalloc<double>(R.f.size());
  cuda_check(cudaMemcpy(s->d_val, csr.val.data(), csr.val.size() * sizeof(double), cudaMemcpyHostToDevice), "copy val");
  cuda_check(cudaMemcpy(s->d_f, R.f.data(), R.f.size() * sizeof(double), cudaMemcpyHostToDevice), "copy f");
  if (s->prec == YT_BF16X3_F32ACC) {
    std::vector<float> f32(R.f.begin(), R.f.end());
    s->d_f32 = dalloc<float>(f32.size());
    cuda_check(cudaMemcpy(s->d_f32, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice), "copy f32");
    std::vector<unsigned char> ol, on;
    tc_operands_local(N, ol);
    tc_operands_neigh(N, on);
    s->d_tc_local = dalloc<unsigned char>(ol.size());
    s->d_tc_neigh = dalloc<unsigned char>(on.size());
    s->d_status = dalloc<int>(1);
    cuda_check(cudaMemcpy(s->d_tc_local, ol.data(), ol.size(), cudaMemcpyHostToDevice), "copy tc operands");
    cuda_check(cudaMemcpy(s->d_tc_neigh, on.data(), on.size(), cudaMemcpyHostToDevice), "copy tc operands");
    cuda_check(cudaMemset(s->d_status, 0, sizeof(int)), "memset status");
    int dev = 0, sms = 0;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    s->tc_grid = (unsigned)std::min<int64_t>(s->ntiles, sms);
    s->d_tc_scratch = dalloc<float>(tc_scratch_floats(N, s->tc_grid));
    if (s->P == kNq) s->d_tc_vol = dalloc<float>((size_t)s->Epad * kNq * s->B);
    if (s->P == kNqVe) {
      // k_theta (FP32): its sparse lists' values, from constant memory too at degree <= 5
      std::vector<float> v32(csr.val.begin(), csr.val.end());
      if (N <= 5) {
        int rc = 0;
        YT_THETA_F32_SWITCH(rc |= ader_upload, v32.data(), v32.size());
        YT_REQUIRE(rc == 0, YT_ERR_CUDA, "upload of constant values failed");
      }
      s->d_val32 = dalloc<float>(v32.size());
      cuda_check(cudaMemcpy(s->d_val32, v32.data(), v32.size() * sizeof(float), cudaMemcpyHostToDevice), "copy val32");
    }
  }
  if (s->prec == YT_F32) {
    std::vector<float> v32(csr.val.begin(), csr.val.end()), f32(R.f.begin(), R.f.end());
    // FP32 values of degrees <= 5 are also read from constant memory (one copy per kernel
    // variant's translation unit)
    if (N <= 5) {
      int rc = 0;
      if (s->P == kNqVe) {
        YT_VARIANT_SWITCH(rc |= ader_upload, vl, v32.data(), v32.size());
        YT_VARIANT_SWITCH(rc |= ader_upload, vn, v32.data(), v32.size());
        YT_VARIANT_SWITCH(rc |= ader_upload, vt, v32.data(), v32.size());
      } else {
        YT_VARIANT_SWITCH(rc |= ader_upload, lf, v32.data(), v32.size());
        YT_VARIANT_SWITCH(rc |= ader_upload, ll, v32.data(), v32.size());
        if (N <= 4) YT_SMALL_SWITCH(rc |= ader_upload, v32.data(), v32.size());
        YT_VARIANT_SWITCH(rc |= ader_upload, nf, v32.data(), v32.size());
        YT_VARIANT_SWITCH(rc |= ader_upload, np, v32.data(), v32.size());
      }
      YT_REQUIRE(rc == 0, YT_ERR_CUDA, "upload of constant values failed");
    }
    s->d_val32 = dalloc<float>(v32.size());
    s->d_f32 = dalloc<float>(f32.size());
    cuda_check(cudaMemcpy(s->d_val32, v32.data(), v32.size() * sizeof(float), cudaMemcpyHostToDevice), "copy val32");
    cuda_check(cudaMemcpy(s->d_f32, f32.data(), f32.size() * sizeof(float), cudaMemcpyHostToDevice), "copy f32");
  }

}

unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

namespace yt {
AderLaunch solver_launch_args(yt_solver* s, cudaStream_t st) { return launch_args(s, st); }

void solver_launch_variant(yt_solver* s, const AderLaunch& L, int variant) {
  YT_REQUIRE(s->prec != YT_BF16X3_F32ACC, YT_ERR_UNSUPPORTED, "tile-table launches: YT_F64 or YT_F32");
  switch (variant) {
    case 0: YT_VARIANT_SWITCH(ader_launch, lf, L); break;
    case 1: YT_VARIANT_SWITCH(ader_launch, ll, L); break;
    case 2: YT_VARIANT_SWITCH(ader_launch, nf, L); break;
    case 3: YT_VARIANT_SWITCH(ader_launch, np, L); break;
    default: throw Error(YT_ERR_INVALID, "kernel variant");
  }
  cuda_check(cudaGetLastError(), "kernel launch");
}

yt_status solver_create_stream_ordered(const yt_mesh_desc* mesh, const yt_scheme_desc* scheme,
                                       cudaStream_t stream, yt_solver** out) {
  t_alloc.async = true;
  t_alloc.stream = stream;
  const yt_status rc = yt_solver_create(mesh, scheme, reinterpret_cast<yt_stream>(stream), out);
  t_alloc = AllocMode{};
  return rc;
}

size_t solver_device_bytes(int order, yt_precision prec, int64_t n_elements) {
  const int N = order - 1;
  const size_t B = n_basis(N), BT = n_face_basis(N);
  const size_t Epad = (size_t)((n_elements + kTile - 1) / kTile) * kTile;
  const size_t rb = prec == YT_F64 ? 8 : 4;
  size_t per = 8 * kNq * B * 3;                        // Q, I, staging
  per += 2 * rb * 4 * kNq * BT;                        // face projections, local products
  per += 8 * (3 * kStarSlots + 8 * 81);                // star matrices, flux solvers
  if (prec != YT_F64) per += 4 * (3 * kStarSlots + 8 * 81);
  per += 4 * 4 + 8 * 12;                               // connectivity, setup inputs
  return Epad * per;
}
}  // namespace yt

extern "C" yt_status yt_solver_create(const yt_mesh_desc* mesh, const yt_scheme_desc* scheme,
                                      yt_stream stream, yt_solver** out) {
  return guarded([&] {
    YT_REQUIRE(mesh && scheme && out, YT_ERR_INVALID, "null argument");
    *out = nullptr;
    YT_REQUIRE(mesh->n_elements > 0 && mesh->material && mesh->jacobian, YT_ERR_INVALID,
               "mesh needs n_elements > 0, material and jacobian");
    YT_REQUIRE((scheme->flags & ~YT_SCHEME_DIAG_EXPIRE_WAIT) == 0, YT_ERR_INVALID, "unknown scheme flags");
    YT_REQUIRE(scheme->flags == 0 || scheme->precision == YT_BF16X3_F32ACC, YT_ERR_INVALID,
               "YT_SCHEME_DIAG_EXPIRE_WAIT needs YT_BF16X3_F32ACC (the kernels with bounded waits)");
    YT_REQUIRE(scheme->order >= 2 && scheme->order <= 7, YT_ERR_INVALID, "order must be 2..7");
    YT_REQUIRE(scheme->precision == YT_F64 || scheme->precision == YT_F32 ||
                   scheme->precision == YT_BF16X3_F32ACC,
               YT_ERR_UNSUPPORTED, "solver precision: YT_F64, YT_F32 or YT_BF16X3_F32ACC");

    YT_REQUIRE(std::isfinite(scheme->dt) && scheme->dt > 0, YT_ERR_INVALID, "dt must be positive");
    YT_REQUIRE(mesh->n_elements < (int64_t(1) << 24), YT_ERR_UNSUPPORTED, "at most 2^24 elements");
    const bool nb = mesh->neighbours != nullptr;
    YT_REQUIRE(!nb || (mesh->faces && mesh->orient), YT_ERR_INVALID, "faces/orient required with neighbours");
    YT_REQUIRE(scheme->quantities == 0 || scheme->quantities == kNq || scheme->quantities == kNqVe,
               YT_ERR_INVALID, "quantities must be 9 or 27");
    const bool ve = scheme->quantities == kNqVe;
    YT_REQUIRE(!ve || mesh->attenuation, YT_ERR_INVALID, "27-quantity solvers need the attenuation parameters");
    YT_REQUIRE(ve || !mesh->attenuation, YT_ERR_INVALID, "attenuation parameters given to a 9-quantity solver");
    YT_REQUIRE(!ve || scheme->precision == YT_F64 || scheme->precision == YT_F32 ||
                   scheme->precision == YT_BF16X3_F32ACC,
               YT_ERR_UNSUPPORTED, "27-quantity solvers: YT_F64, YT_F32 or YT_BF16X3_F32ACC");
    YT_REQUIRE(!ve || nb, YT_ERR_INVALID, "27-quantity solvers need the face connectivity");
    YT_REQUIRE(mesh->n_halo >= 0 && mesh->n_halo < (int64_t(1) << 26), YT_ERR_INVALID, "n_halo out of range");
    YT_REQUIRE(mesh->n_halo == 0 || (nb && !ve && scheme->precision != YT_BF16X3_F32ACC), YT_ERR_UNSUPPORTED,
               "partitioned solves: elastic YT_F64 / YT_F32 with connectivity");
    auto s = std::make_unique<yt_solver>();
    s->alloc_async = t_alloc.async;
    s->alloc_stream = t_alloc.stream;
    s->P = ve ? kNqVe : kNq;
    s->N = scheme->order - 1;
    s->B = n_basis(s->N);
    s->BT = n_face_basis(s->N);
    s->E = mesh->n_elements;
    s->ntiles = (s->E + kTile - 1) / kTile;
    s->Epad = s->ntiles * kTile;
    s->prec = scheme->precision;
    s->real_bytes = s->prec == YT_F64 ? sizeof(double) : sizeof(float);
    s->dt = scheme->dt;
    s->has_neighbours = nb;
    s->diag_expire_wait = (scheme->flags & YT_SCHEME_DIAG_EXPIRE_WAIT) != 0;
    std::vector<int> conn;
    if (nb) {
      conn.assign((size_t)s->Epad * 4, 0);
      for (int64_t e = 0; e < s->E; ++e)
        for (int f = 0; f < 4; ++f) {
          const int64_t n = mesh->neighbours[e * 4 + f];
          const int j = mesh->faces[e * 4 + f], h = mesh->orient[e * 4 + f];
          YT_REQUIRE(j >= 0 && j < 4 && h >= 0 && h < 3, YT_ERR_INVALID, "face/orientation out of range");
          if (n < 0) {
            // halo slot t = -1 - n: group 1, addressed as element t / 4, face t % 4 (the
            // block [slot][9][BT] is then read at ((t/4) * 4 + t%4) * 9 * BT = t * 9 * BT)
            const int64_t t = -1 - n;
            YT_REQUIRE(t < mesh->n_halo, YT_ERR_INVALID, "halo slot out of range");
            conn[e * 4 + f] = (int)(((t >> 2) << 7) | (1 << 4) | ((t & 3) << 2) | h);
          } else {
            YT_REQUIRE(n < s->E, YT_ERR_INVALID, "neighbour index out of range");
            conn[e * 4 + f] = (int)((n << 7) | (j << 2) | h);
          }
        }
    }
    build_tables(s.get());
    YT_REQUIRE(ader_generated_nnz(s->N) == (int)s->n_values, YT_ERR_INVALID,
               "generated kernels do not match the reference matrices (rebuild the library)");
    set_smem(s.get());
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t nq = (size_t)s->Epad * s->P * s->B;
    s->Q = dalloc<double>(nq);
    s->I = dalloc<double>(nq);
    if (ve) {
      s->theta = dalloc<unsigned char>((size_t)s->Epad * kNTheta * s->B * s->real_bytes);
      s->cth = dalloc<double>((size_t)s->Epad * 3 * 3 * kStressSlots);
      s->om = dalloc<double>((size_t)s->Epad * 3);
      s->fthl = dalloc<double>((size_t)s->Epad * 4 * kNTheta * kNq);
      s->fthn = dalloc<double>((size_t)s->Epad * 4 * kNTheta * kNq);
    }
    // face projections: rows of BT values, padded to 8 in the tensor-core form
    const size_t pbytes = (size_t)s->Epad * 4 * kNq *
                          (s->prec == YT_BF16X3_F32ACC ? (size_t)tc::up8(s->BT) : (size_t)s->BT) * s->real_bytes;
    s->Pface = dalloc<unsigned char>(pbytes);
    s->n_halo = mesh->n_halo;
    if (s->n_halo > 0) {
      s->halo = dalloc<unsigned char>((size_t)s->n_halo * kNq * s->BT * s->real_bytes);
      cuda_check(cudaMemsetAsync(s->halo, 0, (size_t)s->n_halo * kNq * s->BT * s->real_bytes, st), "memset halo");
    }
    s->Wloc = dalloc<unsigned char>((size_t)s->Epad * 4 * kNq * s->BT * s->real_bytes);
    s->star = dalloc<double>((size_t)s->Epad * 3 * kStarSlots);
    s->floc = dalloc<double>((size_t)s->Epad * 4 * 81);
    s->fnb = dalloc<double>((size_t)s->Epad * 4 * 81);
    s->conn = dalloc<int>((size_t)s->Epad * 4);
    cuda_check(cudaMemsetAsync(s->Q, 0, nq * sizeof(double), st), "memset Q");
    cuda_check(cudaMemsetAsync(s->I, 0, nq * sizeof(double), st), "memset I");
    cuda_check(cudaMemsetAsync(s->Pface, 0, pbytes, st), "memset P");
    cuda_check(cudaMemsetAsync(s->conn, 0, (size_t)s->Epad * 4 * sizeof(int), st), "memset conn");
    if (nb) cuda_check(cudaMemcpyAsync(s->conn, conn.data(), conn.size() * sizeof(int), cudaMemcpyHostToDevice, st), "copy conn");
    double* dmat = dalloc<double>((size_t)s->E * 3);
    double* djac = dalloc<double>((size_t)s->E * 9);
    double* datt = ve ? dalloc<double>((size_t)s->E * 9) : nullptr;
    cudaError_t e1 = cudaMemcpyAsync(dmat, mesh->material, (size_t)s->E * 3 * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaError_t e2 = cudaMemcpyAsync(djac, mesh->jacobian, (size_t)s->E * 9 * sizeof(double), cudaMemcpyHostToDevice, st);
    if (ve && e2 == cudaSuccess)
      e2 = cudaMemcpyAsync(datt, mesh->attenuation, (size_t)s->E * 9 * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaError_t e3 = cudaMemcpyToSymbolAsync(c_star, &kStar, sizeof(kStar), 0, cudaMemcpyHostToDevice, st);
    cudaError_t e4 = cudaMemcpyToSymbolAsync(c_face_verts, kFaceVerts, sizeof(kFaceVerts), 0, cudaMemcpyHostToDevice, st);
    if (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess && e4 == cudaSuccess) {
      k_setup<<<blocks_for(s->Epad, 128), 128, 0, st>>>(dmat, djac, s->E, s->Epad, s->star, s->floc, s->fnb);
      if (ve)
        k_setup_theta<<<blocks_for(s->Epad, 128), 128, 0, st>>>(dmat, djac, datt, s->E, s->Epad, s->cth, s->om,
                                                                s->fthl, s->fthn);
      e1 = cudaGetLastError();
    }
    if (e1 == cudaSuccess) {
      if (s->prec != YT_F64) {
        const int64_t ns = s->Epad * 3 * kStarSlots, nf = s->Epad * 4 * 81;
        s->star_r = dalloc<float>((size_t)ns);
        s->floc_r = dalloc<float>((size_t)nf);
        s->fnb_r = dalloc<float>((size_t)nf);
        k_to_float<<<blocks_for(ns, 256), 256, 0, st>>>(s->star, static_cast<float*>(s->star_r), ns);
        k_to_float<<<blocks_for(nf, 256), 256, 0, st>>>(s->floc, static_cast<float*>(s->floc_r), nf);
        k_to_float<<<blocks_for(nf, 256), 256, 0, st>>>(s->fnb, static_cast<float*>(s->fnb_r), nf);
        if (ve) {
          const int64_t nc = s->Epad * 3 * 3 * kStressSlots, no = s->Epad * 3, nt = s->Epad * 4 * kNTheta * kNq;
          s->cth_r = dalloc<float>((size_t)nc);
          s->om_r = dalloc<float>((size_t)no);
          s->fthl_r = dalloc<float>((size_t)nt);
          s->fthn_r = dalloc<float>((size_t)nt);
          k_to_float<<<blocks_for(nc, 256), 256, 0, st>>>(s->cth, static_cast<float*>(s->cth_r), nc);
          k_to_float<<<blocks_for(no, 256), 256, 0, st>>>(s->om, static_cast<float*>(s->om_r), no);
          k_to_float<<<blocks_for(nt, 256), 256, 0, st>>>(s->fthl, static_cast<float*>(s->fthl_r), nt);
          k_to_float<<<blocks_for(nt, 256), 256, 0, st>>>(s->fthn, static_cast<float*>(s->fthn_r), nt);
        }
        e1 = cudaGetLastError();
      } else {
        s->star_r = s->star;
        s->floc_r = s->floc;
        s->fnb_r = s->fnb;
        s->cth_r = s->cth;
        s->om_r = s->om;
        s->fthl_r = s->fthl;
        s->fthn_r = s->fthn;
      }
    }
    cudaError_t e5 = cudaStreamSynchronize(st);
    dfree_temp(dmat);
    dfree_temp(djac);
    dfree_temp(datt);
    cuda_check(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : (e3 != cudaSuccess ? e3 : (e4 != cudaSuccess ? e4 : e5))),
               "solver setup");
    *out = s.release();
  });
}

extern "C" yt_status yt_solver_set_dofs(yt_solver* s, const double* dofs, yt_memory where,
                                        yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s && dofs, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(where == YT_MEM_HOST || where == YT_MEM_DEVICE, YT_ERR_INVALID, "where");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = (size_t)s->E * s->P * s->B;
    const double* src = dofs;
    if (where == YT_MEM_HOST) {
      if (!s->staging) s->staging = sdalloc<double>(s, (size_t)s->Epad * s->P * s->B);
      cuda_check(cudaMemcpyAsync(s->staging, dofs, n * sizeof(double), cudaMemcpyHostToDevice, st), "H2D dofs");
      src = s->staging;
    }
    const int64_t total = s->Epad * s->P * s->B;
    k_to_blocked<<<blocks_for(total, 256), 256, 0, st>>>(src, s->Q, s->E, s->Epad, s->B, s->P);
    cuda_check(cudaGetLastError(), "k_to_blocked");
  });
}

extern "C" yt_status yt_solver_get(yt_solver* s, yt_field field, double* out, yt_memory where,
                                   yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s && out, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(field == YT_FIELD_DOFS || field == YT_FIELD_TIME_INTEGRAL, YT_ERR_INVALID, "field");
    YT_REQUIRE(where == YT_MEM_HOST || where == YT_MEM_DEVICE, YT_ERR_INVALID, "where");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = (size_t)s->E * s->P * s->B;
    double* dst = out;
    if (where == YT_MEM_HOST) {
      if (!s->staging) s->staging = sdalloc<double>(s, (size_t)s->Epad * s->P * s->B);
      dst = s->staging;
    }
    k_from_blocked<<<blocks_for((int64_t)n, 256), 256, 0, st>>>(field == YT_FIELD_DOFS ? s->Q : s->I,
                                                                 dst, s->E, s->B, s->P);
    cuda_check(cudaGetLastError(), "k_from_blocked");
    if (where == YT_MEM_HOST)
      cuda_check(cudaMemcpyAsync(out, dst, n * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H");
  });
}

extern "C" yt_status yt_step_local(yt_solver* s, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s, YT_ERR_INVALID, "null solver");
    YT_REQUIRE(s->P == kNq, YT_ERR_UNSUPPORTED, "27-quantity solvers: fused step only (yt_step, yt_step_phase)");
    dispatch_local(s, reinterpret_cast<cudaStream_t>(stream), false);
  });
}

extern "C" yt_status yt_step_neighbour(yt_solver* s, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s, YT_ERR_INVALID, "null solver");
    YT_REQUIRE(s->P == kNq, YT_ERR_UNSUPPORTED, "27-quantity solvers: fused step only (yt_step, yt_step_phase)");
    YT_REQUIRE(s->has_neighbours, YT_ERR_INVALID, "solver was created without neighbours");
    dispatch_neigh(s, reinterpret_cast<cudaStream_t>(stream), false);
  });
}

extern "C" yt_status yt_step_phase(yt_solver* s, int32_t phase, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s, YT_ERR_INVALID, "null solver");
    YT_REQUIRE(phase == 0 || phase == 1, YT_ERR_INVALID, "phase must be 0 or 1");
    YT_REQUIRE(s->has_neighbours, YT_ERR_INVALID, "solver was created without neighbours");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (phase == 0) dispatch_local(s, st, true);
    else dispatch_neigh(s, st, true);
  });
}

extern "C" yt_status yt_step(yt_solver* s, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s, YT_ERR_INVALID, "null solver");
    YT_REQUIRE(s->has_neighbours, YT_ERR_INVALID, "solver was created without neighbours");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    dispatch_local(s, st, true);
    dispatch_neigh(s, st, true);
  });
}

namespace {
// Kernels of one phase over tiles [t0, t0 + nt) (phase 0: k_local of the fused step,
// phase 1: k_neigh of the fused step).
void dispatch_chunk(yt_solver* s, cudaStream_t st, int phase, int64_t t0, int64_t nt) {
  if (s->prec == YT_BF16X3_F32ACC) {
    dispatch_tc_fused(s, st, phase, t0, nt);
  } else {
    const AderLaunch L = chunk_args(launch_args(s, st), s, t0, nt);
    if (s->P == kNqVe) {
      if (phase == 0) {
        YT_VARIANT_SWITCH(ader_launch, vl, L);
      } else {
        YT_VARIANT_SWITCH(ader_launch, vn, L);
        YT_VARIANT_SWITCH(ader_launch, vt, L);
      }
    } else if (phase == 0) {
      YT_VARIANT_SWITCH(ader_launch, lf, L);
    } else {
      YT_VARIANT_SWITCH(ader_launch, nf, L);
    }
  }
  cuda_check(cudaGetLastError(), "chunk launch");
}
}  // namespace

extern "C" yt_status yt_step_host(yt_solver* s, const double* dofs_in, double* dofs_out,
                                  yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s && dofs_in && dofs_out, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(s->has_neighbours, YT_ERR_INVALID, "solver was created without neighbours");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // 16 chunks (measured at 1M tets, order 6: 4 chunks 214-219 ms per step, 8 chunks
    // 210-211, 16 chunks 203: the first upload and the last download, not hidden, shrink
    // with the chunk), each a whole number of waves of one CTA per SM where it can be
    constexpr int kChunks = 16;
    if (!s->staging) s->staging = sdalloc<double>(s, (size_t)s->Epad * s->P * s->B);
    if (!s->copy_stream) {
      cuda_check(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking), "copy stream");
      cuda_check(cudaEventCreateWithFlags(&s->ev_start, cudaEventDisableTiming), "event");
      cuda_check(cudaEventCreateWithFlags(&s->ev_done, cudaEventDisableTiming), "event");
      for (int c = 0; c < kChunks; ++c) {
        cuda_check(cudaEventCreateWithFlags(&s->ev_in[c], cudaEventDisableTiming), "event");
        cuda_check(cudaEventCreateWithFlags(&s->ev_out[c], cudaEventDisableTiming), "event");
      }
    }
    cudaStream_t cp = s->copy_stream;
    int dev = 0, sms = 1;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
    int64_t per = (s->ntiles + kChunks - 1) / kChunks;           // tiles per chunk
    if (per > sms) per = (per + sms - 1) / sms * sms;
    const size_t row = (size_t)s->P * s->B;                      // doubles per element
    cuda_check(cudaEventRecord(s->ev_start, st), "event record");
    cuda_check(cudaStreamWaitEvent(cp, s->ev_start, 0), "stream wait");
    // uploads on the copy stream; layout conversion and local kernel per chunk on `st`
    for (int c = 0; c < kChunks; ++c) {
      const int64_t t0 = c * per, nt = std::min<int64_t>(per, s->ntiles - t0);
      if (nt <= 0) break;
      const int64_t e0 = t0 * kTile, ne = std::min<int64_t>(nt * kTile, s->E - e0);
      cuda_check(cudaMemcpyAsync(s->staging + e0 * row, dofs_in + e0 * row, (size_t)ne * row * sizeof(double),
                                 cudaMemcpyHostToDevice, cp), "H2D chunk");
      cuda_check(cudaEventRecord(s->ev_in[c], cp), "event record");
      cuda_check(cudaStreamWaitEvent(st, s->ev_in[c], 0), "stream wait");
      const int64_t total = nt * kTile * (int64_t)row;
      k_to_blocked<<<blocks_for(total, 256), 256, 0, st>>>(s->staging + e0 * row, s->Q + e0 * row, ne,
                                                           nt * kTile, s->B, s->P);
      cuda_check(cudaGetLastError(), "k_to_blocked");
      dispatch_chunk(s, st, 0, t0, nt);
    }
    // neighbour kernel per chunk (after every local chunk), layout back, downloads
    for (int c = 0; c < kChunks; ++c) {
      const int64_t t0 = c * per, nt = std::min<int64_t>(per, s->ntiles - t0);
      if (nt <= 0) break;
      const int64_t e0 = t0 * kTile, ne = std::min<int64_t>(nt * kTile, s->E - e0);
      dispatch_chunk(s, st, 1, t0, nt);
      k_from_blocked<<<blocks_for(ne * (int64_t)row, 256), 256, 0, st>>>(s->Q + e0 * row,
                                                                         s->staging + e0 * row, ne, s->B, s->P);
      cuda_check(cudaGetLastError(), "k_from_blocked");
      cuda_check(cudaEventRecord(s->ev_out[c], st), "event record");
      cuda_check(cudaStreamWaitEvent(cp, s->ev_out[c], 0), "stream wait");
      cuda_check(cudaMemcpyAsync(dofs_out + e0 * row, s->staging + e0 * row, (size_t)ne * row * sizeof(double),
                                 cudaMemcpyDeviceToHost, cp), "D2H chunk");
    }
    cuda_check(cudaEventRecord(s->ev_done, cp), "event record");
    cuda_check(cudaStreamWaitEvent(st, s->ev_done, 0), "stream wait");
  });
}

namespace {
// out[(i * 9 + q) * BT + m] = Pface[((le_i * 4 + j_i) * 9 + q) * BT + m]
template <typename Real>
__global__ void k_halo_pack(const Real* __restrict__ P, const int* __restrict__ pairs, Real* __restrict__ out,
                            int64_t n, int BT) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * kNq * BT) return;
  const int64_t pair = i / (kNq * BT);
  const int64_t r = i % (kNq * BT);
  out[i] = P[((int64_t)pairs[2 * pair] * 4 + pairs[2 * pair + 1]) * kNq * BT + r];
}
}  // namespace

extern "C" yt_status yt_solver_set_send_list(yt_solver* s, const int32_t* pairs, int64_t n) {
  return guarded([&] {
    YT_REQUIRE(s && (pairs || n == 0) && n >= 0, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(s->P == kNq && s->prec != YT_BF16X3_F32ACC, YT_ERR_UNSUPPORTED,
               "partitioned solves: elastic YT_F64 / YT_F32");
    for (int64_t i = 0; i < n; ++i)
      YT_REQUIRE(pairs[2 * i] >= 0 && pairs[2 * i] < s->E && pairs[2 * i + 1] >= 0 && pairs[2 * i + 1] < 4,
                 YT_ERR_INVALID, "send pair out of range");
    if (s->d_send) s->free_device(s->d_send);
    s->d_send = nullptr;
    s->n_send = n;
    if (n > 0) {
      s->d_send = sdalloc<int>(s, (size_t)(2 * n));
      cuda_check(cudaMemcpy(s->d_send, pairs, (size_t)(2 * n) * sizeof(int), cudaMemcpyHostToDevice), "copy send list");
    }
  });
}

extern "C" yt_status yt_solver_halo_pack(yt_solver* s, void* out, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s && (out || s->n_send == 0), YT_ERR_INVALID, "null argument");
    if (s->n_send == 0) return;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t total = s->n_send * kNq * s->BT;
    if (s->prec == YT_F64)
      k_halo_pack<double><<<blocks_for(total, 256), 256, 0, st>>>(static_cast<const double*>(s->Pface), s->d_send,
                                                                  static_cast<double*>(out), s->n_send, s->BT);
    else
      k_halo_pack<float><<<blocks_for(total, 256), 256, 0, st>>>(static_cast<const float*>(s->Pface), s->d_send,
                                                                 static_cast<float*>(out), s->n_send, s->BT);
    cuda_check(cudaGetLastError(), "k_halo_pack");
  });
}

extern "C" yt_status yt_solver_halo_buffer(yt_solver* s, void** ptr, int64_t* bytes) {
  return guarded([&] {
    YT_REQUIRE(s && ptr, YT_ERR_INVALID, "null argument");
    *ptr = s->halo;
    if (bytes) *bytes = s->n_halo * kNq * s->BT * (int64_t)s->real_bytes;
  });
}

extern "C" yt_status yt_solver_halo_unpack(yt_solver* s, const void* in, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s && (in || s->n_halo == 0), YT_ERR_INVALID, "null argument");
    if (s->n_halo == 0) return;
    cuda_check(cudaMemcpyAsync(s->halo, in, (size_t)s->n_halo * kNq * s->BT * s->real_bytes,
                               cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)), "halo unpack");
  });
}

extern "C" yt_status yt_step_phase_tiles(yt_solver* s, int32_t phase, int64_t t0, int64_t nt, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s, YT_ERR_INVALID, "null solver");
    YT_REQUIRE(phase == 0 || phase == 1, YT_ERR_INVALID, "phase must be 0 or 1");
    YT_REQUIRE(s->has_neighbours, YT_ERR_INVALID, "solver was created without neighbours");
    YT_REQUIRE(t0 >= 0 && nt >= 0 && t0 + nt <= s->ntiles, YT_ERR_INVALID, "tile range out of range");
    if (nt == 0) return;
    dispatch_chunk(s, reinterpret_cast<cudaStream_t>(stream), phase, t0, nt);
  });
}

extern "C" yt_status yt_solver_stats(const yt_solver* s, double* lf, double* nf, double* lb,
                                     double* nbb) {
  return guarded([&] {
    YT_REQUIRE(s, YT_ERR_INVALID, "null solver");
    if (lf) *lf = s->flops_local;
    if (nf) *nf = s->flops_neigh;
    if (lb) *lb = s->bytes_local;
    if (nbb) *nbb = s->bytes_neigh;
  });
}

extern "C" yt_status yt_solver_status(yt_solver* s, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(s, YT_ERR_INVALID, "null solver");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cuda_check(cudaStreamSynchronize(st), "stream synchronize");
    if (!s->d_status) return;
    int v = 0;
    cuda_check(cudaMemcpy(&v, s->d_status, sizeof(int), cudaMemcpyDeviceToHost), "status copy");
    if (v != 0) {
      cuda_check(cudaMemset(s->d_status, 0, sizeof(int)), "status reset");
      throw Error(YT_ERR_TIMEOUT, "a bounded device-side wait of the tensor-core kernels ran out");
    }
  });
}

namespace {
void copy_reference(int N, const char* name, double* out, int64_t* count) {
  YT_REQUIRE(name && count, YT_ERR_INVALID, "null argument");
  const RefMatrices& R = reference_matrices(N);
  const std::vector<double>* v = nullptr;
  const std::string nm(name);
  if (nm == "M") v = &R.M;
  else if (nm == "Khat") v = &R.Khat;
  else if (nm == "Ktilde") v = &R.Ktilde;
  else if (nm == "R") v = &R.R;
  else if (nm == "Rhat") v = &R.Rhat;
  else if (nm == "f") v = &R.f;
  else if (nm == "W") v = &R.W;
  YT_REQUIRE(v, YT_ERR_INVALID, "unknown matrix name");
  *count = (int64_t)v->size();
  if (out) std::memcpy(out, v->data(), v->size() * sizeof(double));
}
}  // namespace

extern "C" yt_status yt_solver_reference_matrix(const yt_solver* s, const char* name,
                                                double* out, int64_t* count) {
  return guarded([&] {
    YT_REQUIRE(s, YT_ERR_INVALID, "null solver");
    copy_reference(s->N, name, out, count);
  });
}

extern "C" yt_status yt_reference_matrix(int32_t order, const char* name, double* out,
                                         int64_t* count) {
  return guarded([&] {
    YT_REQUIRE(order >= 2 && order <= 7, YT_ERR_INVALID, "order must be 2..7");
    copy_reference(order - 1, name, out, count);
  });
}

extern "C" void yt_solver_destroy(yt_solver* s) { delete s; }

// ===================================================================== p-adaptive batch
// Elements of several polynomial degrees: one local-only solver per degree (a "group"),
// neighbour connectivity across groups, and the whole step recorded once as a CUDA graph
// (local kernels of all groups, then neighbour kernels of all groups).
namespace {

__global__ void k_gather_blocked(const double* __restrict__ in, const int64_t* __restrict__ offs,
                                 double* __restrict__ out, int64_t E, int64_t Epad, int B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Epad * kNq * B) return;
  const int lane = (int)(i % kTile);
  const int64_t rest = i / kTile;
  const int k = (int)(rest % B);
  const int q = (int)((rest / B) % kNq);
  const int64_t e = (rest / ((int64_t)B * kNq)) * kTile + lane;
  out[i] = e < E ? in[offs[e] + (int64_t)q * B + k] : 0.0;
}
__global__ void k_scatter_blocked(const double* __restrict__ in, const int64_t* __restrict__ offs,
                                  double* __restrict__ out, int64_t E, int B) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= E * kNq * B) return;
  const int k = (int)(i % B);
  const int q = (int)((i / B) % kNq);
  const int64_t e = i / ((int64_t)B * kNq);
  out[offs[e] + (int64_t)q * B + k] = in[(((e / kTile) * kNq + q) * B + k) * kTile + (e % kTile)];
}

}  // namespace

struct yt_batch {
  yt_precision prec = YT_F64;
  double dt = 0.0;
  int64_t E = 0, total_dofs = 0;
  std::vector<yt_solver*> groups;            // one per degree present
  std::vector<int> group_n;                  // degree of each group
  std::vector<std::vector<int64_t>> members; // batch element ids of each group
  std::vector<int64_t*> d_offs;              // per group: offsets of its elements' DOF blocks
  std::vector<int*> d_conn;                  // per group: packed cross-group connectivity
  FaceGroups faces{};
  double* staging = nullptr;
  cudaStream_t capture = nullptr;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;
  cudaGraphExec_t exec = nullptr;
  // 0: per-group kernels in sequence, 1: per-group kernels on parallel graph branches,
  // 2: the persistent kernel (one cooperative launch per step)
  int mode = 0;
  // persistent kernel: group table, work items of both item orders ([order][phase][items]),
  // claim / barrier counters and the status word, launch shape and chosen parameters
  BatchGroup* d_groups = nullptr;
  int2* d_items[2] = {nullptr, nullptr};
  int n_items = 0;                           // tiles of all groups (per phase)
  int* d_counters = nullptr;                 // [0..2] counters, [3] status
  size_t pers_smem = 0;
  unsigned pers_grid = 0;
  bool pers_coop = true;
  int pers_order = 0, pers_chunk = 1;
  std::string config;                        // the chosen form and the tuner's timings
  double flops = 0.0, bytes = 0.0;
  ~yt_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto* p : d_items) if (p) cudaFree(p);
    if (d_groups) cudaFree(d_groups);
    if (d_counters) cudaFree(d_counters);
    for (auto* g : groups) delete g;
    for (auto* p : d_offs) cudaFree(p);
    for (auto* p : d_conn) cudaFree(p);
    if (staging) cudaFree(staging);
    for (auto st : side) cudaStreamDestroy(st);
    for (auto e : ev) cudaEventDestroy(e);
    if (capture) cudaStreamDestroy(capture);
  }
};

namespace {

AderLaunch batch_launch_args(yt_batch* b, size_t g, cudaStream_t st) {
  AderLaunch L = launch_args(b->groups[g], st);
  L.conn = b->d_conn[g];
  L.groups = b->faces;
  return L;
}

void batch_record(yt_batch* b, cudaStream_t st, int mode) {
  const size_t G = b->groups.size();
  if (mode == 2) {
    cuda_check(cudaMemsetAsync(b->d_counters, 0, 3 * sizeof(int), st), "reset counters");
    BatchArgs A{};
    A.groups = b->d_groups;
    A.faces = b->faces;
    A.items = b->d_items[b->pers_order];
    A.n_items[0] = A.n_items[1] = b->n_items;
    A.chunk = b->pers_chunk;
    A.counters = b->d_counters;
    A.status = b->d_counters + 3;
    A.SP = kStar;
    cuda_check(batch_persistent_launch(b->prec != YT_F64, A, b->pers_grid, b->pers_smem, st, b->pers_coop),
               "persistent batch launch");
    return;
  }
  // (YT_VARIANT_SWITCH dispatches on the degree and precision of the solver named `s`)
  auto local = [&](size_t g, cudaStream_t stream) {
    const AderLaunch L = batch_launch_args(b, g, stream);
    yt_solver* s = b->groups[g];
    YT_VARIANT_SWITCH(ader_launch, lf, L);
  };
  auto neigh = [&](size_t g, cudaStream_t stream) {
    const AderLaunch L = batch_launch_args(b, g, stream);
    yt_solver* s = b->groups[g];
    YT_VARIANT_SWITCH(ader_launch, nf, L);
  };
  if (mode == 0) {
    for (size_t g = 0; g < G; ++g) local(g, st);
    for (size_t g = 0; g < G; ++g) neigh(g, st);
    return;
  }
  // parallel branches: fork after an event on the capture stream, join before the next phase
  for (int phase = 0; phase < 2; ++phase) {
    cuda_check(cudaEventRecord(b->ev[0], st), "fork event");
    for (size_t g = 0; g < G; ++g) {
      cuda_check(cudaStreamWaitEvent(b->side[g], b->ev[0], 0), "fork wait");
      if (phase == 0) local(g, b->side[g]);
      else neigh(g, b->side[g]);
      cuda_check(cudaEventRecord(b->ev[1 + g], b->side[g]), "join event");
      cuda_check(cudaStreamWaitEvent(st, b->ev[1 + g], 0), "join wait");
    }
  }
}

cudaGraphExec_t batch_graph_once(yt_batch* b, int mode) {
  cudaGraph_t graph = nullptr;
  cuda_check(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal), "begin capture");
  try {
    batch_record(b, b->capture, mode);
  } catch (...) {
    cudaStreamEndCapture(b->capture, &graph);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    throw;
  }
  cuda_check(cudaStreamEndCapture(b->capture, &graph), "end capture");
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  cuda_check(e, "graph instantiate");
  return exec;
}

// The persistent kernel is recorded as a cooperative launch (every CTA resident, which
// its grid barrier needs); should capture refuse that, it is recorded as a plain launch
// of the same grid, which the occupancy query sized to fit the device at once.
cudaGraphExec_t batch_graph(yt_batch* b, int mode) {
  if (mode != 2 || !b->pers_coop) return batch_graph_once(b, mode);
  try {
    return batch_graph_once(b, mode);
  } catch (const Error&) {
    b->pers_coop = false;
    return batch_graph_once(b, mode);
  }
}

// Work items (group, tile) of the persistent kernel in two orders: 0 = groups by
// decreasing degree (the longest tiles first), 1 = groups interleaved tile by tile.
void batch_items(yt_batch* b) {
  const size_t G = b->groups.size();
  std::vector<int> by_degree(G);
  for (size_t g = 0; g < G; ++g) by_degree[g] = (int)g;
  std::sort(by_degree.begin(), by_degree.end(), [&](int a, int c) { return b->group_n[a] > b->group_n[c]; });
  std::vector<int2> order0, order1;
  for (int g : by_degree)
    for (int64_t t = 0; t < b->groups[g]->ntiles; ++t) order0.push_back(make_int2(g, (int)t));
  int64_t maxt = 0;
  for (auto* s : b->groups) maxt = std::max<int64_t>(maxt, s->ntiles);
  for (int64_t t = 0; t < maxt; ++t)
    for (int g : by_degree)
      if (t < b->groups[g]->ntiles) order1.push_back(make_int2(g, (int)t));
  b->n_items = (int)order0.size();
  int o = 0;
  for (auto* v : {&order0, &order1}) {
    std::vector<int2> both(*v);
    both.insert(both.end(), v->begin(), v->end());      // local phase, then neighbour phase
    b->d_items[o] = dalloc<int2>(both.size());
    cuda_check(cudaMemcpy(b->d_items[o], both.data(), both.size() * sizeof(int2), cudaMemcpyHostToDevice), "copy items");
    ++o;
  }
}

// Group table, shared memory and grid of the persistent kernel.
void batch_persistent_setup(yt_batch* b) {
  const size_t G = b->groups.size();
  std::vector<BatchGroup> tab(G);
  size_t smem = 0;
  for (size_t g = 0; g < G; ++g) {
    yt_solver* s = b->groups[g];
    BatchGroup& t = tab[g];
    t.N = s->N;
    t.Q = s->Q;
    t.I = s->I;
    t.Pface = s->Pface;
    t.Wloc = s->Wloc;
    t.star = s->star_r;
    t.floc = s->floc_r;
    t.fnb = s->fnb_r;
    t.conn = b->d_conn[g];
    const bool f32 = s->prec != YT_F64;
    t.val = f32 ? (const void*)s->d_val32 : (const void*)s->d_val;
    t.f = f32 ? (const void*)s->d_f32 : (const void*)s->d_f;
    t.dt = s->dt;
    smem = std::max(smem, std::max(s->smem_local, s->smem_neigh));
  }
  b->d_groups = dalloc<BatchGroup>(G);
  cuda_check(cudaMemcpy(b->d_groups, tab.data(), G * sizeof(BatchGroup), cudaMemcpyHostToDevice), "copy groups");
  b->d_counters = dalloc<int>(4);
  cuda_check(cudaMemset(b->d_counters, 0, 4 * sizeof(int)), "memset counters");
  batch_items(b);
  b->pers_smem = smem;
  const int per_sm = batch_persistent_prepare(b->prec != YT_F64, smem);
  cudaGetLastError();
  if (per_sm <= 0) {               // the persistent form is then unavailable (set_form refuses it)
    b->pers_grid = 0;
    return;
  }
  int dev = 0, sms = 0;
  cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  b->pers_grid = (unsigned)std::min<int64_t>((int64_t)per_sm * sms, b->n_items);
}

std::string batch_describe(const yt_batch* b) {
  if (b->mode == 0) return "per-group kernels in sequence (one graph launch per step)";
  if (b->mode == 1) return "per-group kernels on parallel graph branches (one graph launch per step)";
  return "persistent kernel: " + std::string(b->pers_coop ? "cooperative" : "occupancy-sized") +
         " launch of " + std::to_string(b->pers_grid) + " CTAs x 288 threads, " +
         std::to_string(b->pers_smem) + " B shared memory, " + std::to_string(b->pers_chunk) +
         " tile(s) per claim, items " + (b->pers_order == 0 ? "by decreasing degree" : "interleaved across degrees");
}

}  // namespace

extern "C" yt_status yt_batch_create(const yt_mesh_desc* mesh, const int8_t* orders,
                                     const yt_scheme_desc* scheme, yt_stream stream,
                                     yt_batch** out) {
  return guarded([&] {
    YT_REQUIRE(mesh && orders && scheme && out, YT_ERR_INVALID, "null argument");
    *out = nullptr;
    YT_REQUIRE(mesh->neighbours && mesh->faces && mesh->orient && mesh->material && mesh->jacobian,
               YT_ERR_INVALID, "a batch needs material, jacobian and full connectivity");
    YT_REQUIRE(mesh->n_elements > 1 && mesh->n_elements < (int64_t(1) << 24), YT_ERR_INVALID,
               "element count must be 2 .. 2^24-1");
    YT_REQUIRE(scheme->flags == 0, YT_ERR_INVALID, "scheme flags must be 0");
    YT_REQUIRE((scheme->quantities == 0 || scheme->quantities == kNq) && !mesh->attenuation,
               YT_ERR_UNSUPPORTED, "p-adaptive batches: 9 quantities");
    auto b = std::make_unique<yt_batch>();
    b->prec = scheme->precision;
    b->dt = scheme->dt;
    b->E = mesh->n_elements;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<int> group_of_order(8, -1);
    std::vector<int> elem_group(b->E);
    std::vector<int64_t> elem_local(b->E), offs(b->E);
    for (int64_t e = 0; e < b->E; ++e) {
      const int o = orders[e];
      YT_REQUIRE(o >= 2 && o <= 7, YT_ERR_INVALID, "element orders must be 2..7");
      if (group_of_order[o] < 0) {
        group_of_order[o] = (int)b->group_n.size();
        b->group_n.push_back(o - 1);
        b->members.emplace_back();
      }
      const int g = group_of_order[o];
      elem_group[e] = g;
      elem_local[e] = (int64_t)b->members[g].size();
      b->members[g].push_back(e);
      offs[e] = b->total_dofs;
      b->total_dofs += (int64_t)kNq * n_basis(o - 1);
    }
    YT_REQUIRE(b->group_n.size() <= (size_t)kMaxGroups, YT_ERR_UNSUPPORTED, "too many degrees");
    for (size_t g = 0; g < b->group_n.size(); ++g) {
      const auto& mem = b->members[g];
      std::vector<double> mat(mem.size() * 3), jac(mem.size() * 9);
      for (size_t i = 0; i < mem.size(); ++i) {
        std::memcpy(&mat[i * 3], mesh->material + mem[i] * 3, 3 * sizeof(double));
        std::memcpy(&jac[i * 9], mesh->jacobian + mem[i] * 9, 9 * sizeof(double));
      }
      yt_mesh_desc gm{};
      gm.n_elements = (int64_t)mem.size();
      gm.material = mat.data();
      gm.jacobian = jac.data();
      yt_scheme_desc gs = *scheme;
      gs.order = b->group_n[g] + 1;
      yt_solver* sv = nullptr;
      const yt_status rc = yt_solver_create(&gm, &gs, stream, &sv);
      if (rc != YT_OK) throw Error(rc, std::string("group of order ") + std::to_string(gs.order) + ": " + yt_last_error());
      b->groups.push_back(sv);
      b->faces.base[g] = sv->Pface;
      b->faces.bt[g] = sv->BT;
      b->flops += (double)mem.size() * (sv->flops_local + sv->flops_neigh);
      b->bytes += (double)mem.size() * (sv->bytes_local + sv->bytes_neigh);
    }
    for (size_t g = 0; g < b->group_n.size(); ++g) {
      const auto& mem = b->members[g];
      yt_solver* sv = b->groups[g];
      std::vector<int> conn((size_t)sv->Epad * 4, 0);
      std::vector<int64_t> go(mem.size());
      for (size_t i = 0; i < mem.size(); ++i) {
        const int64_t e = mem[i];
        go[i] = offs[e];
        for (int f = 0; f < 4; ++f) {
          const int64_t n = mesh->neighbours[e * 4 + f];
          const int j = mesh->faces[e * 4 + f], h = mesh->orient[e * 4 + f];
          YT_REQUIRE(n >= 0 && n < b->E, YT_ERR_INVALID, "neighbour index out of range");
          YT_REQUIRE(j >= 0 && j < 4 && h >= 0 && h < 3, YT_ERR_INVALID, "face/orientation out of range");
          conn[i * 4 + f] = (int)((elem_local[n] << 7) | (elem_group[n] << 4) | (j << 2) | h);
        }
      }
      // padding lanes point at element 0 of group 0 with zero flux solvers
      b->d_conn.push_back(dalloc<int>(conn.size()));
      cuda_check(cudaMemcpy(b->d_conn.back(), conn.data(), conn.size() * sizeof(int), cudaMemcpyHostToDevice), "copy conn");
      b->d_offs.push_back(dalloc<int64_t>(go.size()));
      cuda_check(cudaMemcpy(b->d_offs.back(), go.data(), go.size() * sizeof(int64_t), cudaMemcpyHostToDevice), "copy offsets");
    }
    b->staging = dalloc<double>((size_t)b->total_dofs);
    cuda_check(cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "stream");
    b->side.resize(b->groups.size());
    for (auto& s : b->side) cuda_check(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
    b->ev.resize(b->groups.size() + 1);
    for (auto& e : b->ev) cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    cuda_check(cudaStreamSynchronize(st), "batch setup");
    batch_persistent_setup(b.get());
    b->exec = batch_graph(b.get(), b->mode);
    b->config = batch_describe(b.get());
    *out = b.release();
  });
}

extern "C" yt_status yt_batch_set_dofs(yt_batch* b, const double* dofs, yt_memory where, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(b && dofs, YT_ERR_INVALID, "null argument");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double* src = dofs;
    if (where == YT_MEM_HOST) {
      cuda_check(cudaMemcpyAsync(b->staging, dofs, (size_t)b->total_dofs * sizeof(double), cudaMemcpyHostToDevice, st), "H2D dofs");
      src = b->staging;
    } else {
      YT_REQUIRE(where == YT_MEM_DEVICE, YT_ERR_INVALID, "where");
    }
    for (size_t g = 0; g < b->groups.size(); ++g) {
      yt_solver* s = b->groups[g];
      const int64_t total = s->Epad * kNq * s->B;
      k_gather_blocked<<<blocks_for(total, 256), 256, 0, st>>>(src, b->d_offs[g], s->Q, s->E, s->Epad, s->B);
    }
    cuda_check(cudaGetLastError(), "k_gather_blocked");
  });
}

extern "C" yt_status yt_batch_get(yt_batch* b, yt_field field, double* out, yt_memory where, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(b && out, YT_ERR_INVALID, "null argument");
    YT_REQUIRE(field == YT_FIELD_DOFS || field == YT_FIELD_TIME_INTEGRAL, YT_ERR_INVALID, "field");
    YT_REQUIRE(where == YT_MEM_HOST || where == YT_MEM_DEVICE, YT_ERR_INVALID, "where");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double* dst = where == YT_MEM_HOST ? b->staging : out;
    for (size_t g = 0; g < b->groups.size(); ++g) {
      yt_solver* s = b->groups[g];
      const int64_t n = s->E * kNq * s->B;
      k_scatter_blocked<<<blocks_for(n, 256), 256, 0, st>>>(field == YT_FIELD_DOFS ? s->Q : s->I,
                                                           b->d_offs[g], dst, s->E, s->B);
    }
    cuda_check(cudaGetLastError(), "k_scatter_blocked");
    if (where == YT_MEM_HOST)
      cuda_check(cudaMemcpyAsync(out, b->staging, (size_t)b->total_dofs * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H");
  });
}

extern "C" yt_status yt_batch_step(yt_batch* b, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(b && b->exec, YT_ERR_INVALID, "null batch");
    cuda_check(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)), "graph launch");
  });
}

extern "C" yt_status yt_batch_tune(yt_batch* b, int32_t repeats, yt_stream stream, int32_t* chosen) {
  return guarded([&] {
    YT_REQUIRE(b, YT_ERR_INVALID, "null batch");
    YT_REQUIRE(repeats > 0 && repeats <= 1000, YT_ERR_INVALID, "repeats must be 1..1000");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // time each candidate on the caller's data and keep the fastest; the DOFs are saved
    // before and restored after, so tuning leaves the state unchanged.  Candidates: the
    // per-group kernels in sequence and on parallel branches, and the persistent kernel
    // with each item order (by decreasing degree / interleaved) and 1, 2 or 4 tiles per
    // claim.
    const size_t G = b->groups.size();
    std::vector<double*> backup(G, nullptr);
    for (size_t g = 0; g < G; ++g) {
      yt_solver* s = b->groups[g];
      const size_t n = (size_t)s->Epad * kNq * s->B;
      backup[g] = dalloc<double>(n);
      cuda_check(cudaMemcpyAsync(backup[g], s->Q, n * sizeof(double), cudaMemcpyDeviceToDevice, st), "backup");
    }
    cudaEvent_t t0, t1;
    cuda_check(cudaEventCreate(&t0), "event");
    cuda_check(cudaEventCreate(&t1), "event");
    struct Cand { int mode, order, chunk; };
    std::vector<Cand> cands = {{0, 0, 1}, {1, 0, 1}};
    if (b->pers_grid > 0)
      for (int order = 0; order < 2; ++order)
        for (int chunk : {1, 2, 4}) cands.push_back({2, order, chunk});
    float best = 0.0f;
    size_t best_i = 0;
    std::string table;
    for (size_t i = 0; i < cands.size(); ++i) {
      b->pers_order = cands[i].order;
      b->pers_chunk = cands[i].chunk;
      cudaGraphExec_t ex = batch_graph(b, cands[i].mode);
      cuda_check(cudaGraphLaunch(ex, st), "warm-up");
      cuda_check(cudaEventRecord(t0, st), "event");
      for (int r = 0; r < repeats; ++r) cuda_check(cudaGraphLaunch(ex, st), "graph launch");
      cuda_check(cudaEventRecord(t1, st), "event");
      cuda_check(cudaEventSynchronize(t1), "sync");
      float ms = 0.0f;
      cuda_check(cudaEventElapsedTime(&ms, t0, t1), "elapsed");
      ms /= (float)repeats;
      table += (i ? "; " : "") + std::string(cands[i].mode == 0 ? "sequence" : (cands[i].mode == 1 ? "branches" : "persistent")) +
               (cands[i].mode == 2 ? std::string(cands[i].order == 0 ? " by-degree" : " interleaved") + " chunk " +
                                         std::to_string(cands[i].chunk)
                                   : std::string()) +
               " " + std::to_string(ms) + " ms";
      if (i == 0 || ms < best) {
        best = ms;
        best_i = i;
      }
      cudaGraphExecDestroy(ex);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    for (size_t g = 0; g < G; ++g) {
      yt_solver* s = b->groups[g];
      const size_t n = (size_t)s->Epad * kNq * s->B;
      cuda_check(cudaMemcpyAsync(s->Q, backup[g], n * sizeof(double), cudaMemcpyDeviceToDevice, st), "restore");
    }
    cuda_check(cudaMemsetAsync(b->d_counters + 3, 0, sizeof(int), st), "status reset");
    cuda_check(cudaStreamSynchronize(st), "restore sync");
    for (auto* p : backup) cudaFree(p);
    b->pers_order = cands[best_i].order;
    b->pers_chunk = cands[best_i].chunk;
    cudaGraphExec_t ex = batch_graph(b, cands[best_i].mode);
    cudaGraphExecDestroy(b->exec);
    b->exec = ex;
    b->mode = cands[best_i].mode;
    b->config = batch_describe(b) + " (tuned: " + table + ")";
    if (chosen) *chosen = b->mode;
  });
}

extern "C" yt_status yt_batch_config(const yt_batch* b, char* out, int32_t capacity) {
  return guarded([&] {
    YT_REQUIRE(b && out && capacity > 0, YT_ERR_INVALID, "null argument");
    std::strncpy(out, b->config.c_str(), (size_t)capacity - 1);
    out[capacity - 1] = '\0';
  });
}

extern "C" yt_status yt_batch_set_form(yt_batch* b, int32_t form, int32_t order, int32_t chunk) {
  return guarded([&] {
    YT_REQUIRE(b, YT_ERR_INVALID, "null batch");
    YT_REQUIRE(form >= 0 && form <= 2 && order >= 0 && order <= 1 && (chunk == 1 || chunk == 2 || chunk == 4),
               YT_ERR_INVALID, "form 0..2, order 0..1, chunk 1, 2 or 4");
    YT_REQUIRE(form != 2 || b->pers_grid > 0, YT_ERR_UNSUPPORTED, "the persistent kernel does not fit an SM");
    b->pers_order = order;
    b->pers_chunk = chunk;
    cudaGraphExec_t ex = batch_graph(b, form);
    cudaGraphExecDestroy(b->exec);
    b->exec = ex;
    b->mode = form;
    b->config = batch_describe(b);
  });
}

extern "C" yt_status yt_batch_status(yt_batch* b, yt_stream stream) {
  return guarded([&] {
    YT_REQUIRE(b, YT_ERR_INVALID, "null batch");
    cuda_check(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)), "stream synchronize");
    int v = 0;
    cuda_check(cudaMemcpy(&v, b->d_counters + 3, sizeof(int), cudaMemcpyDeviceToHost), "status copy");
    if (v != 0) {
      cuda_check(cudaMemset(b->d_counters + 3, 0, sizeof(int)), "status reset");
      throw Error(YT_ERR_TIMEOUT, "the grid barrier of the persistent batch kernel ran out");
    }
  });
}

extern "C" yt_status yt_batch_stats(const yt_batch* b, double* flops, double* bytes, int32_t* n_groups) {
  return guarded([&] {
    YT_REQUIRE(b, YT_ERR_INVALID, "null batch");
    if (flops) *flops = b->flops;
    if (bytes) *bytes = b->bytes;
    if (n_groups) *n_groups = (int32_t)b->groups.size();
  });
}

extern "C" void yt_batch_destroy(yt_batch* b) { delete b; }
