// Internal view of the solver object, shared by the solver, batch and server code.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/yateto_gb300.h"
#include "ader_kernels.cuh"

struct yt_solver {
  int N = 0, B = 0, BT = 0;
  int P = 9;                          // quantities: 9 elastic, 27 viscoelastic-shaped
  int64_t E = 0, Epad = 0, ntiles = 0;
  yt_precision prec = YT_F64;
  double dt = 0.0;
  bool has_neighbours = false;
  double *Q = nullptr, *I = nullptr, *star = nullptr, *floc = nullptr, *fnb = nullptr,
         *staging = nullptr;
  // buffers of the contraction type (double for YT_F64, float for YT_F32 and the
  // tensor-core form YT_BF16X3_F32ACC, whose per-element products run in binary32)
  void *Pface = nullptr, *Wloc = nullptr, *star_r = nullptr, *floc_r = nullptr, *fnb_r = nullptr;
  int* conn = nullptr;
  double* d_val = nullptr;
  double* d_f = nullptr;
  float* d_val32 = nullptr;
  float* d_f32 = nullptr;
  size_t real_bytes = 8;
  double flops_local = 0, flops_neigh = 0, bytes_local = 0, bytes_neigh = 0;
  double flops_local_unfused = 0;
  int64_t n_values = 0;
  size_t smem_local = 0, smem_neigh = 0;
  // tensor-core form: split-bf16 global-matrix operands of the two kernels, persistent
  // grid size and the status word of the bounded device-side waits
  unsigned char *d_tc_local = nullptr, *d_tc_neigh = nullptr;
  float* d_tc_scratch = nullptr;
  int* d_status = nullptr;
  unsigned tc_grid = 0;
  float* d_tc_vol = nullptr;  // tensor-core form: volume increments [tile][9][B][32]
  bool small_local = false;   // yt_step_local on the small-mesh kernel (tiles <= SMs)
  bool diag_expire_wait = false;     // YT_SCHEME_DIAG_EXPIRE_WAIT
  // 27 quantities: anelastic star slots, relaxation frequencies and flux-solver rows (FP64
  // setup copies and the contraction type's), the derivative scratch of the anelastic
  // functions, shared memory of k_theta
  double *cth = nullptr, *om = nullptr, *fthl = nullptr, *fthn = nullptr;
  void *cth_r = nullptr, *om_r = nullptr, *fthl_r = nullptr, *fthn_r = nullptr, *theta = nullptr;
  size_t smem_theta = 0;
  // partitioned solves: halo block [n_halo][9][BT] (contraction type, group 1 of the
  // neighbour gathers) and the send list
  int64_t n_halo = 0, n_send = 0;
  void* halo = nullptr;
  int* d_send = nullptr;
  // device memory from the stream-ordered allocator on alloc_stream (solvers of a server),
  // else from cudaMalloc
  bool alloc_async = false;
  cudaStream_t alloc_stream = nullptr;
  // yt_step_host: copy stream and per-chunk events (created on first use)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_done = nullptr;
  cudaEvent_t ev_in[16] = {}, ev_out[16] = {};
  void free_device(void* p) {
    if (!p) return;
    if (alloc_async) cudaFreeAsync(p, alloc_stream);
    else cudaFree(p);
  }
  ~yt_solver() {
    if (star_r == (void*)star) star_r = floc_r = fnb_r = nullptr;
    if (cth_r == (void*)cth) cth_r = om_r = fthl_r = fthn_r = nullptr;
    for (void* p : {(void*)cth, (void*)om, (void*)fthl, (void*)fthn, cth_r, om_r, fthl_r, fthn_r, theta,
                    halo, (void*)d_send})
      free_device(p);
    for (cudaEvent_t e : ev_in) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ev_out) if (e) cudaEventDestroy(e);
    if (ev_start) cudaEventDestroy(ev_start);
    if (ev_done) cudaEventDestroy(ev_done);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    for (void* p : {(void*)Q, (void*)I, Pface, Wloc, (void*)star, (void*)floc, (void*)fnb, star_r,
                    floc_r, fnb_r, (void*)staging, (void*)conn, (void*)d_val, (void*)d_f,
                    (void*)d_val32, (void*)d_f32, (void*)d_tc_local, (void*)d_tc_neigh, (void*)d_tc_scratch,
                    (void*)d_tc_vol, (void*)d_status})
      free_device(p);
  }
};


namespace yt {
// Launch description of a solver's kernels on `st` (one problem, no tile table).
AderLaunch solver_launch_args(yt_solver* s, cudaStream_t st);
// Kernel variant of the solver's degree and precision: 0 local (fused step), 1 local
// (complete local update), 2 neighbour (fused step), 3 neighbour (after variant 1).
void solver_launch_variant(yt_solver* s, const AderLaunch& L, int variant);
// Device bytes a solver of this order / precision / size allocates (its tables aside).
size_t solver_device_bytes(int order, yt_precision prec, int64_t n_elements);
// yt_solver_create with every device allocation of the solver taken from the
// stream-ordered allocator on `stream` (and freed there by yt_solver_destroy): creating
// and destroying solvers then never waits for work on other streams.
yt_status solver_create_stream_ordered(const yt_mesh_desc* mesh, const yt_scheme_desc* scheme,
                                       cudaStream_t stream, yt_solver** out);
}  // namespace yt
